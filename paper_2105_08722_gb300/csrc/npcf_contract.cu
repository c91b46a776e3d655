// Contraction of per-primary a^b_lm into the raw multiplets (FP32 CUDA-core path)
// and the FP64 cross-block reduction.
//
// 3PCF (Eq. N=3-coeff with App. B halving):
//   zeta_l(b1,b2) = sum_i u_i (l l 0; 0 0 0) sum_{m=-l..l} a^{b1}_{lm} conj(a^{b2}_{lm})
//                 = sum_i u_i (-1)^l / sqrt(2l+1) [a_{l0} a_{l0} + 2 sum_{m>0} Re(a1 conj a2)].
// 4PCF (Eq. simple-NPCF-summation at N=4, Algorithm 3 factorised over b3):
//   P^{L,m3}(b1,b2) = sum_{m1} E C^L_{m1,-m1-m3,m3} a^{b1}_{l1 m1} a^{b2}_{l2,-m1-m3}
//   zeta_L(b1,b2,b3) = sum_i u_i sum_{m3>=0} 2 S(m3) Q_L[P^{L,m3}(b1,b2) a^{b3}_{l3 m3}].
// Each block owns a contiguous chunk of cell-sorted primaries and a set of output rows;
// FP32 sums over the chunk go to a per-chunk FP64 partial, and the reduction adds the
// partials in chunk order, so results do not depend on scheduling.
#include "npcf_device.h"

namespace npcf {
namespace {

constexpr int kTile = 8;   // primaries staged in shared memory at a time

__device__ __forceinline__ void stage_tile(const float2* __restrict__ alm, const float* __restrict__ wp,
                                           int p0, int np, int per, float2* X, float* su) {
    // per = nr * nlm complex values per primary; copy np primaries (contiguous)
    const float2* src = alm + (size_t)p0 * per;
    int total = np * per;
    for (int i = threadIdx.x; i < total; i += blockDim.x) X[i] = src[i];
    for (int i = threadIdx.x; i < np; i += blockDim.x) su[i] = wp[p0 + i];
}

__global__ void k_contract3(const Contract3Args a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int per = a.nr * a.nlm;
    float2* X = reinterpret_cast<float2*>(dsm);
    float* su = reinterpret_cast<float*>(X + kTile * per);
    const int chunk = blockIdx.x;
    const int p0 = chunk * a.chunk;
    const int p1 = min(a.n, p0 + a.chunk);
    const int r = threadIdx.x;
    int l = 0, b1 = 0, b2 = 0, pr = 0;
    if (r < a.nrows) {
        int2 rw = a.rows[r];
        l = rw.x;
        pr = rw.y;
        int2 bb = a.pairs[pr];
        b1 = bb.x;
        b2 = bb.y;
    }
    float acc = 0.f;
    const int lm0 = l * (l + 1) / 2;
    for (int t0 = p0; t0 < p1; t0 += kTile) {
        const int np = min(kTile, p1 - t0);
        __syncthreads();
        stage_tile(a.alm, a.wp, t0, np, per, X, su);
        __syncthreads();
        if (r < a.nrows) {
            for (int q = 0; q < np; ++q) {
                const float2* A1 = X + q * per + b1 * a.nlm + lm0;
                const float2* A2 = X + q * per + b2 * a.nlm + lm0;
                float s = A1[0].x * A2[0].x;
                float s2 = 0.f;
                for (int m = 1; m <= l; ++m) s2 = fmaf(A1[m].x, A2[m].x, fmaf(A1[m].y, A2[m].y, s2));
                acc = fmaf(su[q], fmaf(2.f, s2, s), acc);
            }
        }
    }
    if (r < a.nrows && chunk < a.nchunk)
        a.partial[(size_t)chunk * a.total + a.out_off + l * a.nbins + pr] = (double)a.coef[l] * (double)acc;
}

__global__ void k_contract4(const Contract4Args a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int per = a.nr * a.nlm;
    float4* tc = reinterpret_cast<float4*>(dsm);
    uint32_t* ti = reinterpret_cast<uint32_t*>(tc + a.nterms);
    int4* seg = reinterpret_cast<int4*>(ti + ((a.nterms + 3) & ~3));
    float2* X = reinterpret_cast<float2*>(seg + a.nseg);
    float* su = reinterpret_cast<float*>(X + kTile * per);

    for (int i = threadIdx.x; i < a.nterms; i += blockDim.x) {
        const PairTerm t = a.terms[i];
        tc[i] = make_float4(t.cA, t.cB, t.cC, t.cD);
        ti[i] = (uint32_t)t.lm1 | ((uint32_t)t.lm2 << 16);
    }
    for (int i = threadIdx.x; i < a.nseg; i += blockDim.x)
        seg[i] = make_int4(a.seg_begin[i], a.seg_end[i], a.seg_lm3[i], __float_as_int(a.seg_factor[i]));

    const int chunk = blockIdx.x;
    const int p0 = chunk * a.chunk;
    const int p1 = min(a.n, p0 + a.chunk);
    const int row = blockIdx.y * blockDim.x + threadIdx.x;
    const bool valid = row < a.nrows;
    int4 rw = valid ? a.rows[row] : make_int4(0, 0, 0, 0);
    const int lam = rw.x, b1 = rw.y, b2 = rw.z;
    const int sg0 = valid ? a.lam_seg0[lam] : 0, sg1 = valid ? a.lam_seg0[lam + 1] : 0;
    const bool odd = valid ? a.lam_odd[lam] != 0 : false;

    float acc[kMaxNr];
#pragma unroll
    for (int i = 0; i < kMaxNr; ++i) acc[i] = 0.f;

    for (int t0 = p0; t0 < p1; t0 += kTile) {
        const int np = min(kTile, p1 - t0);
        __syncthreads();
        stage_tile(a.alm, a.wp, t0, np, per, X, su);
        __syncthreads();
        if (!valid) continue;
        for (int q = 0; q < np; ++q) {
            const float u = su[q];
            if (u == 0.f) continue;
            const float2* Xq = X + q * per;
            const float2* A1 = Xq + b1 * a.nlm;
            const float2* A2 = Xq + b2 * a.nlm;
            for (int sg = sg0; sg < sg1; ++sg) {
                const int4 S = seg[sg];
                float pr = 0.f, pim = 0.f;
                for (int t = S.x; t < S.y; ++t) {
                    const float4 c = tc[t];
                    const uint32_t id = ti[t];
                    const float2 x1 = A1[id & 0xffffu];
                    const float2 x2 = A2[id >> 16];
                    pr = fmaf(c.x * x1.x, x2.x, pr);
                    pr = fmaf(c.y * x1.y, x2.y, pr);
                    pim = fmaf(c.z * x1.y, x2.x, pim);
                    pim = fmaf(c.w * x1.x, x2.y, pim);
                }
                const float f = __int_as_float(S.w) * u;
                // even: Re(P a3) = pr x3 - pi y3 ; odd: Im(P a3) = pi x3 + pr y3
                const float A = f * (odd ? pim : pr);
                const float B = f * (odd ? pr : -pim);
#pragma unroll
                for (int b3 = 0; b3 < kMaxNr; ++b3) {
                    if (b3 > b2 && b3 < a.nr) {
                        const float2 x3 = Xq[b3 * a.nlm + S.z];
                        acc[b3] = fmaf(A, x3.x, fmaf(B, x3.y, acc[b3]));
                    }
                }
            }
        }
    }
    if (valid && chunk < a.nchunk) {
        double* dst = a.partial + (size_t)chunk * a.total + rw.w;
#pragma unroll
        for (int b3 = 0; b3 < kMaxNr; ++b3)
            if (b3 > b2 && b3 < a.nr) dst[b3 - b2 - 1] = (double)acc[b3];
    }
}

// FP64 sum over the chunks' partials, times the multiplet's harmonic normalisation
// prod_k sqrt((2 l_k + 1)/(4 pi)) (the contractions work on reduced harmonics).
__global__ void k_reduce(const double* __restrict__ partial, int nchunk, int total,
                         const double* __restrict__ scale, double* __restrict__ zeta) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[(size_t)c * total + e];
    zeta[e] += s * scale[e];
}

}  // namespace

void launch_contract3(const Contract3Args& a, cudaStream_t s) {
    const int per = a.nr * a.nlm;
    size_t smem = (size_t)kTile * per * sizeof(float2) + kTile * sizeof(float);
    int threads = ((a.nrows + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    k_contract3<<<a.nchunk, threads, smem, s>>>(a);
}

size_t contract4_smem_bytes(const Contract4Args& a) {
    const int per = a.nr * a.nlm;
    return (size_t)a.nterms * sizeof(float4) + (size_t)((a.nterms + 3) & ~3) * sizeof(uint32_t) +
           (size_t)a.nseg * sizeof(int4) + (size_t)kTile * per * sizeof(float2) + kTile * sizeof(float);
}

void launch_contract4(const Contract4Args& a, cudaStream_t s) {
    size_t smem = contract4_smem_bytes(a);
    cudaFuncSetAttribute(k_contract4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int threads = 256;
    dim3 grid(a.nchunk, (a.nrows + threads - 1) / threads);
    k_contract4<<<grid, threads, smem, s>>>(a);
}

void launch_reduce(const double* partial, int nchunk, int total, const double* scale, double* zeta,
                   cudaStream_t s) {
    k_reduce<<<(total + 255) / 256, 256, 0, s>>>(partial, nchunk, total, scale, zeta);
}

}  // namespace npcf
