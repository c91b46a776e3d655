// Contraction of per-primary a^b_lm into the raw multiplets (FP32 CUDA-core path)
// and the FP64 cross-block reduction.
//
// 3PCF (Eq. N=3-coeff with App. B halving):
//   zeta_l(b1,b2) = sum_i u_i (l l 0; 0 0 0) sum_{m=-l..l} a^{b1}_{lm} conj(a^{b2}_{lm})
//                 = sum_i u_i (-1)^l / sqrt(2l+1) [a_{l0} a_{l0} + 2 sum_{m>0} Re(a1 conj a2)].
// Each block owns a chunk of cell-sorted primaries (a range within one catalog) and a set
// of output rows; FP32 sums over the chunk go to the chunk's FP64 partial row, and the
// reduction adds a catalog's rows in chunk order, so results do not depend on scheduling.
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
    const int2 C = a.chunks[chunk];   // primaries [C.x, C.y) of one catalog
    const int p0 = C.x, p1 = C.y;
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
    // FP32 sums over one tile of primaries, folded into FP64 after every tile, so the
    // rounding does not grow with the chunk length
    double dacc = 0.0;
    const int lm0 = l * (l + 1) / 2;
    for (int t0 = p0; t0 < p1; t0 += kTile) {
        const int np = min(kTile, p1 - t0);
        __syncthreads();
        stage_tile(a.alm, a.wp, t0, np, per, X, su);
        __syncthreads();
        if (r < a.nrows) {
            float acc = 0.f;
            for (int q = 0; q < np; ++q) {
                const float2* A1 = X + q * per + b1 * a.nlm + lm0;
                const float2* A2 = X + q * per + b2 * a.nlm + lm0;
                float s = A1[0].x * A2[0].x;
                float s2 = 0.f;
                for (int m = 1; m <= l; ++m) s2 = fmaf(A1[m].x, A2[m].x, fmaf(A1[m].y, A2[m].y, s2));
                acc = fmaf(su[q], fmaf(2.f, s2, s), acc);
            }
            dacc += (double)acc;
        }
    }
    if (r < a.nrows && chunk < a.nchunk)
        a.partial[(size_t)chunk * a.total + a.out_off + l * a.nbins + pr] = (double)a.coef[l] * dacc;
}

// Catalog blockIdx.y: its chunks' partial rows in order, times the harmonic scale.
__global__ void k_reduce(const double* __restrict__ partial, const int* __restrict__ cbeg, int total, int off,
                         int count, const double* __restrict__ scale, double* __restrict__ zeta) {
    const int e = off + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= off + count) return;
    const int k = blockIdx.y, r0 = cbeg[k], r1 = cbeg[k + 1];
    double s = 0.0;
    for (int c = r0; c < r1; ++c) s += partial[(size_t)c * total + e];
    zeta[(size_t)k * total + e] += s * scale[e];
}

// Sum of weights of catalog blockIdx.y (the blocks along x share its range), added to
// sumw[k] (only the normalisation uses it).
__global__ void k_sumw(const float* __restrict__ w, const long long* __restrict__ off, double* sumw) {
    const int k = blockIdx.y;
    const long long i0 = off[k], i1 = off[k + 1];
    double s = 0.0;
    for (long long i = i0 + blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (long long)gridDim.x * blockDim.x)
        s += w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
        atomicAdd(&sumw[k], t);
    }
}

// Cached harmonics of data primaries (the re-use of the data part across random splits):
// per-primary rows of `row` float2 and `rc` counts moved between cell order and input order.
__global__ void k_alm_to_input(const float2* __restrict__ alm, const uint32_t* __restrict__ cnt,
                               const uint32_t* __restrict__ idx, int n, int row, int rc, float2* __restrict__ alm_in,
                               uint32_t* __restrict__ cnt_in) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * row;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / row), r = (int)(i - (long long)p * row);
        alm_in[(size_t)idx[p] * row + r] = alm[i];
        if (r < rc) cnt_in[(size_t)idx[p] * rc + r] = cnt[(size_t)p * rc + r];
    }
}

__global__ void k_alm_from_input(const float2* __restrict__ alm_in, const uint32_t* __restrict__ cnt_in,
                                 const uint32_t* __restrict__ idx, int n, int row, int rc, float2* __restrict__ alm,
                                 uint32_t* __restrict__ cnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * row;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / row), r = (int)(i - (long long)p * row);
        alm[i] = alm_in[(size_t)idx[p] * row + r];
        if (r < rc) cnt[(size_t)p * rc + r] = cnt_in[(size_t)idx[p] * rc + r];
    }
}

__global__ void k_add_counts(unsigned long long* dst, const unsigned long long* src, int n) {
    if (threadIdx.x < n) dst[threadIdx.x] += src[threadIdx.x];
}

__global__ void k_set4(long long* dst, long long a, long long b, long long c, long long d) {
    dst[0] = a;
    dst[1] = b;
    dst[2] = c;
    dst[3] = d;
}

}  // namespace

void launch_alm_to_input(const float2* alm, const uint32_t* cnt, const uint32_t* idx, int n, int row, int rc,
                         float2* alm_in, uint32_t* cnt_in, cudaStream_t s) {
    if (n > 0) k_alm_to_input<<<1024, 256, 0, s>>>(alm, cnt, idx, n, row, rc, alm_in, cnt_in);
}

void launch_alm_from_input(const float2* alm_in, const uint32_t* cnt_in, const uint32_t* idx, int n, int row, int rc,
                           float2* alm, uint32_t* cnt, cudaStream_t s) {
    if (n > 0) k_alm_from_input<<<1024, 256, 0, s>>>(alm_in, cnt_in, idx, n, row, rc, alm, cnt);
}

void launch_add_counts(unsigned long long* dst, const unsigned long long* src, int n, cudaStream_t s) {
    k_add_counts<<<1, 32, 0, s>>>(dst, src, n);
}

void launch_set4(long long* dst, long long a, long long b, long long c, long long d, cudaStream_t s) {
    k_set4<<<1, 1, 0, s>>>(dst, a, b, c, d);
}

void launch_contract3(const Contract3Args& a, cudaStream_t s) {
    const int per = a.nr * a.nlm;
    size_t smem = (size_t)kTile * per * sizeof(float2) + kTile * sizeof(float);
    int threads = ((a.nrows + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    k_contract3<<<a.nchunk, threads, smem, s>>>(a);
}

void launch_reduce(const double* partial, const int* cbeg, int ncat, int total, int off, int count,
                   const double* scale, double* zeta, cudaStream_t s) {
    if (count <= 0 || ncat <= 0) return;
    k_reduce<<<dim3((count + 255) / 256, ncat), 256, 0, s>>>(partial, cbeg, total, off, count, scale, zeta);
}

void launch_sumw(const float* w, const long long* off, int ncat, double* sumw, cudaStream_t s) {
    if (ncat > 0) k_sumw<<<dim3(32, ncat), 512, 0, s>>>(w, off, sumw);
}

}  // namespace npcf
