// 4PCF contraction on the CUDA cores, FP32 products, FP64 partials.
//
// Eq. (simple-NPCF-summation) at N = 4, factorised over b3 with the App. B halving in m3:
//   P^{L,m3}(b1,b2) = sum_{m1} E(L) C^L_{m1,-m1-m3,m3} a^{b1}_{l1 m1} a^{b2}_{l2,-m1-m3}
//   zeta_L(b1,b2,b3) += u 2 S(m3) Q_L[P^{L,m3}(b1,b2) a^{b3}_{l3 m3}]     (b1 < b2 < b3)
// (Q_L = Re for parity-even L, Im for parity-odd L).
//
// Lanes are primaries. A block stages the a_lm of 64 primaries in shared memory as
// [lm][b][primary] and its warps take items (L, b1) one at a time. For one item a lane
// holds, for each of its two primaries, P^{L,m3}(b1, b2) of every b2 > b1 in registers
// and contracts it straight away with a^{b3}_{l3 m3} of every b3 > b2 into the item's
// (b2, b3) sums, also in registers. Coupling coefficients, loop bounds and branches are
// the same on every lane, so each coefficient is one broadcast load and no lane waits on
// another; a_lm loads are consecutive across lanes. When the tile is done the warp
// reduces its sums across lanes (transpose-reduction) and adds them to the FP64 partial
// row of the chunk the tile belongs to. Chunks (ranges of primaries within one catalog)
// are taken from a global counter, so blocks stay busy to the end.
#include "npcf_device.h"
#include "npcf_warp.cuh"

#include <algorithm>

namespace npcf {
namespace {

constexpr int kT4 = 64;              // primaries per tile (two per lane)
constexpr int kRS = kT4 + 1;         // float2 stride of one staged (lm, b) row

struct C4Layout {
    size_t X, u, coef, toff, segs, total;
};

__host__ __device__ inline size_t al128(size_t x) { return (x + 127) & ~size_t(127); }

__host__ __device__ inline C4Layout c4_layout(int nr, int nlm, int nterms, int nseg) {
    C4Layout l;
    l.X = 0;
    l.u = al128(l.X + (size_t)nr * nlm * kRS * sizeof(float2));
    l.coef = al128(l.u + kT4 * sizeof(float));
    l.toff = al128(l.coef + (size_t)nterms * sizeof(float4));
    l.segs = al128(l.toff + (size_t)nterms * sizeof(int2));
    l.total = al128(l.segs + (size_t)nseg * sizeof(int4));
    return l;
}

// P of one segment for two primaries (a: lane, b: lane + 32).
// MODE 0: real and imaginary parts; 1: real part only; 2: imaginary part only.
template <int NB2, int MODE>
__device__ __forceinline__ void build_p(const float2* __restrict__ Xl, int b1off, int t0, int t1,
                                        const float4* __restrict__ coef, const int2* __restrict__ toff,
                                        float (&pra)[NB2], float (&pia)[NB2], float (&prb)[NB2],
                                        float (&pib)[NB2]) {
#pragma unroll
    for (int k = 0; k < NB2; ++k) pra[k] = pia[k] = prb[k] = pib[k] = 0.f;
    for (int t = t0; t < t1; ++t) {
        const float4 c = coef[t];
        const int2 o = toff[t];
        const float2* A1 = Xl + o.x + b1off;
        const float2* A2 = Xl + o.y + b1off + kRS;   // shell b1 + 1
        const float2 x1a = A1[0], x1b = A1[32];
        // re += cA x1 x2 + cB y1 y2 ; im += cC y1 x2 + cD x1 y2 (conjugations folded in c)
        const float a0 = c.x * x1a.x, a1 = c.y * x1a.y, a2 = c.z * x1a.y, a3 = c.w * x1a.x;
        const float q0 = c.x * x1b.x, q1 = c.y * x1b.y, q2 = c.z * x1b.y, q3 = c.w * x1b.x;
#pragma unroll
        for (int k = 0; k < NB2; ++k) {
            const float2 ya = A2[k * kRS], yb = A2[k * kRS + 32];
            if (MODE != 2) {
                pra[k] = fmaf(a0, ya.x, fmaf(a1, ya.y, pra[k]));
                prb[k] = fmaf(q0, yb.x, fmaf(q1, yb.y, prb[k]));
            }
            if (MODE != 1) {
                pia[k] = fmaf(a2, ya.x, fmaf(a3, ya.y, pia[k]));
                pib[k] = fmaf(q2, yb.x, fmaf(q3, yb.y, pib[k]));
            }
        }
    }
}

// acc[(b2, b3)] += f Q[P(b1, b2) a3(b3)] for one primary; M0: m3 = 0 (a3 real, one part of P)
template <int NB2, bool M0>
__device__ __forceinline__ void contract_b3(const float2* __restrict__ A3, float f, bool odd,
                                            const float (&pr)[NB2], const float (&pi)[NB2],
                                            float (&acc)[NB2 * (NB2 - 1) / 2]) {
    float2 x3[NB2 - 1];
#pragma unroll
    for (int k = 0; k < NB2 - 1; ++k) x3[k] = A3[k * kRS];
    int e = 0;
#pragma unroll
    for (int k = 0; k < NB2; ++k) {
        if (M0) {
            const float A = f * (odd ? pi[k] : pr[k]);
#pragma unroll
            for (int k3 = k; k3 < NB2 - 1; ++k3, ++e) acc[e] = fmaf(A, x3[k3].x, acc[e]);
        } else {
            // even: Re(P a3) = pr x3 - pi y3 ; odd: Im(P a3) = pi x3 + pr y3
            const float A = f * (odd ? pi[k] : pr[k]);
            const float B = f * (odd ? pr[k] : -pi[k]);
#pragma unroll
            for (int k3 = k; k3 < NB2 - 1; ++k3, ++e) acc[e] = fmaf(A, x3[k3].x, fmaf(B, x3[k3].y, acc[e]));
        }
    }
}

template <int NB2>
__device__ __forceinline__ void c4_item(const int4 item, const float2* __restrict__ X, const float* __restrict__ su,
                                     const float4* __restrict__ coef, const int2* __restrict__ toff,
                                     const int4* __restrict__ segs, double* __restrict__ dst, int lane) {
    constexpr int NOUT = NB2 * (NB2 - 1) / 2;
    const int b1 = item.z & 0xff;
    const bool odd = ((item.z >> 8) & 1) != 0;
    const int b1off = b1 * kRS;
    const float2* Xl = X + lane;
    const float ua = su[lane], ub = su[lane + 32];
    float acc[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) acc[i] = 0.f;
    for (int sg = item.x; sg < item.y; ++sg) {
        const int4 S = segs[sg];   // (first term, end, row of a_{l3 m3} shell 0, 2 S(m3) bits)
        const float f = __int_as_float(S.w);
        const float2* A3 = Xl + S.z + b1off + 2 * kRS;   // shell b1 + 2
        float pra[NB2], pia[NB2], prb[NB2], pib[NB2];
        if (f == 1.f) {   // m3 = 0: a_{l3 0} is real, only one part of P contributes
            if (odd)
                build_p<NB2, 2>(Xl, b1off, S.x, S.y, coef, toff, pra, pia, prb, pib);
            else
                build_p<NB2, 1>(Xl, b1off, S.x, S.y, coef, toff, pra, pia, prb, pib);
            contract_b3<NB2, true>(A3, f * ua, odd, pra, pia, acc);
            contract_b3<NB2, true>(A3 + 32, f * ub, odd, prb, pib, acc);
        } else {
            build_p<NB2, 0>(Xl, b1off, S.x, S.y, coef, toff, pra, pia, prb, pib);
            contract_b3<NB2, false>(A3, f * ua, odd, pra, pia, acc);
            contract_b3<NB2, false>(A3 + 32, f * ub, odd, prb, pib, acc);
        }
    }
    using R = warp::TR<NOUT>;
    R::run(acc, lane);
#pragma unroll
    for (int i = 0; i < R::F; ++i) {
        const int e = R::origin(i, lane);
        if (e >= 0) dst[item.w + e] += (double)acc[i];
    }
}

template <int NBMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_contract4w(const Contract4WArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const C4Layout lay = c4_layout(a.nr, a.nlm, a.nterms, a.nseg);
    float2* X = reinterpret_cast<float2*>(dsm + lay.X);
    float* su = reinterpret_cast<float*>(dsm + lay.u);
    float4* coef = reinterpret_cast<float4*>(dsm + lay.coef);
    int2* toff = reinterpret_cast<int2*>(dsm + lay.toff);
    int4* segs = reinterpret_cast<int4*>(dsm + lay.segs);
    __shared__ int chunk_s, item_next;

    const int tid = threadIdx.x, lane = tid & 31;
    const int rows = a.nr * a.nlm;
    for (int i = tid; i < a.nterms; i += blockDim.x) {
        const PairTerm t = a.terms[i];
        coef[i] = make_float4(t.cA, t.cB, t.cC, t.cD);
        toff[i] = make_int2(t.lm1 * a.nr * kRS, t.lm2 * a.nr * kRS);
    }
    for (int i = tid; i < a.nseg; i += blockDim.x) {
        const int4 S = a.segs[i];   // (first term, end, lm of a_{l3 m3}, 2 S(m3) bits)
        segs[i] = make_int4(S.x, S.y, S.z * a.nr * kRS, S.w);
    }
    // chunks (primary ranges of one catalog) are taken dynamically; chunk c sums into row c
    for (;;) {
        if (tid == 0) chunk_s = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        const int c = chunk_s;
        if (c >= a.nchunk) break;
        const int2 C = a.chunks[c];
        double* dst = a.partial + (size_t)c * a.total;
        for (int i = tid; i < a.nout; i += blockDim.x) dst[a.out_off + i] = 0.0;
        for (int p0 = C.x; p0 < C.y; p0 += kT4) {
        const int np = min(kT4, C.y - p0);
        if (tid == 0) item_next = 0;
        // stage [lm][b][q] from the pair kernel's [q][b][lm]
        const float2* src = a.alm + (size_t)p0 * rows;
        for (int i = tid; i < kT4 * rows; i += blockDim.x) {
            const int q = i / rows, r = i - q * rows;   // r = b * nlm + lm
            const int b = r / a.nlm, lm = r - b * a.nlm;
            X[(lm * a.nr + b) * kRS + q] = q < np ? src[i] : make_float2(0.f, 0.f);
        }
        if (tid < kT4) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
        __syncthreads();   // also orders the row's zeroing before the first sums
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(&item_next, 1);
            it = __shfl_sync(warp::kFullMask, it, 0);
            if (it >= a.nitem) break;
            const int4 item = a.items[it];
            switch ((item.z >> 16) & 0xff) {
#define NPCF_C4_CASE(K) \
    case K:             \
        if (K <= NBMAX) c4_item<(K <= NBMAX ? K : 2)>(item, X, su, coef, toff, segs, dst, lane); \
        break;
                NPCF_C4_CASE(2) NPCF_C4_CASE(3) NPCF_C4_CASE(4) NPCF_C4_CASE(5) NPCF_C4_CASE(6)
                NPCF_C4_CASE(7) NPCF_C4_CASE(8) NPCF_C4_CASE(9) NPCF_C4_CASE(10) NPCF_C4_CASE(11)
                NPCF_C4_CASE(12) NPCF_C4_CASE(13) NPCF_C4_CASE(14) NPCF_C4_CASE(15)
#undef NPCF_C4_CASE
                default: break;
            }
        }
        __syncthreads();
        }
        __syncthreads();   // every thread has read chunk_s before it is taken again
    }
}

}  // namespace

size_t contract4w_smem_bytes(const Contract4WArgs& a) {
    return c4_layout(a.nr, a.nlm, a.nterms, a.nseg).total;
}

int contract4w_blocks(int nsm, int nchunk) { return std::max(1, std::min(nsm, nchunk)); }

void launch_contract4w(const Contract4WArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = contract4w_smem_bytes(a);
    // up to 10 shells: 16 warps of <= 128 registers; more shells hold more sums per lane
    if (a.nr <= 10) {
        cudaFuncSetAttribute(k_contract4w<9, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract4w<9, 512><<<nblocks, 512, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_contract4w<15, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract4w<15, 256><<<nblocks, 256, smem, s>>>(a);
    }
}

}  // namespace npcf
