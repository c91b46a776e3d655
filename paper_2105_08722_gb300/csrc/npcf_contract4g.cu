// 4PCF contraction for high lmax, FP32 products, FP64 partials: one primary per lane, the
// coupling terms read through L1.
//
// Eq. (simple-NPCF-summation) at N = 4, factorised over b3 with the App. B halving in m3:
//   P^{L,m3}(b1,b2) = sum_{m1} E(L) C^L_{m1,-m1-m3,m3} a^{b1}_{l1 m1} a^{b2}_{l2,-m1-m3}
//   zeta_L(b1,b2,b3) += u 2 S(m3) Q_L[P^{L,m3}(b1,b2) a^{b3}_{l3 m3}]     (b1 < b2 < b3)
// (Q_L = Re for parity-even L, Im for parity-odd L).
//
// The kernel of npcf_contract4.cu keeps the coupling terms and a tile of 64 primaries in
// shared memory, which bounds it to lmax <= 6 (Table 2 of the paper also runs lmax = 10).
// This one stages only a tile of 32 primaries ([lm][b][primary]) and reads the terms with
// warp-uniform loads through L1, so shared memory holds nr (lmax + 1)(lmax + 2) / 2 x 33
// float2 (174 KB at lmax 10 and 10 shells). To use each loaded a^{b2} value more than once,
// the segments m3 of a multiplet are taken two at a time and their terms grouped by the
// stored a^{b2}_{l2 |m2|} they read (the sign of m2 and the conjugation folded into the
// coefficients); a lane holds both segments' P(b2) in registers and contracts them with
// a^{b3} of every b3 > b2 straight away.
#include "npcf_device.h"
#include "npcf_warp.cuh"

#include <algorithm>

namespace npcf {
namespace {

constexpr int kTG = 32;            // primaries per tile (one per lane)
constexpr int kRG = kTG + 1;       // float2 stride of one staged (lm, b) row

__host__ __device__ inline size_t al128g(size_t x) { return (x + 127) & ~size_t(127); }
__host__ __device__ inline size_t c4g_u_offset(int nr, int nlm) {
    return al128g((size_t)nr * nlm * kRG * sizeof(float2));
}

// acc[(b2, b3)] += f Q[P(b1, b2) a3(b3)] (NB2 values of b2, b3 > b2); M0: m3 = 0, a3 real
template <int NB2, bool M0>
__device__ __forceinline__ void contract_b3g(const float2* __restrict__ A3, float f, bool odd,
                                             const float (&pr)[NB2], const float (&pi)[NB2],
                                             float (&acc)[NB2 * (NB2 - 1) / 2]) {
    float2 x3[NB2 - 1];
#pragma unroll
    for (int k = 0; k < NB2 - 1; ++k) x3[k] = A3[k * kRG];
    int e = 0;
#pragma unroll
    for (int k = 0; k < NB2; ++k) {
        // even: Re(P a3) = pr x3 - pi y3 ; odd: Im(P a3) = pi x3 + pr y3
        const float A = f * (odd ? pi[k] : pr[k]);
        if (M0) {
#pragma unroll
            for (int k3 = k; k3 < NB2 - 1; ++k3, ++e) acc[e] = fmaf(A, x3[k3].x, acc[e]);
        } else {
            const float B = f * (odd ? pr[k] : -pi[k]);
#pragma unroll
            for (int k3 = k; k3 < NB2 - 1; ++k3, ++e) acc[e] = fmaf(A, x3[k3].x, fmaf(B, x3[k3].y, acc[e]));
        }
    }
}

// P of the two segments of a pair for one primary. MODE: how the first segment sums
// (0: both parts; 1: real part only; 2: imaginary part only, both for m3 = 0).
template <int NB2, int MODE>
__device__ __forceinline__ void build_pair(const float2* __restrict__ Xl, int g0, int g1, int lmstride,
                                           const Contract4GArgs& a, float (&ar)[NB2], float (&ai)[NB2],
                                           float (&br)[NB2], float (&bi)[NB2]) {
#pragma unroll
    for (int k = 0; k < NB2; ++k) ar[k] = ai[k] = br[k] = bi[k] = 0.f;
    for (int g = g0; g < g1; ++g) {
        const int4 G = __ldg(&a.groups[g]);   // terms of segment 0 [x, y), of segment 1 [y, z), lm2
        float2 y[NB2];
#pragma unroll
        for (int k = 0; k < NB2; ++k) y[k] = Xl[G.w * lmstride + (k + 1) * kRG];
        // re += cA x1 x2 + cB y1 y2 ; im += cC y1 x2 + cD x1 y2 (conjugations folded in c)
        for (int t = G.x; t < G.y; ++t) {
            const float4 c = __ldg(&a.coef[t]);
            const float2 x1 = Xl[__ldg(&a.tlm[t]) * lmstride];
            const float a0 = c.x * x1.x, a1 = c.y * x1.y, a2 = c.z * x1.y, a3 = c.w * x1.x;
#pragma unroll
            for (int k = 0; k < NB2; ++k) {
                if (MODE != 2) ar[k] = fmaf(a0, y[k].x, fmaf(a1, y[k].y, ar[k]));
                if (MODE != 1) ai[k] = fmaf(a2, y[k].x, fmaf(a3, y[k].y, ai[k]));
            }
        }
        for (int t = G.y; t < G.z; ++t) {
            const float4 c = __ldg(&a.coef[t]);
            const float2 x1 = Xl[__ldg(&a.tlm[t]) * lmstride];
            const float a0 = c.x * x1.x, a1 = c.y * x1.y, a2 = c.z * x1.y, a3 = c.w * x1.x;
#pragma unroll
            for (int k = 0; k < NB2; ++k) {
                br[k] = fmaf(a0, y[k].x, fmaf(a1, y[k].y, br[k]));
                bi[k] = fmaf(a2, y[k].x, fmaf(a3, y[k].y, bi[k]));
            }
        }
    }
}

template <int NB2>
__device__ __forceinline__ void c4g_item(const int4 item, const float2* __restrict__ X, float u, int lmstride,
                                         const Contract4GArgs& a, double* __restrict__ dst, int lane) {
    constexpr int NOUT = NB2 * (NB2 - 1) / 2;
    const int b1 = item.z & 0xff;
    const bool odd = ((item.z >> 8) & 1) != 0;
    const float2* Xl = X + lane + b1 * kRG;
    float acc[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) acc[i] = 0.f;
    for (int q = item.x; q < item.y; ++q) {
        const int4 P0 = __ldg(&a.pairs[2 * q]);       // groups [x, y), lm3 of the two segments (w < 0: one)
        const int4 P1 = __ldg(&a.pairs[2 * q + 1]);   // 2 S(m3) of both (bits), m3 = 0 of the first
        float ar[NB2], ai[NB2], br[NB2], bi[NB2];
        const float2* A3 = Xl + P0.z * lmstride + 2 * kRG;
        if (P1.z == 0) {
            build_pair<NB2, 0>(Xl, P0.x, P0.y, lmstride, a, ar, ai, br, bi);
            contract_b3g<NB2, false>(A3, u * __int_as_float(P1.x), odd, ar, ai, acc);
        } else {
            if (odd)
                build_pair<NB2, 2>(Xl, P0.x, P0.y, lmstride, a, ar, ai, br, bi);
            else
                build_pair<NB2, 1>(Xl, P0.x, P0.y, lmstride, a, ar, ai, br, bi);
            contract_b3g<NB2, true>(A3, u * __int_as_float(P1.x), odd, ar, ai, acc);
        }
        if (P0.w >= 0)
            contract_b3g<NB2, false>(Xl + P0.w * lmstride + 2 * kRG, u * __int_as_float(P1.y), odd, br, bi, acc);
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
__global__ void __launch_bounds__(THREADS, 1) k_contract4g(const Contract4GArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    float2* X = reinterpret_cast<float2*>(dsm);
    float* su = reinterpret_cast<float*>(dsm + c4g_u_offset(a.nr, a.nlm));
    __shared__ int chunk_s, item_next;

    const int tid = threadIdx.x, lane = tid & 31;
    const int rows = a.nr * a.nlm;
    const int lmstride = a.nr * kRG;   // one harmonic row of every shell
    // chunks (primary ranges of one catalog) are taken dynamically; chunk c sums into row c
    for (;;) {
        if (tid == 0) chunk_s = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        const int c = chunk_s;
        if (c >= a.nchunk) break;
        const int2 C = a.chunks[c];
        double* dst = a.partial + (size_t)c * a.total;
        for (int i = tid; i < a.nout; i += blockDim.x) dst[a.out_off + i] = 0.0;
        for (int p0 = C.x; p0 < C.y; p0 += kTG) {
            const int np = min(kTG, C.y - p0);
            if (tid == 0) item_next = 0;
            // stage [lm][b][q] from the pair kernel's [q][b][lm]
            const float2* src = a.alm + (size_t)p0 * rows;
            for (int i = tid; i < kTG * rows; i += blockDim.x) {
                const int q = i / rows, r = i - q * rows;   // r = b * nlm + lm
                const int b = r / a.nlm, lm = r - b * a.nlm;
                X[(lm * a.nr + b) * kRG + q] = q < np ? src[i] : make_float2(0.f, 0.f);
            }
            if (tid < kTG) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
            __syncthreads();   // also orders the row's zeroing before the first sums
            const float u = su[lane];
            for (;;) {
                int it = 0;
                if (lane == 0) it = atomicAdd(&item_next, 1);
                it = __shfl_sync(warp::kFullMask, it, 0);
                if (it >= a.nitem) break;
                const int4 item = __ldg(&a.items[it]);
                switch ((item.z >> 16) & 0xff) {
#define NPCF_C4G_CASE(K) \
    case K:              \
        if (K <= NBMAX) c4g_item<(K <= NBMAX ? K : 2)>(item, X, u, lmstride, a, dst, lane); \
        break;
                    NPCF_C4G_CASE(2) NPCF_C4G_CASE(3) NPCF_C4G_CASE(4) NPCF_C4G_CASE(5) NPCF_C4G_CASE(6)
                    NPCF_C4G_CASE(7) NPCF_C4G_CASE(8) NPCF_C4G_CASE(9) NPCF_C4G_CASE(10) NPCF_C4G_CASE(11)
                    NPCF_C4G_CASE(12) NPCF_C4G_CASE(13) NPCF_C4G_CASE(14) NPCF_C4G_CASE(15)
#undef NPCF_C4G_CASE
                    default: break;
                }
            }
            __syncthreads();
        }
        __syncthreads();   // every thread has read chunk_s before it is taken again
    }
}

}  // namespace

size_t contract4g_smem_bytes(int nr, int nlm) {
    return al128g(c4g_u_offset(nr, nlm) + kTG * sizeof(float));
}

void launch_contract4g(const Contract4GArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = contract4g_smem_bytes(a.nr, a.nlm);
    // up to 10 shells: 16 warps of <= 128 registers; more shells hold more sums per lane
    if (a.nr <= 10) {
        cudaFuncSetAttribute(k_contract4g<9, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract4g<9, 512><<<nblocks, 512, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_contract4g<15, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract4g<15, 256><<<nblocks, 256, smem, s>>>(a);
    }
}

}  // namespace npcf
