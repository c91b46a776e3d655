// 5PCF contraction on the CUDA cores, FP32 products, FP64 partials; primaries on the lanes.
//
// For L = (l1, l2, l12, l3, l4), Eq. (basis-coupling) at N = 5 couples two pairs of
// harmonic coefficients through an intermediate m12:
//   E C^L_M = sqrt(2 l12 + 1) (-1)^{l12-m12} (l1 l2 l12; m1 m2 -m12) (l12 l3 l4; m12 m3 m4),
// so the sum over M of Eq. (NPCF-mult-discrete-binned-estimator) factorises into
//   sqrt(2 l12 + 1) sum_{m12} (-1)^{l12-m12} P12^{m12}(b1,b2) P34^{m12}(b3,b4),
// with only m12 >= 0 summed (App. B: 2 S(m12) and Q_L = Re / Im).
//
// A block stages the a_lm of 32 primaries as [lm][b][primary]; its warps take items
// (up to G multiplets L that share (l12 l3 l4), beta) with b2 = beta. For an item each lane
// (one primary) builds in registers P34^{m12}(b3, b4) for every beta < b3 < b4 once, then
// for each of the item's multiplets P12^{m12}(b1, beta) for every b1 < beta, and
// accumulates their products over m12 into that multiplet's (b1, b3, b4) sums. Coupling
// terms (in shared memory), loop bounds and branches are the same on every lane. After the
// tile the warp reduces its sums across lanes and adds them to the chunk's FP64 row.
#include "npcf_device.h"
#include "npcf_warp.cuh"

#include <algorithm>

namespace npcf {
namespace {

struct C5Layout {
    size_t X, u, c12, o12, c34, o34, s12, s34, binq, total;
};

__host__ __device__ inline size_t al128_5(size_t x) { return (x + 127) & ~size_t(127); }

__host__ __device__ inline C5Layout c5_layout(int nr, int nlm, int nt12, int nt34, int ns12, int ns34) {
    C5Layout l;
    l.X = 0;
    l.u = al128_5(l.X + (size_t)nr * nlm * kRS5 * sizeof(float2));
    l.c12 = al128_5(l.u + kT5 * sizeof(float));
    l.o12 = al128_5(l.c12 + (size_t)nt12 * sizeof(float4));
    l.c34 = al128_5(l.o12 + (size_t)nt12 * sizeof(uint32_t));
    l.o34 = al128_5(l.c34 + (size_t)nt34 * sizeof(float4));
    l.s12 = al128_5(l.o34 + (size_t)nt34 * sizeof(uint32_t));
    l.s34 = al128_5(l.s12 + (size_t)ns12 * sizeof(int2));
    l.binq = al128_5(l.s34 + (size_t)ns34 * sizeof(int2));
    l.total = al128_5(l.binq + (size_t)nr * nr * sizeof(int));
    return l;
}

struct C5Shared {
    const int4* partners;
    const float2* X;
    const float* su;
    const float4* c12;
    const uint32_t* o12;
    const float4* c34;
    const uint32_t* o34;
    const int2* s12;
    const int2* s34;
    const int* binq;
};

// Item for one tile: NB = beta rows b1 < beta, M = nr - 1 - beta shells after beta (NP =
// M (M - 1) / 2 pairs b3 < b4), g <= G multiplets sharing (l12 l3 l4). item = (first P34
// segment of (l12 l3 l4), l12 | beta << 8 | g << 16, first partner, 0); partner = (first
// P12 segment of (l1 l2 l12), first output of L, odd, 0).
template <int NB, int M>
__device__ __forceinline__ void c5_item(const int4 item, const C5Shared& s, int nr, double* __restrict__ dst,
                                        int lane) {
    constexpr int NP = M * (M - 1) / 2;
    constexpr int NOUT = NB * NP;
    constexpr int G = c5_group(NB, M);
    const int l12 = item.y & 0xff;
    const int g = (item.y >> 16) & 0xff;
    const float rcf = sqrtf((float)(2 * l12 + 1));
    const float2* Xl = s.X + lane;
    const float u = s.su[lane];
    int seg12[G], out0[G];
    bool odd[G];
#pragma unroll
    for (int h = 0; h < G; ++h) {
        const int4 P = h < g ? s.partners[item.z + h] : make_int4(0, 0, 0, 0);
        seg12[h] = P.x;
        out0[h] = P.y;
        odd[h] = P.z != 0;
    }
    float acc[G][NOUT];
#pragma unroll
    for (int h = 0; h < G; ++h)
#pragma unroll
        for (int i = 0; i < NOUT; ++i) acc[h][i] = 0.f;
    for (int m12 = 0; m12 <= l12; ++m12) {
        // P34(b3, b4) for beta < b3 < b4, pairs in lexicographic order
        float p34r[NP], p34i[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) p34r[p] = p34i[p] = 0.f;
        const int2 S34 = s.s34[item.x + m12];
        for (int k = S34.x; k < S34.y; ++k) {
            const float4 c = s.c34[k];
            const uint32_t o = s.o34[k];
            const float2* X3 = Xl + (o & 0xffffu) + (NB + 1) * kRS5;
            const float2* X4 = Xl + (o >> 16) + (NB + 1) * kRS5;
            float2 x4[M];
#pragma unroll
            for (int q = 1; q < M; ++q) x4[q] = X4[q * kRS5];
            int p = 0;
#pragma unroll
            for (int i = 0; i + 1 < M; ++i) {
                const float2 x3 = X3[i * kRS5];
                const float a0 = c.x * x3.x, a1 = c.y * x3.y, a2 = c.z * x3.y, a3 = c.w * x3.x;
#pragma unroll
                for (int q = i + 1; q < M; ++q, ++p) {
                    p34r[p] = fmaf(a0, x4[q].x, fmaf(a1, x4[q].y, p34r[p]));
                    p34i[p] = fmaf(a2, x4[q].x, fmaf(a3, x4[q].y, p34i[p]));
                }
            }
        }
        // u 2 S(m12) (-1)^{l12 - m12} sqrt(2 l12 + 1)
        const float cm = u * (m12 == 0 ? 1.f : 2.f) * (((l12 - m12) & 1) ? -1.f : 1.f) * rcf;
#pragma unroll
        for (int h = 0; h < G; ++h) {
            if (h >= g) break;
            // P12(b1, beta) for b1 < beta; the b2 factor is the same for every b1
            float p12r[NB], p12i[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) p12r[j] = p12i[j] = 0.f;
            const int2 S12 = s.s12[seg12[h] + m12];
            for (int k = S12.x; k < S12.y; ++k) {
                const float4 c = s.c12[k];
                const uint32_t o = s.o12[k];
                const float2 x2 = Xl[(o >> 16) + NB * kRS5];
                // re += cA x1 x2 + cB y1 y2 ; im += cC y1 x2 + cD x1 y2 (conjugations folded in c)
                const float a0 = c.x * x2.x, a1 = c.y * x2.y, a2 = c.z * x2.x, a3 = c.w * x2.y;
                const float2* X1 = Xl + (o & 0xffffu);
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const float2 x1 = X1[j * kRS5];
                    p12r[j] = fmaf(a0, x1.x, fmaf(a1, x1.y, p12r[j]));
                    p12i[j] = fmaf(a2, x1.y, fmaf(a3, x1.x, p12i[j]));
                }
            }
            // Re (even L) or Im (odd L) of P12 P34
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const float A = cm * (odd[h] ? p12i[j] : p12r[j]);
                const float B = cm * (odd[h] ? p12r[j] : -p12i[j]);
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    acc[h][j * NP + p] = fmaf(A, p34r[p], fmaf(B, p34i[p], acc[h][j * NP + p]));
            }
        }
    }
    using R = warp::TR<NOUT>;
#pragma unroll
    for (int h = 0; h < G; ++h) {
        if (h >= g) break;
        R::run(acc[h], lane);
#pragma unroll
        for (int i = 0; i < R::F; ++i) {
            const int e = R::origin(i, lane);
            if (e >= 0) {
                const int j = e / NP, p = e - j * NP;
                dst[out0[h] + s.binq[j * nr + NB] + p] += (double)acc[h][i];
            }
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(256, 2) k_contract5w(const Contract5WArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const C5Layout lay = c5_layout(NR, a.nlm, a.nterms12, a.nterms34, a.nseg12, a.nseg34);
    float2* X = reinterpret_cast<float2*>(dsm + lay.X);
    float* su = reinterpret_cast<float*>(dsm + lay.u);
    float4* c12 = reinterpret_cast<float4*>(dsm + lay.c12);
    uint32_t* o12 = reinterpret_cast<uint32_t*>(dsm + lay.o12);
    float4* c34 = reinterpret_cast<float4*>(dsm + lay.c34);
    uint32_t* o34 = reinterpret_cast<uint32_t*>(dsm + lay.o34);
    int2* s12 = reinterpret_cast<int2*>(dsm + lay.s12);
    int2* s34 = reinterpret_cast<int2*>(dsm + lay.s34);
    int* binq = reinterpret_cast<int*>(dsm + lay.binq);
    __shared__ int chunk_s, item_next;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < a.nterms12; i += blockDim.x) { c12[i] = a.c12[i]; o12[i] = a.o12[i]; }
    for (int i = tid; i < a.nterms34; i += blockDim.x) { c34[i] = a.c34[i]; o34[i] = a.o34[i]; }
    for (int i = tid; i < a.nseg12; i += blockDim.x) s12[i] = a.segs12[i];
    for (int i = tid; i < a.nseg34; i += blockDim.x) s34[i] = a.segs34[i];
    for (int i = tid; i < NR * NR; i += blockDim.x) binq[i] = a.binq[i];
    const C5Shared sh{a.partners, X, su, c12, o12, c34, o34, s12, s34, binq};
    const int rows = NR * a.nlm;

    // chunks (primary ranges of one catalog) taken dynamically; chunk c sums into row c
    for (;;) {
        if (tid == 0) chunk_s = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        const int c = chunk_s;
        if (c >= a.nchunk) break;
        const int2 C = a.chunks[c];
        double* dst = a.partial + (size_t)c * a.total;
        for (int i = tid; i < a.nout; i += blockDim.x) dst[a.out_off + i] = 0.0;
        for (int p0 = C.x; p0 < C.y; p0 += kT5) {
            const int np = min(kT5, C.y - p0);
            if (tid == 0) item_next = 0;
            // stage [lm][b][q] from the pair kernel's [q][b][lm]
            const float2* src = a.alm + (size_t)p0 * rows;
            for (int i = tid; i < kT5 * rows; i += blockDim.x) {
                const int q = i / rows, r = i - q * rows;   // r = b * nlm + lm
                const int b = r / a.nlm, lm = r - b * a.nlm;
                X[(lm * NR + b) * kRS5 + q] = q < np ? src[i] : make_float2(0.f, 0.f);
            }
            if (tid < kT5) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
            __syncthreads();   // also orders the row's zeroing before the first sums
            for (;;) {
                int it = 0;
                if (lane == 0) it = atomicAdd(&item_next, 1);
                it = __shfl_sync(warp::kFullMask, it, 0);
                if (it >= a.nitem) break;
                const int4 item = a.items[it];
                switch ((item.y >> 8) & 0xff) {   // beta
#define NPCF_C5_CASE(B) \
    case B:             \
        if (B <= NR - 3) c5_item<(B <= NR - 3 ? B : 1), (B <= NR - 3 ? NR - 1 - B : 2)>(item, sh, NR, dst, lane); \
        break;
                    NPCF_C5_CASE(1) NPCF_C5_CASE(2) NPCF_C5_CASE(3) NPCF_C5_CASE(4)
                    NPCF_C5_CASE(5) NPCF_C5_CASE(6) NPCF_C5_CASE(7)
#undef NPCF_C5_CASE
                    default: break;
                }
            }
            __syncthreads();
        }
        __syncthreads();   // every thread has read chunk_s before it is taken again
    }
}

template <int NR>
void launch_nr(const Contract5WArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = contract5w_smem_bytes(a);
    cudaFuncSetAttribute(k_contract5w<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_contract5w<NR><<<nblocks, 256, smem, s>>>(a);
}

}  // namespace

size_t contract5w_smem_bytes(const Contract5WArgs& a) {
    return c5_layout(a.nr, a.nlm, a.nterms12, a.nterms34, a.nseg12, a.nseg34).total;
}

void launch_contract5w(const Contract5WArgs& a, int nblocks, cudaStream_t s) {
    switch (a.nr) {
        case 4: launch_nr<4>(a, nblocks, s); break;
        case 5: launch_nr<5>(a, nblocks, s); break;
        case 6: launch_nr<6>(a, nblocks, s); break;
        case 7: launch_nr<7>(a, nblocks, s); break;
        case 8: launch_nr<8>(a, nblocks, s); break;
        case 9: launch_nr<9>(a, nblocks, s); break;
        case 10: launch_nr<10>(a, nblocks, s); break;
        default: break;
    }
}

}  // namespace npcf
