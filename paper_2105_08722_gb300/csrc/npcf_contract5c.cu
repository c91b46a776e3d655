// 5PCF contraction with P34 built once per block and tile: FP32 products, FP64 partials,
// primaries on the lanes.
//
// Eq. (basis-coupling) at N = 5 through the intermediate m12 (App. B halving over m12):
//   zeta_L(b1,b2,b3,b4) += u sqrt(2 l12 + 1) sum_{m12 >= 0} 2 S(m12) (-1)^{l12-m12}
//                          Q_L[P12^{m12}(b1,b2) P34^{m12}(b3,b4)]
//   P12^{m12}(b1,b2) = sum_{m1} (l1 l2 l12; m1, m12 - m1, -m12) a^{b1}_{l1 m1} a^{b2}_{l2,m12-m1}
//   P34^{m12}(b3,b4) = sum_{m3} (l12 l3 l4; m12, m3, -m12 - m3) a^{b3}_{l3 m3} a^{b4}_{l4,-m12-m3}.
//
// P34 depends on the right triple (l12 l3 l4), m12 and (b3, b4) only, but every multiplet
// of that triple and every b2 < b3 uses it. The register-only kernel (npcf_contract5w.cu)
// builds it again for every b2 and every item of at most two multiplets. Here a block
// builds P34 of a group of right triples once per tile of 32 primaries into shared memory
// ([m12][pair (b3 < b4), b3 >= 2][primary]); its warps then take items (left triple
// (l1 l2 l12), b2, up to four multiplets of that left triple whose right triples are in the
// group): each lane builds P12(b1, b2) for every b1 < b2 once in registers and multiplies it
// with the cached P34 of every pair after b2 of each multiplet into that multiplet's
// (b1, b3, b4) sums. Two cache slots alternate: in one phase the warps take, from one work
// list, the P34 builds of group g (writing one slot) and the items of group g - 1 (reading
// the other), so one block barrier separates the phases. The coupling terms are staged in
// shared memory where they fit beside the slots (one block of 512 threads per SM), else
// read through L1 (two blocks of 256 threads per SM where the slots allow, else one of 512).
#include "npcf_device.h"
#include "npcf_warp.cuh"

#include <algorithm>

namespace npcf {
namespace {

constexpr int kC5CThreads = 256;

struct C5CLayout {
    size_t X, u, cache, c12, o12, c34, o34, s12, s34, total;
};

__host__ __device__ inline size_t al128c(size_t x) { return (x + 127) & ~size_t(127); }

// tables: the coupling terms and segments staged in shared memory too (else read through L1)
__host__ __device__ inline C5CLayout c5c_layout(int nr, int nlm, int slot_entries, bool tables, int nt12, int nt34,
                                                int ns12, int ns34) {
    C5CLayout l;
    l.X = 0;
    l.u = al128c(l.X + (size_t)nr * nlm * kRS5 * sizeof(float2));
    l.cache = al128c(l.u + kT5 * sizeof(float));
    l.c12 = al128c(l.cache + (size_t)2 * slot_entries * kT5 * sizeof(float2));
    if (!tables) nt12 = nt34 = ns12 = ns34 = 0;
    l.o12 = al128c(l.c12 + (size_t)nt12 * sizeof(float4));
    l.c34 = al128c(l.o12 + (size_t)nt12 * sizeof(uint32_t));
    l.o34 = al128c(l.c34 + (size_t)nt34 * sizeof(float4));
    l.s12 = al128c(l.o34 + (size_t)nt34 * sizeof(uint32_t));
    l.s34 = al128c(l.s12 + (size_t)ns12 * sizeof(int2));
    l.total = al128c(l.s34 + (size_t)ns34 * sizeof(int2));
    return l;
}

// where the kernel reads the coupling terms: shared memory (TS) or global memory through L1
struct C5CTabs {
    const float4* c12;
    const uint32_t* o12;
    const float4* c34;
    const uint32_t* o34;
    const int2* s12;
    const int2* s34;
};

template <bool TS, typename T>
__device__ __forceinline__ T tld(const T* p) {
    if constexpr (TS) return *p;
    else return __ldg(p);
}

// first pair (b3, b3 + 1) of shell b3 >= 2 in the cache's pair order (lexicographic)
__host__ __device__ constexpr int pair_off(int nr, int b3) { return (b3 - 2) * (2 * nr - 3 - b3) / 2; }
static_assert(pair_off(8, 2) == 0 && pair_off(8, 3) == 5 && pair_off(8, 6) == 14 && pair_off(8, 7) == 15,
              "pairs (b3, b4), 2 <= b3 < b4 < 8, in lexicographic order");

// P34^{m12}(b3, b4) of one (triple, m12) for every b4 > b3 into the cache.
template <int NR, bool TS>
__device__ __forceinline__ void c5c_build34(const int4 w, const C5CTabs& tb, const float2* __restrict__ X,
                                            float2* __restrict__ cache, int lane) {
    constexpr int MX = NR - 3;   // b3 >= 2: at most NR - 3 shells after it
    const int b3 = w.y & 0xff;
    const int nb4 = NR - 1 - b3;
    float pr[MX], pi[MX];
#pragma unroll
    for (int q = 0; q < MX; ++q) pr[q] = pi[q] = 0.f;
    const int2 S = tld<TS>(&tb.s34[w.x]);
    const float2* Xl = X + lane;
    for (int k = S.x; k < S.y; ++k) {
        const float4 c = tld<TS>(&tb.c34[k]);
        const uint32_t o = tld<TS>(&tb.o34[k]);
        const float2 x3 = Xl[(o & 0xffffu) + b3 * kRS5];
        const float2* X4 = Xl + (o >> 16) + (b3 + 1) * kRS5;
        // re += cA x3 x4 + cB y3 y4 ; im += cC y3 x4 + cD x3 y4 (conjugations folded in c)
        const float a0 = c.x * x3.x, a1 = c.y * x3.y, a2 = c.z * x3.y, a3 = c.w * x3.x;
#pragma unroll
        for (int q = 0; q < MX; ++q) {
            if (q < nb4) {
                const float2 x4 = X4[q * kRS5];
                pr[q] = fmaf(a0, x4.x, fmaf(a1, x4.y, pr[q]));
                pi[q] = fmaf(a2, x4.x, fmaf(a3, x4.y, pi[q]));
            }
        }
    }
    float2* dst = cache + (size_t)(w.z + pair_off(NR, b3)) * kT5 + lane;
#pragma unroll
    for (int q = 0; q < MX; ++q)
        if (q < nb4) dst[q * kT5] = make_float2(pr[q], pi[q]);
}

// Item (left triple, beta = b2, g <= GM partners): the multiplets (l1 l2 l12 l3 l4) of one
// left triple (l1 l2 l12) whose right triples sit in the same group share P12, so a lane
// builds P12(b1, beta) for every b1 < beta once per m12 and multiplies it with the cached
// P34 of each partner into that partner's sums. NB = beta shells b1 < beta, M = NR - 1 -
// beta shells after it (NP = M (M - 1) / 2 pairs b3 < b4).
template <int NR, int NB, int M, bool TS>
__device__ __forceinline__ void c5c_item(const int4 w, const C5CTabs& tb, const int4* __restrict__ partners,
                                         const float2* __restrict__ X, const float2* __restrict__ cache, float u,
                                         const int* __restrict__ binq, double* __restrict__ dst, int lane) {
    constexpr int NP = M * (M - 1) / 2;
    constexpr int NOUT = NB * NP;
    constexpr int NPALL = (NR - 3) * (NR - 2) / 2;
    constexpr int GM = c5c_group(NB, M);
    const int l12 = (w.y >> 16) & 0xff;
    const int g = ((w.y >> 26) & 3) + 1;
    const float rcf = sqrtf((float)(2 * l12 + 1));
    const float2* Xl = X + lane;
    const float2* C34[GM];
    bool odd[GM];
    int out0[GM];
#pragma unroll
    for (int h = 0; h < GM; ++h) {
        const int4 P = h < g ? __ldg(&partners[w.z + h]) : make_int4(0, 0, 0, 0);   // (P34 block, output, odd)
        C34[h] = cache + (size_t)(P.x + pair_off(NR, NB + 1)) * kT5 + lane;
        out0[h] = P.y;
        odd[h] = P.z != 0;
    }
    float acc[GM][NOUT];
#pragma unroll
    for (int h = 0; h < GM; ++h)
#pragma unroll
        for (int i = 0; i < NOUT; ++i) acc[h][i] = 0.f;
    for (int m12 = 0; m12 <= l12; ++m12) {
        // P12(b1, beta) for b1 < beta; the b2 factor is the same for every b1
        float p12r[NB], p12i[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) p12r[j] = p12i[j] = 0.f;
        const int2 S12 = tld<TS>(&tb.s12[w.x + m12]);
        for (int k = S12.x; k < S12.y; ++k) {
            const float4 c = tld<TS>(&tb.c12[k]);
            const uint32_t o = tld<TS>(&tb.o12[k]);
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
        // u 2 S(m12) (-1)^{l12 - m12} sqrt(2 l12 + 1); Re (even L) or Im (odd L) of P12 P34
        const float cm = u * (m12 == 0 ? 1.f : 2.f) * (((l12 - m12) & 1) ? -1.f : 1.f) * rcf;
#pragma unroll
        for (int h = 0; h < GM; ++h) {
            if (h >= g) break;
            float A[NB], B[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                A[j] = cm * (odd[h] ? p12i[j] : p12r[j]);
                B[j] = cm * (odd[h] ? p12r[j] : -p12i[j]);
            }
            const float2* P34 = C34[h] + (size_t)m12 * NPALL * kT5;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float2 q = P34[p * kT5];
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    acc[h][j * NP + p] = fmaf(A[j], q.x, fmaf(B[j], q.y, acc[h][j * NP + p]));
            }
        }
    }
    using R = warp::TR<NOUT>;
#pragma unroll
    for (int h = 0; h < GM; ++h) {
        if (h >= g) break;
        R::run(acc[h], lane);
#pragma unroll
        for (int i = 0; i < R::F; ++i) {
            const int e = R::origin(i, lane);
            if (e >= 0) {
                const int j = e / NP, p = e - j * NP;
                dst[out0[h] + binq[j * NR + NB] + p] += (double)acc[h][i];
            }
        }
    }
}

template <int NR, int THREADS, int MINB, bool TS>
__global__ void __launch_bounds__(THREADS, MINB) k_contract5c(const Contract5CArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const C5CLayout lay = c5c_layout(NR, a.nlm, a.slot_entries, TS, a.nterms12, a.nterms34, a.nseg12, a.nseg34);
    float2* X = reinterpret_cast<float2*>(dsm + lay.X);
    float* su = reinterpret_cast<float*>(dsm + lay.u);
    float2* cache = reinterpret_cast<float2*>(dsm + lay.cache);
    __shared__ int chunk_s, next[2];
    __shared__ int binq[NR * NR];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < NR * NR; i += blockDim.x) binq[i] = a.binq[i];
    C5CTabs tb{a.c12, a.o12, a.c34, a.o34, a.segs12, a.segs34};
    if constexpr (TS) {
        float4* c12 = reinterpret_cast<float4*>(dsm + lay.c12);
        uint32_t* o12 = reinterpret_cast<uint32_t*>(dsm + lay.o12);
        float4* c34 = reinterpret_cast<float4*>(dsm + lay.c34);
        uint32_t* o34 = reinterpret_cast<uint32_t*>(dsm + lay.o34);
        int2* s12 = reinterpret_cast<int2*>(dsm + lay.s12);
        int2* s34 = reinterpret_cast<int2*>(dsm + lay.s34);
        for (int i = tid; i < a.nterms12; i += blockDim.x) { c12[i] = a.c12[i]; o12[i] = a.o12[i]; }
        for (int i = tid; i < a.nterms34; i += blockDim.x) { c34[i] = a.c34[i]; o34[i] = a.o34[i]; }
        for (int i = tid; i < a.nseg12; i += blockDim.x) s12[i] = a.segs12[i];
        for (int i = tid; i < a.nseg34; i += blockDim.x) s34[i] = a.segs34[i];
        tb = C5CTabs{c12, o12, c34, o34, s12, s34};
    }
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
            // stage [lm][b][q] from the pair kernel's [q][b][lm]
            const float2* src = a.alm + (size_t)p0 * rows;
            for (int i = tid; i < kT5 * rows; i += blockDim.x) {
                const int q = i / rows, r = i - q * rows;   // r = b * nlm + lm
                const int b = r / a.nlm, lm = r - b * a.nlm;
                X[(lm * NR + b) * kRS5 + q] = q < np ? src[i] : make_float2(0.f, 0.f);
            }
            if (tid < kT5) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
            if (tid == 0) next[0] = next[1] = 0;
            __syncthreads();   // also orders the row's zeroing before the first sums
            const float u = su[lane];
            for (int ph = 0; ph < a.nphase; ++ph) {
                const int w0 = __ldg(&a.phase_begin[ph]), nw = __ldg(&a.phase_begin[ph + 1]) - w0;
                if (tid == 0) next[(ph + 1) & 1] = 0;   // nobody uses it in this phase
                for (;;) {
                    int it = 0;
                    if (lane == 0) it = atomicAdd(&next[ph & 1], 1);
                    it = __shfl_sync(warp::kFullMask, it, 0);
                    if (it >= nw) break;
                    const int4 w = __ldg(&a.work[w0 + it]);
                    float2* slot = cache + (size_t)((w.y >> 24) & 1) * a.slot_entries * kT5;
                    if (w.y & (1 << 30)) {
                        c5c_build34<NR, TS>(w, tb, X, slot, lane);
                    } else {
                        switch (w.y & 0xff) {   // beta
#define NPCF_C5C_CASE(B) \
    case B:              \
        if (B <= NR - 3) c5c_item<NR, (B <= NR - 3 ? B : 1), (B <= NR - 3 ? NR - 1 - B : 2), TS>(w, tb, a.partners, X, slot, u, binq, dst, lane); \
        break;
                            NPCF_C5C_CASE(1) NPCF_C5C_CASE(2) NPCF_C5C_CASE(3) NPCF_C5C_CASE(4)
                            NPCF_C5C_CASE(5) NPCF_C5C_CASE(6) NPCF_C5C_CASE(7)
#undef NPCF_C5C_CASE
                            default: break;
                        }
                    }
                }
                __syncthreads();   // the slot written in this phase is read in the next
            }
        }
        __syncthreads();   // every thread has read chunk_s before it is taken again
    }
}

template <int NR>
void launch_nr_c(const Contract5CArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = contract5c_smem_bytes(a);
    if (a.tables_smem) {   // one block of 512 threads per SM, coupling terms in shared memory
        cudaFuncSetAttribute(k_contract5c<NR, 512, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract5c<NR, 512, 1, true><<<nblocks, 512, smem, s>>>(a);
    } else if (a.blocks_per_sm >= 2) {
        cudaFuncSetAttribute(k_contract5c<NR, kC5CThreads, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_contract5c<NR, kC5CThreads, 2, false><<<nblocks, kC5CThreads, smem, s>>>(a);
    } else {   // one block per SM: 512 threads
        cudaFuncSetAttribute(k_contract5c<NR, 512, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_contract5c<NR, 512, 1, false><<<nblocks, 512, smem, s>>>(a);
    }
}

}  // namespace

size_t contract5c_smem_bytes(const Contract5CArgs& a) {
    return c5c_layout(a.nr, a.nlm, a.slot_entries, a.tables_smem != 0, a.nterms12, a.nterms34, a.nseg12, a.nseg34)
        .total;
}

size_t contract5c_static_smem() { return 1024; }

void launch_contract5c(const Contract5CArgs& a, int nblocks, cudaStream_t s) {
    switch (a.nr) {
        case 4: launch_nr_c<4>(a, nblocks, s); break;
        case 5: launch_nr_c<5>(a, nblocks, s); break;
        case 6: launch_nr_c<6>(a, nblocks, s); break;
        case 7: launch_nr_c<7>(a, nblocks, s); break;
        case 8: launch_nr_c<8>(a, nblocks, s); break;
        case 9: launch_nr_c<9>(a, nblocks, s); break;
        case 10: launch_nr_c<10>(a, nblocks, s); break;
        default: break;
    }
}

}  // namespace npcf
