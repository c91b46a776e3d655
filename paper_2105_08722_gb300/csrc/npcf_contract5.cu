// 5PCF contraction on the CUDA cores (FP32 products, per-chunk FP64 partials).
//
// For L = (l1, l2, l12, l3, l4), Eq. (basis-coupling) at N = 5 couples two pairs of
// harmonic coefficients through an intermediate m12:
//   E C^L_M = sqrt(2 l12 + 1) (-1)^{l12-m12} (l1 l2 l12; m1 m2 -m12) (l12 l3 l4; m12 m3 m4),
// so the sum over M of Eq. (NPCF-mult-discrete-binned-estimator) factorises into
//   sqrt(2 l12 + 1) sum_{m12} (-1)^{l12-m12} P12^{m12}(b1,b2) P34^{m12}(b3,b4),
// and with the App. B symmetry only m12 >= 0 is summed, with 2 S(m12) and Q_L = Re / Im.
//
// Block (row block, chunk of primaries): per primary the block tabulates P34 of its
// (l12, l3, l4) triples over every shell pair (b3 < b4) in shared memory (a warp per
// (triple, m12) segment, lanes over the pairs); each thread owns one row (L, b1, b2),
// builds P12^{m12} in registers and accumulates over exactly the (b3, b4) pairs that
// follow b2 (rows sorted by b2 within a block keep that count uniform across a warp).
#include "npcf_device.h"

namespace npcf {
namespace {

constexpr int kTile5 = 8;     // primaries staged per pass
constexpr int kThreads5 = 256;
constexpr int kFold5 = 4;     // tiles between folds of the FP32 sums into FP64

// One coupling term c x1 x2 with conjugations folded into c (cA..cD): re += cA x1 x2 +
// cB y1 y2, im += cC y1 x2 + cD x1 y2.
__device__ __forceinline__ void pair_product(const float4 c, float2 x1, float2 x2, float& pr, float& pi) {
    pr = fmaf(c.x * x1.x, x2.x, pr);
    pr = fmaf(c.y * x1.y, x2.y, pr);
    pi = fmaf(c.z * x1.y, x2.x, pi);
    pi = fmaf(c.w * x1.x, x2.y, pi);
}

// acc[k] += Ar Re(P34[k]) + Ai Im(P34[k]) over the NP (b3, b4) pairs after b2.
template <int NP>
__device__ __forceinline__ void products(const float2* __restrict__ P34, float Ar, float Ai,
                                         float (&acc)[kMaxPairs5]) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 y = P34[k];
        acc[k] = fmaf(Ar, y.x, fmaf(Ai, y.y, acc[k]));
    }
}

__global__ void __launch_bounds__(kThreads5, 4) k_contract5(const Contract5Args a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int per = a.nr * a.nlm;
    const int nm = a.l12max + 1;
    float2* X = reinterpret_cast<float2*>(dsm);                        // [tile][b][lm]
    float2* T34 = X + kTile5 * per;                                     // [kMaxT34][nm][npairs]
    float* su = reinterpret_cast<float*>(T34 + (size_t)kMaxT34 * nm * a.npairs);
    __shared__ int t34s[kMaxT34];
    __shared__ int nt34;

    const int4 B = a.blocks[blockIdx.y];
    if (threadIdx.x < kMaxT34) t34s[threadIdx.x] = a.blk_t34[blockIdx.y * kMaxT34 + threadIdx.x];
    if (threadIdx.x == 0) nt34 = B.z;
    const int chunk = blockIdx.x;
    const int2 C = a.chunks[chunk];   // primaries [C.x, C.y) of one catalog
    const int p0 = C.x, p1 = C.y;
    const bool valid = threadIdx.x < B.y;
    const int row = B.x + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int4 ra = make_int4(0, 0, 0, 0), rb = make_int4(0, 0, 0, 0);
    float2 rc = make_float2(0.f, 0.f);
    if (valid) { ra = a.rowsA[row]; rb = a.rowsB[row]; rc = a.rowsC[row]; }
    const int t12 = rb.x, tl34 = rb.y, q0 = rb.z, np = rb.w;
    // the triple (l1 l2 l12) has one segment per m12 = 0..l12
    const int l12 = valid ? a.t12_seg0[t12 + 1] - a.t12_seg0[t12] - 1 : 0;
    const bool odd = rc.y != 0.f;

    float acc[kMaxPairs5];
#pragma unroll
    for (int k = 0; k < kMaxPairs5; ++k) acc[k] = 0.f;
    // this thread's outputs in the chunk's FP64 row: the FP32 sums are added there every
    // kFold5 tiles, so the rounding does not grow with the chunk length
    double* dst = a.partial + (size_t)chunk * a.total + ra.w;
    if (valid && chunk < a.nchunk)
        for (int k = 0; k < np; ++k) dst[k] = 0.0;
    int tiles = 0;
    __syncthreads();
    const int nseg34 = nt34 * nm;   // (triple, m12) segments of the block's P34 table

    for (int s0 = p0; s0 < p1; s0 += kTile5) {
        const int nt = min(kTile5, p1 - s0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt * per; i += kThreads5) X[i] = a.alm[(size_t)s0 * per + i];
        for (int i = threadIdx.x; i < nt; i += kThreads5) su[i] = a.wp[s0 + i];
        __syncthreads();
        for (int q = 0; q < nt; ++q) {
            const float u = su[q];
            if (u == 0.f) continue;   // uniform: the primary adds nothing
            const float2* Xq = X + q * per;
            // ---- P34 of this block's triples: one warp per (triple, m12) segment, so the
            // coupling terms are the same on every lane; lanes run over the shell pairs
            for (int sgi = warp; sgi < nseg34; sgi += kThreads5 / 32) {
                const int t = sgi / nm, m12 = sgi - t * nm;
                const int tg = t34s[t];
                const int sg = a.t34_seg0[tg] + m12;
                if (sg >= a.t34_seg0[tg + 1]) continue;   // m12 > l12 of the triple: never read
                const int2 S = a.segs34[sg];
                for (int pq = lane; pq < a.npairs; pq += 32) {
                    const int2 bb = a.pairs[pq];
                    const float2* A3 = Xq + bb.x * a.nlm;
                    const float2* A4 = Xq + bb.y * a.nlm;
                    float pr = 0.f, pim = 0.f;
                    for (int k = S.x; k < S.y; ++k) {
                        const uint32_t id = a.i34[k];
                        pair_product(a.c34[k], A3[id & 0xffffu], A4[id >> 16], pr, pim);
                    }
                    T34[(size_t)sgi * a.npairs + pq] = make_float2(pr, pim);
                }
            }
            __syncthreads();
            if (valid) {
                const float2* A1 = Xq + ra.y * a.nlm;
                const float2* A2 = Xq + ra.z * a.nlm;
                const int sg0 = a.t12_seg0[t12];
                for (int m12 = 0; m12 <= l12; ++m12) {
                    const int2 S = a.segs12[sg0 + m12];
                    float pr = 0.f, pim = 0.f;
                    for (int k = S.x; k < S.y; ++k) {
                        const uint32_t id = a.i12[k];
                        pair_product(a.c12[k], A1[id & 0xffffu], A2[id >> 16], pr, pim);
                    }
                    // u 2 S(m12) (-1)^{l12 - m12} sqrt(2 l12 + 1), then Re or Im of P12 P34
                    const float c = u * (m12 == 0 ? 1.f : 2.f) * (((l12 - m12) & 1) ? -1.f : 1.f) * rc.x;
                    const float Ar = c * (odd ? pim : pr), Ai = c * (odd ? pr : -pim);
                    const float2* P34 = T34 + ((size_t)tl34 * nm + m12) * a.npairs + q0;
                    // the pairs after b2 number C(nr - 1 - b2, 2); rows are sorted by b2 in a
                    // block, so a warp mostly takes one of these cases
                    switch (np) {
                        case 1: products<1>(P34, Ar, Ai, acc); break;
                        case 3: products<3>(P34, Ar, Ai, acc); break;
                        case 6: products<6>(P34, Ar, Ai, acc); break;
                        case 10: products<10>(P34, Ar, Ai, acc); break;
                        case 15: products<15>(P34, Ar, Ai, acc); break;
                        case 21: products<21>(P34, Ar, Ai, acc); break;
                        default: products<28>(P34, Ar, Ai, acc); break;
                    }
                }
            }
            __syncthreads();
        }
        if (++tiles == kFold5 || s0 + kTile5 >= p1) {
            if (valid && chunk < a.nchunk) {
#pragma unroll
                for (int k = 0; k < kMaxPairs5; ++k)
                    if (k < np) {
                        dst[k] += (double)acc[k];
                        acc[k] = 0.f;
                    }
            }
            tiles = 0;
        }
    }
}

}  // namespace

size_t contract5_smem_bytes(const Contract5Args& a) {
    const int per = a.nr * a.nlm;
    return (size_t)kTile5 * per * sizeof(float2) + (size_t)kMaxT34 * (a.l12max + 1) * a.npairs * sizeof(float2) +
           kTile5 * sizeof(float);
}

void launch_contract5(const Contract5Args& a, cudaStream_t s) {
    const size_t smem = contract5_smem_bytes(a);
    cudaFuncSetAttribute(k_contract5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(a.nchunk, a.nblocks);
    k_contract5<<<grid, kThreads5, smem, s>>>(a);
}

}  // namespace npcf
