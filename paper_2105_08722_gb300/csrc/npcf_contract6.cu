// 6PCF contraction on the CUDA cores, FP32 products, FP64 partials; primaries on the lanes.
//
// For L = (l1, l2, l12, l3, l123, l4, l5), Eq. (basis-coupling) at N = 6 couples the five
// harmonic coefficients through two intermediates m12 = m1 + m2 and m123 = m12 + m3:
//   E C^L_M = sqrt((2 l12 + 1)(2 l123 + 1)) (-1)^{l12 - m12 + l123 - m123}
//             (l1 l2 l12; m1 m2 -m12) (l12 l3 l123; m12 m3 -m123) (l123 l4 l5; m123 m4 m5)
// (the (-1)^{sum of l} of C^L_M cancels against E(L)), so the sum over M of
// Eq. (NPCF-mult-discrete-binned-estimator) factorises as
//   sqrt(...) sum_{m123} Q^{m123}(b1, b2, b3) P45^{m123}(b4, b5),
//   Q^{m123}(b1,b2,b3) = sum_{m12} (-1)^{l123-m123} (l12 l3 l123; m12, m123-m12, -m123)
//                        P12^{m12}(b1,b2) a^{b3}_{l3, m123-m12},
//   P12^{m12}(b1,b2) = sum_{m1} (-1)^{l12-m12} (l1 l2 l12; m1, m12-m1, -m12) a^{b1}_{l1 m1} a^{b2}_{l2, m12-m1},
//   P45^{m123}(b4,b5) = sum_{m4} (l123 l4 l5; m123, m4, -m123-m4) a^{b4}_{l4 m4} a^{b5}_{l5, -m123-m4},
// with only m123 >= 0 summed (App. B: the terms of -M are those of M conjugated, times
// E(L); factor 2 S(m123), then Re for parity-even L and Im for parity-odd L).
//
// A block stages the a_lm of 32 primaries as complex [l^2 + l + m][b][primary] for
// m = -l..l (a_{l,-m} = (-1)^m conj(a_{lm})), so every product is a plain complex product.
// Its warps take items (L, b3); each lane (one primary) forms, for every m123 >= 0, the
// P45 of every b3 < b4 < b5 and the Q of every b1 < b2 < b3 (P12 formed again for every
// m123: the kernel keeps its sums in registers and serves the order's correctness more
// than its speed), and adds Re or Im of their products into its (b1, b2, b4, b5) sums; after
// the tile the warp reduces the sums across lanes into the chunk's FP64 row.
#include "npcf_device.h"
#include "npcf_warp.cuh"

namespace npcf {
namespace {

constexpr int kT6 = 32;
constexpr int kRS6 = kT6 + 1;

template <int NB, int M>
__device__ __forceinline__ void c6_item(const int2 item, const Contract6Args& a, const float2* X, float u,
                                        const int* binq, int nr, double* __restrict__ dst, int lane) {
    constexpr int NQ = NB * (NB - 1) / 2;   // pairs b1 < b2 < b3 = NB
    constexpr int NP = M * (M - 1) / 2;     // pairs b3 < b4 < b5
    constexpr int NOUT = NQ * NP;
    const int L = item.x;
    const int4 i1 = __ldg(&a.lam[L]);   // l12, l123, odd, first output of L
    const int4 i2 = __ldg(&a.lam2[L]);  // first P12 segment, first (Q, P45) segment, bits of the prefactor
    const int l123 = i1.y;
    const bool odd = i1.z != 0;
    const float pref = __int_as_float(i2.z);
    const int rowb = nr * kRS6;         // stride of one harmonic row
    const float2* Xl = X + lane;
    float acc[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) acc[i] = 0.f;
    for (int m123 = 0; m123 <= l123; ++m123) {
        // P45(b4, b5) for NB < b4 < b5, pairs in lexicographic order
        float p45r[NP], p45i[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) p45r[p] = p45i[p] = 0.f;
        const int2 s3 = __ldg(&a.seg3[i2.y + m123]);
        for (int k = s3.x; k < s3.y; ++k) {
            const int4 t = __ldg(&a.terms3[k]);   // lm of (l4, m4), lm of (l5, m5), coefficient
            const float c = __int_as_float(t.z);
            const float2* X4 = Xl + t.x * rowb + (NB + 1) * kRS6;
            const float2* X5 = Xl + t.y * rowb + (NB + 1) * kRS6;
            float2 x5[M];
#pragma unroll
            for (int q = 1; q < M; ++q) x5[q] = X5[q * kRS6];
            int p = 0;
#pragma unroll
            for (int i = 0; i + 1 < M; ++i) {
                const float2 x4 = X4[i * kRS6];
                const float cr = c * x4.x, ci = c * x4.y;
#pragma unroll
                for (int q = i + 1; q < M; ++q, ++p) {
                    p45r[p] = fmaf(cr, x5[q].x, fmaf(-ci, x5[q].y, p45r[p]));
                    p45i[p] = fmaf(cr, x5[q].y, fmaf(ci, x5[q].x, p45i[p]));
                }
            }
        }
        // Q(b1, b2) for b1 < b2 < NB
        float qr[NQ], qi[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) qr[j] = qi[j] = 0.f;
        const int2 s2 = __ldg(&a.seg2[i2.y + m123]);
        for (int e = s2.x; e < s2.y; ++e) {
            const int4 t2 = __ldg(&a.terms2[e]);   // P12 segment of m12, lm of (l3, m3), coefficient
            const float c2 = __int_as_float(t2.z);
            const float2 x3 = Xl[t2.y * rowb + NB * kRS6];
            const float a3r = c2 * x3.x, a3i = c2 * x3.y;
            float pr[NQ], pim[NQ];
#pragma unroll
            for (int j = 0; j < NQ; ++j) pr[j] = pim[j] = 0.f;
            const int2 s1 = __ldg(&a.seg1[t2.x]);
            for (int k = s1.x; k < s1.y; ++k) {
                const int4 t = __ldg(&a.terms1[k]);   // lm of (l1, m1), lm of (l2, m2), coefficient
                const float c = __int_as_float(t.z);
                const float2* X1 = Xl + t.x * rowb;
                const float2* X2 = Xl + t.y * rowb;
                float2 x2[NB];
#pragma unroll
                for (int q = 1; q < NB; ++q) x2[q] = X2[q * kRS6];
                int j = 0;
#pragma unroll
                for (int i = 0; i + 1 < NB; ++i) {
                    const float2 x1 = X1[i * kRS6];
                    const float cr = c * x1.x, ci = c * x1.y;
#pragma unroll
                    for (int q = i + 1; q < NB; ++q, ++j) {
                        pr[j] = fmaf(cr, x2[q].x, fmaf(-ci, x2[q].y, pr[j]));
                        pim[j] = fmaf(cr, x2[q].y, fmaf(ci, x2[q].x, pim[j]));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                qr[j] = fmaf(pr[j], a3r, fmaf(-pim[j], a3i, qr[j]));
                qi[j] = fmaf(pr[j], a3i, fmaf(pim[j], a3r, qi[j]));
            }
        }
        // u 2 S(m123) sqrt((2 l12 + 1)(2 l123 + 1)) times Re (even L) or Im (odd L) of Q P45
        const float w = u * (m123 == 0 ? 1.f : 2.f) * pref;
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const float A = w * (odd ? qi[j] : qr[j]);
            const float B = w * (odd ? qr[j] : -qi[j]);
#pragma unroll
            for (int p = 0; p < NP; ++p) acc[j * NP + p] = fmaf(A, p45r[p], fmaf(B, p45i[p], acc[j * NP + p]));
        }
    }
    using R = warp::TR<NOUT>;
    R::run(acc, lane);
#pragma unroll
    for (int i = 0; i < R::F; ++i) {
        const int e = R::origin(i, lane);
        if (e >= 0) {
            const int j = e / NP, p = e - j * NP;
            // pair j = (b1, b2) in lexicographic order
            int b1 = 0, rem = j;
            while (rem >= NB - 1 - b1) {
                rem -= NB - 1 - b1;
                ++b1;
            }
            const int b2 = b1 + 1 + rem;
            dst[i1.w + binq[(b1 * nr + b2) * nr + NB] + p] += (double)acc[i];
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(256, 2) k_contract6(const Contract6Args a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const int nlmf = (a.lmax + 1) * (a.lmax + 1);
    float2* X = reinterpret_cast<float2*>(dsm);                              // [nlmf][NR][kRS6]
    int* binq = reinterpret_cast<int*>(dsm + (size_t)nlmf * NR * kRS6 * sizeof(float2));   // [NR][NR][NR]
    __shared__ float su[kT6];
    __shared__ int chunk_s, item_next;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < NR * NR * NR; i += blockDim.x) binq[i] = a.binq[i];
    const int rows = NR * a.nlm;
    for (;;) {
        if (tid == 0) chunk_s = atomicAdd(a.chunk_counter, 1);
        __syncthreads();
        const int c = chunk_s;
        if (c >= a.nchunk) break;
        const int2 C = a.chunks[c];
        double* dst = a.partial + (size_t)c * a.total;
        for (int i = tid; i < a.nout; i += blockDim.x) dst[a.out_off + i] = 0.0;
        for (int p0 = C.x; p0 < C.y; p0 += kT6) {
            const int np = min(kT6, C.y - p0);
            if (tid == 0) item_next = 0;
            // stage [l^2 + l + m][b][q] for m = -l..l from the pair kernel's [q][b][lm], m >= 0
            const float2* src = a.alm + (size_t)p0 * rows;
            for (int i = tid; i < kT6 * rows; i += blockDim.x) {
                const int q = i / rows, r = i - q * rows;   // r = b * nlm + lm
                const int b = r / a.nlm, lm = r - b * a.nlm;
                int l = 0, m = lm;
                while (m > l) { m -= l + 1; ++l; }
                const float2 v = q < np ? src[i] : make_float2(0.f, 0.f);
                X[((l * l + l + m) * NR + b) * kRS6 + q] = v;
                if (m > 0) {
                    const float s = (m & 1) ? -1.f : 1.f;   // a_{l,-m} = (-1)^m conj(a_{lm})
                    X[((l * l + l - m) * NR + b) * kRS6 + q] = make_float2(s * v.x, -s * v.y);
                }
            }
            if (tid < kT6) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
            __syncthreads();   // also orders the row's zeroing before the first sums
            for (;;) {
                int it = 0;
                if (lane == 0) it = atomicAdd(&item_next, 1);
                it = __shfl_sync(warp::kFullMask, it, 0);
                if (it >= a.nitem) break;
                const int2 item = __ldg(&a.items[it]);
                const float u = su[lane];
                switch (item.y) {   // b3
#define NPCF_C6_CASE(B)                                                                              \
    case B:                                                                                          \
        if (B >= 2 && B <= NR - 3)                                                                   \
            c6_item<(B >= 2 && B <= NR - 3 ? B : 2), (B >= 2 && B <= NR - 3 ? NR - 1 - B : 2)>(item, a, X, u, \
                                                                                       binq, NR, dst, lane); \
        break;
                    NPCF_C6_CASE(2) NPCF_C6_CASE(3) NPCF_C6_CASE(4) NPCF_C6_CASE(5)
#undef NPCF_C6_CASE
                    default: break;
                }
            }
            __syncthreads();
        }
        __syncthreads();   // every thread has read chunk_s before it is taken again
    }
}

template <int NR>
void launch_nr6(const Contract6Args& a, int nblocks, cudaStream_t s) {
    const size_t smem = contract6_smem_bytes(a);
    cudaFuncSetAttribute(k_contract6<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_contract6<NR><<<nblocks, 256, smem, s>>>(a);
}

}  // namespace

size_t contract6_smem_bytes(const Contract6Args& a) {
    const size_t nlmf = (size_t)(a.lmax + 1) * (a.lmax + 1);
    return nlmf * a.nr * kRS6 * sizeof(float2) + (size_t)a.nr * a.nr * a.nr * sizeof(int);
}

void launch_contract6(const Contract6Args& a, int nblocks, cudaStream_t s) {
    switch (a.nr) {
        case 5: launch_nr6<5>(a, nblocks, s); break;
        case 6: launch_nr6<6>(a, nblocks, s); break;
        case 7: launch_nr6<7>(a, nblocks, s); break;
        case 8: launch_nr6<8>(a, nblocks, s); break;
        default: break;
    }
}

}  // namespace npcf
