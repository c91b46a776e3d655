// 4PCF contraction on the 5th-generation tensor cores, split bf16 with fp32 accumulation.
//
// The sum over primaries p of Eq. (simple-NPCF-summation) at N=4 is a dense contraction:
//   zeta_L(b1,b2,b3) = sum_{p, m3, c} A[(L,b1,b2)][(p,m3,c)] * B[(p,m3,c)][b3]
// with A = the coupled product P^{L,m3}(b1,b2;p) = sum_{m1} E C^L_M a^{b1}_{l1 m1} a^{b2}_{l2 m2}
// (real or imaginary part c) and B = u_p 2 S(m3) times the matching part of a^{b3}_{l3 m3}
// (the sign and the part depend on the parity of L: Q_L of App. B). Rows are grouped by
// (l3, parity) so that one B serves a whole group.
//
// One block per chunk of primaries keeps every 128 x 16 accumulator tile of the output in
// tensor memory. Per step of 16 primaries: the block stages their a_lm in shared memory,
// builds the B slabs (one 16 x 16 K-major slab per (m3, c) and group), then for every tile
// computes P in FP32 on the CUDA cores, splits it into three bf16 terms v ~ hi + mid + lo
// (residual ~2^-24 |v|) and writes one 128 x 16 K-major slab per (m3, c) and term; one
// thread issues the tcgen05 MMAs hi.hi + hi.mid + mid.hi + hi.lo + lo.hi + mid.mid into the
// tile's accumulator (the dropped products are below 2^-24 of |A B|) and commits them to
// an mbarrier, which the block waits on (bounded) before it overwrites the operands. The
// B slabs of a group are built when its first tile of the step comes up.
#include "npcf_device.h"
#include "npcf_tc.cuh"

#include <cuda_bf16.h>

namespace npcf {
namespace {

constexpr int kKStep = 16;        // primaries per K slab
constexpr int kThreads = 512;
constexpr uint32_t kIdesc = tc::idesc_bf16(128, 16);
constexpr uint32_t kATerm = 4096, kASlab = 3 * kATerm;   // 128 x 16 bf16 per term
constexpr uint32_t kBTerm = 512, kBSlab = 3 * kBTerm;    // 16 x 16 bf16 per term

struct TCLayout {
    size_t X, u, A, B, tc, ti, segs, lamseg, combos, cbin, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 127) & ~size_t(127); }

__host__ __device__ inline TCLayout tc_layout(const Contract4TCArgs& a) {
    TCLayout l;
    l.A = 0;                                                       // maxcomp x (hi, mid, lo: 4 KB each)
    l.B = al16(l.A + (size_t)a.maxcomp * kASlab);                  // maxcomp x (hi, mid, lo: 512 B each)
    l.X = al16(l.B + (size_t)a.maxcomp * kBSlab);                  // [b][lm][p] float2
    l.u = al16(l.X + (size_t)a.nr * a.nlm * kKStep * 8);
    l.tc = al16(l.u + kKStep * 4);
    l.ti = al16(l.tc + (size_t)a.nterms * 16);
    l.segs = al16(l.ti + (size_t)a.nterms * 4);
    l.lamseg = al16(l.segs + (size_t)a.nseg * 16);
    l.combos = al16(l.lamseg + (size_t)(a.nlam + 1) * 4);
    l.cbin = al16(l.combos + (size_t)a.ncombo * 8);
    l.total = al16(l.cbin + (size_t)a.ncombo * 4);
    return l;
}

// v ~ hi + mid + lo in bf16, stored at slab + off + {0, term, 2 term}
__device__ __forceinline__ void split_store(unsigned char* slab, uint32_t off, float v, uint32_t term) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    *reinterpret_cast<__nv_bfloat16*>(slab + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(slab + term + off) = mid;
    *reinterpret_cast<__nv_bfloat16*>(slab + 2 * term + off) = lo;
}

// P of a run of N rows (multiplet L, b1, b2 = b2first .. b2first + N - 1) for primary k of
// the step, every segment m3 of L, written as three bf16 terms into the A slabs: the
// coupling term and a^{b1} are loaded once per term for all N rows.
template <int N>
__device__ __forceinline__ void p_run(const int4 R, const float2* __restrict__ X, int nlm, int k,
                                      const float4* __restrict__ tcoef, const uint32_t* __restrict__ tidx,
                                      const int4* __restrict__ segs, const int* __restrict__ lamseg,
                                      unsigned char* Abuf, bool odd) {
    const int b1 = R.w & 0xff, b2 = R.w >> 8;
    const float2* A1 = X + (size_t)b1 * nlm * kKStep + k;
    const float2* A2 = X + (size_t)b2 * nlm * kKStep + k;
    const int lam = R.z, sg0 = lamseg[lam], sg1 = lamseg[lam + 1];
    for (int sg = sg0; sg < sg1; ++sg) {
        const int4 S = segs[sg];
        float pr[N], pim[N];
#pragma unroll
        for (int j = 0; j < N; ++j) pr[j] = pim[j] = 0.f;
        for (int q = S.x; q < S.y; ++q) {
            const float4 c = tcoef[q];
            const uint32_t id = tidx[q];
            const float2 x1 = A1[(id & 0xffffu) * kKStep];
            const float a0 = c.x * x1.x, a1 = c.y * x1.y, a2 = c.z * x1.y, a3 = c.w * x1.x;
            const float2* B2 = A2 + (id >> 16) * kKStep;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float2 x2 = B2[(size_t)j * nlm * kKStep];
                pr[j] = fmaf(a0, x2.x, fmaf(a1, x2.y, pr[j]));
                pim[j] = fmaf(a2, x2.x, fmaf(a3, x2.y, pim[j]));
            }
        }
        const int m3 = sg - sg0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const uint32_t off = tc::kmajor16_offset(R.x + j, k);
            if (m3 == 0) {
                split_store(Abuf, off, odd ? pim[j] : pr[j], kATerm);
            } else {
                split_store(Abuf + (size_t)(2 * m3 - 1) * kASlab, off, pr[j], kATerm);
                split_store(Abuf + (size_t)(2 * m3) * kASlab, off, pim[j], kATerm);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_contract4_tc(const Contract4TCArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    const TCLayout lay = tc_layout(a);
    unsigned char* Abuf = dsm + lay.A;
    unsigned char* Bbuf = dsm + lay.B;
    float2* X = reinterpret_cast<float2*>(dsm + lay.X);
    float* su = reinterpret_cast<float*>(dsm + lay.u);
    float4* tcoef = reinterpret_cast<float4*>(dsm + lay.tc);
    uint32_t* tidx = reinterpret_cast<uint32_t*>(dsm + lay.ti);
    int4* segs = reinterpret_cast<int4*>(dsm + lay.segs);
    int* lamseg = reinterpret_cast<int*>(dsm + lay.lamseg);
    int2* combos = reinterpret_cast<int2*>(dsm + lay.combos);
    int* cbin = reinterpret_cast<int*>(dsm + lay.cbin);
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int4 groups[32];
    __shared__ int gbslab[32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < a.nterms; i += kThreads) {
        const PairTerm t = a.terms[i];
        tcoef[i] = make_float4(t.cA, t.cB, t.cC, t.cD);
        tidx[i] = (uint32_t)t.lm1 | ((uint32_t)t.lm2 << 16);
    }
    for (int i = tid; i < a.nseg; i += kThreads) segs[i] = a.segs[i];
    for (int i = tid; i <= a.nlam; i += kThreads) lamseg[i] = a.lam_seg0[i];
    for (int i = tid; i < a.ncombo; i += kThreads) { combos[i] = a.combos[i]; cbin[i] = a.combo_bin[i]; }
    if (tid < a.ngroup) { groups[tid] = a.groups[tid]; gbslab[tid] = a.group_bslab[tid]; }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    const int2 C = a.chunks[blockIdx.x];   // primaries [C.x, C.y) of one catalog
    const int p0 = C.x, p1 = C.y;
    const int per = a.nr * a.nlm;
    uint32_t ncommit = 0;   // commits issued so far (thread 0 issues, every thread counts)
    bool ok = true;
    bool fresh = true;      // accumulators hold nothing since the last drain
    bool first_drain = true;
    int steps_since_drain = 0;
    double* dst = a.partial + (size_t)blockIdx.x * a.total;
    const int quarter = warp & 3;

    // Tensor memory -> FP64 partials of this block (= on the first drain, += after), so
    // that no accumulator sums more than drain_steps steps of MMAs before it is rounded
    // into FP64.
    auto drain = [&](bool have) {
        for (int t = warp >> 2; t < a.ntile; t += kThreads / 128) {
            const int4 T = a.tiles[t];
            const int4 G = groups[T.x];
            float v[16];
            if (have) {
                tc::tmem_ld16(tbase + ((uint32_t)(32 * quarter) << 16) + 16u * (uint32_t)t, v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            const int rr = 32 * quarter + lane;
            if (rr < T.z) {
                const int grow = T.y + rr;
                const int lam = a.group_lams[G.z + grow / a.ncombo];
                const int combo = grow % a.ncombo;
                const int2 bb = combos[combo];
                const int e0 = a.off4 + lam * a.nb4 + cbin[combo];
#pragma unroll
                for (int b3 = 0; b3 < 16; ++b3)
                    if (b3 > bb.y && b3 < a.nr) {
                        double* q = dst + e0 + b3 - bb.y - 1;
                        *q = first_drain ? (double)v[b3] : *q + (double)v[b3];
                    }
            }
        }
        first_drain = false;
    };

    for (int s0 = p0; s0 < p1 && ok; s0 += kKStep) {
        const int np = min(kKStep, p1 - s0);
        // ---- operands of the previous step must be consumed before they are overwritten
        if (ncommit > 0 && !tc::mbar_wait(&bar, (ncommit - 1) & 1u)) ok = false;
        if (__syncthreads_or(ok ? 0 : 1)) { ok = false; break; }
        // ---- stage a_lm of the step as [b][lm][p]
        for (int i = tid; i < kKStep * per; i += kThreads) {
            const int q = i / per, r = i % per;   // r = b * nlm + lm
            X[r * kKStep + q] = q < np ? a.alm[(size_t)(s0 + q) * per + r] : make_float2(0.f, 0.f);
        }
        if (tid < kKStep) su[tid] = tid < np ? a.wp[s0 + tid] : 0.f;
        __syncthreads();
        // ---- one tile at a time: P-build into A, then the MMAs
        for (int t = 0; t < a.ntile; ++t) {
            const int4 T = a.tiles[t];
            const int4 G = groups[T.x];
            const int ncomp = 2 * G.x + 1;
            if (t > 0 || ncommit > 0) {
                // A and B are free once the previous tile's MMAs have completed
                if (ncommit > 0 && !tc::mbar_wait(&bar, (ncommit - 1) & 1u)) ok = false;
                if (__syncthreads_or(ok ? 0 : 1)) { ok = false; break; }
            }
            if (t == 0 || a.tiles[t - 1].x != T.x) {
                // B slabs of this group: u 2S(m3) times the part of a^{b3}_{l3 m3} that meets
                // component j (m3 = (j+1)/2; j = 0: real part for even L, imaginary for odd L;
                // j odd: real part; j even > 0: imaginary part)
                const int l3 = G.x, odd = G.y;
                for (int i = tid; i < ncomp * 256; i += kThreads) {
                    const int j = i >> 8, e = i & 255, n = e >> 4, kk = e & 15;
                    const int m3 = (j + 1) >> 1;
                    const bool imc = (j == 0) ? (odd != 0) : ((j & 1) == 0);
                    float v = 0.f;
                    if (n < a.nr) {
                        const float2 x3 = X[(n * a.nlm + l3 * (l3 + 1) / 2 + m3) * kKStep + kk];
                        const float f = (m3 == 0 ? 1.f : 2.f) * su[kk];
                        v = odd ? f * (imc ? x3.x : x3.y) : f * (imc ? -x3.y : x3.x);
                    }
                    split_store(Bbuf + (size_t)j * kBSlab, tc::kmajor16_offset(n, kk), v, kBTerm);
                }
            }
            // 16 lanes per group of threads, one primary (K column) each
            const int k = tid & 15, g16 = tid >> 4;
            for (int rr = T.z + g16; rr < 128; rr += kThreads / 16)   // rows past the tile's end
                for (int j = 0; j < ncomp; ++j)
                    split_store(Abuf + (size_t)j * kASlab, tc::kmajor16_offset(rr, k), 0.f, kATerm);
            for (int r = a.tile_run0[t] + g16; r < a.tile_run0[t + 1]; r += kThreads / 16) {
                const int4 R = a.runs[r];
                switch (R.y) {
                    case 1: p_run<1>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 2: p_run<2>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 3: p_run<3>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 4: p_run<4>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 5: p_run<5>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 6: p_run<6>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    case 7: p_run<7>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                    default: p_run<8>(R, X, a.nlm, k, tcoef, tidx, segs, lamseg, Abuf, G.y != 0); break;
                }
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t d = tbase + 16u * (uint32_t)t;
                const uint32_t a0 = tc::smem_addr(Abuf), b0 = tc::smem_addr(Bbuf);
                for (int j = 0; j < ncomp; ++j) {
                    uint64_t ad[3], bd[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        ad[q] = tc::desc_kmajor(a0 + kASlab * j + kATerm * q, 128, 256);
                        bd[q] = tc::desc_kmajor(b0 + kBSlab * j + kBTerm * q, 128, 256);
                    }
                    tc::mma_bf16(d, ad[0], bd[0], kIdesc, (!fresh || j > 0) ? 1u : 0u);    // hi.hi
                    tc::mma_bf16(d, ad[0], bd[1], kIdesc, 1u);                               // hi.mid
                    tc::mma_bf16(d, ad[1], bd[0], kIdesc, 1u);                               // mid.hi
                    tc::mma_bf16(d, ad[0], bd[2], kIdesc, 1u);                               // hi.lo
                    tc::mma_bf16(d, ad[2], bd[0], kIdesc, 1u);                               // lo.hi
                    tc::mma_bf16(d, ad[1], bd[1], kIdesc, 1u);                               // mid.mid
                }
                tc::mma_commit(&bar);
            }
            ++ncommit;
        }
        if (!ok) break;
        fresh = false;
        if (++steps_since_drain >= a.drain_steps && s0 + kKStep < p1) {
            if (!tc::mbar_wait(&bar, (ncommit - 1) & 1u)) ok = false;
            if (__syncthreads_or(ok ? 0 : 1)) { ok = false; break; }
            tc::fence_after_sync();
            drain(true);
            tc::fence_before_sync();
            __syncthreads();
            fresh = true;
            steps_since_drain = 0;
        }
    }

    // ---- epilogue: every MMA done, tensor memory to FP64 partials
    if (ok && ncommit > 0 && !tc::mbar_wait(&bar, (ncommit - 1) & 1u)) ok = false;
    const bool good = !__syncthreads_or(ok ? 0 : 1);
    tc::fence_after_sync();
    if (!fresh || first_drain) drain(good && !fresh);
    if (!good) {
        if (tid == 0) atomicOr(a.err, 2);
        // MMAs may still be in flight: give them one more bounded wait before freeing TMEM
        if (ncommit > 0) tc::mbar_wait(&bar, (ncommit - 1) & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

}  // namespace

size_t contract4_tc_smem_bytes(const Contract4TCArgs& a) { return tc_layout(a).total; }

void launch_contract4_tc(const Contract4TCArgs& a, int nchunk, cudaStream_t s) {
    const size_t smem = contract4_tc_smem_bytes(a);
    cudaFuncSetAttribute(k_contract4_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_contract4_tc<<<nchunk, kThreads, smem, s>>>(a);
}

}  // namespace npcf
