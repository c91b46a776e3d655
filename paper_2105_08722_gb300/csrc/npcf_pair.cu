// Pair kernel: for every primary i the binned harmonic coefficients
//   a^b_lm(s_i) = sum_j w_j Y_lm(unit(r_j - s_i)) Theta^b(|r_j - s_i|)
// (Eq. binned-discrete-alm without 1/v_b; Algorithm 1 lines over secondaries and
// Algorithm 2).
//
// Like Algorithm 2 the harmonics come from Cartesian powers of the unit separation
// (x, y, z), accumulated per shell and converted to a_lm afterwards. Instead of all
// (lmax+1)(lmax+2)(lmax+3)/6 monomials x^p y^q z^r, the kernel accumulates the
// (lmax+1)^2 real components of S_{m,k} = sum_j w_j (x + i y)^m T_k(z), m + k <= lmax
// (T_k Chebyshev polynomials), which span exactly the Y_lm with m >= 0, since
// Y_lm = N_lm (-1)^m (x+iy)^m P_l^{(m)}(z) with P_l^{(m)} a polynomial of degree l - m.
// The Chebyshev basis keeps the conversion coefficients O(1), so FP32 sums do not lose
// accuracy to cancellation at high l as plain powers z^k would.
//
// One warp owns one primary at a time (dynamic schedule over cell-sorted primaries):
//   pass 0: scan the neighbour cells, apply the exact FP32 neighbour/shell rule and
//           count neighbours per shell;
//   pass 1: scan again and write neighbour indices into a shared-memory list ordered
//           by shell (only as many as fit; primaries with more neighbours repeat
//           pass 1 for the next slice);
//   accumulate: per shell, lanes take neighbours in parallel and accumulate the
//           S_{m,k} in registers; a shuffle transpose-reduction gives the per-shell
//           sums, which are converted to a_lm and written once per (primary, shell).
#include "npcf_device.h"
#include "npcf_rules.cuh"

namespace npcf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 16;

__host__ __device__ constexpr int ncomp(int L) { return (L + 1) * (L + 1); }
__host__ __device__ constexpr int nlmc(int L) { return (L + 1) * (L + 2) / 2; }
// position of Re S_{m,k} in the accumulator array (Im S_{m,k} follows for m > 0)
__host__ __device__ constexpr int s_index(int L, int m, int k) {
    return m == 0 ? k : (L + 1) + (m - 1) * (2 * L + 2 - m) + 2 * k;
}

template <int L>
__device__ __forceinline__ void harm_accumulate(float (&acc)[ncomp(L)], float x, float y, float z,
                                                float w) {
    float c[L + 1], s[L + 1], wz[L + 1];
    c[0] = 1.f;
    s[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        c[m] = fmaf(c[m - 1], x, -s[m - 1] * y);
        s[m] = fmaf(s[m - 1], x, c[m - 1] * y);
    }
    // w T_k(z): T_0 = 1, T_1 = z, T_{k+1} = 2 z T_k - T_{k-1}
    float t[L + 1];
    t[0] = 1.f;
    if (L >= 1) t[1] = z;
    const float z2 = z + z;
#pragma unroll
    for (int k = 2; k <= L; ++k) t[k] = fmaf(z2, t[k - 1], -t[k - 2]);
    wz[0] = w;
#pragma unroll
    for (int k = 1; k <= L; ++k) wz[k] = w * t[k];
#pragma unroll
    for (int k = 0; k <= L; ++k) acc[k] += wz[k];
#pragma unroll
    for (int m = 1; m <= L; ++m) {
#pragma unroll
        for (int k = 0; k + m <= L; ++k) {
            acc[s_index(L, m, k)] = fmaf(c[m], wz[k], acc[s_index(L, m, k)]);
            acc[s_index(L, m, k) + 1] = fmaf(s[m], wz[k], acc[s_index(L, m, k) + 1]);
        }
    }
}

// One halving step of the warp transpose-reduction: values [0, C) pair with
// [H, 2H); lanes with bit O set keep the upper half.
template <int C, int O>
__device__ __forceinline__ void tr_step(float* v, int lane) {
    constexpr int H = (C + 1) / 2;
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float lo = v[i];
        float hi = (i + H < C) ? v[i + H] : 0.f;
        float send = up ? lo : hi;
        float keep = up ? hi : lo;
        v[i] = keep + __shfl_xor_sync(kFull, send, O);
    }
}

template <int V>
struct TR {
    static constexpr int C0 = V, C1 = (C0 + 1) / 2, C2 = (C1 + 1) / 2, C3 = (C2 + 1) / 2,
                         C4 = (C3 + 1) / 2, C5 = (C4 + 1) / 2;
    static constexpr int F = C5;   // values left per lane
    __device__ static void run(float* v, int lane) {
        tr_step<C0, 16>(v, lane);
        tr_step<C1, 8>(v, lane);
        tr_step<C2, 4>(v, lane);
        tr_step<C3, 2>(v, lane);
        tr_step<C4, 1>(v, lane);
    }
    // original index of final slot i on this lane, or -1 for a padding slot
    __device__ static int origin(int i, int lane) {
        const int Cs[5] = {C0, C1, C2, C3, C4};
        const int Os[5] = {16, 8, 4, 2, 1};
        int idx = i;
        for (int st = 4; st >= 0; --st) {
            int H = (Cs[st] + 1) / 2;
            if (lane & Os[st]) idx += H;
            if (idx >= Cs[st]) return -1;
        }
        return idx;
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 21); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The neighbour rows of one cell as segments of the cell-sorted point array:
// (global start, count, offset in the staging buffer, shift code 2 bits per axis).
// Computed by one warp; returns (number of segments, total points) via shared memory.
__device__ void build_segments(const PairArgs& a, const int4* rows, int cx, int cy, int cz,
                               int4* segs, int* out_nseg, int* out_total, int lane) {
    const GridInfo& g = a.g;
    int nseg = 0, total = 0;
    for (int r0 = 0; r0 < a.nrows; r0 += 32) {
        const int r = r0 + lane;
        int cnt[2] = {0, 0}, beg[2] = {0, 0}, code[2] = {0, 0}, ns = 0;
        if (r < a.nrows) {
            const int4 rw = rows[r];
            int yy = cy + rw.x, zz = cz + rw.y, cyz = 0;
            bool ok = true;
            if (g.periodic) {
                if (yy < 0) { yy += g.gy; cyz |= 1 << 2; } else if (yy >= g.gy) { yy -= g.gy; cyz |= 2 << 2; }
                if (zz < 0) { zz += g.gz; cyz |= 1 << 4; } else if (zz >= g.gz) { zz -= g.gz; cyz |= 2 << 4; }
            } else {
                ok = yy >= 0 && yy < g.gy && zz >= 0 && zz < g.gz;
            }
            if (ok) {
                const int base = (zz * g.gy + yy) * g.gx;
                int x0 = cx + rw.z, x1 = cx + rw.w;
                if (g.periodic) {
                    if (x0 < 0) {
                        beg[ns] = (int)a.cell_start[base + x0 + g.gx];
                        cnt[ns] = (int)a.cell_start[base + g.gx] - beg[ns];
                        code[ns++] = cyz | 1;
                        x0 = 0;
                    }
                    if (x1 >= g.gx) {
                        beg[ns] = (int)a.cell_start[base];
                        cnt[ns] = (int)a.cell_start[base + x1 - g.gx + 1] - beg[ns];
                        code[ns++] = cyz | 2;
                        x1 = g.gx - 1;
                    }
                } else {
                    x0 = x0 < 0 ? 0 : x0;
                    x1 = x1 >= g.gx ? g.gx - 1 : x1;
                }
                if (x0 <= x1 && ns < 2) {
                    beg[ns] = (int)a.cell_start[base + x0];
                    cnt[ns] = (int)a.cell_start[base + x1 + 1] - beg[ns];
                    code[ns++] = cyz;
                }
            }
        }
        // drop empty segments, then a warp scan of segment and point counts
        int k = 0, pts = 0;
        for (int q = 0; q < ns; ++q)
            if (cnt[q] > 0) { beg[k] = beg[q]; cnt[k] = cnt[q]; code[k] = code[q]; pts += cnt[q]; ++k; }
        int ks = k, ps = pts;
        for (int o = 1; o < 32; o <<= 1) {
            int a1 = __shfl_up_sync(kFull, ks, o), a2 = __shfl_up_sync(kFull, ps, o);
            if (lane >= o) { ks += a1; ps += a2; }
        }
        int sidx = nseg + ks - k, soff = total + ps - pts;
        for (int q = 0; q < k; ++q) {
            segs[sidx + q] = make_int4(beg[q], cnt[q], soff, code[q]);
            soff += cnt[q];
        }
        nseg += __shfl_sync(kFull, ks, 31);
        total += __shfl_sync(kFull, ps, 31);
    }
    if (lane == 0) { *out_nseg = nseg; *out_total = total; }
}

// Per-warp state for the primary loop (shared memory).
struct WarpState {
    uint32_t hist[kMaxNr];
    uint32_t cur[kMaxNr];
    int rlo[kMaxNr], rhi[kMaxNr], gofs[kMaxNr];
    int next[4];
};

template <int L>
__global__ void __launch_bounds__(256, 1) k_pair(const PairArgs a) {
    constexpr int NC = ncomp(L);
    constexpr int NLM = nlmc(L);
    using R = TR<NC>;
    constexpr int kW = 8;  // warps per block
    extern __shared__ __align__(128) unsigned char dsm[];
    float4* cand = reinterpret_cast<float4*>(dsm);                       // staged neighbour points
    int4* segs = reinterpret_cast<int4*>(cand + a.cand_cap);             // segment table
    int4* rows = segs + 2 * a.nrows;                                      // neighbour rows
    uint16_t* lists = reinterpret_cast<uint16_t*>(rows + a.nrows);       // per-warp neighbour lists
    __shared__ WarpState ws[kW];
    __shared__ float red[kW][NC];
    __shared__ float kmat[NLM * (L + 1)];
    __shared__ float e2[kMaxNr + 1];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int unit[4];   // cell, nseg, total, overflow

    for (int i = threadIdx.x; i < a.nrows; i += blockDim.x) rows[i] = a.rows[i];
    for (int i = threadIdx.x; i < NLM * (L + 1); i += blockDim.x) kmat[i] = a.kmat[i];
    if (threadIdx.x <= a.nr) e2[threadIdx.x] = a.e2[threadIdx.x];
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nr = a.nr;
    const GridInfo& g = a.g;
    WarpState& W = ws[warp];
    uint16_t* list16 = lists + (size_t)warp * a.cap;
    uint32_t* list32 = reinterpret_cast<uint32_t*>(list16);

    int slot_org[R::F];
#pragma unroll
    for (int i = 0; i < R::F; ++i) slot_org[i] = R::origin(i, lane);
    uint32_t parity = 0;

    for (;;) {
        if (threadIdx.x == 0) unit[0] = atomicAdd(a.work, 1);
        __syncthreads();
        const int cell = unit[0];
        if (cell >= g.ncell) break;
        const int pbeg = (int)a.cell_start[cell], pend = (int)a.cell_start[cell + 1];
        if (pbeg == pend) {
            __syncthreads();
            continue;
        }
        const int cx = cell % g.gx, cy = (cell / g.gx) % g.gy, cz = cell / (g.gx * g.gy);
        if (warp == 0) build_segments(a, rows, cx, cy, cz, segs, &unit[1], &unit[2], lane);
        __syncthreads();
        const int nseg = unit[1], total = unit[2];
        const bool staged = total <= a.cand_cap;
        if (staged && total > 0) {
            // stage the neighbour points with bulk asynchronous copies (one mbarrier)
            if (threadIdx.x == 0) {
                const uint32_t b = smem_u32(&bar);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                             "r"((uint32_t)total * 16u)
                             : "memory");
                for (int s = 0; s < nseg; ++s) {
                    const int4 sg = segs[s];
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                            "r"(smem_u32(cand + sg.z)),
                        "l"(a.pts + sg.x), "r"((uint32_t)sg.y * 16u), "r"(b)
                        : "memory");
                }
            }
            const bool ok = mbar_wait_bounded(smem_u32(&bar), parity);
            // the whole block leaves together if any thread's wait gave up
            if (__syncthreads_or(ok ? 0 : 1)) {
                if (threadIdx.x == 0) atomicOr(a.err, 2);
                mbar_wait_bounded(smem_u32(&bar), parity);  // give in-flight copies a last chance to land
                break;
            }
            parity ^= 1u;
        }
        const int cap = staged ? a.cap : a.cap / 2;   // 16-bit staged or 32-bit global indices

        for (int p = pbeg + warp; p < pend; p += kW) {
            float2* out = a.alm + (size_t)p * nr * NLM;
            const float u = a.wp[p];
            if (u == 0.f) {  // primary not evaluated
                for (int i = lane; i < nr * NLM; i += 32) out[i] = make_float2(0.f, 0.f);
                if (lane < nr) a.cnt[(size_t)p * nr + lane] = 0u;
                continue;
            }
            const float4 pi = a.pts[p];

            // ---- pass 0: neighbour counts per shell
            if (lane < kMaxNr) W.hist[lane] = 0u;
            __syncwarp();
            for (int s = 0; s < nseg; ++s) {
                const int4 sg = segs[s];
                const float sx = shift_of(sg.w & 3, g.L), sy = shift_of((sg.w >> 2) & 3, g.L),
                            sz = shift_of((sg.w >> 4) & 3, g.L);
                for (int j = lane; j < sg.y; j += 32) {
                    const float4 pj = staged ? cand[sg.z + j] : a.pts[sg.x + j];
                    const int b = shell_of(pj, pi, sx, sy, sz, e2, nr);
                    if (b >= 0) atomicAdd(&W.hist[b], 1u);
                }
            }
            __syncwarp();
            if (lane < nr) {
                const uint32_t c = W.hist[lane];
                a.cnt[(size_t)p * nr + lane] = c;
                if (c) atomicAdd(&a.counts[lane], (unsigned long long)c);
            }

            float acc[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) acc[i] = 0.f;

            int s_next = 0, r_next = 0;
            while (s_next < nr) {
                // ---- slice of the shell-ordered list: shells [g_first, g_last]
                if (lane == 0) {
                    for (int q = 0; q < kMaxNr; ++q) { W.rlo[q] = 0; W.rhi[q] = -1; W.cur[q] = 0u; }
                    int used = 0, t = s_next, r = r_next, last = s_next;
                    while (t < nr) {
                        const int avail = (int)W.hist[t] - r;
                        const int take = avail < cap - used ? avail : cap - used;
                        W.rlo[t] = r;
                        W.rhi[t] = r + take;
                        W.gofs[t] = used;
                        used += take;
                        last = t;
                        if (take < avail) { r += take; break; }  // shell t continues in the next slice
                        ++t;
                        r = 0;
                        if (used >= cap) break;
                    }
                    W.next[0] = used;
                    W.next[1] = last;
                    W.next[2] = t;
                    W.next[3] = r;
                }
                __syncwarp();
                const int g_first = s_next;
                const int used = W.next[0];
                const int g_last = W.next[1];
                s_next = W.next[2];
                r_next = W.next[3];

                // ---- pass 1: write the slice's neighbour indices in shell order
                if (used > 0) {
                    for (int s = 0; s < nseg; ++s) {
                        const int4 sg = segs[s];
                        const float sx = shift_of(sg.w & 3, g.L), sy = shift_of((sg.w >> 2) & 3, g.L),
                                    sz = shift_of((sg.w >> 4) & 3, g.L);
                        for (int j0 = 0; j0 < sg.y; j0 += 32) {
                            const int j = j0 + lane;
                            int key = -1;
                            if (j < sg.y) {
                                const float4 pj = staged ? cand[sg.z + j] : a.pts[sg.x + j];
                                const int b = shell_of(pj, pi, sx, sy, sz, e2, nr);
                                if (b >= g_first && b <= g_last) key = b;
                            }
                            if (__ballot_sync(kFull, key >= 0) == 0u) continue;
                            const unsigned m = __match_any_sync(kFull, key);
                            const int leader = __ffs(m) - 1;
                            uint32_t b0 = 0u;
                            if (key >= 0 && lane == leader) b0 = atomicAdd(&W.cur[key], (uint32_t)__popc(m));
                            b0 = __shfl_sync(kFull, b0, leader);
                            if (key >= 0) {
                                const int rank = (int)b0 + __popc(m & ((1u << lane) - 1u));
                                if (rank >= W.rlo[key] && rank < W.rhi[key]) {
                                    const int slot = W.gofs[key] + rank - W.rlo[key];
                                    if (staged) list16[slot] = (uint16_t)(sg.z + j);
                                    else list32[slot] = (uint32_t)(sg.x + j);
                                }
                            }
                        }
                    }
                }
                __syncwarp();

                // ---- accumulate the slice, finish the shells it completes
                for (int t = g_first; t <= g_last; ++t) {
                    const int k0 = W.gofs[t];
                    const int kn = W.rhi[t] - W.rlo[t];
                    for (int k = lane; k < kn; k += 32) {
                        const float4 pj = staged ? cand[list16[k0 + k]] : a.pts[list32[k0 + k]];
                        float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                        if (g.periodic) {
                            dx = dx > g.hL ? dx - g.L : (dx < -g.hL ? dx + g.L : dx);
                            dy = dy > g.hL ? dy - g.L : (dy < -g.hL ? dy + g.L : dy);
                            dz = dz > g.hL ? dz - g.L : (dz < -g.hL ? dz + g.L : dz);
                        }
                        const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                        harm_accumulate<L>(acc, dx * inv, dy * inv, dz * inv, pj.w);
                    }
                    if (W.rhi[t] == (int)W.hist[t]) {
                        R::run(acc, lane);
#pragma unroll
                        for (int i = 0; i < R::F; ++i)
                            if (slot_org[i] >= 0) red[warp][slot_org[i]] = acc[i];
                        __syncwarp();
                        for (int q = lane; q < NLM; q += 32) {
                            int l = 0, m = q;
                            while (m > l) { m -= l + 1; ++l; }
                            float re = 0.f, im = 0.f;
                            for (int k = l - m; k >= 0; k -= 2) {
                                const float kk = kmat[q * (L + 1) + k];
                                const int si = s_index(L, m, k);
                                re = fmaf(kk, red[warp][si], re);
                                if (m > 0) im = fmaf(kk, red[warp][si + 1], im);
                            }
                            out[t * NLM + q] = make_float2(re, im);
                        }
#pragma unroll
                        for (int i = 0; i < NC; ++i) acc[i] = 0.f;
                        __syncwarp();
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();   // every warp is done with the staged points of this cell
    }
}

template <int L>
void launch_L(const PairArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = pair_dynamic_smem(a);
    cudaFuncSetAttribute(k_pair<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair<L><<<nblocks, 8 * 32, smem, s>>>(a);
}

}  // namespace

size_t pair_dynamic_smem(const PairArgs& a) {
    return (size_t)a.cand_cap * sizeof(float4) + (size_t)3 * a.nrows * sizeof(int4) +
           (size_t)8 * a.cap * sizeof(uint16_t);
}

void launch_pair(const PairArgs& a, int nblocks, cudaStream_t s) {
    switch (a.lmax) {
        case 0: launch_L<0>(a, nblocks, s); break;
        case 1: launch_L<1>(a, nblocks, s); break;
        case 2: launch_L<2>(a, nblocks, s); break;
        case 3: launch_L<3>(a, nblocks, s); break;
        case 4: launch_L<4>(a, nblocks, s); break;
        case 5: launch_L<5>(a, nblocks, s); break;
        case 6: launch_L<6>(a, nblocks, s); break;
        case 7: launch_L<7>(a, nblocks, s); break;
        case 8: launch_L<8>(a, nblocks, s); break;
        case 9: launch_L<9>(a, nblocks, s); break;
        case 10: launch_L<10>(a, nblocks, s); break;
        default: break;
    }
}

}  // namespace npcf
