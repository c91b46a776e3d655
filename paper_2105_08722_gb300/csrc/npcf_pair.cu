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
// A persistent block (2 groups of 8 warps) takes work units, runs of x-adjacent cells of
// one catalog's grid, from a device counter. For a unit, warp 0 lists the neighbour rows
// (rows of cells within r_max of the run) and one thread stages their points into shared
// memory with bulk asynchronous copies, in passes of rows that fit the buffer. A group
// then takes the unit's primaries one at a time:
//   cut: every staged row is cut to the primary's x-window and the kept rows form one
//        flat index space, split evenly over the group's warps;
//   scan: each lane tests candidates with the exact FP32 neighbour/shell rule; accepted
//        pairs go to the warp's sub-list (16-bit staged index, shell), shells counted;
//   sort: a counting sort orders the group's slice by shell (a full sub-list ends the
//        slice early; the scan then resumes where it stopped);
//   accumulate: each warp takes an equal run of 32-entry packets of the sorted slice,
//        accumulates the S_{m,k} of each shell in registers and reduces them across
//        lanes with a shuffle transpose-reduction; the per-shell sums, folded in warp
//        order, are converted to a_lm (added to the earlier passes' a_lm, if any).
#include "npcf_device.h"
#include "npcf_rules.cuh"
#include "npcf_warp.cuh"

namespace npcf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
using warp::TR;

__host__ __device__ constexpr int ncomp(int L) { return (L + 1) * (L + 1); }
__host__ __device__ constexpr int nlmc(int L) { return (L + 1) * (L + 2) / 2; }
// position of Re S_{m,k} in the accumulator array (Im S_{m,k} follows for m > 0)
__host__ __device__ constexpr int s_index(int L, int m, int k) {
    return m == 0 ? k : (L + 1) + (m - 1) * (2 * L + 2 - m) + 2 * k;
}

template <int L>
__device__ __forceinline__ void harm_accumulate(float (&acc)[ncomp(L)], float x, float y, float z,
                                                float w) {
    // c_m + i s_m = (x + i y)^m ; wt_k = w T_k(z) with T_0 = 1, T_1 = z,
    // T_{k+1} = 2 z T_k - T_{k-1} (the weight rides along the recurrence)
    float c[L + 1], s[L + 1], wt[L + 1];
    c[0] = 1.f;
    s[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        c[m] = fmaf(c[m - 1], x, -s[m - 1] * y);
        s[m] = fmaf(s[m - 1], x, c[m - 1] * y);
    }
    wt[0] = w;
    if (L >= 1) wt[1] = w * z;
    const float z2 = z + z;
#pragma unroll
    for (int k = 2; k <= L; ++k) wt[k] = fmaf(z2, wt[k - 1], -wt[k - 2]);
#pragma unroll
    for (int k = 0; k <= L; ++k) acc[k] += wt[k];
#pragma unroll
    for (int m = 1; m <= L; ++m) {
#pragma unroll
        for (int k = 0; k + m <= L; ++k) {
            acc[s_index(L, m, k)] = fmaf(c[m], wt[k], acc[s_index(L, m, k)]);
            acc[s_index(L, m, k) + 1] = fmaf(s[m], wt[k], acc[s_index(L, m, k) + 1]);
        }
    }
}

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

// The exact FP32 neighbour rule (same operations as shell_of in npcf_rules.cuh) followed
// by the shell lookup; -1 for a rejected pair. No loops: the range test is a predicate
// and linear edges take a direct estimate with one correction. e2lo = e2[0], e2hi = e2[nr].
// (A variant that skips the edge loads when the estimate is far from an edge measured
// slower: its branch keeps the independent candidates of a step from interleaving.)
__device__ __forceinline__ int pair_shell_fast(const float4 pj, const float4 pi, float sx, float sy, float sz,
                                               const float* e2, int nr, float e2lo, float e2hi, int linear,
                                               float r0, float inv_w) {
    const float dx = __fsub_rn(__fsub_rn(pj.x, pi.x), sx);
    const float dy = __fsub_rn(__fsub_rn(pj.y, pi.y), sy);
    const float dz = __fsub_rn(__fsub_rn(pj.z, pi.z), sz);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const bool ok = (r2 > 0.f) & (r2 >= e2lo) & (r2 < e2hi);
    int b;
    if (linear) {
        // the estimate is within one shell of the rule's shell (shells are wider than 1e-3
        // r_max when linear is set, far above the FP32 error of the estimate), so one
        // correction against both of its edges, loaded together, is exact
        b = (int)((r2 * rsqrtf(r2) - r0) * inv_w);
        b = min(max(b, 0), nr - 1);
        const float lo = e2[b], hi = e2[b + 1];
        b += (r2 >= hi ? 1 : 0) - (r2 < lo ? 1 : 0);
    } else {
        b = 0;
#pragma unroll
        for (int step = 8; step >= 1; step >>= 1)
            if (b + step < nr && r2 >= e2[b + step]) b += step;
    }
    return ok ? b : -1;
}

// The neighbour rows of a run of cells (x-adjacent, same y and z) as segments of the
// cell-sorted point array: (global start, count, offset in the staging buffer, code).
// code bits 0-5: periodic shift, 2 bits per axis; bits 6-18: the row's y cell; bits 19-31:
// its z cell. Computed by one warp; the totals go to shared memory.
__device__ void build_segments(const PairArgs& a, const int4* rows, int cbase, int cx, int cy, int cz, int run,
                               int4* segs, int* out_nseg, int* out_total, int* out_maxseg, int lane) {
    const GridInfo& g = a.g;
    int nseg = 0, total = 0, maxseg = 0;
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
                const int base = cbase + (zz * g.gy + yy) * g.gx;
                cyz |= (yy << 6) | (zz << 19);   // the row's cell (y, z) rides along for the x-window cut
                int x0 = cx + rw.z, x1 = cx + run - 1 + rw.w;
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
            if (cnt[q] > 0) {
                beg[k] = beg[q];
                cnt[k] = cnt[q];
                code[k] = code[q];
                pts += cnt[q];
                maxseg = max(maxseg, cnt[q]);
                ++k;
            }
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
    for (int o = 16; o > 0; o >>= 1) maxseg = max(maxseg, __shfl_xor_sync(kFull, maxseg, o));
    if (lane == 0) { *out_nseg = nseg; *out_total = total; *out_maxseg = maxseg; }
}

constexpr int kW = 8;             // warps per group; a group works on one primary
constexpr int kG = 2;             // groups per block
constexpr int kShiftCodes = 64;   // 2 bits per axis

// Byte offsets of the pair kernel's dynamic shared memory (host and device agree).
// cap is the neighbour-list capacity of one group in 16-bit entries.
struct PairLayout {
    size_t cand, segs, rows, tpref, tdc, tstart, tcode, ulist, ushell, slist, part, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Floats of one group's partial area: nr + kW - 1 slots for the slice's per-warp sums
// (warp w's share of shell t goes to slot t + w: the warps' equal runs of packets of the
// shell-sorted slice are ordered, so these never collide) and nr per-shell sums.
__host__ __device__ constexpr int part_floats(int nr, int nc) { return (2 * nr + kW - 1) * nc; }

__host__ __device__ inline PairLayout pair_layout(int cand_cap, int nrows, int cap, int nr, int nc) {
    PairLayout l;
    l.cand = 0;
    l.segs = align16(l.cand + (size_t)cand_cap * 16);
    l.rows = align16(l.segs + (size_t)2 * nrows * 16);
    // per group: flat-index prefix and (staging offset minus prefix, shift code) of each
    // kept row; per-row scratch of the cut (staging start, code and count)
    l.tpref = align16(l.rows + (size_t)nrows * 16);
    l.tdc = align16(l.tpref + (size_t)kG * (2 * nrows + 1) * 4);
    l.tstart = align16(l.tdc + (size_t)kG * 2 * nrows * 4);
    l.tcode = align16(l.tstart + (size_t)kG * 2 * nrows * 4);
    l.ulist = align16(l.tcode + (size_t)kG * 2 * nrows * 4);
    l.ushell = align16(l.ulist + (size_t)kG * cap * 2);
    l.slist = align16(l.ushell + (size_t)kG * cap);
    // per group: the slice's (warp, shell) partials in slots shell + warp, then the
    // primary's per-shell sums
    l.part = align16(l.slist + (size_t)kG * cap * 2);
    l.total = align16(l.part + (size_t)kG * part_floats(nr, nc) * 4);
    return l;
}

// Shared state of one group.
struct GroupShared {
    uint32_t hist[kW][kMaxNr];     // per-warp shell counts of the current slice
    uint32_t base[kW][kMaxNr];     // where each warp scatters each shell
    uint32_t off[kMaxNr + 1];      // shell offsets of the sorted slice
    uint32_t pk[kMaxNr + 1];       // first 32-entry packet of each shell (packets never straddle shells)
    uint32_t tot[kMaxNr];          // shell totals of the current primary
    int done[kW];
    int wtot[kW];                  // per-warp sums of the row-trimming prefix
};

template <int L>
struct PairShared {
    float4 shift[kShiftCodes];     // (sx, sy, sz) of each periodic shift code
    float kmat[nlmc(L) * (L + 1)];
    float e2[kMaxNr + 1];
    GroupShared grp[kG];
    int unit[4];
};

__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(kW * 32) : "memory");
}

// Both ends of the staged row at 'base' (n points, sorted by x) that fall in [vlo, vhi]:
// the first index with x >= vlo and the first with x > vhi. The two searches run in
// lockstep without branches: the answer is built bit by bit from the highest power of
// two <= n, each bit kept if the predicate holds at the probed index.
__device__ __forceinline__ int2 x_bounds(const float4* cand, int base, int n, float vlo, float vhi) {
    int a = 0, b = 0;
    if (n > 0) {
        for (int step = 1 << (31 - __clz(n)); step > 0; step >>= 1) {
            const float xa = cand[base + min(a + step, n) - 1].x;
            const float xb = cand[base + min(b + step, n) - 1].x;
            a += (a + step <= n && xa < vlo) ? step : 0;
            b += (b + step <= n && !(xb > vhi)) ? step : 0;
        }
    }
    return make_int2(a, b);
}

// The part of every staged row this primary can reach, as one flat index space over
// the rows left non-empty: row s covers flat [tpref[s], tpref[s+1]), its staged index is
// flat + (tdc[s] >> 6) and its periodic shift code tdc[s] & 63. With trim, a row keeps
// only the points whose x lies within sqrt(r_max^2 - d_yz^2) (plus a margin) of the
// primary, d_yz the distance from the primary to the row's (y, z) cell square; the exact
// FP32 rule is applied to what remains. Rows are sorted by x (cells in x order, members
// sorted by x). tstart and tcode are scratch. Returns the flat total; *nrow = rows kept.
template <int L>
__device__ __forceinline__ int trim_rows(const PairArgs& a, const PairShared<L>& sh, const float4* cand,
                                         const int4* segs, int nseg, int zbase, const float4 pi, int* tpref,
                                         int* tdc, int* tstart, int* tcode, int* wtot, bool trim, int grp,
                                         int warp, int lane, int* nrow) {
    const int gt = warp * 32 + lane;
    const int per = (nseg + kW * 32 - 1) / (kW * 32);   // rows per thread
    const int s0 = min(nseg, gt * per), s1 = min(nseg, s0 + per);
    const float R2 = sh.e2[a.nr], m = a.trim_margin, c = a.cell;
    int cnt_local = 0, rows_local = 0;
    for (int s = s0; s < s1; ++s) {
        const int4 sg = segs[s];
        int lo = 0, hi = sg.y;
        if (trim) {
            const float4 sf = sh.shift[sg.w & 63];
            const int yy = (sg.w >> 6) & 8191, zz = (int)((unsigned)sg.w >> 19);
            const float ylo = a.g.oy + (float)yy * c - sf.y - m, yhi = ylo + c + 2.f * m;
            const float zlo = a.g.oz + (float)zz * c - sf.z - m, zhi = zlo + c + 2.f * m;
            const float dy = fmaxf(0.f, fmaxf(ylo - pi.y, pi.y - yhi));
            const float dz = fmaxf(0.f, fmaxf(zlo - pi.z, pi.z - zhi));
            const float d2 = dy * dy + dz * dz;
            if (d2 >= R2 * (1.f + 1e-5f)) {
                hi = 0;
            } else {
                const float h = sqrtf(fmaxf(R2 * (1.f + 1e-5f) - d2, 0.f)) + m;
                const float xc = pi.x + sf.x;
                const int2 ab = x_bounds(cand, sg.z - zbase, sg.y, xc - h, xc + h);
                lo = ab.x;
                hi = ab.y;
            }
        }
        tstart[s] = sg.z - zbase + lo;
        tcode[s] = (sg.w & 63) | ((hi - lo) << 8);
        cnt_local += hi - lo;
        rows_local += hi > lo ? 1 : 0;
    }
    // exclusive prefix over the group's threads of (rows kept << 16 | points); both fit
    // in 16 bits: points <= staging capacity, rows <= 2 nrows
    const int v = (rows_local << 16) | cnt_local;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    group_sync(grp);
    int base = incl - v;
    for (int w = 0; w < warp; ++w) base += wtot[w];
    int total = 0;
    for (int w = 0; w < kW; ++w) total += wtot[w];
    int pb = base & 0xffff, rb = base >> 16;
    for (int s = s0; s < s1; ++s) {
        const int cs = tcode[s] >> 8;
        if (cs > 0) {
            tpref[rb] = pb;
            tdc[rb] = ((tstart[s] - pb) << 6) | (tcode[s] & 63);   // staged start >= flat start
            ++rb;
            pb += cs;
        }
    }
    *nrow = total >> 16;
    total &= 0xffff;
    if (gt == 0) tpref[*nrow] = total;
    group_sync(grp);
    return total;
}

// One primary, processed by one group of kW warps. Neighbours are split evenly over the
// warps (flat index space of the cut staged rows, or segments round-robin for the
// global-memory path); each warp appends accepted neighbours (index, shell) to its own
// sub-list; a counting sort orders the slice by shell (ranks from __match_any_sync); each
// warp takes an equal run of 32-entry packets of the sorted slice and its per-shell sums
// go to per-warp partials, which give a_lm at the end (added to the a_lm of earlier
// staging passes when add is set). Sub-lists that fill up end the slice early, and the
// scan resumes where it stopped.
template <int L, bool STAGED>
__device__ __forceinline__ void one_primary(const PairArgs& a, PairShared<L>& sh, const float4* cand,
                                            const int4* segs, int nseg, int zbase, int total,
                                            int* tpref, int* tdc, int* tstart, int* tcode, bool trim,
                                            uint16_t* ulist, uint8_t* ushell, uint16_t* slist, float* part,
                                            int p, int cat, bool add, int grp, int warp, int lane,
                                            const int* slot_org) {
    constexpr int NC = ncomp(L);
    constexpr int NLM = nlmc(L);
    using R = TR<NC>;
    GroupShared& G = sh.grp[grp];
    const int nr = a.nr;
    const int gt = warp * 32 + lane;   // thread index in the group
    const GridInfo& g = a.g;
    float2* out = a.alm + (size_t)p * nr * NLM;
    // A primary of weight 0 adds nothing to zeta, but its neighbours are still counted
    // (every primary's pairs enter the counts) unless separate primary weights select a
    // sample of primaries: then a weight of 0 means "not in the sample".
    if (a.skip_zero && a.wp[p] == 0.f) {  // primary not evaluated
        if (!add) {
            for (int i = gt; i < nr * NLM; i += kW * 32) out[i] = make_float2(0.f, 0.f);
            if (gt < nr) a.cnt[(size_t)p * nr + gt] = 0u;
        }
        return;
    }
    const float4 pi = a.pts[p];
    float* slot = part;                          // [nr + kW - 1][NC], rewritten every slice
    float* psum = part + (nr + kW - 1) * NC;     // [nr][NC] sums of the primary
    for (int i = gt; i < nr * NC; i += kW * 32) psum[i] = 0.f;
    if (gt < kMaxNr) G.tot[gt] = 0u;

    // this warp's share of the neighbours and its sub-list
    const int capw = STAGED ? a.cap / kW : a.cap / (2 * kW);
    // sub-list entries: 16-bit staged index (staged) or 32-bit point index (global), shell
    uint16_t* ul16 = ulist + (size_t)warp * (a.cap / kW);
    uint32_t* ul32 = reinterpret_cast<uint32_t*>(ul16);
    uint8_t* us = ushell + (size_t)warp * (a.cap / kW);
    const float e2lo = sh.e2[0], e2hi = sh.e2[nr];
    uint32_t* sl32 = reinterpret_cast<uint32_t*>(slist);
    // staged: the rows cut to this primary's x-window, one flat index space split evenly
    int nrow = 0;
    const int T = STAGED ? trim_rows<L>(a, sh, cand, segs, nseg, zbase, pi, tpref, tdc, tstart, tcode, G.wtot,
                                        trim, grp, warp, lane, &nrow)
                         : total;
    const int per = (T + kW - 1) / kW;
    int cursor = STAGED ? min(T, warp * per) : 0;
    const int kend = STAGED ? min(T, cursor + per) : 0;
    int seg = warp, segpos = 0;   // global-memory path: segments warp, warp + kW, ...
    const unsigned lt = (1u << lane) - 1u;
    // staged: the row of flat index cursor (first s with tpref[s + 1] > cursor), the same
    // in every lane
    int srow = 0;
    if (STAGED && cursor < kend) {
        const int k0 = cursor;
        int lo = 0, n = nrow;
        while (n > 0) {
            const int half = n >> 1;
            if (tpref[lo + half + 1] <= k0) {
                lo += half + 1;
                n -= half + 1;
            } else {
                n = half;
            }
        }
        srow = lo;
    }
    group_sync(grp);   // partials zeroed before any warp adds to them

    for (;;) {
        // ---- scan: append accepted neighbours while the sub-list has room, counting shells
        int cw = 0;
        if (lane < kMaxNr) G.hist[warp][lane] = 0u;
        __syncwarp();
        if (STAGED) {
            // candidates per lane per step (independent chains). A step appends up to
            // 32 KC entries, so capw >= 32 KC is required for progress: the host admits
            // list capacities of at least 1024 (capw >= 128).
            constexpr int KC = 4;
            while (cw + 32 * KC <= capw && cursor < kend) {
                // Rows of the step's flat indices cursor + o, o < 32 KC, without per-lane
                // searches: lane i loads the end of row srow + i (rows are non-empty, so the
                // ends increase strictly); a bitmap of the ends' offsets in the step gives
                // each offset's row as srow + the ends at or below it. The step stops at the
                // last loaded end, so no row beyond the loaded ones is met.
                const int d = tpref[min(srow + 1 + lane, nrow)] - cursor;   // >= 1
                const int lim = min(min(32 * KC, kend - cursor), __shfl_sync(kFull, d, 31));
                unsigned W[KC];
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const unsigned o = (unsigned)(d - 32 * j);
                    W[j] = __reduce_or_sync(kFull, o < 32u ? 1u << o : 0u);
                }
                const unsigned le = 0xffffffffu >> (31 - lane);   // offsets 32 j .. 32 j + lane
                int q[KC], b[KC];
                float4 sf[KC];
                int below = 0;
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const int row = min(srow + below + __popc(W[j] & le), nrow - 1);
                    below += __popc(W[j]);
                    const int dc = tdc[row];
                    q[j] = 32 * j + lane < lim ? cursor + 32 * j + lane + (dc >> 6) : 0;
                    sf[j] = sh.shift[dc & 63];
                }
                float4 c[KC];
#pragma unroll
                for (int j = 0; j < KC; ++j) c[j] = cand[q[j]];
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const int r = pair_shell_fast(c[j], pi, sf[j].x, sf[j].y, sf[j].z, sh.e2, nr, e2lo, e2hi,
                                                  a.linear, a.lin_r0, a.lin_inv_w);
                    b[j] = (32 * j + lane < lim) ? r : -1;
                }
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    const unsigned m = __ballot_sync(kFull, b[j] >= 0);
                    if (b[j] >= 0) {
                        const int pos = cw + __popc(m & lt);
                        ul16[pos] = (uint16_t)q[j];
                        us[pos] = (uint8_t)b[j];
                    }
                    cw += __popc(m);
                    const unsigned gm = __match_any_sync(kFull, b[j]);
                    if (b[j] >= 0 && lane == __ffs(gm) - 1) atomicAdd(&G.hist[warp][b[j]], (uint32_t)__popc(gm));
                }
                srow += __popc(__ballot_sync(kFull, d <= lim));   // the row of cursor + lim
                cursor += lim;
            }
        } else {
            while (seg < nseg && cw + 32 <= capw) {
                const int4 sg = segs[seg];
                const float4 sf = sh.shift[sg.w & 63];
                const int k = segpos + lane;
                int b = -1;
                if (k < sg.y)
                    b = pair_shell_fast(a.pts[sg.x + k], pi, sf.x, sf.y, sf.z, sh.e2, nr, e2lo, e2hi, a.linear,
                                        a.lin_r0, a.lin_inv_w);
                const unsigned m = __ballot_sync(kFull, b >= 0);
                if (b >= 0) {
                    const int pos = cw + __popc(m & lt);
                    ul32[pos] = (uint32_t)(sg.x + k);
                    us[pos] = (uint8_t)b;
                }
                cw += __popc(m);
                const unsigned gm = __match_any_sync(kFull, b);
                if (b >= 0 && lane == __ffs(gm) - 1) atomicAdd(&G.hist[warp][b], (uint32_t)__popc(gm));
                segpos += 32;
                if (segpos >= sg.y) { seg += kW; segpos = 0; }
            }
        }
        const bool done = STAGED ? (cursor >= kend) : (seg >= nseg);
        if (lane == 0) G.done[warp] = done ? 1 : 0;
        group_sync(grp);
        int all_done = 1;
        for (int w = 0; w < kW; ++w) all_done &= G.done[w];

        // ---- shell offsets of the slice and each warp's scatter bases
        if (warp == 0) {
            uint32_t tsum = 0u;
            if (lane < nr)
                for (int w = 0; w < kW; ++w) tsum += G.hist[w][lane];
            uint32_t incl = tsum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            // packets of 32 entries per shell, and their prefix
            const uint32_t npk = (tsum + 31u) / 32u;
            uint32_t pincl = npk;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, pincl, o);
                if (lane >= o) pincl += y;
            }
            if (lane < nr) {
                uint32_t bw = incl - tsum;
                G.off[lane] = bw;
                G.pk[lane] = pincl - npk;
                for (int w = 0; w < kW; ++w) { G.base[w][lane] = bw; bw += G.hist[w][lane]; }
                G.tot[lane] += tsum;
            }
            if (lane == nr - 1) {
                G.off[nr] = incl;
                G.pk[nr] = pincl;
            }
        }
        group_sync(grp);

        // ---- scatter the sub-list into shell order (stable within a warp)
        for (int k0 = 0; k0 < cw; k0 += 32) {
            const bool ok = k0 + lane < cw;
            const int shk = ok ? (int)us[k0 + lane] : -1;
            const uint32_t idx = ok ? (STAGED ? (uint32_t)ul16[k0 + lane] : ul32[k0 + lane]) : 0u;
            const unsigned m = __match_any_sync(kFull, shk);
            const uint32_t b0 = ok ? G.base[warp][shk] : 0u;
            __syncwarp();
            if (ok) {
                const uint32_t pos = b0 + (uint32_t)__popc(m & lt);
                if (STAGED) slist[pos] = (uint16_t)idx;
                else sl32[pos] = idx;
                if (lane == __ffs(m) - 1) G.base[warp][shk] = b0 + (uint32_t)__popc(m);
            }
            __syncwarp();
        }
        group_sync(grp);

        // ---- accumulate an equal run of 32-entry packets of the sorted slice, per shell
        // (a packet holds one shell's entries, so only a shell's last packet has idle lanes)
        {
            const int npk = (int)G.pk[nr];
            const int per = (npk + kW - 1) / kW;
            const int q0 = min(npk, warp * per), q1 = min(npk, q0 + per);
            for (int t = 0; t < nr; ++t) {
                const int pa = max(q0, (int)G.pk[t]), pb = min(q1, (int)G.pk[t + 1]);
                if (pa >= pb) continue;
                const int base = (int)G.off[t] - 32 * (int)G.pk[t], hi = (int)G.off[t + 1];
                float acc[NC];
                const float invL = 1.f / g.L;
#pragma unroll
                for (int i = 0; i < NC; ++i) acc[i] = 0.f;
                for (int q = pa; q < pb; ++q) {
                    const int k = base + 32 * q + lane;
                    if (k >= hi) continue;
                    float dx, dy, dz, wj;
                    // accepted pairs are closer than r_max < L/3: the minimum image is the
                    // image the neighbour rule accepted (taken without branches)
                    const float4 pj = STAGED ? cand[slist[k]] : a.pts[sl32[k]];
                    dx = pj.x - pi.x;
                    dy = pj.y - pi.y;
                    dz = pj.z - pi.z;
                    wj = pj.w;
                    if (g.periodic) {
                        dx = fmaf(-g.L, rintf(dx * invL), dx);
                        dy = fmaf(-g.L, rintf(dy * invL), dy);
                        dz = fmaf(-g.L, rintf(dz * invL), dz);
                    }
                    const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    harm_accumulate<L>(acc, dx * inv, dy * inv, dz * inv, wj);
                }
                R::run(acc, lane);
                float* pw = slot + (size_t)(t + warp) * NC;
#pragma unroll
                for (int i = 0; i < R::F; ++i)
                    if (slot_org[i] >= 0) pw[slot_org[i]] = acc[i];
            }
        }
        group_sync(grp);   // lists are rewritten by the next slice
        // fold the slice's slots into the primary's sums, warps in order (deterministic);
        // the next slice writes slots only after its next group barrier
        {
            const int npk = (int)G.pk[nr];
            const int per = (npk + kW - 1) / kW;
            for (int i = gt; i < nr * NC; i += kW * 32) {
                const int t = i / NC, c = i - t * NC;
                const int o0 = (int)G.pk[t], o1 = (int)G.pk[t + 1];
                float v = 0.f;
                for (int w = 0; w < kW; ++w) {
                    const int q0 = min(npk, w * per), q1 = min(npk, q0 + per);
                    if (max(q0, o0) < min(q1, o1)) v += slot[(t + w) * NC + c];
                }
                psum[i] += v;
            }
        }
        if (all_done) break;
    }
    group_sync(grp);   // every fold is done before the sums are read

    // ---- combine the per-warp partials and convert to a_lm
    for (int i = gt; i < nr * NLM; i += kW * 32) {
        const int t = i / NLM, q = i % NLM;
        int l = 0, m = q;
        while (m > l) { m -= l + 1; ++l; }
        float re = 0.f, im = 0.f;
        for (int k = l - m; k >= 0; k -= 2) {
            const int si = s_index(L, m, k);
            const float sr = psum[t * NC + si];
            const float sim = m > 0 ? psum[t * NC + si + 1] : 0.f;
            const float kk = sh.kmat[q * (L + 1) + k];
            re = fmaf(kk, sr, re);
            im = fmaf(kk, sim, im);
        }
        if (add) {   // a later staging pass of the unit: a_lm is linear in the sums
            const float2 o = out[i];
            re += o.x;
            im += o.y;
        }
        out[i] = make_float2(re, im);
    }
    if (gt < nr) {
        const uint32_t c = G.tot[gt];
        a.cnt[(size_t)p * nr + gt] = add ? a.cnt[(size_t)p * nr + gt] + c : c;
        if (c) atomicAdd(&a.counts[(size_t)cat * nr + gt], (unsigned long long)c);
    }
    group_sync(grp);   // partials and totals are reset by the next primary
}

template <int L>
__global__ void __launch_bounds__(kG * kW * 32, 1) k_pair(const PairArgs a) {
    using R = TR<ncomp(L)>;
    extern __shared__ __align__(128) unsigned char dsm[];
    const PairLayout lay = pair_layout(a.cand_cap, a.nrows, a.cap, a.nr, ncomp(L));
    float4* cand = reinterpret_cast<float4*>(dsm + lay.cand);
    int4* segs = reinterpret_cast<int4*>(dsm + lay.segs);
    int4* rows = reinterpret_cast<int4*>(dsm + lay.rows);
    __shared__ PairShared<L> sh;
    __shared__ __align__(8) uint64_t bar;

    const GridInfo& g = a.g;
    for (int i = threadIdx.x; i < a.nrows; i += blockDim.x) rows[i] = a.rows[i];
    for (int i = threadIdx.x; i < nlmc(L) * (L + 1); i += blockDim.x) sh.kmat[i] = a.kmat[i];
    if (threadIdx.x <= a.nr) sh.e2[threadIdx.x] = a.e2[threadIdx.x];
    if (threadIdx.x < kShiftCodes) {
        const int c = threadIdx.x;
        sh.shift[c] = make_float4(shift_of(c & 3, g.L), shift_of((c >> 2) & 3, g.L),
                                  shift_of((c >> 4) & 3, g.L), 0.f);
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int wblk = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = wblk / kW, warp = wblk % kW;
    uint16_t* ulist = reinterpret_cast<uint16_t*>(dsm + lay.ulist) + (size_t)grp * a.cap;
    uint8_t* ushell = dsm + lay.ushell + (size_t)grp * a.cap;
    uint16_t* slist = reinterpret_cast<uint16_t*>(dsm + lay.slist) + (size_t)grp * a.cap;
    float* part = reinterpret_cast<float*>(dsm + lay.part) + (size_t)grp * part_floats(a.nr, ncomp(L));
    int* tpref = reinterpret_cast<int*>(dsm + lay.tpref) + (size_t)grp * (2 * a.nrows + 1);
    int* tdc = reinterpret_cast<int*>(dsm + lay.tdc) + (size_t)grp * 2 * a.nrows;
    int* tstart = reinterpret_cast<int*>(dsm + lay.tstart) + (size_t)grp * 2 * a.nrows;
    int* tcode = reinterpret_cast<int*>(dsm + lay.tcode) + (size_t)grp * 2 * a.nrows;
    // the x-window cut needs every cell sorted by x (binning flags bit 8 otherwise)
    const bool trim = a.trim != 0 && (*(volatile int*)a.err & 8) == 0;
    int slot_org[R::F];
#pragma unroll
    for (int i = 0; i < R::F; ++i) slot_org[i] = R::origin(i, lane);
    uint32_t parity = 0;
    const int upr = (g.gx + a.run - 1) / a.run;   // units per row of cells
    const int ucat = upr * g.gy * g.gz;           // units per catalog
    const int nunits = ucat * a.ncat;

    for (;;) {
        if (threadIdx.x == 0) sh.unit[0] = atomicAdd(a.work, 1);
        __syncthreads();
        const int u = sh.unit[0];
        if (u >= nunits) break;
        // unit u: catalog u / ucat, then a run of x-adjacent cells of that catalog's grid
        const int cat = u / ucat, uc = u - cat * ucat;
        const int cbase = cat * g.ncell;
        const int row = uc / upr, cx = (uc % upr) * a.run;
        const int run = min(a.run, g.gx - cx);
        const int cy = row % g.gy, cz = row / g.gy;
        const int c0 = cbase + (cz * g.gy + cy) * g.gx + cx;
        const int pbeg = (int)a.cell_start[c0], pend = (int)a.cell_start[c0 + run];
        if (pbeg == pend) {
            __syncthreads();
            continue;
        }
        if (wblk == 0)
            build_segments(a, rows, cbase, cx, cy, cz, run, segs, &sh.unit[1], &sh.unit[2], &sh.unit[3], lane);
        __syncthreads();
        const int nseg = sh.unit[1], total = sh.unit[2];
        if (sh.unit[3] > a.cand_cap) {
            // a row longer than the staging buffer: neighbours straight from global memory
            for (int p = pbeg + grp; p < pend; p += kG)
                one_primary<L, false>(a, sh, cand, segs, nseg, 0, total, tpref, tdc, tstart, tcode, trim, ulist,
                                      ushell, slist, part, p, cat, false, grp, warp, lane, slot_org);
            __syncthreads();
            continue;
        }
        // Staged in passes of consecutive rows that fit the staging buffer (one pass unless
        // the unit's neighbourhood is larger); each pass adds its sums to the primaries'
        // a_lm and counts. A pass of the rows [s0, s1) is staged with bulk asynchronous
        // copies (one mbarrier); row s sits at sg.z - segs[s0].z in the buffer.
        bool failed = false;
        for (int s0 = 0, pass = 0; pass == 0 || s0 < nseg; ++pass) {
            // every thread plans the pass (the same search over the shared row list)
            int s1 = s0, ptotal = 0;
            const int zbase = s0 < nseg ? segs[s0].z : 0;
            if (s0 < nseg) {
                // the most rows from s0 whose points fit (staging offsets increase)
                int lo = s0 + 1, n = nseg - s0 - 1;   // answer in [s0 + 1, nseg]
                while (n > 0) {
                    const int half = n >> 1;
                    const int4 sg = segs[lo + half];
                    if (sg.z + sg.y - zbase <= a.cand_cap) {
                        lo += half + 1;
                        n -= half + 1;
                    } else {
                        n = half;
                    }
                }
                s1 = lo;
                ptotal = segs[s1 - 1].z + segs[s1 - 1].y - zbase;
            }
            if (threadIdx.x == 0 && ptotal > 0) {
                const uint32_t b = smem_u32(&bar);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                             "r"((uint32_t)ptotal * 16u)
                             : "memory");
                for (int q = s0; q < s1; ++q) {
                    const int4 sg = segs[q];
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                        "[%3];" ::"r"(smem_u32(cand + (sg.z - zbase))),
                        "l"(a.pts + sg.x), "r"((uint32_t)sg.y * 16u), "r"(b)
                        : "memory");
                }
            }
            if (ptotal > 0) {
                const bool ok = mbar_wait_bounded(smem_u32(&bar), parity);
                // the whole block leaves together if any thread's wait gave up
                if (__syncthreads_or(ok ? 0 : 1)) {
                    if (threadIdx.x == 0) atomicOr(a.err, 2);
                    mbar_wait_bounded(smem_u32(&bar), parity);  // give in-flight copies a last chance to land
                    failed = true;
                    break;
                }
                parity ^= 1u;
            }
            for (int p = pbeg + grp; p < pend; p += kG)
                one_primary<L, true>(a, sh, cand, segs + s0, s1 - s0, zbase, ptotal, tpref, tdc, tstart, tcode,
                                     trim, ulist, ushell, slist, part, p, cat, pass > 0, grp, warp, lane,
                                     slot_org);
            __syncthreads();   // both groups are done with this pass's staged points
            s0 = s1;
        }
        if (failed) break;
    }
}

template <int L>
void launch_L(const PairArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = pair_dynamic_smem(a);
    cudaFuncSetAttribute(k_pair<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair<L><<<nblocks, kG * kW * 32, smem, s>>>(a);
}

}  // namespace

template <int L>
size_t static_L() {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_pair<L>) != cudaSuccess) return 16 * 1024;
    return fa.sharedSizeBytes;
}

size_t pair_static_smem(int lmax) {
    switch (lmax) {
        case 0: return static_L<0>();
        case 1: return static_L<1>();
        case 2: return static_L<2>();
        case 3: return static_L<3>();
        case 4: return static_L<4>();
        case 5: return static_L<5>();
        case 6: return static_L<6>();
        case 7: return static_L<7>();
        case 8: return static_L<8>();
        case 9: return static_L<9>();
        case 10: return static_L<10>();
        default: return 16 * 1024;
    }
}

size_t pair_dynamic_smem(const PairArgs& a) {
    return pair_layout(a.cand_cap, a.nrows, a.cap, a.nr, ncomp(a.lmax)).total;
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
