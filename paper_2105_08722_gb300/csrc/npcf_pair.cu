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
// A persistent block of kPairWarps independent warps takes work units, runs of
// x-adjacent cells of one catalog's grid, from a device counter. For a unit, warp 0 lists
// the neighbour rows (rows of cells within r_max of the run) and one thread stages their
// points into shared memory with bulk asynchronous copies, in passes of rows that fit the
// buffer. Each warp then takes the unit's primaries one at a time from a shared counter
// and runs the whole primary alone, so no warp waits for another between the phases of a
// primary (the scan of one warp overlaps the accumulation of another):
//   cut: every staged row is cut to the primary's x-window and the kept rows form one
//        flat index space;
//   scan: each lane tests four candidates a step with the exact FP32 neighbour/shell
//        rule; accepted pairs go straight to per-shell buckets (a private region of
//        global scratch per warp, sized by shell volume and resident in L2) as
//        (staged index, periodic shift code);
//   accumulate: a full bucket, and at the end every non-empty one, is summed into the
//        S_{m,k} of its shell in registers and reduced across lanes with a shuffle
//        transpose-reduction; the per-shell sums are converted to a_lm (added to the
//        earlier passes' a_lm, if any).
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

constexpr int kShiftCodes = 64;   // 2 bits per axis
constexpr int kKC = 4;            // candidates per lane per scan step (independent chains)
constexpr int kShellTab = kPairShellTab;

// Byte offsets of the pair kernel's dynamic shared memory (host and device agree).
struct PairLayout {
    size_t cand, segs, rows, tpref, tdc, psum, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline PairLayout pair_layout(int cand_cap, int nrows, int nr, int nc) {
    PairLayout l;
    l.cand = 0;
    l.segs = align16(l.cand + (size_t)cand_cap * 16);
    l.rows = align16(l.segs + (size_t)2 * nrows * 16);
    // per warp: flat-index prefix and (staging offset minus prefix, shift code) of each
    // kept row of the current primary, then the primary's per-shell sums
    l.tpref = align16(l.rows + (size_t)nrows * 16);
    l.tdc = align16(l.tpref + (size_t)kPairWarps * (2 * nrows + 1) * 4);
    l.psum = align16(l.tdc + (size_t)kPairWarps * 2 * nrows * 4);
    l.total = align16(l.psum + (size_t)kPairWarps * nr * nc * 4);
    return l;
}

template <int L>
struct PairShared {
    float4 shift[kShiftCodes];       // (sx, sy, sz) of each periodic shift code
    int4 stab[kShellTab];            // shell of r2 by bins of r2 (valid when the table is on)
    float kmat[nlmc(L) * (L + 1)];
    float e2[kMaxNr + 1];
    int boff[kMaxNr + 1];            // bucket of shell t: entries [boff[t], boff[t+1]) of a warp's region
    int2 ne[kPairWarps][kMaxNr + 1]; // per warp and shell: next free entry, end of the bucket;
                                     // slot kMaxNr takes rejected candidates and never fills
    uint32_t tot[kPairWarps][kMaxNr];// accepted pairs of the warp's current primary, per shell
    int unit[4];
    int next;                        // next primary of the current pass (dynamic over warps)
};

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

// The exact FP32 neighbour rule (same operations as shell_of in npcf_rules.cuh), its
// shell read from a table over bins of r2: bin i = [i, i + 1) / scale with scale a power
// of two, so i = floor(r2 scale) is exact; the host has checked that no bin holds more
// than one point where the rule's shell changes (r2 > 0, the edges e2[b]), and entry i
// gives the shell below and above that point. -1 for a rejected pair.
__device__ __forceinline__ int pair_shell_tab(const float4 pj, const float4 pi, float sx, float sy, float sz,
                                              const int4* tab, float scale, int nbin) {
    const float dx = __fsub_rn(__fsub_rn(pj.x, pi.x), sx);
    const float dy = __fsub_rn(__fsub_rn(pj.y, pi.y), sy);
    const float dz = __fsub_rn(__fsub_rn(pj.z, pi.z), sz);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const int i = min(__float2int_rz(__fmul_rn(r2, scale)), nbin - 1);   // NaN gives 0
    const int4 e = tab[i];
    return r2 >= __int_as_float(e.z) ? e.y : e.x;
}

// The part of every staged row this primary can reach, as one flat index space over the
// rows left non-empty (one warp): row s covers flat [tpref[s], tpref[s+1]), its staged
// index is flat + (tdc[s] >> 6) and its periodic shift code tdc[s] & 63. With trim, a row
// keeps only the points whose x lies within sqrt(r_max^2 - d_yz^2) (plus a margin) of the
// primary, d_yz the distance from the primary to the row's (y, z) cell square; the exact
// FP32 rule is applied to what remains. Rows are sorted by x (cells in x order, members
// sorted by x). Returns the flat total; *nrow = rows kept.
template <int L>
__device__ __forceinline__ int cut_rows(const PairArgs& a, const PairShared<L>& sh, const float4* cand,
                                        const int4* segs, int nseg, int zbase, const float4 pi, int* tpref,
                                        int* tdc, bool trim, int lane, int* nrow) {
    const float R2 = sh.e2[a.nr], m = a.trim_margin, c = a.cell;
    int rows_acc = 0, pts_acc = 0;
    for (int k0 = 0; k0 < nseg; k0 += 32) {
        const int s = k0 + lane;
        int lo = 0, hi = 0, start = 0, code = 0;
        if (s < nseg) {
            const int4 sg = segs[s];
            hi = sg.y;
            code = sg.w & 63;
            if (trim) {
                const float4 sf = sh.shift[code];
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
            start = sg.z - zbase + lo;
        }
        const int cnt = hi - lo;
        // inclusive prefix of (kept rows << 16 | points): points <= staging capacity < 2^16
        const int v = ((cnt > 0 ? 1 : 0) << 16) | cnt;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int ex = incl - v;
        if (cnt > 0) {
            const int rb = rows_acc + (ex >> 16), pb = pts_acc + (ex & 0xffff);
            tpref[rb] = pb;
            tdc[rb] = ((start - pb) << 6) | code;   // staged start >= flat start
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        rows_acc += tot >> 16;
        pts_acc += tot & 0xffff;
    }
    if (lane == 0) tpref[rows_acc] = pts_acc;
    __syncwarp();
    *nrow = rows_acc;
    return pts_acc;
}

// n accepted pairs of one shell into that shell's sums pw[0 .. ncomp(L)) (one warp; all
// lanes call it together): the lanes take consecutive entries and accumulate
// S_{m,k} = sum w (x + i y)^m T_k(z) in registers (T_k Chebyshev, m + k <= lmax); a
// shuffle transpose-reduction adds the lanes' sums to pw. Staged entries hold (staged
// index | shift code << 16): the separation is the one the neighbour rule accepted,
// (p_j - p_i) - shift. Global entries hold the point index; the periodic image is then the
// minimum image (accepted pairs are closer than L/3). Not inlined: a scan calls it only
// when a bucket fills, and once per non-empty shell at the end of a primary.
template <int L, bool STAGED>
__device__ __noinline__ void sum_bucket(const float4* cand, const float4* pts, const float4* shift,
                                        const uint32_t* e, int n, float4 pi, float boxL, float* pw, int lane) {
    constexpr int NC = ncomp(L);
    using R = TR<NC>;
    float acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.f;
    const float invL = boxL > 0.f ? 1.f / boxL : 0.f;
    uint32_t cur = lane < n ? __ldcg(e + lane) : 0u;
    for (int i = lane; i - lane < n; i += 32) {
        const uint32_t nxt = i + 32 < n ? __ldcg(e + i + 32) : 0u;
        if (i < n) {
            float dx, dy, dz, wj;
            if (STAGED) {
                const float4 pj = cand[cur & 0xffffu];
                const float4 sf = shift[cur >> 16];
                dx = (pj.x - pi.x) - sf.x;
                dy = (pj.y - pi.y) - sf.y;
                dz = (pj.z - pi.z) - sf.z;
                wj = pj.w;
            } else {
                const float4 pj = pts[cur];
                dx = pj.x - pi.x;
                dy = pj.y - pi.y;
                dz = pj.z - pi.z;
                wj = pj.w;
                dx = fmaf(-boxL, rintf(dx * invL), dx);
                dy = fmaf(-boxL, rintf(dy * invL), dy);
                dz = fmaf(-boxL, rintf(dz * invL), dz);
            }
            const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            harm_accumulate<L>(acc, dx * inv, dy * inv, dz * inv, wj);
        }
        cur = nxt;
    }
    R::run(acc, lane);
#pragma unroll
    for (int i = 0; i < R::F; ++i) {
        const int o = R::origin(i, lane);
        if (o >= 0) pw[o] += acc[i];
    }
    __syncwarp();
}

// Shell t's bucket of the warp into the shell's sums; the bucket is then empty.
template <int L, bool STAGED>
__device__ __forceinline__ void flush_shell(const PairArgs& a, PairShared<L>& sh, const float4* cand,
                                            const uint32_t* bucket, float* psum, int t, float4 pi, int warp,
                                            int lane) {
    __syncwarp();   // the entries written by every lane are visible
    const int b0 = sh.boff[t];
    const int n = sh.ne[warp][t].x - b0;
    sum_bucket<L, STAGED>(cand, a.pts, sh.shift, bucket + b0, n, pi, a.g.periodic ? a.g.L : 0.f,
                          psum + t * ncomp(L), lane);
    if (lane == 0) {
        sh.tot[warp][t] += (uint32_t)n;
        sh.ne[warp][t].x = b0;
    }
    __syncwarp();
}

// Append one accepted pair per lane (shell b, -1 for none) to the warp's per-shell
// buckets; a bucket that cannot take its lanes' entries is summed and emptied first.
template <int L, bool STAGED>
__device__ __forceinline__ void bucket_insert(const PairArgs& a, PairShared<L>& sh, const float4* cand,
                                              uint32_t* bucket, float* psum, int b, uint32_t entry, float4 pi,
                                              int warp, int lane, unsigned lt) {
    const unsigned gm = __match_any_sync(kFull, b);
    const int rank = __popc(gm & lt);
    const int bi = b < 0 ? kMaxNr : b;
    int2 ne = sh.ne[warp][bi];
    if (__any_sync(kFull, ne.x + rank >= ne.y)) {   // rare: some lane's bucket is full
        const unsigned fullm = __reduce_or_sync(kFull, ne.x + rank >= ne.y ? 1u << bi : 0u);
        for (unsigned mm = fullm; mm; mm &= mm - 1)
            flush_shell<L, STAGED>(a, sh, cand, bucket, psum, __ffs(mm) - 1, pi, warp, lane);
        ne = sh.ne[warp][bi];
    }
    if (b >= 0) bucket[ne.x + rank] = entry;
    __syncwarp();
    if (b >= 0 && rank == 0) sh.ne[warp][bi].x = ne.x + __popc(gm);
    __syncwarp();
}

// One primary, processed by one warp (no other warp waits for it). Staged: the rows of
// the staging pass are cut to the primary's x-window and form one flat index space that
// the lanes scan kKC candidates at a time with the exact FP32 neighbour rule; global: the
// rows are read from global memory, 32 candidates a step. Accepted pairs go straight to
// per-shell buckets (a private region of global scratch, L2-resident); a full bucket and,
// at the end, every non-empty one are summed into the per-shell sums, which give a_lm
// (added to the a_lm of earlier staging passes when add is set).
template <int L, bool STAGED>
__device__ void one_primary(const PairArgs& a, PairShared<L>& sh, const float4* cand, const int4* segs,
                            int nseg, int zbase, int* tpref, int* tdc, float* psum, uint32_t* bucket, bool trim,
                            int p, int cat, bool add, int warp, int lane) {
    constexpr int NC = ncomp(L);
    constexpr int NLM = nlmc(L);
    const int nr = a.nr;
    float2* out = a.alm + (size_t)p * nr * NLM;
    // A primary of weight 0 adds nothing to zeta, but its neighbours are still counted
    // (every primary's pairs enter the counts) unless separate primary weights select a
    // sample of primaries: then a weight of 0 means "not in the sample".
    if (a.skip_zero && a.wp[p] == 0.f) {
        if (!add) {
            for (int i = lane; i < nr * NLM; i += 32) out[i] = make_float2(0.f, 0.f);
            if (lane < nr) a.cnt[(size_t)p * nr + lane] = 0u;
        }
        return;
    }
    const float4 pi = a.pts[p];
    for (int i = lane; i < nr * NC; i += 32) psum[i] = 0.f;
    if (lane < nr) {
        sh.ne[warp][lane] = make_int2(sh.boff[lane], sh.boff[lane + 1]);
        sh.tot[warp][lane] = 0u;
    }
    __syncwarp();
    const float e2lo = sh.e2[0], e2hi = sh.e2[nr];
    const bool tab = a.tab_ok != 0;
    const unsigned lt = (1u << lane) - 1u;
    if (STAGED) {
        int nrow = 0;
        const int T = cut_rows<L>(a, sh, cand, segs, nseg, zbase, pi, tpref, tdc, trim, lane, &nrow);
        int cursor = 0, srow = 0;
        while (cursor < T) {
            // Rows of the step's flat indices cursor + o, o < 32 kKC, without per-lane
            // searches: lane i loads the end of row srow + i (rows are non-empty, so the
            // ends increase strictly); a bitmap of the ends' offsets in the step gives each
            // offset's row as srow + the ends at or below it. The step stops at the last
            // loaded end, so no row beyond the loaded ones is met.
            const int d = tpref[min(srow + 1 + lane, nrow)] - cursor;   // >= 1
            const int lim = min(min(32 * kKC, T - cursor), __shfl_sync(kFull, d, 31));
            unsigned W[kKC];
#pragma unroll
            for (int j = 0; j < kKC; ++j) {
                const unsigned o = (unsigned)(d - 32 * j);
                W[j] = __reduce_or_sync(kFull, o < 32u ? 1u << o : 0u);
            }
            const unsigned le = 0xffffffffu >> (31 - lane);   // offsets 32 j .. 32 j + lane
            int q[kKC], b[kKC], code[kKC];
            float4 sf[kKC];
            int below = 0;
#pragma unroll
            for (int j = 0; j < kKC; ++j) {
                const int row = min(srow + below + __popc(W[j] & le), nrow - 1);
                below += __popc(W[j]);
                const int dc = tdc[row];
                q[j] = 32 * j + lane < lim ? cursor + 32 * j + lane + (dc >> 6) : 0;
                code[j] = dc & 63;
                sf[j] = sh.shift[code[j]];
            }
            float4 c[kKC];
#pragma unroll
            for (int j = 0; j < kKC; ++j) c[j] = cand[q[j]];
            if (tab) {
#pragma unroll
                for (int j = 0; j < kKC; ++j) {
                    const int r = pair_shell_tab(c[j], pi, sf[j].x, sf[j].y, sf[j].z, sh.stab, a.tab_scale,
                                                 a.tab_n);
                    b[j] = (32 * j + lane < lim) ? r : -1;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kKC; ++j) {
                    const int r = pair_shell_fast(c[j], pi, sf[j].x, sf[j].y, sf[j].z, sh.e2, nr, e2lo, e2hi,
                                                  a.linear, a.lin_r0, a.lin_inv_w);
                    b[j] = (32 * j + lane < lim) ? r : -1;
                }
            }
            srow += __popc(__ballot_sync(kFull, d <= lim));   // the row of cursor + lim
            cursor += lim;
#pragma unroll
            for (int j = 0; j < kKC; ++j)
                bucket_insert<L, true>(a, sh, cand, bucket, psum, b[j], (uint32_t)q[j] | ((uint32_t)code[j] << 16),
                                       pi, warp, lane, lt);
        }
    } else {
        for (int s = 0; s < nseg; ++s) {
            const int4 sg = segs[s];
            const float4 sf = sh.shift[sg.w & 63];
            for (int k0 = 0; k0 < sg.y; k0 += 32) {
                const int k = k0 + lane;
                int b = -1;
                if (k < sg.y)
                    b = tab ? pair_shell_tab(a.pts[sg.x + k], pi, sf.x, sf.y, sf.z, sh.stab, a.tab_scale, a.tab_n)
                            : pair_shell_fast(a.pts[sg.x + k], pi, sf.x, sf.y, sf.z, sh.e2, nr, e2lo, e2hi,
                                              a.linear, a.lin_r0, a.lin_inv_w);
                bucket_insert<L, false>(a, sh, cand, bucket, psum, b, (uint32_t)(sg.x + k), pi, warp, lane, lt);
            }
        }
    }
    for (int t = 0; t < nr; ++t)
        if (sh.ne[warp][t].x > sh.boff[t]) flush_shell<L, STAGED>(a, sh, cand, bucket, psum, t, pi, warp, lane);
    __syncwarp();

    // ---- per-shell sums to a_lm
    for (int i = lane; i < nr * NLM; i += 32) {
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
    if (lane < nr) {
        const uint32_t c = sh.tot[warp][lane];
        a.cnt[(size_t)p * nr + lane] = add ? a.cnt[(size_t)p * nr + lane] + c : c;
        if (c) atomicAdd(&a.counts[(size_t)cat * nr + lane], (unsigned long long)c);
    }
    __syncwarp();   // psum, ne and tot are reset by the next primary
}

template <int L>
__global__ void __launch_bounds__(kPairWarps * 32, 1) k_pair(const PairArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const PairLayout lay = pair_layout(a.cand_cap, a.nrows, a.nr, ncomp(L));
    float4* cand = reinterpret_cast<float4*>(dsm + lay.cand);
    int4* segs = reinterpret_cast<int4*>(dsm + lay.segs);
    int4* rows = reinterpret_cast<int4*>(dsm + lay.rows);
    __shared__ PairShared<L> sh;
    __shared__ __align__(8) uint64_t bar;

    const GridInfo& g = a.g;
    for (int i = threadIdx.x; i < a.nrows; i += blockDim.x) rows[i] = a.rows[i];
    for (int i = threadIdx.x; i < nlmc(L) * (L + 1); i += blockDim.x) sh.kmat[i] = a.kmat[i];
    if (threadIdx.x <= a.nr) {
        sh.e2[threadIdx.x] = a.e2[threadIdx.x];
        sh.boff[threadIdx.x] = a.boff[threadIdx.x];
    }
    if (a.tab_ok)
        for (int i = threadIdx.x; i < a.tab_n; i += blockDim.x) sh.stab[i] = a.tab[i];
    if (threadIdx.x < kPairWarps) sh.ne[threadIdx.x][kMaxNr] = make_int2(0, 0x7fffffff);
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

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tpref = reinterpret_cast<int*>(dsm + lay.tpref) + (size_t)warp * (2 * a.nrows + 1);
    int* tdc = reinterpret_cast<int*>(dsm + lay.tdc) + (size_t)warp * 2 * a.nrows;
    float* psum = reinterpret_cast<float*>(dsm + lay.psum) + (size_t)warp * a.nr * ncomp(L);
    uint32_t* bucket = a.bucket + ((size_t)blockIdx.x * kPairWarps + warp) * a.boff[a.nr];
    // the x-window cut needs every cell sorted by x (binning flags bit 8 otherwise)
    const bool trim = a.trim != 0 && (*(volatile int*)a.err & 8) == 0;
    uint32_t parity = 0;
    const int upr = (g.gx + a.run - 1) / a.run;   // units per row of cells
    const int ucat = upr * g.gy * g.gz;           // units per catalog
    const int nunits = ucat * a.ncat;

    for (;;) {
        if (threadIdx.x == 0) {
            sh.unit[0] = atomicAdd(a.work, 1);
            sh.next = 0;
        }
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
        if (warp == 0)
            build_segments(a, rows, cbase, cx, cy, cz, run, segs, &sh.unit[1], &sh.unit[2], &sh.unit[3], lane);
        __syncthreads();
        const int nseg = sh.unit[1];
        if (sh.unit[3] > a.cand_cap) {
            // a row longer than the staging buffer: neighbours straight from global memory
            for (;;) {
                int p = 0;
                if (lane == 0) p = pbeg + atomicAdd(&sh.next, 1);
                p = __shfl_sync(kFull, p, 0);
                if (p >= pend) break;
                one_primary<L, false>(a, sh, cand, segs, nseg, 0, tpref, tdc, psum, bucket, trim, p, cat, false,
                                      warp, lane);
            }
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
            for (;;) {
                int p = 0;
                if (lane == 0) p = pbeg + atomicAdd(&sh.next, 1);
                p = __shfl_sync(kFull, p, 0);
                if (p >= pend) break;
                one_primary<L, true>(a, sh, cand, segs + s0, s1 - s0, zbase, tpref, tdc, psum, bucket, trim, p,
                                     cat, pass > 0, warp, lane);
            }
            __syncthreads();   // every warp is done with this pass's staged points
            if (threadIdx.x == 0) sh.next = 0;
            __syncthreads();
            s0 = s1;
        }
        if (failed) break;
    }
}

template <int L>
void launch_L(const PairArgs& a, int nblocks, cudaStream_t s) {
    const size_t smem = pair_dynamic_smem(a);
    cudaFuncSetAttribute(k_pair<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair<L><<<nblocks, kPairWarps * 32, smem, s>>>(a);
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
    return pair_layout(a.cand_cap, a.nrows, a.nr, ncomp(a.lmax)).total;
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
