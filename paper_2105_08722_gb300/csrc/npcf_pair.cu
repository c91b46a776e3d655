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
// A persistent block of kPairWarps independent warps per SM takes chunks of consecutive
// primaries (cell-sorted, so spatially close) from a global counter; each warp takes one
// primary at a time from its block's chunks and runs it alone, so no warp waits for
// another (the scan of one warp overlaps the accumulation of another, and there is no
// barrier at which a block idles):
//   cut: the primary's neighbour rows (cells within r_max, read as runs of the cell-sorted
//        points) are cut to its x-window and form one flat index space;
//   scan: each lane tests eight candidates a step with the exact FP32 neighbour/shell
//        rule, reading them through L1 (the neighbourhoods of a block's primaries
//        overlap); accepted pairs go straight to per-shell buckets (a private region of
//        global scratch per warp, sized by shell volume and resident in L2) as (point
//        index, periodic shift code);
//   accumulate: a full bucket, and at the end every non-empty one, is summed into the
//        S_{m,k} of its shell in registers and reduced across lanes with a shuffle
//        transpose-reduction; the per-shell sums are converted to a_lm.
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

// Two pairs at once (same sums): the two recurrences are independent chains, so their
// instructions interleave and hide each other's latency.
template <int L>
__device__ __forceinline__ void harm_accumulate2(float (&acc)[ncomp(L)], float xa, float ya, float za, float wa,
                                                 float xb, float yb, float zb, float wb) {
    float ca[L + 1], sa[L + 1], ta[L + 1], cb[L + 1], sb[L + 1], tb[L + 1];
    ca[0] = cb[0] = 1.f;
    sa[0] = sb[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        ca[m] = fmaf(ca[m - 1], xa, -sa[m - 1] * ya);
        sa[m] = fmaf(sa[m - 1], xa, ca[m - 1] * ya);
        cb[m] = fmaf(cb[m - 1], xb, -sb[m - 1] * yb);
        sb[m] = fmaf(sb[m - 1], xb, cb[m - 1] * yb);
    }
    ta[0] = wa;
    tb[0] = wb;
    if (L >= 1) {
        ta[1] = wa * za;
        tb[1] = wb * zb;
    }
    const float za2 = za + za, zb2 = zb + zb;
#pragma unroll
    for (int k = 2; k <= L; ++k) {
        ta[k] = fmaf(za2, ta[k - 1], -ta[k - 2]);
        tb[k] = fmaf(zb2, tb[k - 1], -tb[k - 2]);
    }
#pragma unroll
    for (int k = 0; k <= L; ++k) acc[k] += ta[k] + tb[k];
#pragma unroll
    for (int m = 1; m <= L; ++m) {
#pragma unroll
        for (int k = 0; k + m <= L; ++k) {
            acc[s_index(L, m, k)] = fmaf(cb[m], tb[k], fmaf(ca[m], ta[k], acc[s_index(L, m, k)]));
            acc[s_index(L, m, k) + 1] = fmaf(sb[m], tb[k], fmaf(sa[m], ta[k], acc[s_index(L, m, k) + 1]));
        }
    }
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


constexpr int kShiftCodes = 64;   // 2 bits per axis
constexpr int kKC = kPairKC;      // candidates per lane per scan step (independent chains)
constexpr int kShellTab = kPairShellTab;
// Chunk ring of a block (tagged entries). Each warp holds at most one position whose
// chunk it has not read yet, and a position fetches at most one chunk (two ahead), so at
// most kPairWarps + 2 chunks are live at a time, whatever the chunk size: 64 slots are
// never overwritten before they are read.
constexpr int kRing = 64;
constexpr int kIdxBits = 26;      // bucket entry: point index (26 bits) | shift code << 26

// Byte offsets of the pair kernel's dynamic shared memory (host and device agree): per
// warp, the flat-index prefix of the kept rows of its current primary, each kept row's
// (first point minus flat start, shift code), and the primary's per-shell sums.
struct PairLayout {
    size_t rows, tpref, tdc, psum, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline PairLayout pair_layout(int nrows, int nr, int nc) {
    PairLayout l;
    l.rows = 0;
    l.tpref = align16(l.rows + (size_t)nrows * 16);
    l.tdc = align16(l.tpref + (size_t)kPairWarps * (2 * nrows + 1) * 4);
    l.psum = align16(l.tdc + (size_t)kPairWarps * 2 * nrows * 8);
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
    unsigned long long ring[kRing];  // chunks of this block: chunk id << 32 | first primary
    int take;                        // next position in this block's stream of primaries
};

// Both ends of the cell-sorted row pts[base, base + n) (sorted by x) that fall in
// [vlo, vhi]: the first index with x >= vlo and the first with x > vhi. The two searches
// run in lockstep without branches: the answer is built bit by bit from the highest power
// of two <= n, each bit kept if the predicate holds at the probed index.
__device__ __forceinline__ int2 x_bounds(const float4* __restrict__ pts, int base, int n, float vlo, float vhi) {
    int a = 0, b = 0;
    if (n > 0) {
        for (int step = 1 << (31 - __clz(n)); step > 0; step >>= 1) {
            const float xa = __ldg(&pts[base + min(a + step, n) - 1].x);
            const float xb = __ldg(&pts[base + min(b + step, n) - 1].x);
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

// The neighbourhood of primary pi in cell (cx, cy, cz) of catalog grid cbase, as one flat
// index space over the non-empty parts of its neighbour rows (one warp; lane r takes rows
// r, r + 32, ...). A neighbour row (cells within r_max of the primary's cell, same y and z)
// is one or two runs of the cell-sorted points (two where the periodic grid wraps in x);
// with trim, a run keeps only the points whose x lies within sqrt(r_max^2 - d_yz^2) (plus
// a margin) of the primary, d_yz the distance from the primary to the row's (y, z) cell
// square (runs are sorted by x: cells in x order, members sorted by x); the exact FP32
// rule is applied to what remains. Kept run s covers flat [tpref[s], tpref[s+1]); its
// points are pts[flat + tdc[s].x] and its periodic shift code is tdc[s].y. Returns the flat
// total; *nrow = runs kept.
template <int L>
__device__ __forceinline__ int cut_rows(const PairArgs& a, const PairShared<L>& sh, const int4* rows, int cbase,
                                        int cx, int cy, int cz, const float4 pi, int* tpref, int2* tdc, bool trim,
                                        int lane, int* nrow) {
    const GridInfo& g = a.g;
    const float R2 = sh.e2[a.nr], m = a.trim_margin, c = a.cell;
    int rows_acc = 0, pts_acc = 0;
    for (int k0 = 0; k0 < a.nrows; k0 += 32) {
        const int r = k0 + lane;
        int beg[2] = {0, 0}, cnt[2] = {0, 0}, code[2] = {0, 0};
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
                int x0 = cx + rw.z, x1 = cx + rw.w, ns = 0;
                if (g.periodic) {
                    if (x0 < 0) {
                        beg[ns] = (int)__ldg(&a.cell_start[base + x0 + g.gx]);
                        cnt[ns] = (int)__ldg(&a.cell_start[base + g.gx]) - beg[ns];
                        code[ns++] = cyz | 1;
                        x0 = 0;
                    }
                    if (x1 >= g.gx) {
                        beg[ns] = (int)__ldg(&a.cell_start[base]);
                        cnt[ns] = (int)__ldg(&a.cell_start[base + x1 - g.gx + 1]) - beg[ns];
                        code[ns++] = cyz | 2;
                        x1 = g.gx - 1;
                    }
                } else {
                    x0 = x0 < 0 ? 0 : x0;
                    x1 = x1 >= g.gx ? g.gx - 1 : x1;
                }
                if (x0 <= x1 && ns < 2) {
                    beg[ns] = (int)__ldg(&a.cell_start[base + x0]);
                    cnt[ns] = (int)__ldg(&a.cell_start[base + x1 + 1]) - beg[ns];
                    code[ns++] = cyz;
                }
                if (trim) {
                    // the row's (y, z) cell square, and the primary's distance to it
                    const float4 sf = sh.shift[cyz];
                    const float ylo = g.oy + (float)yy * c - sf.y - m, yhi = ylo + c + 2.f * m;
                    const float zlo = g.oz + (float)zz * c - sf.z - m, zhi = zlo + c + 2.f * m;
                    const float dy = fmaxf(0.f, fmaxf(ylo - pi.y, pi.y - yhi));
                    const float dz = fmaxf(0.f, fmaxf(zlo - pi.z, pi.z - zhi));
                    const float d2 = dy * dy + dz * dz;
                    if (d2 >= R2 * (1.f + 1e-5f)) {
                        cnt[0] = cnt[1] = 0;
                    } else {
                        const float h = sqrtf(fmaxf(R2 * (1.f + 1e-5f) - d2, 0.f)) + m;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            if (cnt[q] > 0) {
                                const float xc = pi.x + sh.shift[code[q]].x;
                                const int2 ab = x_bounds(a.pts, beg[q], cnt[q], xc - h, xc + h);
                                beg[q] += ab.x;
                                cnt[q] = ab.y - ab.x;
                            }
                        }
                    }
                }
            }
        }
        // inclusive prefixes of kept runs and of their points over the lanes
        int kr = (cnt[0] > 0) + (cnt[1] > 0), kp = cnt[0] + cnt[1];
        int ir = kr, ip = kp;
        for (int o = 1; o < 32; o <<= 1) {
            const int yr = __shfl_up_sync(kFull, ir, o), yp = __shfl_up_sync(kFull, ip, o);
            if (lane >= o) {
                ir += yr;
                ip += yp;
            }
        }
        int rb = rows_acc + ir - kr, pb = pts_acc + ip - kp;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (cnt[q] > 0) {
                tpref[rb] = pb;
                tdc[rb] = make_int2(beg[q] - pb, code[q]);
                ++rb;
                pb += cnt[q];
            }
        rows_acc += __shfl_sync(kFull, ir, 31);
        pts_acc += __shfl_sync(kFull, ip, 31);
    }
    if (lane == 0) tpref[rows_acc] = pts_acc;
    __syncwarp();
    *nrow = rows_acc;
    return pts_acc;
}

// n accepted pairs of one shell into that shell's sums pw[0 .. ncomp(L)) (one warp; all
// lanes call it together): the lanes take consecutive entries and accumulate
// S_{m,k} = sum w (x + i y)^m T_k(z) in registers (T_k Chebyshev, m + k <= lmax); a
// shuffle transpose-reduction adds the lanes' sums to pw. An entry holds (point index |
// shift code << 26): the separation is the one the neighbour rule accepted,
// (p_j - p_i) - shift. Called once per non-empty shell at the end of a primary, and
// during a scan only when a bucket fills; inlined for lmax 4 to 8 (fewer spills and no call
// frame, measured 2 % faster at lmax 5), called for the other lmax (sum_bucket_call).
template <int L>
__device__ __forceinline__ void sum_bucket(const float4* __restrict__ pts, const float4* shift, const uint32_t* e,
                                           int n, float4 pi, float* pw, int lane) {
    constexpr int NC = ncomp(L);
    using R = TR<NC>;
    float acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.f;
    auto sep = [&](uint32_t c, float& x, float& y, float& z, float& w) {
        const float4 pj = __ldg(&pts[c & ((1u << kIdxBits) - 1u)]);
        const float4 sf = shift[c >> kIdxBits];
        const float dx = (pj.x - pi.x) - sf.x;
        const float dy = (pj.y - pi.y) - sf.y;
        const float dz = (pj.z - pi.z) - sf.z;
        w = pj.w;
        const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        x = dx * inv;
        y = dy * inv;
        z = dz * inv;
    };
    // Lane takes entries i and i + 32 of each block of 64, two pairs at once; the entries
    // of the next block are in flight meanwhile (L2 latency).
    uint32_t a0 = lane < n ? __ldcg(e + lane) : 0u, b0 = lane + 32 < n ? __ldcg(e + lane + 32) : 0u;
    uint32_t a1 = lane + 64 < n ? __ldcg(e + lane + 64) : 0u, b1 = lane + 96 < n ? __ldcg(e + lane + 96) : 0u;
    for (int i = lane; i - lane < n; i += 64) {
        const uint32_t ca = a0, cb = b0;
        a0 = a1;
        b0 = b1;
        a1 = i + 128 < n ? __ldcg(e + i + 128) : 0u;
        b1 = i + 160 < n ? __ldcg(e + i + 160) : 0u;
        if (i + 32 < n) {
            float xa, ya, za, wa, xb, yb, zb, wb;
            sep(ca, xa, ya, za, wa);
            sep(cb, xb, yb, zb, wb);
            harm_accumulate2<L>(acc, xa, ya, za, wa, xb, yb, zb, wb);
        } else if (i < n) {
            float xa, ya, za, wa;
            sep(ca, xa, ya, za, wa);
            harm_accumulate<L>(acc, xa, ya, za, wa);
        }
    }
    R::run(acc, lane);
#pragma unroll
    for (int i = 0; i < R::F; ++i) {
        const int o = R::origin(i, lane);
        if (o >= 0) pw[o] += acc[i];
    }
    __syncwarp();
}

template <int L>
__device__ __noinline__ void sum_bucket_call(const float4* __restrict__ pts, const float4* shift, const uint32_t* e,
                                             int n, float4 pi, float* pw, int lane) {
    sum_bucket<L>(pts, shift, e, n, pi, pw, lane);
}

// Shell t's bucket of the warp into the shell's sums; the bucket is then empty.
template <int L>
__device__ __forceinline__ void flush_shell(const PairArgs& a, PairShared<L>& sh, const uint32_t* bucket,
                                            float* psum, int t, float4 pi, int warp, int lane) {
    __syncwarp();   // the entries written by every lane are visible
    const int b0 = sh.boff[t];
    const int n = sh.ne[warp][t].x - b0;
    if constexpr (L >= 4 && L <= 8)
        sum_bucket<L>(a.pts, sh.shift, bucket + b0, n, pi, psum + t * ncomp(L), lane);
    else
        sum_bucket_call<L>(a.pts, sh.shift, bucket + b0, n, pi, psum + t * ncomp(L), lane);
    if (lane == 0) {
        sh.tot[warp][t] += (uint32_t)n;
        sh.ne[warp][t].x = b0;
    }
    __syncwarp();
}

// Append one accepted pair per lane (shell b, -1 for none) to the warp's per-shell
// buckets. The caller has made room: every bucket takes at least a scan step's entries.
template <int L>
__device__ __forceinline__ void bucket_insert(PairShared<L>& sh, uint32_t* bucket, int b, uint32_t entry, int warp,
                                              unsigned lt) {
    const unsigned gm = __match_any_sync(kFull, b);
    const int rank = __popc(gm & lt);
    const int bi = b < 0 ? kMaxNr : b;
    const int nx = sh.ne[warp][bi].x;
    if (b >= 0) __stcg(bucket + nx + rank, entry);
    __syncwarp();
    if (b >= 0 && rank == 0) sh.ne[warp][bi].x = nx + __popc(gm);
    __syncwarp();
}

// One primary, processed by one warp (no other warp waits for it): its neighbour rows cut
// to its x-window form one flat index space that the lanes scan kKC candidates at a time
// with the exact FP32 neighbour rule (candidates read through L1: the block's warps work
// on nearby primaries, whose neighbourhoods overlap); accepted pairs go straight to
// per-shell buckets (a private region of global scratch, L2-resident); a full bucket and,
// at the end, every non-empty one are summed into the per-shell sums, which give a_lm.
template <int L>
__device__ void one_primary(const PairArgs& a, PairShared<L>& sh, const int4* rows, int* tpref, int2* tdc,
                            float* psum, uint32_t* bucket, bool trim, int p, int warp, int lane) {
    constexpr int NC = ncomp(L);
    constexpr int NLM = nlmc(L);
    const int nr = a.nr;
    float2* out = a.alm + (size_t)p * nr * NLM;
    // A primary of weight 0 adds nothing to zeta, but its neighbours are still counted
    // (every primary's pairs enter the counts) unless separate primary weights select a
    // sample of primaries: then a weight of 0 means "not in the sample".
    if (a.skip_zero && a.pwp[p] == 0.f) {
        if (!a.add) {
            for (int i = lane; i < nr * NLM; i += 32) out[i] = make_float2(0.f, 0.f);
            if (lane < nr) a.cnt[(size_t)p * nr + lane] = 0u;
        }
        return;
    }
    const GridInfo& g = a.g;
    const float4 pi = __ldg(&a.ppts[p]);
    const int cell = (int)__ldg(&a.pcell[p]);
    const int cat = cell / g.ncell, lc = cell - cat * g.ncell;
    const int cx = lc % g.gx, cy = (lc / g.gx) % g.gy, cz = lc / (g.gx * g.gy);
    for (int i = lane; i < nr * NC; i += 32) psum[i] = 0.f;
    if (lane < nr) {
        sh.ne[warp][lane] = make_int2(sh.boff[lane], sh.boff[lane + 1]);
        sh.tot[warp][lane] = 0u;
    }
    __syncwarp();
    const float e2lo = sh.e2[0], e2hi = sh.e2[nr];
    const bool tab = a.tab_ok != 0;
    const unsigned lt = (1u << lane) - 1u;
    int nrow = 0;
    const int T = cut_rows<L>(a, sh, rows, cat * g.ncell, cx, cy, cz, pi, tpref, tdc, trim, lane, &nrow);
    int cursor = 0, srow = 0;
    while (cursor < T) {
        // Rows of the step's flat indices cursor + o, o < 32 kKC, without per-lane
        // searches: lane i loads the end of run srow + i (runs are non-empty, so the ends
        // increase strictly); a bitmap of the ends' offsets in the step gives each offset's
        // run as srow + the ends at or below it. The step stops at the last loaded end, so
        // no run beyond the loaded ones is met.
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
            const int2 dc = tdc[row];
            q[j] = 32 * j + lane < lim ? cursor + 32 * j + lane + dc.x : 0;
            code[j] = dc.y;
            sf[j] = sh.shift[code[j]];
        }
        float4 c[kKC];
#pragma unroll
        for (int j = 0; j < kKC; ++j) c[j] = __ldg(&a.pts[q[j]]);
        if (tab) {
#pragma unroll
            for (int j = 0; j < kKC; ++j) {
                const int r = pair_shell_tab(c[j], pi, sf[j].x, sf[j].y, sf[j].z, sh.stab, a.tab_scale, a.tab_n);
                b[j] = (32 * j + lane < lim) ? r : -1;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kKC; ++j) {
                const int r = pair_shell_fast(c[j], pi, sf[j].x, sf[j].y, sf[j].z, sh.e2, nr, e2lo, e2hi, a.linear,
                                              a.lin_r0, a.lin_inv_w);
                b[j] = (32 * j + lane < lim) ? r : -1;
            }
        }
        srow += __popc(__ballot_sync(kFull, d <= lim));   // the run of cursor + lim
        cursor += lim;
        {
            // a step adds at most 32 kKC entries to a bucket: sum and empty (rarely) every
            // bucket with less room left (each holds at least kPairBucketMin = 2 x 32 kKC)
            const int2 ne = sh.ne[warp][lane < nr ? lane : kMaxNr];
            for (unsigned lowm = __ballot_sync(kFull, lane < nr && ne.y - ne.x < 32 * kKC); lowm; lowm &= lowm - 1)
                flush_shell<L>(a, sh, bucket, psum, __ffs(lowm) - 1, pi, warp, lane);
        }
#pragma unroll
        for (int j = 0; j < kKC; ++j)
            bucket_insert<L>(sh, bucket, b[j], (uint32_t)q[j] | ((uint32_t)code[j] << kIdxBits), warp, lt);
    }
    for (int t = 0; t < nr; ++t)
        if (sh.ne[warp][t].x > sh.boff[t]) flush_shell<L>(a, sh, bucket, psum, t, pi, warp, lane);
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
        if (a.add) {   // a further pass over another list of secondaries: a_lm is linear in them
            const float2 o = out[i];
            re += o.x;
            im += o.y;
        }
        __stcs(&out[i], make_float2(re, im));
    }
    if (lane < nr) {
        const uint32_t c = sh.tot[warp][lane];
        a.cnt[(size_t)p * nr + lane] = a.add ? a.cnt[(size_t)p * nr + lane] + c : c;
        if (c) atomicAdd(&a.counts[(size_t)cat * nr + lane], (unsigned long long)c);
    }
    __syncwarp();   // psum, ne and tot are reset by the next primary
}

// Bounded wait for chunk k of the block's stream (its ring entry carries the chunk id);
// returns the chunk's first primary, or -1 if the wait gave up.
__device__ __forceinline__ int chunk_base(const unsigned long long* ring, int k) {
    const volatile unsigned long long* r = ring + (k % kRing);
    for (int it = 0; it < (1 << 22); ++it) {
        const unsigned long long v = *r;
        if ((int)(v >> 32) == k) return (int)(v & 0xffffffffu);
        __nanosleep(64);
    }
    return -1;
}

// Chunk k of the block's stream: its first primary from the global counter, published
// with the chunk id.
__device__ __forceinline__ void fetch_chunk(const PairArgs& a, unsigned long long* ring, int k) {
    const int base = atomicAdd(a.work, a.chunk);
    atomicExch(ring + (k % kRing), ((unsigned long long)(unsigned)k << 32) | (unsigned)base);
}

template <int L>
__global__ void __launch_bounds__(kPairWarps * 32, 1) k_pair(const PairArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const PairLayout lay = pair_layout(a.nrows, a.nr, ncomp(L));
    int4* rows = reinterpret_cast<int4*>(dsm + lay.rows);
    __shared__ PairShared<L> sh;

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
    if (threadIdx.x < kRing) sh.ring[threadIdx.x] = ~0ull;   // no chunk yet
    if (threadIdx.x == 0) sh.take = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        fetch_chunk(a, sh.ring, 0);
        fetch_chunk(a, sh.ring, 1);
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tpref = reinterpret_cast<int*>(dsm + lay.tpref) + (size_t)warp * (2 * a.nrows + 1);
    int2* tdc = reinterpret_cast<int2*>(dsm + lay.tdc) + (size_t)warp * 2 * a.nrows;
    float* psum = reinterpret_cast<float*>(dsm + lay.psum) + (size_t)warp * a.nr * ncomp(L);
    uint32_t* bucket = a.bucket + ((size_t)blockIdx.x * kPairWarps + warp) * a.boff[a.nr];
    // the x-window cut needs every cell sorted by x (binning flags bit 8 otherwise)
    const bool trim = a.trim != 0 && (*(volatile int*)a.err & 8) == 0;

    // The block's warps take positions of the block's stream of primaries, chunks of
    // a.chunk consecutive (cell-sorted, so nearby) primaries from the global counter. The
    // warp that takes a chunk's first position fetches the chunk two ahead, so a chunk is
    // normally published long before a warp needs it.
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&sh.take, 1);
        t = __shfl_sync(kFull, t, 0);
        const int k = t / a.chunk, r = t - k * a.chunk;
        if (r == 0 && lane == 0) fetch_chunk(a, sh.ring, k + 2);
        int base = 0;
        if (lane == 0) base = chunk_base(sh.ring, k);
        base = __shfl_sync(kFull, base, 0);
        if (base < 0) {   // gave up waiting (never expected): report and stop
            if (lane == 0) atomicOr(a.err, 2);
            break;
        }
        if (base >= a.np) break;   // past the last primary: so is every later chunk
        const int p = base + r;
        if (p >= a.np) continue;
        one_primary<L>(a, sh, rows, tpref, tdc, psum, bucket, trim, p, warp, lane);
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
    return pair_layout(a.nrows, a.nr, ncomp(a.lmax)).total;
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
