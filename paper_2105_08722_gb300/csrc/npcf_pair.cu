// Pair kernel: for every primary i the binned harmonic coefficients
//   a^b_lm(s_i) = sum_j w_j Y_lm(unit(r_j - s_i)) Theta^b(|r_j - s_i|)
// (Eq. binned-discrete-alm without 1/v_b; Algorithm 1 lines over secondaries and
// Algorithm 2).
//
// Like Algorithm 2 the harmonics come from Cartesian powers of the unit separation
// (x, y, z), accumulated per shell and converted to a_lm afterwards. Instead of all
// (lmax+1)(lmax+2)(lmax+3)/6 monomials x^p y^q z^r, the kernel accumulates the
// (lmax+1)^2 real components of S_{m,k} = sum_j w_j (x + i y)^m z^k, m + k <= lmax,
// which span exactly the Y_lm with m >= 0: Y_lm = N_lm (-1)^m (x+iy)^m P_l^{(m)}(z).
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

// The neighbour/shell rule in IEEE FP32 round-to-nearest, never fused; (sx,sy,sz)
// is the periodic image shift of the cell row (0 or +-L), applied as d - s exactly
// as the rule's d - L / d + L.
__device__ __forceinline__ int shell_of(const float4 pj, const float4 pi, float sx, float sy,
                                        float sz, const float* e2, int nr) {
    float dx = __fsub_rn(__fsub_rn(pj.x, pi.x), sx);
    float dy = __fsub_rn(__fsub_rn(pj.y, pi.y), sy);
    float dz = __fsub_rn(__fsub_rn(pj.z, pi.z), sz);
    float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (!(r2 > 0.f) || !(r2 >= e2[0]) || !(r2 < e2[nr])) return -1;
    int b = 0;
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1)
        if (b + step < nr && r2 >= e2[b + step]) b += step;
    return b;
}

// Visit the point ranges of every neighbour cell row of cell (cx, cy, cz).
template <class F>
__device__ __forceinline__ void for_segments(const PairArgs& a, const int4* rows, int cx, int cy,
                                             int cz, F&& f) {
    const GridInfo& g = a.g;
    for (int r = 0; r < a.nrows; ++r) {
        const int4 rw = rows[r];
        int yy = cy + rw.x, zz = cz + rw.y;
        float sy = 0.f, sz = 0.f;
        if (g.periodic) {
            if (yy < 0) { yy += g.gy; sy = g.L; } else if (yy >= g.gy) { yy -= g.gy; sy = -g.L; }
            if (zz < 0) { zz += g.gz; sz = g.L; } else if (zz >= g.gz) { zz -= g.gz; sz = -g.L; }
        } else if (yy < 0 || yy >= g.gy || zz < 0 || zz >= g.gz) {
            continue;
        }
        const int base = (zz * g.gy + yy) * g.gx;
        int x0 = cx + rw.z, x1 = cx + rw.w;
        if (g.periodic) {
            if (x0 < 0) {
                f((int)a.cell_start[base + x0 + g.gx], (int)a.cell_start[base + g.gx], g.L, sy, sz);
                x0 = 0;
            }
            if (x1 >= g.gx) {
                f((int)a.cell_start[base], (int)a.cell_start[base + x1 - g.gx + 1], -g.L, sy, sz);
                x1 = g.gx - 1;
            }
        } else {
            x0 = x0 < 0 ? 0 : x0;
            x1 = x1 >= g.gx ? g.gx - 1 : x1;
        }
        if (x0 <= x1) f((int)a.cell_start[base + x0], (int)a.cell_start[base + x1 + 1], 0.f, sy, sz);
    }
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
    wz[0] = w;
#pragma unroll
    for (int k = 1; k <= L; ++k) wz[k] = wz[k - 1] * z;
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

template <int L>
__global__ void __launch_bounds__(512) k_pair(const PairArgs a) {
    constexpr int NC = ncomp(L);
    constexpr int NLM = nlmc(L);
    using R = TR<NC>;
    extern __shared__ __align__(16) unsigned char dsm[];
    int4* rows = reinterpret_cast<int4*>(dsm);
    uint32_t* ent_all = reinterpret_cast<uint32_t*>(rows + a.nrows);
    __shared__ uint32_t hist[kMaxWarps][kMaxNr];
    __shared__ uint32_t cur[kMaxWarps][kMaxNr];
    __shared__ int rlo[kMaxWarps][kMaxNr], rhi[kMaxWarps][kMaxNr], gofs[kMaxWarps][kMaxNr];
    __shared__ int gnext[kMaxWarps][4];
    __shared__ float red[kMaxWarps][NC];
    __shared__ float kmat[NLM * (L + 1)];
    __shared__ float e2[kMaxNr + 1];

    for (int i = threadIdx.x; i < a.nrows; i += blockDim.x) rows[i] = a.rows[i];
    for (int i = threadIdx.x; i < NLM * (L + 1); i += blockDim.x) kmat[i] = a.kmat[i];
    if (threadIdx.x <= a.nr) e2[threadIdx.x] = a.e2[threadIdx.x];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* ent = ent_all + (size_t)warp * a.cap;
    const int nr = a.nr;
    const GridInfo& g = a.g;

    int slot_org[R::F];
#pragma unroll
    for (int i = 0; i < R::F; ++i) slot_org[i] = R::origin(i, lane);
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(a.work, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= a.n) break;
        float2* out = a.alm + (size_t)p * nr * NLM;
        const float u = a.wp[p];
        if (u == 0.f) {  // primary not evaluated
            for (int i = lane; i < nr * NLM; i += 32) out[i] = make_float2(0.f, 0.f);
            if (lane < nr) a.cnt[(size_t)p * nr + lane] = 0u;
            continue;
        }
        const float4 pi = a.pts[p];
        const uint32_t cell = a.cell_of[p];
        const int cx = (int)(cell % (uint32_t)g.gx);
        const int cy = (int)((cell / (uint32_t)g.gx) % (uint32_t)g.gy);
        const int cz = (int)(cell / ((uint32_t)g.gx * (uint32_t)g.gy));

        // ---- pass 0: neighbour counts per shell
        if (lane < kMaxNr) hist[warp][lane] = 0u;
        __syncwarp();
        for_segments(a, rows, cx, cy, cz, [&](int j0, int j1, float sx, float sy, float sz) {
            for (int j = j0 + lane; j < j1; j += 32) {
                int b = shell_of(a.pts[j], pi, sx, sy, sz, e2, nr);
                if (b >= 0) atomicAdd(&hist[warp][b], 1u);
            }
        });
        __syncwarp();
        if (lane < nr) {
            uint32_t c = hist[warp][lane];
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
                for (int q = 0; q < kMaxNr; ++q) { rlo[warp][q] = 0; rhi[warp][q] = -1; cur[warp][q] = 0u; }
                int used = 0, t = s_next, r = r_next, last = s_next;
                while (t < nr) {
                    int avail = (int)hist[warp][t] - r;
                    int take = avail < a.cap - used ? avail : a.cap - used;
                    rlo[warp][t] = r;
                    rhi[warp][t] = r + take;
                    gofs[warp][t] = used;
                    used += take;
                    last = t;
                    if (take < avail) { r += take; break; }  // shell t continues in the next slice
                    ++t;
                    r = 0;
                    if (used >= a.cap) break;
                }
                gnext[warp][0] = used;
                gnext[warp][1] = last;
                gnext[warp][2] = t;
                gnext[warp][3] = r;
            }
            __syncwarp();
            const int g_first = s_next;
            const int used = gnext[warp][0];
            const int g_last = gnext[warp][1];
            s_next = gnext[warp][2];
            r_next = gnext[warp][3];

            // ---- pass 1: write the slice's neighbour indices in shell order
            if (used > 0) {
                for_segments(a, rows, cx, cy, cz, [&](int j0, int j1, float sx, float sy, float sz) {
                    for (int base = j0; base < j1; base += 32) {
                        const int j = base + lane;
                        int key = -1;
                        if (j < j1) {
                            int b = shell_of(a.pts[j], pi, sx, sy, sz, e2, nr);
                            if (b >= g_first && b <= g_last) key = b;
                        }
                        if (__ballot_sync(kFull, key >= 0) == 0u) continue;
                        const unsigned m = __match_any_sync(kFull, key);
                        const int leader = __ffs(m) - 1;
                        uint32_t b0 = 0u;
                        if (key >= 0 && lane == leader) b0 = atomicAdd(&cur[warp][key], (uint32_t)__popc(m));
                        b0 = __shfl_sync(kFull, b0, leader);
                        if (key >= 0) {
                            int rank = (int)b0 + __popc(m & ((1u << lane) - 1u));
                            if (rank >= rlo[warp][key] && rank < rhi[warp][key])
                                ent[gofs[warp][key] + rank - rlo[warp][key]] = (uint32_t)j;
                        }
                    }
                });
            }
            __syncwarp();

            // ---- accumulate the slice, finish the shells it completes
            for (int t = g_first; t <= g_last; ++t) {
                const int k0 = gofs[warp][t];
                const int kn = rhi[warp][t] - rlo[warp][t];
                for (int k = lane; k < kn; k += 32) {
                    const float4 pj = a.pts[ent[k0 + k]];
                    float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    if (g.periodic) {
                        dx = dx > g.hL ? dx - g.L : (dx < -g.hL ? dx + g.L : dx);
                        dy = dy > g.hL ? dy - g.L : (dy < -g.hL ? dy + g.L : dy);
                        dz = dz > g.hL ? dz - g.L : (dz < -g.hL ? dz + g.L : dz);
                    }
                    const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    harm_accumulate<L>(acc, dx * inv, dy * inv, dz * inv, pj.w);
                }
                if (rhi[warp][t] == (int)hist[warp][t]) {
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
}

template <int L>
void launch_L(const PairArgs& a, int nblocks, cudaStream_t s) {
    size_t smem = (size_t)a.nrows * sizeof(int4) + (size_t)a.warps * a.cap * sizeof(uint32_t);
    cudaFuncSetAttribute(k_pair<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair<L><<<nblocks, a.warps * 32, smem, s>>>(a);
}

}  // namespace

size_t pair_smem_bytes(int warps, int cap) {
    return (size_t)warps * cap * sizeof(uint32_t);
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
