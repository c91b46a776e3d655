// Cell-list construction (counting sort of particles into a Cartesian grid), the
// neighbour-search structure of the pair kernel (Sec. 5.1 / Fig. 5: particles are
// placed on a Cartesian grid before the pair search).
//
// Stages: per-point cell id + histogram -> exclusive scan -> scatter into cell order
// as float4 (x, y, z, w) -> per-cell sort by (x, input index). The order is
// deterministic, so every sum that follows it is too, and a run of x-adjacent cells is
// sorted by x as a whole, which lets the pair kernel cut each row of neighbour cells to
// the x-window of one primary by binary search.
#include "npcf_device.h"

#include <cfloat>

namespace npcf {

namespace {

__device__ __forceinline__ int cell_coord(float x, float o, float inv, int g) {
    int c = (int)floorf((x - o) * inv);
    return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__global__ void k_bbox(const float* __restrict__ pos, int n, float* __restrict__ part) {
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float v = pos[3 * i + a];
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
    __shared__ float sh[6][32];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) { sh[a][warp] = mn[a]; sh[3 + a][warp] = mx[a]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int a = threadIdx.x;
        float v = sh[a][0];
        for (int k = 1; k < nw; ++k) v = (a < 3) ? fminf(v, sh[a][k]) : fmaxf(v, sh[a][k]);
        part[blockIdx.x * 6 + a] = v;
    }
}

__global__ void k_assign(BinArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2];
    bool bad = !(x == x && y == y && z == z);
    if (a.g.periodic)
        bad |= !(x >= 0.f && x < a.g.L && y >= 0.f && y < a.g.L && z >= 0.f && z < a.g.L);
    if (bad) atomicOr(a.err, 1);
    int cx = cell_coord(x, a.g.ox, a.g.inv_cell, a.g.gx);
    int cy = cell_coord(y, a.g.oy, a.g.inv_cell, a.g.gy);
    int cz = cell_coord(z, a.g.oz, a.g.inv_cell, a.g.gz);
    // catalog of point i: last k with off[k] <= i (binary search over the batch offsets)
    int lo = 0, hi = a.ncat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.off[mid] <= (long long)i) lo = mid;
        else hi = mid - 1;
    }
    uint32_t c = (uint32_t)lo * (uint32_t)a.g.ncell + (uint32_t)((cz * a.g.gy + cy) * a.g.gx + cx);
    a.cid[i] = c;
    atomicAdd(&a.count[c], 1u);
}

// Single-block exclusive scan of the cell histogram (ncell is at most a few million).
__global__ void k_scan(const uint32_t* __restrict__ count, uint32_t* __restrict__ start,
                       uint32_t* __restrict__ cursor, int ncell) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < ncell ? count[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        uint32_t excl = carry + (warp > 0 ? warp_tot[warp - 1] : 0u) + x - v;
        if (i < ncell) { start[i] = excl; cursor[i] = excl; }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k_scatter(BinArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    uint32_t c = a.cid[i];
    uint32_t k = atomicAdd(&a.cursor[c], 1u);
    a.pts[k] = make_float4(a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2], a.w[i]);
    a.wp[k] = a.wprim ? a.wprim[i] : a.w[i];
    a.idx[k] = (uint32_t)i;
    a.cell_of[k] = c;
}

// Order each cell's members by (x, input index), one warp per cell: the members are
// loaded into shared memory and each goes to its rank among the cell's keys (the keys are
// distinct: the input index breaks ties), written back in order. Cells longer than
// kSortCap are ordered by insertion sort in place by one lane; above 4096 members they stay
// in scatter order and flag error bit 8, which turns the pair kernel's x-window cut off.
constexpr int kSortWarps = 4;
constexpr int kSortCap = 384;

__device__ __forceinline__ bool key_less(float xa, uint32_t ia, float xb, uint32_t ib) {
    return xa < xb || (xa == xb && ia < ib);
}

__global__ void __launch_bounds__(kSortWarps * 32) k_cell_order(BinArgs a) {
    __shared__ float4 sp[kSortWarps][kSortCap];
    __shared__ uint32_t si[kSortWarps][kSortCap];
    __shared__ float sw[kSortWarps][kSortCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncells = a.g.ncell * a.ncat;
    for (int c = blockIdx.x * kSortWarps + warp; c < ncells; c += gridDim.x * kSortWarps) {
        const uint32_t s0 = a.start[c], s1 = a.start[c + 1];
        const int n = (int)(s1 - s0);
        if (n <= 1) continue;
        if (n <= kSortCap) {
            for (int i = lane; i < n; i += 32) {
                sp[warp][i] = a.pts[s0 + i];
                si[warp][i] = a.idx[s0 + i];
                sw[warp][i] = a.wp[s0 + i];
            }
            __syncwarp();
            for (int i = lane; i < n; i += 32) {
                const float xi = sp[warp][i].x;
                const uint32_t ii = si[warp][i];
                int rank = 0;
                for (int j = 0; j < n; ++j) rank += key_less(sp[warp][j].x, si[warp][j], xi, ii) ? 1 : 0;
                a.pts[s0 + rank] = sp[warp][i];
                a.idx[s0 + rank] = ii;
                a.wp[s0 + rank] = sw[warp][i];
            }
            __syncwarp();
            continue;
        }
        if (lane != 0) continue;
        if (n > 4096) {  // keep the quadratic sort bounded
            atomicOr(a.err, 8);
            continue;
        }
        for (uint32_t k = s0 + 1; k < s1; ++k) {
            const uint32_t key = a.idx[k];
            const float4 p = a.pts[k];
            const float u = a.wp[k];
            uint32_t j = k;
            while (j > s0) {
                const float xj = a.pts[j - 1].x;
                if (!key_less(p.x, key, xj, a.idx[j - 1])) break;
                a.idx[j] = a.idx[j - 1];
                a.pts[j] = a.pts[j - 1];
                a.wp[j] = a.wp[j - 1];
                --j;
            }
            a.idx[j] = key;
            a.pts[j] = p;
            a.wp[j] = u;
        }
    }
}

}  // namespace

void launch_bbox(const float* pos, int n, float* part, int nblocks, cudaStream_t s) {
    k_bbox<<<nblocks, 256, 0, s>>>(pos, n, part);
}

void launch_bin(const BinArgs& a, cudaStream_t s) {
    const int nbp = (a.n + 255) / 256;
    if (a.n > 0) k_assign<<<nbp, 256, 0, s>>>(a);
    const int cells = a.g.ncell * a.ncat;
    k_scan<<<1, 1024, 0, s>>>(a.count, a.start, a.cursor, cells);
    if (a.n > 0) k_scatter<<<nbp, 256, 0, s>>>(a);
    const int nb = (cells + kSortWarps - 1) / kSortWarps;
    k_cell_order<<<nb < 4096 ? nb : 4096, kSortWarps * 32, 0, s>>>(a);
}

}  // namespace npcf
