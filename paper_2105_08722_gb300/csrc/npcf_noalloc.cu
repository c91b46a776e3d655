// Exact per-shell pair counts without any device allocation.
//
// Some callers cannot call cudaMalloc: hosts whose device memory belongs entirely to
// another allocator (a framework's caching pool that must not be bypassed, a real-time
// pipeline that forbids allocation after start-up), or plug-ins that must not change the
// process's memory footprint per call. For them npcf_pair_counts_noalloc computes the same
// neighbour counts as the context-based path (npcf_accumulate + npcf_pair_counts) but
// keeps every scratch buffer -- the cell list and the counters -- in one file-scope device
// array of fixed size; the few neighbour-row offsets travel in the kernel's arguments.
//
// That array (kScratchBytes, about 13 MiB) is held by every GPU that loads the library
// until the process exits. It bounds the catalog to kMaxPoints points and the grid to
// kMaxCells cells. All calls share the array and it keeps the last call's contents, so
// everything that must start at zero is cleared by each call, and calls that overlap on
// the GPU (different streams or threads without ordering) race on it.
#include "encore_gpu.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "npcf_device.h"
#include "npcf_rules.cuh"

namespace npcf {
void set_global_error(const char* msg);   // npcf_capi.cu: text for npcf_last_error(NULL)
}

namespace {

using namespace npcf;

constexpr int64_t kMaxPoints = 1 << 18;    // 262,144 particles
constexpr int kMaxCells = 1 << 18;         // neighbour-grid cells
constexpr int kMaxRows = 128;              // neighbour rows of the grid (4 cells per r_max: 77)
constexpr int kBBoxBlocks = 64;
constexpr int kWarps = 8;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// scratch layout: byte offsets of each region
constexpr size_t kOffPts = 0;
constexpr size_t kOffW = align256(kOffPts + 16 * kMaxPoints);
constexpr size_t kOffCid = align256(kOffW + 4 * kMaxPoints);
constexpr size_t kOffIdx = align256(kOffCid + 4 * kMaxPoints);
constexpr size_t kOffCellOf = align256(kOffIdx + 4 * kMaxPoints);
constexpr size_t kOffWp = align256(kOffCellOf + 4 * kMaxPoints);
constexpr size_t kOffCount = align256(kOffWp + 4 * kMaxPoints);
constexpr size_t kOffStart = align256(kOffCount + 4 * (size_t)kMaxCells);
constexpr size_t kOffCursor = align256(kOffStart + 4 * ((size_t)kMaxCells + 1));
constexpr size_t kOffBBox = align256(kOffCursor + 4 * (size_t)kMaxCells);
constexpr size_t kOffMisc = align256(kOffBBox + 4 * 6 * (size_t)kBBoxBlocks);
constexpr size_t kScratchBytes = align256(kOffMisc + 256);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, resolved once with that device current.
std::mutex g_mu;
void* g_addr[64] = {};

npcf_status scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return NPCF_ECUDA;
    }
    if (dev < 0 || dev >= 64) {
        set_global_error("device index outside the 64 devices the scratch table tracks");
        return NPCF_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            std::string m = std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                            cudaGetErrorString(e);
            set_global_error(m.c_str());
            return NPCF_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return NPCF_OK;
}

struct CountArgs {
    const float4* pts;
    const uint32_t* cell_of;
    const uint32_t* cell_start;
    int4 rows[kMaxRows];       // (dy, dz, dx_lo, dx_hi), by value: no host buffer to copy
    int nrows;
    GridInfo g;
    float e2[kMaxNr + 1];
    int nr;
    int n;
    int* work;
    const int* err;            // error bits of the binning (1: position outside the box or NaN)
    unsigned long long* counts;
};

__global__ void k_set_range(long long* off, long long n) {
    off[0] = 0;
    off[1] = n;
}

__global__ void k_fill_ones(float* w, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = 1.0f;
}

// Count-only variant of the pair kernel: one warp per primary, neighbour cells read from
// global memory, per-warp shared histograms flushed once per warp at the end. If the
// binning flagged a position outside the periodic box or a NaN position, no pair is
// counted and every count is set to UINT64_MAX instead (a value no count reaches).
__global__ void __launch_bounds__(kWarps * 32) k_count(const CountArgs a) {
    if (*(volatile const int*)a.err & 1) {
        if (blockIdx.x == 0 && threadIdx.x < a.nr) a.counts[threadIdx.x] = ~0ull;
        return;
    }
    __shared__ uint32_t hist[kWarps][kMaxNr];
    __shared__ float e2[kMaxNr + 1];
    if (threadIdx.x <= a.nr) e2[threadIdx.x] = a.e2[threadIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kMaxNr) hist[warp][lane] = 0u;
    __syncthreads();
    const GridInfo& g = a.g;
    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(a.work, 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= a.n) break;
        const float4 pi = a.pts[p];
        const int cell = (int)a.cell_of[p];
        const int cx = cell % g.gx, cy = (cell / g.gx) % g.gy, cz = cell / (g.gx * g.gy);
        for (int r = 0; r < a.nrows; ++r) {
            const int4 rw = a.rows[r];
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
            int segb[3], sege[3];
            float segs[3];
            int ns = 0;
            if (g.periodic) {
                if (x0 < 0) {
                    segb[ns] = (int)a.cell_start[base + x0 + g.gx];
                    sege[ns] = (int)a.cell_start[base + g.gx];
                    segs[ns++] = g.L;
                    x0 = 0;
                }
                if (x1 >= g.gx) {
                    segb[ns] = (int)a.cell_start[base];
                    sege[ns] = (int)a.cell_start[base + x1 - g.gx + 1];
                    segs[ns++] = -g.L;
                    x1 = g.gx - 1;
                }
            } else {
                x0 = x0 < 0 ? 0 : x0;
                x1 = x1 >= g.gx ? g.gx - 1 : x1;
            }
            if (x0 <= x1) {
                segb[ns] = (int)a.cell_start[base + x0];
                sege[ns] = (int)a.cell_start[base + x1 + 1];
                segs[ns++] = 0.f;
            }
            for (int q = 0; q < ns; ++q)
                for (int j = segb[q] + lane; j < sege[q]; j += 32) {
                    const int b = shell_of(a.pts[j], pi, segs[q], sy, sz, e2, a.nr);
                    if (b >= 0) atomicAdd(&hist[warp][b], 1u);
                }
        }
    }
    __syncwarp();
    if (lane < a.nr && hist[warp][lane]) atomicAdd(&a.counts[lane], (unsigned long long)hist[warp][lane]);
}

npcf_status bad(npcf_status s, const char* msg) {
    set_global_error(msg);
    return s;
}

#define CUN(call)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);    \
            set_global_error(m_.c_str());                                            \
            return NPCF_ECUDA;                                                       \
        }                                                                            \
    } while (0)

}  // namespace

extern "C" npcf_status npcf_pair_counts_noalloc(const float* d_pos, int64_t n, int nr,
                                                const double* edges, double box,
                                                uint64_t* d_counts, void* stream) {
    if (nr < 1 || nr > kMaxNr) return bad(NPCF_EINVAL, "nr outside [1, 16]");
    if (!edges || !d_counts) return bad(NPCF_EINVAL, "null edges or output pointer");
    if (n < 0) return bad(NPCF_EINVAL, "negative particle count");
    if (n > kMaxPoints) {
        char m[160];
        snprintf(m, sizeof(m), "%lld particles exceed the %lld this entry point's fixed scratch holds",
                 (long long)n, (long long)kMaxPoints);
        return bad(NPCF_EINVAL, m);
    }
    if (n > 0 && !d_pos) return bad(NPCF_EINVAL, "null position pointer");
    for (int i = 0; i <= nr; ++i)
        if (!std::isfinite(edges[i]) || edges[i] < 0 || (i > 0 && !(edges[i] > edges[i - 1])))
            return bad(NPCF_EINVAL, "edges must be finite, >= 0 and strictly increasing");
    if (!(box >= 0) || !std::isfinite(box)) return bad(NPCF_EINVAL, "box must be >= 0");
    if (box > 0 && !(edges[nr] * 3.0 < box)) return bad(NPCF_EINVAL, "periodic box must exceed 3 r_max");

    unsigned char* base = nullptr;
    npcf_status st = scratch_address(&base);
    if (st != NPCF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUN(cudaMemsetAsync(d_counts, 0, nr * sizeof(uint64_t), s));
    if (n == 0) return NPCF_OK;

    const double rmax = edges[nr];
    GridInfo g{};
    std::vector<int> rows;
    if (box > 0) {
        if (!plan_periodic_grid(box, rmax, 4, kMaxCells, &g, &rows))
            return bad(NPCF_EINVAL, "no neighbour grid fits the fixed scratch for this box and r_max");
    } else {
        float* bb = reinterpret_cast<float*>(base + kOffBBox);
        launch_bbox(d_pos, (int)n, bb, kBBoxBlocks, s);
        CUN(cudaGetLastError());
        float part[6 * kBBoxBlocks];
        CUN(cudaMemcpyAsync(part, bb, sizeof(part), cudaMemcpyDeviceToHost, s));
        CUN(cudaStreamSynchronize(s));
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) {
            mn[a] = part[a];
            mx[a] = part[3 + a];
            for (int b = 1; b < kBBoxBlocks; ++b) {
                mn[a] = std::min(mn[a], part[b * 6 + a]);
                mx[a] = std::max(mx[a], part[b * 6 + 3 + a]);
            }
            if (!std::isfinite(mn[a]) || !std::isfinite(mx[a])) return bad(NPCF_EINVAL, "non-finite positions");
        }
        plan_open_grid(mn, mx, rmax, 4, kMaxCells, &g, &rows);
    }
    const int nrows = (int)rows.size() / 4;
    if (nrows > kMaxRows || g.ncell > kMaxCells) return bad(NPCF_EINVAL, "neighbour grid exceeds the fixed scratch");

    uint32_t* count = reinterpret_cast<uint32_t*>(base + kOffCount);
    int* misc = reinterpret_cast<int*>(base + kOffMisc);   // [0] error bits, [1] work counter
    CUN(cudaMemsetAsync(count, 0, (size_t)g.ncell * sizeof(uint32_t), s));
    CUN(cudaMemsetAsync(misc, 0, 2 * sizeof(int), s));
    float* w = reinterpret_cast<float*>(base + kOffW);
    k_fill_ones<<<(int)((n + 255) / 256), 256, 0, s>>>(w, (int)n);
    long long* d_off = reinterpret_cast<long long*>(base + kOffMisc + 64);   // one catalog: {0, n}
    k_set_range<<<1, 1, 0, s>>>(d_off, (long long)n);

    BinArgs b{};
    b.pos = d_pos;
    b.w = w;
    b.wprim = nullptr;
    b.n = (int)n;
    b.g = g;
    b.cid = reinterpret_cast<uint32_t*>(base + kOffCid);
    b.count = count;
    b.start = reinterpret_cast<uint32_t*>(base + kOffStart);
    b.cursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
    b.pts = reinterpret_cast<float4*>(base + kOffPts);
    b.wp = reinterpret_cast<float*>(base + kOffWp);
    b.idx = reinterpret_cast<uint32_t*>(base + kOffIdx);
    b.cell_of = reinterpret_cast<uint32_t*>(base + kOffCellOf);
    b.err = misc;
    b.off = d_off;
    b.ncat = 1;
    launch_bin(b, s);
    CUN(cudaGetLastError());

    CountArgs c{};
    c.pts = b.pts;
    c.cell_of = b.cell_of;
    c.cell_start = b.start;
    for (int r = 0; r < nrows; ++r)
        c.rows[r] = make_int4(rows[4 * r], rows[4 * r + 1], rows[4 * r + 2], rows[4 * r + 3]);
    c.nrows = nrows;
    c.g = g;
    for (int i = 0; i <= nr; ++i) c.e2[i] = (float)(edges[i] * edges[i]);
    c.nr = nr;
    c.n = (int)n;
    c.work = misc + 1;
    c.err = misc;
    c.counts = reinterpret_cast<unsigned long long*>(d_counts);
    int dev = 0, nsm = 0;
    CUN(cudaGetDevice(&dev));
    CUN(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    k_count<<<2 * nsm, kWarps * 32, 0, s>>>(c);
    CUN(cudaGetLastError());
    return NPCF_OK;
}
