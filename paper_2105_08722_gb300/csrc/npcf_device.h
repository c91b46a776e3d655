// Argument blocks and launch wrappers shared by the kernels of libencore_gpu.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "npcf_tables.h"

namespace npcf {

// Cartesian cell grid of the neighbour search (cells sorted x fastest, then y, z). A batch
// of catalogs uses one grid per catalog: cell c of catalog k has the global id k ncell + c.
struct GridInfo {
    int gx, gy, gz, ncell;     // ncell: cells of one catalog's grid
    float ox, oy, oz;      // origin of cell (0,0,0)
    float inv_cell;        // 1 / cell side
    int periodic;
    float L, hL;           // periodic side and float(L/2)
};

// Host: neighbour-grid planning (npcf_grid.cpp). Rows are (dy, dz, dx_lo, dx_hi).
std::vector<int> neighbour_rows(float cell, double rmax, int* reach);
bool plan_periodic_grid(double L, double rmax, int cells_per_rmax, int max_cells, GridInfo* g,
                        std::vector<int>* rows);
void plan_open_grid(const float mn[3], const float mx[3], double rmax, int cells_per_rmax,
                    int max_cells, GridInfo* g, std::vector<int>* rows);
// Table of the neighbour rule's shell over bins of r2 of width 2^-k (at most max_bins
// bins up to e2[nr]): entry i = (shell below, shell above, bits of the float r2 where it
// changes, 0), valid when no bin holds two changes; *scale = 2^k. False if none fits.
bool build_shell_table(const float* e2, int nr, int max_bins, std::vector<int4>* tab, float* scale);

// ---------------------------------------------------------------- cell list (a1)
struct BinArgs {
    const float* pos;      // [n][3] input order
    const float* w;        // [n]
    const float* wprim;    // [n] or nullptr (= w)
    int n;
    GridInfo g;
    uint32_t* cid;         // [n] cell of each input point
    uint32_t* count;       // [ncell] histogram (zeroed by caller)
    uint32_t* start;       // [ncell + 1] exclusive scan
    uint32_t* cursor;      // [ncell] scatter cursors
    float4* pts;           // [n] sorted (x, y, z, w)
    float* wp;             // [n] sorted primary weights
    uint32_t* idx;         // [n] sorted -> input index
    uint32_t* cell_of;     // [n] sorted -> cell
    int* err;              // error bits (1: position outside the periodic box / NaN)
    float* bbox_part;      // [nblocks][6] partial min/max (non-periodic)
    const long long* off;  // [ncat + 1] first point of each catalog (device)
    int ncat;
};

void launch_bbox(const float* pos, int n, float* part, int nblocks, cudaStream_t s);
void launch_bin(const BinArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- pair kernel (a2 + a3)
constexpr int kPairWarps = 16;     // independent warps per pair-kernel block (one block per SM)
constexpr int kPairShellTab = 512; // bins of r2 of the pair kernel's shell table
constexpr int kPairKC = 8;         // pair kernel: candidates per lane per scan step
// smallest per-shell bucket: twice the entries one scan step can add to a shell
constexpr int kPairBucketMin = 2 * 32 * kPairKC;
struct PairArgs {
    const float4* pts;         // secondaries: (x, y, z, w) in cell order
    const float* wp;
    const uint32_t* cell_of;
    const uint32_t* cell_start;// cell starts of the secondaries
    const float4* ppts;        // primaries in cell order (the same list as pts, or another one
    const float* pwp;          //   binned on the same grid), their weights u and cells
    const uint32_t* pcell;
    int np;                    // primaries
    int add;                   // add to a_lm and cnt (another pass over other secondaries)
    const int4* rows;          // (dy, dz, dx_lo, dx_hi) neighbour rows
    int nrows;
    GridInfo g;
    float e2[kMaxNr + 1];
    int nr;
    int lmax;
    const float* kmat;         // [nlm][lmax + 1] Y_lm conversion matrix
    float2* alm;               // [n][nr][nlm]
    uint32_t* cnt;             // [n][nr]
    unsigned long long* counts;// [ncat][nr]
    int ncat;                  // catalogs; work units run over catalogs x cell runs
    int n;
    int* work;                 // global counter of primaries handed out in chunks (zeroed by caller)
    int* err;                  // error bits (2: a bounded wait gave up)
    int skip_zero;             // separate primary weights given: a primary of weight 0 is
                               // not evaluated (no a_lm, no counts); else every primary is
    uint32_t* bucket;          // [blocks][kPairWarps][boff[nr]] per-shell buckets of accepted pairs
    int boff[kMaxNr + 1];      // shell t's bucket: entries [boff[t], boff[t+1]) of a warp's region
    int chunk;                 // primaries per chunk a block takes from the global counter
    int linear;                // edges are linear in r: shell estimated from sqrt(r2)
    float lin_r0, lin_inv_w;   // first edge and 1 / shell width of linear edges
    int tab_ok;                // the shell table below is valid (else the estimate above)
    int tab_n;                 // bins of the table
    float tab_scale;           // bin of r2: floor(r2 tab_scale), a power of two
    const int4* tab;           // [tab_n] (shell below, shell above, bits of float r2 where it changes, 0)
    int trim;                  // cut staged rows to each primary's x-window (cells sorted by x)
    float cell;                // cell side of the grid
    float trim_margin;         // slack of the cut (covers FP32 rounding of the cell bounds)
};

void launch_pair(const PairArgs& a, int nblocks, cudaStream_t s);
// dynamic shared memory of the pair kernel for a given capacity setting
size_t pair_dynamic_smem(const PairArgs& a);
size_t pair_static_smem(int lmax);   // static shared memory of the pair kernel for lmax

// ---------------------------------------------------------------- contraction (a4 + a5)
struct Contract3Args {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;
    int n, nr, nlm, lmax;
    const int2* chunks;        // [nchunk] primary ranges, none crossing a catalog (one block each)
    int nchunk;
    const int4* items;         // (l, l(l+1)/2, b1 | (nr - 1 - b1) << 16, output of (l, b1, b1 + 1) in the order)
    int nitem;
    const float* coef;         // per l: (l l 0; 0 0 0)
    double* partial;           // [nchunk][total]
    int total, out_off;        // entries of the whole output, first entry of this order
    int nout;                  // entries of this order
};

// 4PCF contraction, FP32 on the CUDA cores: lanes are primaries, warps take items
// (multiplet, b1); see npcf_contract4.cu.
struct Contract4WArgs {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;           // [n] primary weights
    int n, nr, nlm;
    const PairTerm* terms;
    int nterms;
    const int4* segs;          // per (multiplet, m3): term range, lm of a_{l3 m3}, 2 S(m3) bits
    int nseg;
    const int4* items;         // (first segment, end, b1 | odd << 8 | (nr - 1 - b1) << 16, first output)
    int nitem;
    const int2* chunks;        // [nchunk] primary ranges, none crossing a catalog
    int nchunk;
    double* partial;           // [nchunk][total]: chunk c sums into row c
    int total, out_off, nout;  // this order's entries: [out_off, out_off + nout)
    int* chunk_counter;        // zeroed before the launch
};
void launch_contract4w(const Contract4WArgs& a, int nblocks, cudaStream_t s);
size_t contract4w_smem_bytes(const Contract4WArgs& a);
int contract4w_blocks(int nsm, int nchunk);

// 4PCF contraction for lmax beyond what the kernel above stages (npcf_contract4g.cu):
// one primary per lane, coupling terms read through L1, two m3 segments at a time with
// their terms grouped by the a^{b2} row they read.
struct Contract4GArgs {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;           // [n] primary weights
    int n, nr, nlm;
    const float4* coef;        // per term (cA, cB, cC, cD)
    const int* tlm;            // per term: lm of a^{b1}_{l1 |m1|}
    const int4* groups;        // (first term of segment 0, of segment 1, end, lm of a^{b2}_{l2 |m2|})
    const int4* pairs;         // per segment pair: (first group, end, lm of a_{l3 m3} of segment 0,
                               //   of segment 1 or -1), (2 S(m3) bits of both, m3 == 0 of segment 0, 0)
    const int4* items;         // (first pair of L, end, b1 | odd << 8 | (nr - 1 - b1) << 16, first output)
    int nitem;
    const int2* chunks;        // [nchunk] primary ranges, none crossing a catalog
    int nchunk;
    double* partial;           // [nchunk][total]: chunk c sums into row c
    int total, out_off, nout;
    int* chunk_counter;        // zeroed before the launch
};
void launch_contract4g(const Contract4GArgs& a, int nblocks, cudaStream_t s);
size_t contract4g_smem_bytes(int nr, int nlm);

// 4PCF contraction on the tensor cores (split bf16, fp32 accumulation in tensor memory).
// Rows (multiplet, b1, b2) are grouped by (l3, parity); each group's rows form 128-row
// tiles whose 128 x 16 (b3) accumulators stay in tensor memory for a block's whole chunk
// of primaries.
struct Contract4TCArgs {
    const float2* alm;
    const float* wp;
    int n, nr, nlm;
    const int2* chunks;        // one primary range per block, none crossing a catalog
    const PairTerm* terms;
    int nterms;
    const int4* segs;          // per (multiplet, m3): term range, lm of a_{l3 m3}, 2 S(m3)
    int nseg;
    const int* lam_seg0;       // first segment of each multiplet (n_lambda + 1)
    int nlam;
    const int4* groups;        // (l3, odd, first multiplet in group_lams, multiplets)
    const int* group_lams;
    int ngroup;
    const int4* tiles;         // (group, first row in the group, rows, first B slab)
    int ntile;
    const int4* runs;          // (first row in the tile, rows <= 8, multiplet, b1 | first b2 << 8)
    const int* tile_run0;      // first run of each tile (ntile + 1)
    const int2* combos;        // (b1, b2), b1 < b2 <= nr - 2
    const int* combo_bin;      // bin-tuple index of (b1, b2, b2 + 1)
    int ncombo;
    const int* group_bslab;    // first B slab of each group
    int nbslab;                // B slabs in total (sum of 2 l3 + 1)
    int maxcomp;               // largest 2 l3 + 1
    int off4, nb4;
    int drain_steps;           // steps of 16 primaries between drains of tensor memory
    double* partial;           // [nchunk][total]
    int total;
    int* err;
};

void launch_contract4_tc(const Contract4TCArgs& a, int nchunk, cudaStream_t s);


// 5PCF contraction (FP32 CUDA cores, npcf_contract5w.cu). For L = (l1, l2, l12, l3, l4):
//   P12^{m12}(b1,b2) = sum_{m1} (l1 l2 l12; m1, m12-m1, -m12) a^{b1}_{l1 m1} a^{b2}_{l2, m12-m1}
//   P34^{m12}(b3,b4) = sum_{m3} (l12 l3 l4; m12, m3, -m12-m3) a^{b3}_{l3 m3} a^{b4}_{l4, -m12-m3}
//   zeta_L(b1..b4) += u sqrt(2 l12 + 1) sum_{m12>=0} 2 S(m12) (-1)^{l12-m12} Q_L[P12 P34].
// Tiles of kT5 primaries staged as [lm][b][primary] with row stride kRS5; warps take
// items (L, beta = b2), one primary per lane.
constexpr int kT5 = 32;
constexpr int kRS5 = kT5 + 1;
struct Contract5WArgs {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;
    int n, nr, nlm;
    const float4* c12;         // P12 terms (cA, cB, cC, cD)
    const uint32_t* o12;       // staged offsets lm1 nr kRS5 | lm2 nr kRS5 << 16
    const float4* c34;
    const uint32_t* o34;
    const int2* segs12;        // term range of each (l1 l2 l12 triple, m12)
    const int2* segs34;
    int nterms12, nterms34, nseg12, nseg34;
    const int* binq;           // [nr][nr]: bin index of (b1, b2, b2 + 1, b2 + 2)
    const int4* items;         // (P34 segment of m12 = 0, l12 | beta << 8 | partners << 16, first partner, 0)
    int nitem;
    const int4* partners;      // (P12 segment of m12 = 0, first output of L, odd, 0) per multiplet L of an item
    int npartner;
    const int2* chunks;        // primary ranges, none crossing a catalog
    int nchunk;
    double* partial;           // [nchunk][total]
    int total, out_off, nout;
    int* chunk_counter;        // zeroed before the launch
};
// Multiplets (l1 l2 l12 l3 l4) of one 5PCF item: they share (l12 l3 l4) and so the P34
// build. Two while their sums fit in 64 registers, else one (measured: three or four per
// item ran slower, the kernel's register cap of 128 leaving too little room).
__host__ __device__ constexpr int c5_group(int nb, int m) {
    const int g = 64 / (nb * m * (m - 1) / 2);
    return g < 1 ? 1 : (g > 2 ? 2 : g);
}
void launch_contract5w(const Contract5WArgs& a, int nblocks, cudaStream_t s);
// 5PCF contraction with P34 built once per block and tile into shared memory
// (npcf_contract5c.cu). The work list of each phase holds P34 builds, (segment of the
// (triple, m12), b3 | slot << 24 | 1 << 30, cache entry of the (triple, m12) block, 0), and
// items, (P12 segment of m12 = 0 of a left triple, beta | l12 << 16 | slot << 24 | (g - 1)
// << 26, first of its g partners, 0); a partner is (cache entry of its right triple's
// m12 = 0 block, first output of the multiplet, odd, 0); a cache entry is kT5 float2.
// Partners per item: as many as their sums fit in about 64 registers, at most 4.
__host__ __device__ constexpr int c5c_group(int nb, int m) {
    const int g = 64 / (nb * m * (m - 1) / 2);
    return g < 1 ? 1 : (g > 4 ? 4 : g);
}
struct Contract5CArgs {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;
    int n, nr, nlm;
    const float4* c12;         // P12 terms (cA, cB, cC, cD)
    const uint32_t* o12;       // staged offsets lm1 nr kRS5 | lm2 nr kRS5 << 16
    const float4* c34;
    const uint32_t* o34;
    const int2* segs12;        // term range of each (l1 l2 l12 triple, m12)
    const int2* segs34;
    const int* binq;           // [nr][nr]: bin index of (b1, b2, b2 + 1, b2 + 2)
    const int4* work;          // the phases' work lists, back to back
    const int4* partners;      // the items' partners
    const int* phase_begin;    // [nphase + 1]
    int nphase;
    int slot_entries;          // entries of one cache slot
    int blocks_per_sm;         // 2 where two blocks' shared memory fits on an SM, else 1
    int tables_smem;           // 1: one block of 512 threads per SM, coupling terms in shared memory
    int nterms12, nterms34, nseg12, nseg34;
    const int2* chunks;        // primary ranges, none crossing a catalog
    int nchunk;
    double* partial;           // [nchunk][total]
    int total, out_off, nout;
    int* chunk_counter;        // zeroed before the launch
};
void launch_contract5c(const Contract5CArgs& a, int nblocks, cudaStream_t s);
size_t contract5c_smem_bytes(const Contract5CArgs& a);
size_t contract5c_static_smem();

size_t contract5w_smem_bytes(const Contract5WArgs& a);
size_t contract4_tc_smem_bytes(const Contract4TCArgs& a);

// 6PCF contraction (FP32 CUDA cores, npcf_contract6.cu): Eq. basis-coupling at N = 6
// through m12 and m123, primaries on the lanes, items (L, b3); 5 <= nr <= 8.
struct Contract6Args {
    const float2* alm;         // [n][nr][nlm]
    const float* wp;
    int n, nr, nlm, lmax;
    const int4* lam;           // per multiplet: (l12, l123, odd, first output of L)
    const int4* lam2;          // per multiplet: (first P12 segment, first m123 segment, prefactor bits, 0)
    const int2* seg1;          // P12 segments: term range of (L, m12)
    const int4* terms1;        // (lm of (l1, m1), lm of (l2, m2), coefficient bits, 0); lm = l^2 + l + m
    const int2* seg2;          // per (L, m123): range of Q terms
    const int4* terms2;        // (P12 segment of m12, lm of (l3, m3), coefficient bits, 0)
    const int2* seg3;          // per (L, m123): range of P45 terms
    const int4* terms3;        // (lm of (l4, m4), lm of (l5, m5), coefficient bits, 0)
    const int* binq;           // [nr][nr][nr]: bin index of (b1, b2, b3, b3 + 1, b3 + 2)
    const int2* items;         // (multiplet, b3)
    int nitem;
    const int2* chunks;        // primary ranges, none crossing a catalog
    int nchunk;
    double* partial;           // [nchunk][total]
    int total, out_off, nout;
    int* chunk_counter;        // zeroed before the launch
};
void launch_contract6(const Contract6Args& a, int nblocks, cudaStream_t s);
size_t contract6_smem_bytes(const Contract6Args& a);

void launch_contract3(const Contract3Args& a, cudaStream_t s);

// ---------------------------------------------------------------- gridded fields (FFT)
// a_lm of a density field on a periodic n^3 mesh by FFT (npcf_fftgrid.cu).
struct GridFFTArgs {
    float e2[kMaxNr + 1];      // squared shell edges of the FP32 rule
    int nr, lmax;
};
struct GridFFT;
GridFFT* gridfft_create();
void gridfft_destroy(GridFFT* g);
// alm [n^3][nr][nlm] (cells x fastest) and wp [n^3] = delta; 0 on success, 2 (out of
// memory) or 3 (CUDA or cuFFT error) with a message in err.
int gridfft_alm(GridFFT* G, const float* delta, int n, float box, const GridFFTArgs& a, float2* alm, float* wp,
                cudaStream_t s, char* err, size_t errlen);

// ---------------------------------------------------------------- edge correction (a7)
struct EdgeArgs {
    const double* nraw;        // [nl][nb] raw multiplets of the data-minus-randoms run
    const double* rraw;        // [nl][nb] raw multiplets of the randoms-only run
    int nl, nb;
    const int* tptr;           // [nl * nl + 1] entries of M[L''][L] in the sparse table
    const int* tlp;            // L' of each entry
    const double* tg;          // G^{L L' L''} of each entry
    double* out;               // [nl][nb] edge-corrected zeta
    int* err;                  // error bits (4: a singular system)
};
void launch_edge_solve(const EdgeArgs& a, cudaStream_t s);
size_t edge_smem_bytes(int nl);

// ---------------------------------------------------------------- FP64 reduction (a6)
// For every catalog k (grid row): zeta[k][e] += scale[e] * sum_{cbeg[k] <= c < cbeg[k+1]}
// partial[c][e], e in [off, off + count); zeta rows are total long.
void launch_reduce(const double* partial, const int* cbeg, int ncat, int total, int off, int count,
                   const double* scale, double* zeta, cudaStream_t s);
void launch_sumw(const float* w, const long long* off, int ncat, double* sumw, cudaStream_t s);
// Per-primary a_lm rows (row float2) and shell counts (rc) between cell order (p) and input
// order (idx[p]): the cached data harmonics of npcf_cache_data / npcf_accumulate_split.
void launch_alm_to_input(const float2* alm, const uint32_t* cnt, const uint32_t* idx, int n, int row, int rc,
                         float2* alm_in, uint32_t* cnt_in, cudaStream_t s);
void launch_alm_from_input(const float2* alm_in, const uint32_t* cnt_in, const uint32_t* idx, int n, int row, int rc,
                           float2* alm, uint32_t* cnt, cudaStream_t s);
void launch_add_counts(unsigned long long* dst, const unsigned long long* src, int n, cudaStream_t s);
// dst[0..3] = (a, b, c, d), stream-ordered (offset tables written without host buffers)
void launch_set4(long long* dst, long long a, long long b, long long c, long long d, cudaStream_t s);

}  // namespace npcf
