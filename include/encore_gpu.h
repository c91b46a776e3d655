/*
 * encore_gpu.h -- C ABI of libencore_gpu, a single-GPU (sm_103a) implementation of
 * the isotropic N-point correlation function estimator of Philcox, Slepian, Hou,
 * Warner, Cahn & Eisenstein, "ENCORE: an O(N_g^2) estimator for galaxy N-point
 * correlation functions" (arXiv:2105.08722).
 *
 * What one accumulate call computes (all of it on the GPU):
 *   1. cell list: particles binned into a Cartesian grid for the neighbour search
 *      (Sec. 5.1 / Fig. 5 "placing particles onto a Cartesian grid");
 *   2. for every primary i, the binned harmonic coefficients
 *         a^b_lm(s_i) = sum_j w_j Y_lm(unit(r_j - s_i)) Theta^b(|r_j - s_i|),
 *      Eq. (binned-discrete-alm) without the 1/v_b factor, from Cartesian powers of
 *      the unit separation (Algorithm 2);
 *   3. the raw multiplets
 *         zeta^B_L += sum_i u_i sum_M E(L) C^L_M prod_k a^{b_k}_{l_k m_k}(s_i),
 *      Eq. (NPCF-mult-discrete-binned-estimator) without 1/V, summed with the
 *      m_{N-1} >= 0 halving of App. B (Eq. simple-NPCF-summation), for N = 3, 4, 5, 6
 *      (for N = 6 the halving runs over the second intermediate m123).
 *
 * Conventions shared with the documentation:
 *  - Y_lm orthonormal, Condon-Shortley phase (Sec. 2.1). Separation r_j - s_i.
 *  - Neighbour/shell rule, evaluated in IEEE FP32 round-to-nearest without fused
 *    multiply-add so that pair counts are exact and reproducible:
 *      d = p_j - p_i per axis; periodic side L > 0: d > L/2 -> d - L,
 *      d < -L/2 -> d + L; r2 = (dx*dx + dy*dy) + dz*dz; e2[k] = float(edge_k^2);
 *      pair accepted iff r2 > 0 and e2[0] <= r2 < e2[nr]; shell b with
 *      e2[b] <= r2 < e2[b+1]. Bins are distinct and ordered, b1 < b2 < ... (Sec. 3.2.1).
 *  - Multiplets L: l1 outer, then l2, [l12], l3, [l123], l4, [l5], last index fastest;
 *    N=3: (l, l), l = 0..lmax; N=4: |l1-l2| <= l3 <= min(l1+l2, lmax);
 *    N=5: |l1-l2| <= l12 <= l1+l2, |l12-l3| <= l4 <= min(l12+l3, lmax);
 *    N=6: |l1-l2| <= l12 <= l1+l2,
 *    |l12-l3| <= l123 <= l12+l3, |l123-l4| <= l5 <= min(l123+l4, lmax).
 *    Parity-even only (sum of principal l even) unless allparity != 0 (Table 1).
 *  - Output of npcf_finalize: orders ascending; for each order an array
 *    [n_multiplets][n_bin_tuples], bin tuples lexicographic with the last index
 *    fastest. Parity-even multiplets are real; parity-odd ones are purely imaginary
 *    (Sec. 3.1) and their imaginary part is stored.
 *
 * Threading: a context is not thread-safe; use one context per host thread.
 * Errors: every call returns an npcf_status and never aborts; npcf_last_error gives
 * a message. Device-side waits are bounded and report NPCF_ETIMEOUT.
 */
#ifndef ENCORE_GPU_H
#define ENCORE_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct npcf_ctx npcf_ctx;

typedef enum {
    NPCF_OK = 0,
    NPCF_EINVAL = 1,        /* bad argument (null pointer, bad size, bad edges ...) */
    NPCF_ENOMEM = 2,        /* device or host allocation failed */
    NPCF_ECUDA = 3,         /* a CUDA runtime call failed */
    NPCF_EUNSUPPORTED = 4,  /* valid request this build does not implement */
    NPCF_ETIMEOUT = 5       /* a bounded device-side wait gave up */
} npcf_status;

/* Arithmetic of the contraction over primaries (step 3). FP32: CUDA-core FP32
 * products and sums. SPLIT_BF16: each FP32 operand v is split into three bf16 terms
 * v ~ hi + mid + lo and the tensor cores (tcgen05) form the six products
 * hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid with FP32 accumulation.
 * Cross-block sums are FP64. */
typedef enum {
    NPCF_FP32 = 0,
    NPCF_SPLIT_BF16 = 1
} npcf_precision;

/* Create a context.
 *   lmax        maximum l of every principal angular momentum, 0 <= lmax <= 10
 *               (Sec. 3.1: the l_i <= lmax truncation).
 *   order_mask  bit N set to compute the N-point function; N in {3, 4, 5, 6}. The 6PCF
 *               takes at most 8 shells (NPCF_EUNSUPPORTED above; with fewer than 5 it has
 *               no bin tuple and an empty output) and (lmax + 1)^2 x nr x 264 bytes of
 *               shared memory (NPCF_EUNSUPPORTED beyond the device's limit). The FP32
 *               4PCF needs nr (lmax + 1)(lmax + 2) / 2 x 264 bytes of shared memory (every
 *               lmax <= 10 up to 10 shells); the split-BF16 4PCF stages more and takes
 *               lmax <= 5 (NPCF_EUNSUPPORTED beyond, with the byte count).
 *   nr, edges   nr radial shells (1 <= nr <= 16) with host edges[nr+1] strictly
 *               increasing, edges[0] >= 0 (the binning functions Theta^b, Sec. 3.2).
 *   box         > 0: periodic cube of that side (Table 1 "periodic"); positions must
 *               lie in [0, box) and edges[nr] < box / 3. 0: no periodicity.
 *   prec        contraction arithmetic (npcf_precision).
 *   allparity   non-zero: parity-odd multiplets too (Table 1 "allparity").
 * The context owns every device buffer it needs; npcf_destroy frees them. On failure
 * *out is NULL and npcf_last_error(NULL) describes the problem. */
npcf_status npcf_create(npcf_ctx** out, int lmax, unsigned order_mask, int nr,
                        const double* edges, double box, int prec, int allparity);

/* Accumulate the multiplets of one catalog into the context (adds to previous calls,
 * so random-catalog splits co-add, Sec. 4.2).
 *   d_pos   device float32 [n][3] positions (x, y, z), caller-owned
 *   d_w     device float32 [n] weights w_j (secondaries, and primaries unless d_wprim)
 *   d_wprim nullable device float32 [n] primary weights u_i. When given, a primary with
 *           u_i == 0 is skipped entirely: its a_lm are not formed and its neighbours
 *           are not counted (so a seeded sample of primaries can be evaluated against
 *           the full catalog; npcf_pair_counts then counts the sample's pairs only).
 *           Without d_wprim, u_i = w_i and every primary's neighbours are counted,
 *           including those of primaries of weight 0 (which add nothing to zeta).
 *   n       number of particles, 0 <= n < 2^26 (NPCF_EUNSUPPORTED above)
 *   stream  cudaStream_t to enqueue on (0 = legacy default stream)
 * Work is enqueued asynchronously; caller buffers must stay valid until the stream
 * reaches it. For box == 0 the call reads the bounding box back to the host (one
 * stream synchronisation). */
npcf_status npcf_accumulate(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n,
                            void* stream);
npcf_status npcf_accumulate_ex(npcf_ctx* ctx, const float* d_pos, const float* d_w,
                               const float* d_wprim, int64_t n, void* stream);

/* Same as npcf_accumulate, from HOST buffers: copies them to the device inside the
 * call (stream-ordered) and synchronises the stream before returning. */
npcf_status npcf_accumulate_host(npcf_ctx* ctx, const float* h_pos, const float* h_w,
                                 int64_t n, void* stream);

/* Random splits with the data harmonics kept (Sec. 4.2: the data particles' contributions
 * to a_lm are the same in every data-minus-randoms split, so they are formed once).
 * npcf_cache_data: for every data point as a primary, its a_lm from the data as secondaries
 * and its per-shell counts, and the data-data pair counts, kept in the context with a device
 * copy of the data (d_pos, d_w as in npcf_accumulate, 1 <= n < 2^26; a new call replaces
 * them). It does not touch the accumulators.
 * npcf_accumulate_split: adds what npcf_accumulate would add for the catalog made of the
 * cached data followed by this split's randoms (d_pos, d_w, n as in npcf_accumulate, n >= 0;
 * random weights typically -N_D/N_R), without searching the data-data pairs again: a data
 * primary takes its cached a_lm plus the randoms as secondaries, a random primary takes the
 * data and the randoms as secondaries; the counts include the cached data-data pairs. Calls
 * on the same context are stream-ordered (use one stream, or synchronise between streams);
 * single catalogs only (NPCF_EINVAL when the accumulators hold a batch); NPCF_EINVAL
 * before npcf_cache_data. With box == 0 each call reads a bounding box back to the host
 * (one stream synchronisation); the grid covers the data and the randoms. */
npcf_status npcf_cache_data(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream);
npcf_status npcf_accumulate_split(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n,
                                  void* stream);

/* Gridded data (Sec. 3.2.2, Eq. alm-binned-def-fft): a density field delta on a periodic
 * ngrid^3 mesh over the context's box (cell side h = box / ngrid; d_delta: device float32
 * [ngrid^3], cells x fastest, then y, z; caller-owned; 1 <= ngrid <= 406). Adds to the
 * accumulators the multiplets of the field with every cell a primary and a secondary of
 * weight delta at its centre: the harmonic coefficients of every cell come from FFTs (the
 * correlation of delta with the kernel Y_lm(unit(r)) Theta^b(r) sampled on cell offsets,
 * whose shell is the FP32 rule on the offset's separation), then the same contractions
 * as for particles. Equal, up to FP32 rounding, to npcf_accumulate of the cell centres with
 * weights delta when the cell-centre coordinates are exact in FP32. Raw sums (the
 * normalisation of npcf_finalize is for particle catalogs); pair counts and the sum of
 * weights are not updated. Keeps the kernel spectra of the mesh in the context (nr x
 * (lmax+1)(lmax+2)/2 x ngrid^3 x 8 bytes, plus one shell's field set and one spectrum of
 * delta as work space); FP32 transforms by cuFFT (their rounding is about 1e-6 of the RMS
 * of the a_lm). NPCF_EUNSUPPORTED without a periodic box; NPCF_ENOMEM when the spectra do
 * not fit. */
npcf_status npcf_accumulate_grid(npcf_ctx* ctx, const float* d_delta, int ngrid, void* stream);

/* Number of doubles npcf_finalize writes. */
npcf_status npcf_output_size(const npcf_ctx* ctx, size_t* len);

/* Multiplet and bin-tuple tables of one order (N in the context's mask). lambdas
 * (nullable) receives n_lambda x {2,3,5} ints, bins (nullable) n_bins x (N-1). */
npcf_status npcf_layout(const npcf_ctx* ctx, int order, int* n_lambda, int* n_bins,
                        int* lambdas, int* bins);

/* Copy the FP64 multiplets accumulated so far to host out[out_len] (synchronises;
 * NPCF_EINVAL when the context holds a batch of several catalogs).
 * normalize = 0: raw sums as defined above. normalize = 1 (periodic only): divide by
 * V prod_k v_{b_k} (Eq. NPCF-mult-discrete-binned-estimator, Eq. alm-binned-def with
 * v_b = 4 pi (r_{b+1}^3 - r_b^3) / 3, V = box^3) and by R_0 = (4pi)^{-(N-1)/2} nbar^N
 * with nbar = sum w / V (Eq. R-periodic-form). */
npcf_status npcf_finalize(npcf_ctx* ctx, double* out, size_t out_len, int normalize);

/* Batch of catalogs in one call (a8): catalog k is points offsets[k] .. offsets[k+1]-1 of
 * d_pos / d_w (device, caller-owned, as in npcf_accumulate); offsets: host int64
 * [ncat+1], offsets[0] = 0, non-decreasing; 1 <= ncat <= 65535. Periodic boxes only (every
 * catalog uses the same grid shape; NPCF_EUNSUPPORTED otherwise). All catalogs run through
 * the same kernels in one pass: the cell lists of all catalogs are built together (cell
 * ids offset per catalog), the pair kernel takes work units over (catalog, cell run) from
 * one device counter, the contractions take chunks of primaries that never cross a
 * catalog, and each catalog keeps its own FP64 multiplets (read with
 * npcf_finalize_batch), sums of weights and pair counts. The device work of a call is
 * captured into a CUDA graph on the first call with a given shape and replayed by later
 * calls with the same pointers, offsets, tuning and context buffers (a launch on the legacy
 * default stream is enqueued directly: that stream cannot be captured). The first
 * accumulate call after npcf_create or npcf_reset fixes the number of catalogs the
 * accumulators hold; later calls must use the same number (they co-add per catalog). */
npcf_status npcf_accumulate_batch(npcf_ctx* ctx, const float* d_pos, const float* d_w,
                                  const int64_t* offsets, int ncat, void* stream);

/* Same as npcf_accumulate_batch with separate primary weights (as npcf_accumulate_ex):
 * d_wprim device float32 [n], nullable (then d_w); primaries with weight 0 are skipped, so
 * a seeded sample of primaries of every catalog can be evaluated against full catalogs. */
npcf_status npcf_accumulate_batch_ex(npcf_ctx* ctx, const float* d_pos, const float* d_w,
                                     const float* d_wprim, const int64_t* offsets, int ncat,
                                     void* stream);

/* Multiplets of every catalog, host out[ncat][npcf_output_size] (synchronises);
 * normalize as in npcf_finalize, catalog k with its own sum of weights. */
npcf_status npcf_finalize_batch(npcf_ctx* ctx, double* out, size_t out_len, int normalize);

/* Per-catalog pair counts, host uint64 out[ncat][nr] (synchronises). */
npcf_status npcf_pair_counts_batch(npcf_ctx* ctx, uint64_t* out, size_t out_len);

/* Autotuner: runs the pipeline on the catalog (d_pos, d_w, n as in npcf_accumulate) for
 * candidate settings and keeps the fastest: pair kernel (median of three timed runs after a
 * warm-up) over cells per r_max {2, ..., 6} x primaries per chunk {8, 16, 32, 64} x bucket
 * entries per warp {4096, 8192}, then the contractions over primaries per chunk (1, 2, 4 or 8 waves of
 * chunks over the SMs). The accumulators must be empty (fresh context or npcf_reset) and
 * are reset afterwards. chosen (nullable, host int[4]) receives the settings: tuning keys
 * 0, 5, 3 and 2. Synchronises the stream; takes some tens of pipeline runs. */
npcf_status npcf_autotune(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream,
                          int* chosen);

/* Catalogs the accumulators hold (0 before the first accumulate call) and how many batch
 * calls were run as CUDA-graph launches. Either pointer may be NULL. */
npcf_status npcf_batch_info(const npcf_ctx* ctx, int* ncat, int64_t* graph_launches);

/* Per-shell pair counts accumulated so far (uint64 [nr], exact; synchronises). */
npcf_status npcf_pair_counts(npcf_ctx* ctx, uint64_t* out);

/* Zero every accumulator of the context. */
npcf_status npcf_reset(npcf_ctx* ctx);

/* Diagnostics: a^b_lm and per-shell neighbour counts of selected primaries from the
 * LAST accumulate call (synchronises). idx: host int64 [k] input indices.
 * alm: host float [k][nr][(lmax+1)(lmax+2)] as (re, im) pairs for l = 0..lmax,
 * m = 0..l (index l(l+1)/2 + m); counts: host uint32 [k][nr] (nullable). */
npcf_status npcf_debug_alm(npcf_ctx* ctx, const int64_t* idx, int64_t k, float* alm,
                           uint32_t* counts);

/* Tuning knobs (the autotuner sets these): key 0 = cells per r_max (1..8; the cell
 * side of the neighbour grid is about r_max / key0; 0, the default, picks 2 below ~630
 * mean neighbours within r_max and 3 above), key 2 = contraction primaries
 * per chunk, rounded up to a multiple of 64, for every contraction kernel (0 = automatic:
 * about n / (4 x SMs) for the 3PCF and 5PCF, n / SMs for the 4PCF), key 3 = pair kernel:
 * entries of each warp's per-shell buckets of accepted pairs (multiple of 256 in
 * max(1024, 512 x shells)..65536, default 8192; every shell gets at least 512, the rest in
 * proportion to the shell volumes; a bucket with room for less than one scan step (256
 * entries) is summed early, so larger buckets mean fewer reductions for dense primaries;
 * device scratch of SMs x 16 x 4 bytes per entry),
 * key 4 = FP32 4PCF contraction: 0 (default) stages the coupling terms with a tile of 64
 * primaries in shared memory where they fit (lmax <= 6 at 4 shells) and takes the
 * high-lmax kernel (tiles of 32 primaries, terms read through L1) beyond; 1 takes the
 * high-lmax kernel always, key 5 = pair kernel: consecutive (cell-sorted) primaries per
 * chunk that a block takes from the global counter (1..1024, default 16; small chunks keep
 * a block's warps on nearby primaries, whose neighbourhoods then share L1), key 6 =
 * split-bf16 contraction:
 * steps of 16 primaries between drains of the tensor-memory accumulators into FP64 (>= 1;
 * fewer steps bound the accumulation error of the tensor cores more tightly), key 7 = pair
 * kernel: cut each neighbour row to the primary's x-window (1, default) or scan whole rows
 * (0), key 8 = pair kernel: read the shell of each candidate from a table over bins of r2
 * (1, default, used when no bin holds two shell edges) or compute it from sqrt(r2) and the
 * edges (0); both apply the same exact FP32 rule; key 9 = 5PCF contraction: 0 (default)
 * builds P34 once per block and tile into shared memory where it fits, with the coupling
 * terms in shared memory too where they also fit, else read through L1; 1 takes the
 * register-only kernel, 2 the P34 cache with the terms read through L1, 3 the P34 cache
 * with the terms in shared memory (where they do not fit: the register-only kernel). */
npcf_status npcf_set_tuning(npcf_ctx* ctx, int key, int value);

/* Device time in ms of the stages of the last accumulate call:
 * [0] cell list, [1] pair kernel, [2] contraction, [3] FP64 reduction. */
npcf_status npcf_get_timings(npcf_ctx* ctx, float* ms4);

/* Exact per-shell pair counts of one catalog, computed without allocating any device
 * memory. The paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc: processes whose device memory belongs entirely to another allocator (a
 * framework's caching pool, a pipeline that forbids allocation after start-up), and
 * plug-ins that must not grow their memory footprint per call.
 *   d_pos    device float32 [n][3] positions, caller-owned; in [0, box) when periodic
 *   n        0 <= n <= 262144 (larger catalogs are rejected with NPCF_EINVAL)
 *   nr, edges, box   as in npcf_create (host edges[nr+1]; box > 3 edges[nr] or 0)
 *   d_counts device uint64 [nr], caller-owned; overwritten with the counts of this call
 *   stream   cudaStream_t the work is enqueued on
 * Counts are the same as npcf_accumulate + npcf_pair_counts give for the catalog (the
 * same FP32 neighbour rule, every particle a primary). A position outside [0, box) when
 * periodic, or a NaN position, is found on the device after the call has returned: then
 * every entry of d_counts is set to UINT64_MAX (a value no count reaches) instead of a
 * count. All scratch lives in one fixed device array of about 13 MiB that every GPU
 * loading the library keeps until the process exits. The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress). Calls share the array: each clears
 * what must start at zero, and calls that overlap on the GPU race. With box == 0 the call
 * reads the bounding box back to the host (one stream synchronisation); with box > 0 it
 * only enqueues work. Errors found on the host are reported through
 * npcf_last_error(NULL). */
npcf_status npcf_pair_counts_noalloc(const float* d_pos, int64_t n, int nr, const double* edges,
                                     double box, uint64_t* d_counts, void* stream);

/* Edge correction (Sec. 3.3, Eq. edge-corrected-NPCF; Sec. 4.2). For every order and
 * bin tuple B it solves, in FP64 on the GPU,
 *   sum_L zeta_L(B) M_{L L''}(B) = N_{L''}(B) / R_0(B),
 *   M_{L L''}(B) = sum_{L'} (R_{L'}(B) / R_0(B)) E(L'') G^{L L' L''},
 * with N the raw multiplets accumulated in nctx (data weighted +1, randoms -N_D/N_R),
 * R those accumulated in rctx (randoms only, weighted +N_D/N_R) and G the generalized
 * Gaunt integrals of App. A (see npcf_gaunt). Both contexts must have the same lmax,
 * orders, shells and box, be parity-even (allparity = 0; E(L'') = +1) and hold orders 3
 * and 4 only (NPCF_EUNSUPPORTED for 5). One block per bin tuple, Gaussian elimination
 * with partial pivoting. Writes host out[npcf_output_size] in the layout of
 * npcf_finalize; a bin tuple whose system is singular (R_0 = 0, no pivot) gets NaN and
 * the call returns NPCF_EINVAL. Synchronises the device. */
npcf_status npcf_edge_correct(npcf_ctx* nctx, npcf_ctx* rctx, double* out);

/* Truncation to a smaller lmax (Sec. 3.3: N and R are measured with an lmax one larger than
 * the output's, so that the edge correction of the multiplets near the output lmax is
 * accurate). in: host double[in_len] in this context's output layout (npcf_finalize,
 * one catalog's row of npcf_finalize_batch, or npcf_edge_correct); out: host
 * double[out_len] in the layout a context with lmax_out (same orders, shells, parity)
 * would have: of every order, the multiplets whose l's are all <= lmax_out (for the 5PCF
 * also l12 <= 2 lmax_out), in the same order, with all their bin tuples. in_len must be
 * npcf_output_size(ctx). out_len: with out == NULL it receives the length of the smaller
 * layout (in may then be NULL too); otherwise it must hold that length. NPCF_EINVAL for a
 * length mismatch or an lmax_out that is negative or above the context's lmax. Host only;
 * does not touch the device. */
npcf_status npcf_truncate(const npcf_ctx* ctx, const double* in, size_t in_len, int lmax_out, double* out,
                          size_t* out_len);

/* Generalized Gaunt integral G^{L1 L2 L3} = int dR P_L1 P_L2 P_L3 (Eq. generalized-gaunt-def)
 * from the closed forms of App. A (Wigner 3-j and 9-j symbols), the values the edge
 * correction uses. Host-only (no device work). L1, L2, L3: host int multiplets of order
 * N = 3, 4 or 5 laid out as npcf_layout gives them ({l, l}, {l1, l2, l3},
 * {l1, l2, l12, l3, l4}); *out receives the value. */
npcf_status npcf_gaunt(int N, const int* L1, const int* L2, const int* L3, double* out);

/* Multiplets L of order N = 3..6 (Sec. 2.2: the triangle conditions of the 3-j symbols of
 * Eq. basis-coupling, principal l's <= lmax, intermediates over their natural range; the
 * parity-even ones, sum of principal l's even, unless allparity), in the output order of
 * npcf_finalize (lexicographic in the l's with the last entry fastest, the order of the
 * edge-correction matrices of the mock-catalog figures, Sec. 5.4). Layout per multiplet: {l, l},
 * {l1, l2, l3}, {l1, l2, l12, l3, l4}, {l1, l2, l12, l3, l123, l4, l5}. *count receives
 * their number; out (nullable) receives count x (2, 3, 5, 7) ints. Host-only. lmax in
 * [0, 10]. */
npcf_status npcf_multiplets(int N, int lmax, int allparity, int* count, int* out);

/* Coupling coefficient C^L_M of Eq. basis-coupling (Eq. N=3-coeff and N=4-coeff for N = 3,
 * 4; one intermediate for N = 5, two for N = 6); L laid out as npcf_multiplets gives it,
 * M = {m_1, ..., m_{N-1}} (host ints). *out receives the value (0 where the 3-j symbols
 * vanish). Host-only; NPCF_EINVAL for N outside 3..6 or an l outside [0, 40]. */
npcf_status npcf_coupling(int N, const int* L, const int* M, double* out);

/* FP32 CUDA-core throughput of the current device, measured: the peak that the FP32
 * roofline fractions of the pair kernel and the FP32 contractions are taken against (the
 * paper has no counterpart). Launches fused multiply-add chains on every SM (four blocks
 * of 256 threads per SM, eight independent chains per thread), times five launches after a
 * warm-up with CUDA events on the legacy default stream and keeps the fastest.
 * *tflops receives 2 x FMAs / time in TFLOP/s; ms (nullable) that launch's time.
 * Synchronises the device; allocates a small output buffer; errors through
 * npcf_last_error(NULL). */
npcf_status npcf_probe_fp32_peak(double* tflops, double* ms);

/* Message of the last failed call on ctx; with ctx == NULL, of the last failed
 * npcf_create or npcf_pair_counts_noalloc on this thread. */
const char* npcf_last_error(const npcf_ctx* ctx);
void npcf_destroy(npcf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
