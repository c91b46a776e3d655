// C ABI of libencore_gpu (include/encore_gpu.h): context management and the
// accumulate / finalize pipeline. Host code only enqueues work; every step of the
// estimator runs in the kernels of npcf_bin.cu, npcf_pair.cu and npcf_contract.cu.
#include "encore_gpu.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "npcf_device.h"
#include "npcf_tables.h"

using namespace npcf;

namespace {

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t count) {
        if (count <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) n = count;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
};

thread_local std::string g_create_error;

}  // namespace

namespace npcf {
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace npcf

struct npcf_ctx {
    int lmax = 0, nr = 0, prec = 0, allparity = 0;
    unsigned mask = 0;
    double box = 0.0;
    std::vector<double> edges;
    float e2[kMaxNr + 1] = {};
    std::string err;

    std::vector<OrderTable> orders;
    std::vector<int> order_off;
    int total = 0;
    int nlm = 0;

    // cell-list tuning and geometry
    int cells_per_rmax = 0;    // 0: chosen per call from the catalog's density
    int pair_chunk = 16;       // pair kernel: consecutive primaries per chunk a block takes
    int pair_cap = 8192;       // pair kernel: bucket entries per warp (all shells)
    int drain_steps = 2;       // tensor-core contraction: steps of 16 primaries per TMEM drain
    int trim = 1;              // pair kernel: cut staged rows to each primary's x-window
    int use_stab = 1;          // pair kernel: shell by table lookup when the table is valid
    int c4g_force = 0;         // FP32 4PCF: the high-lmax contraction even where the staged one fits
    int c5_mode = 0;           // 5PCF: 0 automatic, 1 register-only, 2 P34 cache with the terms read
                               // through L1, 3 P34 cache with the terms in shared memory
    int chunk_target = 0;      // primaries per contraction chunk (0 = automatic)
    GridInfo grid{};
    std::vector<int> rows_host;
    float rows_cell = -1.f;

    // device tables
    DevBuf<float> kmat;
    DevBuf<int4> rows;
    DevBuf<int4> c3items;
    DevBuf<float> c3coef;
    int c3nitem = 0;
    DevBuf<PairTerm> c4terms;
    DevBuf<int4> c4segs, c4items;
    DevBuf<int> c4lamseg0;
    int c4nitem = 0, c4nterms = 0, c4nseg = 0, c4nlam = 0;
    // high-lmax FP32 4PCF contraction (npcf_contract4g.cu): used where the kernel above
    // does not fit in shared memory, or when tuning key 4 asks for it
    DevBuf<float4> c4g_coef;
    DevBuf<int> c4g_tlm;
    DevBuf<int4> c4g_groups, c4g_pairs, c4g_items;
    bool c4g_needed = false;
    // tensor-core (split bf16) 4PCF contraction tables
    DevBuf<int4> tc_groups, tc_tiles, tc_runs;
    DevBuf<int> tc_tile_run0;
    DevBuf<int> tc_group_lams, tc_group_bslab, tc_combo_bin;
    DevBuf<int2> tc_combos;
    int tc_ngroup = 0, tc_ntile = 0, tc_ncombo = 0, tc_nbslab = 0, tc_maxcomp = 0;
    int off4 = 0, nb4 = 0;
    // 5PCF contraction tables
    DevBuf<float4> c5c12, c5c34;
    DevBuf<uint32_t> c5i12, c5i34;
    DevBuf<int> c5binq;
    DevBuf<int4> c5items;
    int c5nitem = 0;
    DevBuf<int4> c5parts;        // multiplets of each item
    int c5npart = 0;
    DevBuf<int2> c5segs12, c5segs34;
    // 5PCF contraction with the P34 cache (npcf_contract5c.cu), where its shared memory fits
    DevBuf<int4> c5c_work;
    DevBuf<int> c5c_phase;
    DevBuf<int4> c5c_partners;
    int c5c_nphase = 0, c5c_slot = 0, c5c_bps = 0;
    bool c5c_ok = false, c5c_tabs_fit = false;   // tabs_fit: the tables fit in shared memory too
    int c5nterms12 = 0, c5nterms34 = 0, c5nseg12 = 0, c5nseg34 = 0;
    // 6PCF contraction tables
    DevBuf<int4> c6lam, c6lam2, c6terms1, c6terms2, c6terms3;
    DevBuf<int2> c6seg1, c6seg2, c6seg3, c6items;
    DevBuf<int> c6binq;
    int c6nitem = 0;

    // working buffers
    DevBuf<float4> pts;
    DevBuf<float> wp;
    DevBuf<uint32_t> idx, cell_of, cid;
    DevBuf<float2> alm;
    DevBuf<uint32_t> cnt;
    DevBuf<uint32_t> bucket;   // pair kernel: per-warp per-shell buckets of accepted pairs
    DevBuf<int4> stab;         // pair kernel: shell of r2 by bins (when stab_ok)
    int stab_ok = 0, stab_n = 0;
    float stab_scale = 0.f;
    DevBuf<uint32_t> count, start, cursor;
    DevBuf<double> partial, zeta, sumw, zscale;
    DevBuf<unsigned long long> counts;
    DevBuf<int> errflag, work;
    DevBuf<float> bbox;
    DevBuf<float> hpos_stage, hw_stage;
    // data harmonics kept across random splits (npcf_cache_data): the data positions and
    // weights (input order), their a_lm from the data alone and per-shell counts (input
    // order) and the data-data pair counts
    DevBuf<float> sd_pos, sd_w;
    DevBuf<float2> sd_alm;
    DevBuf<uint32_t> sd_cnt;
    DevBuf<unsigned long long> sd_counts;
    DevBuf<long long> sd_off;      // {0, n_data, 0, n_randoms}
    int64_t sd_n = 0;              // data points cached (0: none)
    // gridded fields: FFT plans, kernel spectra and work fields (created on first use)
    GridFFT* gfft = nullptr;
    // catalogs the accumulators hold (0: none yet; fixed by the first accumulate call)
    int ncat = 0;
    // tables of the current batch (host copies decide whether an upload is needed)
    DevBuf<long long> d_off;
    std::vector<long long> h_off;
    DevBuf<int2> chunks;
    std::vector<int2> h_chunks;
    DevBuf<int> cbeg;
    std::vector<int> h_cbeg;
    DevBuf<int2> chunks4;          // coarser chunks of the FP32 4PCF kernel
    std::vector<int2> h_chunks4;
    DevBuf<int> cbeg4;
    std::vector<int> h_cbeg4;
    // CUDA graph of the last batch shape
    cudaGraphExec_t gexec = nullptr;
    std::vector<uintptr_t> gsig;
    long long graph_launches = 0;
    // edge correction: sparse generalized Gaunt tables per order (built on first use)
    DevBuf<int> e_tptr[3], e_tlp[3];
    DevBuf<double> e_tg[3], e_out;
    bool edge_ready = false;
    int64_t last_n = 0;
    int nsm = 0;

    cudaEvent_t ev[5] = {};
    bool timed = false;
};

namespace {

npcf_status fail(npcf_ctx* c, npcf_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CU(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? NPCF_ENOMEM : NPCF_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                     \
    } while (0)

template <class T>
cudaError_t upload(DevBuf<T>& b, const std::vector<T>& v) {
    cudaError_t e = b.ensure(v.size());
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Tables of the tensor-core 4PCF contraction: rows (multiplet, b1, b2) grouped by
// (l3, parity), cut into 128-row tiles; one B slab per (group, component).
npcf_status setup_tc_tables(npcf_ctx* ctx, const OrderTable& o, const ContractTable4& t) {
    const int nr = ctx->nr;
    std::vector<int2> combos;
    std::vector<int> cbin;
    for (int b = 0; b < o.n_bins(); ++b) {
        const int* B = &o.bins[3 * b];
        if (B[2] != B[1] + 1) continue;
        combos.push_back(make_int2(B[0], B[1]));
        cbin.push_back(b);
    }
    std::vector<int4> groups, tiles;
    std::vector<int> glams, gbslab;
    int nbslab = 0, maxcomp = 0;
    for (int l3 = 0; l3 <= ctx->lmax; ++l3)
        for (int odd = 0; odd <= 1; ++odd) {
            std::vector<int> lams;
            for (int a = 0; a < o.n_lambda(); ++a)
                if (o.lam[3 * a + 2] == l3 && (int)o.odd(a) == odd) lams.push_back(a);
            if (lams.empty()) continue;
            const int g = (int)groups.size();
            const int ncomp = 2 * l3 + 1;
            groups.push_back(make_int4(l3, odd, (int)glams.size(), (int)lams.size()));
            gbslab.push_back(nbslab);
            glams.insert(glams.end(), lams.begin(), lams.end());
            const int rows = (int)lams.size() * (int)combos.size();
            for (int r0 = 0; r0 < rows; r0 += 128)
                tiles.push_back(make_int4(g, r0, std::min(128, rows - r0), nbslab));
            nbslab += ncomp;
            maxcomp = std::max(maxcomp, ncomp);
        }
    if (tiles.size() * 16 > 512 || groups.size() > 32)
        return fail(ctx, NPCF_EUNSUPPORTED, "split-bf16 4PCF: %zu accumulator tiles exceed tensor memory "
                    "(at most 32; use fewer shells, a lower lmax or parity-even multiplets)", tiles.size());
    (void)nr;
    // runs of a tile's rows sharing (multiplet, b1) with consecutive b2 (at most 4): the
    // P-build loads coefficients and a^{b1} once per run
    std::vector<int4> runs;
    std::vector<int> tile_run0;
    for (const int4& T : tiles) {
        tile_run0.push_back((int)runs.size());
        const int4& G = groups[T.x];
        int4 cur = make_int4(-1, 0, -1, -1);
        int prev_b2 = -1;
        for (int rr = 0; rr < T.z; ++rr) {
            const int grow = T.y + rr;
            const int lam = glams[G.z + grow / (int)combos.size()];
            const int2 bb = combos[grow % combos.size()];
            const bool same = cur.x >= 0 && cur.z == lam && (cur.w & 0xff) == bb.x && bb.y == prev_b2 + 1 &&
                              cur.y < 4;
            if (same) {
                ++cur.y;
            } else {
                if (cur.x >= 0) runs.push_back(cur);
                cur = make_int4(rr, 1, lam, bb.x | (bb.y << 8));
            }
            prev_b2 = bb.y;
        }
        if (cur.x >= 0) runs.push_back(cur);
        // longest first: groups take runs round-robin, so this keeps their row counts even
        std::stable_sort(runs.begin() + tile_run0.back(), runs.end(),
                         [](const int4& x, const int4& y) { return x.y > y.y; });
    }
    tile_run0.push_back((int)runs.size());
    CU(upload(ctx->tc_runs, runs));
    CU(upload(ctx->tc_tile_run0, tile_run0));
    ctx->tc_ngroup = (int)groups.size();
    ctx->tc_ntile = (int)tiles.size();
    ctx->tc_ncombo = (int)combos.size();
    ctx->tc_nbslab = nbslab;
    ctx->tc_maxcomp = maxcomp;
    CU(upload(ctx->tc_groups, groups));
    CU(upload(ctx->tc_tiles, tiles));
    CU(upload(ctx->tc_group_lams, glams));
    CU(upload(ctx->tc_group_bslab, gbslab));
    CU(upload(ctx->tc_combos, combos));
    CU(upload(ctx->tc_combo_bin, cbin));
    return NPCF_OK;
}

// Tables of the 5PCF contraction: the P12 and P34 coupling terms with their offsets in the
// staged tile, and items (multiplet, beta = b2 <= nr - 3) grouped by beta.
npcf_status setup_c5_tables(npcf_ctx* ctx, const OrderTable& o, int off) {
    const int nr = ctx->nr;
    if (nr > 10)
        return fail(ctx, NPCF_EUNSUPPORTED, "the 5PCF contraction supports at most 10 shells");
    ContractTable5 t = make_contract5(o);
    const int nb = o.n_bins();
    auto bin_index = [&](int b1, int b2, int b3, int b4) {
        for (int b = 0; b < nb; ++b) {
            const int* B = &o.bins[4 * b];
            if (B[0] == b1 && B[1] == b2 && B[2] == b3 && B[3] == b4) return b;
        }
        return -1;
    };
    // coupling terms with the offsets of their factors in the staged [lm][b][primary] tile
    std::vector<float4> c12, c34;
    std::vector<uint32_t> o12, o34;
    auto pack = [&](const std::vector<PairTerm>& in, std::vector<float4>& c, std::vector<uint32_t>& o) {
        for (const PairTerm& q : in) {
            c.push_back(make_float4(q.cA, q.cB, q.cC, q.cD));
            o.push_back((uint32_t)(q.lm1 * nr * kRS5) | ((uint32_t)(q.lm2 * nr * kRS5) << 16));
        }
    };
    pack(t.terms12, c12, o12);
    pack(t.terms34, c34, o34);
    std::vector<int2> s12, s34;
    for (size_t i = 0; i < t.seg12_begin.size(); ++i) s12.push_back(make_int2(t.seg12_begin[i], t.seg12_end[i]));
    for (size_t i = 0; i < t.seg34_begin.size(); ++i) s34.push_back(make_int2(t.seg34_begin[i], t.seg34_end[i]));
    // bin of (b1, b2, b2 + 1, b2 + 2): the first of the (b3, b4) pairs after b2
    std::vector<int> binq((size_t)nr * nr, 0);
    for (int b2 = 1; b2 + 2 < nr; ++b2)
        for (int b1 = 0; b1 < b2; ++b1) binq[(size_t)b1 * nr + b2] = bin_index(b1, b2, b2 + 1, b2 + 2);
    // items (up to c5_group multiplets sharing (l12 l3 l4), beta = b2), grouped by beta
    // (the kernel's specialisation), heaviest first
    std::vector<std::vector<int>> by34;
    for (int a = 0; a < o.n_lambda(); ++a) {
        const int t34 = t.lam_t34[a];
        if ((int)by34.size() <= t34) by34.resize(t34 + 1);
        by34[t34].push_back(a);
    }
    struct Item5 {
        double key;
        int4 head;
        std::vector<int4> parts;
    };
    std::vector<Item5> items;
    for (int t34 = 0; t34 < (int)by34.size(); ++t34) {
        const std::vector<int>& mult = by34[t34];
        if (mult.empty()) continue;
        const int l12 = o.lam[(size_t)mult[0] * 5 + 2];
        for (int beta = 1; beta + 2 < nr; ++beta) {
            const int m = nr - 1 - beta, G = c5_group(beta, m);
            for (size_t h0 = 0; h0 < mult.size(); h0 += G) {
                Item5 I;
                I.key = 0;
                const size_t h1 = std::min(mult.size(), h0 + G);
                for (int m12 = 0; m12 <= l12; ++m12) {
                    const int k34 = t.seg34_end[t.t34_seg0[t34] + m12] - t.seg34_begin[t.t34_seg0[t34] + m12];
                    I.key += k34 * m * (m - 1) / 2.0;
                    for (size_t h = h0; h < h1; ++h) {
                        const int t12 = t.lam_t12[mult[h]];
                        const int k12 = t.seg12_end[t.t12_seg0[t12] + m12] - t.seg12_begin[t.t12_seg0[t12] + m12];
                        I.key += k12 * beta + beta * m * (m - 1) / 2.0;
                    }
                }
                I.key += 1e12 * beta;
                I.head = make_int4(t.t34_seg0[t34], l12 | (beta << 8) | ((int)(h1 - h0) << 16), 0, 0);
                for (size_t h = h0; h < h1; ++h) {
                    const int a = mult[h];
                    I.parts.push_back(make_int4(t.t12_seg0[t.lam_t12[a]], off + a * nb, o.odd(a) ? 1 : 0, 0));
                }
                items.push_back(std::move(I));
            }
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const Item5& x, const Item5& y) { return x.key > y.key; });
    std::vector<int4> it, parts;
    for (Item5& x : items) {
        x.head.z = (int)parts.size();
        it.push_back(x.head);
        parts.insert(parts.end(), x.parts.begin(), x.parts.end());
    }
    {
        Contract5WArgs c{};
        c.nr = nr;
        c.nlm = ctx->nlm;
        c.nterms12 = (int)c12.size();
        c.nterms34 = (int)c34.size();
        c.nseg12 = (int)s12.size();
        c.nseg34 = (int)s34.size();
        int dev = 0, optin = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (!it.empty() && contract5w_smem_bytes(c) + 1024 > (size_t)optin)
            return fail(ctx, NPCF_EUNSUPPORTED, "5PCF: coupling tables and staged harmonics need %zu B of shared "
                        "memory (limit %d)", contract5w_smem_bytes(c), optin);
    }
    // P34-cache kernel: right triples packed into groups whose P34^{m12}(b3 < b4, b3 >= 2)
    // fit one cache slot; phase g holds the items of group g - 1 and the P34 builds of
    // group g (slots alternate), each list heaviest first
    ctx->c5c_ok = false;
    if (!it.empty()) {
        const int npall = (nr - 3) * (nr - 2) / 2;
        int maxsize = 0;
        for (int t34 = 0; t34 < (int)by34.size(); ++t34)
            if (!by34[t34].empty()) maxsize = std::max(maxsize, (t.t34_l12[t34] + 1) * npall);
        int dev = 0, optin = 0, per_sm = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CU(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        Contract5CArgs cc{};
        cc.nr = nr;
        cc.nlm = ctx->nlm;
        cc.slot_entries = 0;
        cc.nterms12 = (int)c12.size();
        cc.nterms34 = (int)c34.size();
        cc.nseg12 = (int)s12.size();
        cc.nseg34 = (int)s34.size();
        const long long base = (long long)contract5c_smem_bytes(cc) + (long long)contract5c_static_smem() + 1024;
        const long long entry2 = 2LL * kT5 * sizeof(float2);   // one entry in both slots
        const long long slot2 = (per_sm / 2 - base) / entry2, slot1 = (optin - base) / entry2;
        int slot = 0, bps = 0;
        if (slot2 >= maxsize) {
            slot = (int)slot2;
            bps = 2;
        } else if (slot1 >= maxsize) {
            slot = (int)slot1;
            bps = 1;
        }
        {
            // with the coupling terms in shared memory too (one block per SM), the slots take
            // the rest of the block's shared memory
            cc.tables_smem = 1;
            const long long baset = (long long)contract5c_smem_bytes(cc) + (long long)contract5c_static_smem() + 1024;
            const long long slott = (optin - baset) / entry2;
            ctx->c5c_tabs_fit = slott >= maxsize && maxsize > 0;
            if (ctx->c5c_tabs_fit) {
                slot = (int)slott;
                bps = (long long)2 * (base + entry2 * slott) <= per_sm ? 2 : 1;   // for the L1-terms kernel
            }
        }
        if (slot > 0 && maxsize > 0) {
            // right triples in order of l12, so that a group holds triples of one l12 and the
            // multiplets of a left triple in a group can share its P12
            std::vector<int> order34;
            for (int t34 = 0; t34 < (int)by34.size(); ++t34)
                if (!by34[t34].empty()) order34.push_back(t34);
            std::stable_sort(order34.begin(), order34.end(),
                             [&](int x, int y) { return t.t34_l12[x] < t.t34_l12[y]; });
            std::vector<std::vector<std::pair<double, int4>>> phase(1);
            std::vector<std::vector<int>> members(1);   // right triples of each group
            std::vector<int> tb34(by34.size(), 0);      // cache entry of each right triple
            int g = 0, used = 0;
            for (int t34 : order34) {
                const int l12 = t.t34_l12[t34], size = (l12 + 1) * npall;
                if (used + size > slot) {
                    ++g;
                    used = 0;
                    phase.emplace_back();
                    members.emplace_back();
                }
                tb34[t34] = used;
                used += size;
                members[g].push_back(t34);
                for (int m12 = 0; m12 <= l12; ++m12) {
                    const int sg = t.t34_seg0[t34] + m12;
                    const int k34 = t.seg34_end[sg] - t.seg34_begin[sg];
                    for (int b3 = 2; b3 + 1 < nr; ++b3)
                        phase[g].push_back({(double)k34 * (nr - 1 - b3),
                                            make_int4(sg, b3 | ((g & 1) << 24) | (1 << 30), tb34[t34] + m12 * npall, 0)});
                }
            }
            phase.resize(g + 2);
            std::vector<int4> partners;
            for (int gg = 0; gg <= g; ++gg) {
                // the group's multiplets by left triple
                std::vector<std::vector<int>> by12;
                for (int t34 : members[gg])
                    for (int a : by34[t34]) {
                        const int t12 = t.lam_t12[a];
                        if ((int)by12.size() <= t12) by12.resize(t12 + 1);
                        by12[t12].push_back(a);
                    }
                for (int t12 = 0; t12 < (int)by12.size(); ++t12) {
                    const std::vector<int>& mult = by12[t12];
                    if (mult.empty()) continue;
                    const int l12 = o.lam[(size_t)mult[0] * 5 + 2];
                    const int p0 = (int)partners.size();
                    for (int a : mult)
                        partners.push_back(make_int4(tb34[t.lam_t34[a]], off + a * nb, o.odd(a) ? 1 : 0, 0));
                    for (int beta = 1; beta + 2 < nr; ++beta) {
                        const int m = nr - 1 - beta, GM = c5c_group(beta, m);
                        double c12cost = 0;
                        for (int m12 = 0; m12 <= l12; ++m12) {
                            const int sg = t.t12_seg0[t12] + m12;
                            c12cost += 2.0 * (t.seg12_end[sg] - t.seg12_begin[sg]) * beta;
                        }
                        for (int h0 = 0; h0 < (int)mult.size(); h0 += GM) {
                            const int gcount = std::min(GM, (int)mult.size() - h0);
                            const double cost = c12cost + (l12 + 1) * gcount * beta * m * (m - 1) / 2.0;
                            phase[gg + 1].push_back(
                                {cost, make_int4(t.t12_seg0[t12], beta | (l12 << 16) | ((gg & 1) << 24) |
                                                                      ((gcount - 1) << 26),
                                                 p0 + h0, 0)});
                        }
                    }
                }
            }
            std::vector<int4> work;
            std::vector<int> pb;
            for (auto& ph : phase) {
                // P34 builds first, then the items by b2 (each b2 is its own specialisation of
                // the kernel: warps that run at the same time then share one code path in the
                // instruction cache), heaviest first within each
                auto kind = [](const int4& w) { return (w.y & (1 << 30)) ? 0 : 1 + (w.y & 0xff); };
                std::stable_sort(ph.begin(), ph.end(),
                                 [&](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                                     const int kx = kind(x.second), ky = kind(y.second);
                                     return kx != ky ? kx < ky : x.first > y.first;
                                 });
                pb.push_back((int)work.size());
                for (const auto& x : ph) work.push_back(x.second);
            }
            pb.push_back((int)work.size());
            ctx->c5c_nphase = (int)phase.size();
            ctx->c5c_slot = slot;
            ctx->c5c_bps = bps;
            CU(upload(ctx->c5c_work, work));
            CU(upload(ctx->c5c_phase, pb));
            CU(upload(ctx->c5c_partners, partners));
            ctx->c5c_ok = true;
        }
    }
    ctx->c5nitem = (int)it.size();
    ctx->c5npart = (int)parts.size();
    CU(upload(ctx->c5parts, parts));
    ctx->c5nterms12 = (int)c12.size();
    ctx->c5nterms34 = (int)c34.size();
    ctx->c5nseg12 = (int)s12.size();
    ctx->c5nseg34 = (int)s34.size();
    CU(upload(ctx->c5c12, c12));
    CU(upload(ctx->c5i12, o12));
    CU(upload(ctx->c5c34, c34));
    CU(upload(ctx->c5i34, o34));
    CU(upload(ctx->c5segs12, s12));
    CU(upload(ctx->c5segs34, s34));
    CU(upload(ctx->c5binq, binq));
    CU(upload(ctx->c5items, it));
    return NPCF_OK;
}

// 6PCF tables (npcf_contract6.cu): per multiplet L = (l1, l2, l12, l3, l123, l4, l5) the
// P12 terms of every m12, and for every m123 >= 0 the Q terms (m12, m3) and the P45 terms
// (m4, m5), with the 3-j symbols of Eq. basis-coupling and the phases (-1)^{l12 - m12}
// (in the P12 terms) and (-1)^{l123 - m123} (in the Q terms); harmonic rows lm = l^2 + l + m.
npcf_status setup_c6_tables(npcf_ctx* ctx, const OrderTable& o, int off) {
    const int nr = ctx->nr, nb = o.n_bins();
    if (nb == 0) return NPCF_OK;
    if (nr > 8) return fail(ctx, NPCF_EUNSUPPORTED, "6PCF: %d shells (the contraction takes at most 8)", nr);
    {
        Contract6Args c{};
        c.lmax = ctx->lmax;
        c.nr = nr;
        int dev = 0, optin = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (contract6_smem_bytes(c) + 1024 > (size_t)optin)
            return fail(ctx, NPCF_EUNSUPPORTED, "6PCF: lmax %d with %d shells needs %zu B of shared memory",
                        ctx->lmax, nr, contract6_smem_bytes(c));
    }
    auto lmf = [](int l, int m) { return l * l + l + m; };
    auto bits = [](double v) {
        const float f = (float)v;
        int b;
        std::memcpy(&b, &f, 4);
        return b;
    };
    std::vector<int4> lam, lam2, t1, t2, t3;
    std::vector<int2> seg1, seg2, seg3;
    for (int a = 0; a < o.n_lambda(); ++a) {
        const int* L = &o.lam[(size_t)a * 7];
        const int l1 = L[0], l2 = L[1], l12 = L[2], l3 = L[3], l123 = L[4], l4 = L[5], l5 = L[6];
        const int s1base = (int)seg1.size(), s23base = (int)seg2.size();
        for (int m12 = -l12; m12 <= l12; ++m12) {
            const int b = (int)t1.size();
            for (int m1 = -l1; m1 <= l1; ++m1) {
                const int m2 = m12 - m1;
                if (std::abs(m2) > l2) continue;
                const double c = (((l12 - m12) & 1) ? -1.0 : 1.0) * wigner3j(l1, l2, l12, m1, m2, -m12);
                if (c != 0.0) t1.push_back(make_int4(lmf(l1, m1), lmf(l2, m2), bits(c), 0));
            }
            seg1.push_back(make_int2(b, (int)t1.size()));
        }
        for (int m123 = 0; m123 <= l123; ++m123) {
            const int b2 = (int)t2.size();
            for (int m12 = -l12; m12 <= l12; ++m12) {
                const int m3 = m123 - m12;
                if (std::abs(m3) > l3) continue;
                const double c = (((l123 - m123) & 1) ? -1.0 : 1.0) * wigner3j(l12, l3, l123, m12, m3, -m123);
                if (c != 0.0) t2.push_back(make_int4(s1base + m12 + l12, lmf(l3, m3), bits(c), 0));
            }
            seg2.push_back(make_int2(b2, (int)t2.size()));
            const int b3 = (int)t3.size();
            for (int m4 = -l4; m4 <= l4; ++m4) {
                const int m5 = -m123 - m4;
                if (std::abs(m5) > l5) continue;
                const double c = wigner3j(l123, l4, l5, m123, m4, m5);
                if (c != 0.0) t3.push_back(make_int4(lmf(l4, m4), lmf(l5, m5), bits(c), 0));
            }
            seg3.push_back(make_int2(b3, (int)t3.size()));
        }
        lam.push_back(make_int4(l12, l123, o.odd(a) ? 1 : 0, off + a * nb));
        lam2.push_back(make_int4(s1base, s23base, bits(std::sqrt((2.0 * l12 + 1.0) * (2.0 * l123 + 1.0))), 0));
    }
    // bin index of (b1, b2, b3, b3 + 1, b3 + 2); the (b4, b5) pairs after b3 follow in order
    std::vector<int> binq((size_t)nr * nr * nr, 0);
    for (int b = 0; b < nb; ++b) {
        const int* B = &o.bins[(size_t)b * 5];
        if (B[3] == B[2] + 1 && B[4] == B[2] + 2) binq[((size_t)B[0] * nr + B[1]) * nr + B[2]] = b;
    }
    // items (L, b3), grouped by b3 (the kernel's specialisation), heaviest multiplets first
    std::vector<std::pair<double, int2>> items;
    for (int a = 0; a < o.n_lambda(); ++a) {
        double cost = 0.0;
        for (int q = lam2[a].y; q < lam2[a].y + lam[a].y + 1; ++q) {
            cost += seg3[q].y - seg3[q].x;
            for (int e = seg2[q].x; e < seg2[q].y; ++e) cost += 1 + seg1[t2[e].x].y - seg1[t2[e].x].x;
        }
        for (int b3 = 2; b3 <= nr - 3; ++b3) items.push_back({1e12 * (nr - b3) + cost, make_int2(a, b3)});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) { return x.first > y.first; });
    std::vector<int2> it;
    for (const auto& x : items) it.push_back(x.second);
    ctx->c6nitem = (int)it.size();
    CU(upload(ctx->c6lam, lam));
    CU(upload(ctx->c6lam2, lam2));
    CU(upload(ctx->c6seg1, seg1));
    CU(upload(ctx->c6seg2, seg2));
    CU(upload(ctx->c6seg3, seg3));
    CU(upload(ctx->c6terms1, t1));
    CU(upload(ctx->c6terms2, t2));
    CU(upload(ctx->c6terms3, t3));
    CU(upload(ctx->c6binq, binq));
    CU(upload(ctx->c6items, it));
    return NPCF_OK;
}

npcf_status setup_tables(npcf_ctx* ctx) {
    ctx->nlm = nlm(ctx->lmax);
    // Y_lm conversion matrix
    std::vector<double> K = ylm_chebyshev_matrix(ctx->lmax);
    std::vector<float> Kf(K.begin(), K.end());
    CU(upload(ctx->kmat, Kf));
    ctx->total = 0;
    for (int N = 3; N <= 6; ++N) {
        if (!(ctx->mask & (1u << N))) continue;
        ctx->orders.push_back(make_order(N, ctx->lmax, ctx->nr, ctx->allparity != 0));
        ctx->order_off.push_back(ctx->total);
        const OrderTable& o = ctx->orders.back();
        ctx->total += o.n_lambda() * o.n_bins();
    }
    // per output entry: the harmonic normalisation of its multiplet's N-1 factors
    std::vector<double> zs;
    zs.reserve(ctx->total);
    for (const OrderTable& o : ctx->orders)
        for (int L = 0; L < o.n_lambda(); ++L) {
            const int* l = &o.lam[(size_t)L * o.width];
            double f = 1.0;
            for (int k = 0; k < o.width; ++k)
                if (!((o.N == 5 && k == 2) || (o.N == 6 && (k == 2 || k == 4))))
                    f *= ylm_l_norm(l[k]);   // l12 and l123 couple, they are no harmonics
            zs.insert(zs.end(), o.n_bins(), f);
        }
    CU(upload(ctx->zscale, zs));
    for (size_t k = 0; k < ctx->orders.size(); ++k) {
        const OrderTable& o = ctx->orders[k];
        const int off = ctx->order_off[k];
        if (o.N == 3) {
            // items (l, b1) over the shells b2 > b1; the bins (b1, b2) are in lexicographic
            // order, so those of one b1 are consecutive
            // items ordered by b1 (the kernel's specialisation on the shells after b1), so
            // that warps running at the same time share one code path
            std::vector<int4> items;
            std::vector<float> coef;
            for (int l = 0; l <= ctx->lmax; ++l)
                // E(L) C^{ll}_{m,-m} (-1)^m = (l l 0; 0 0 0) for every m (Eq. N=3-coeff)
                coef.push_back((float)wigner3j(l, l, 0, 0, 0, 0));
            for (int b1 = 0; b1 + 1 < ctx->nr; ++b1)
                for (int l = 0; l <= ctx->lmax; ++l) {
                    int first = -1;
                    for (int b = 0; b < o.n_bins() && first < 0; ++b)
                        if (o.bins[2 * b] == b1 && o.bins[2 * b + 1] == b1 + 1) first = b;
                    const int nb2 = ctx->nr - 1 - b1;
                    for (int k = 0; k < nb2; ++k)
                        if (first < 0 || o.bins[2 * (first + k)] != b1 || o.bins[2 * (first + k) + 1] != b1 + 1 + k)
                            return fail(ctx, NPCF_EINVAL, "3PCF bins are not in lexicographic order");
                    items.push_back(make_int4(l, l * (l + 1) / 2, b1 | (nb2 << 16), l * o.n_bins() + first));
                }
            ctx->c3nitem = (int)items.size();
            CU(upload(ctx->c3items, items));
            CU(upload(ctx->c3coef, coef));
            (void)off;
        } else if (o.N == 4) {
            ContractTable4 t = make_contract4(o);
            const int nb = o.n_bins();
            std::vector<int4> segs;
            for (size_t i = 0; i < t.seg_begin.size(); ++i) {
                float f = t.seg_factor[i];
                int fb;
                std::memcpy(&fb, &f, 4);
                segs.push_back(make_int4(t.seg_begin[i], t.seg_end[i], t.seg_lm3[i], fb));
            }
            // items (multiplet, b1) with at least one (b2, b3) after b1, ordered by the number
            // of shells after b1 (the kernel's specialisation: warps that run at the same time
            // share one code path in the instruction cache), heaviest first within it
            std::vector<std::pair<double, int4>> items;
            for (int a = 0; a < o.n_lambda(); ++a)
                for (int b1 = 0; b1 + 2 < ctx->nr; ++b1) {
                    int first = -1;
                    for (int b = 0; b < nb && first < 0; ++b)
                        if (o.bins[3 * b] == b1 && o.bins[3 * b + 1] == b1 + 1 && o.bins[3 * b + 2] == b1 + 2)
                            first = b;
                    const int nb2 = ctx->nr - 1 - b1;
                    double cost = 0;
                    for (int sg = t.lam_seg0[a]; sg < t.lam_seg0[a + 1]; ++sg)
                        cost += 10.0 * nb2 * (t.seg_end[sg] - t.seg_begin[sg]) + 2.0 * nb2 * (nb2 - 1);
                    items.push_back({1e12 * nb2 + cost, make_int4(t.lam_seg0[a], t.lam_seg0[a + 1],
                                                     b1 | ((o.odd(a) ? 1 : 0) << 8) | (nb2 << 16),
                                                     off + a * nb + first)});
                }
            std::stable_sort(items.begin(), items.end(),
                             [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                                 return x.first > y.first;
                             });
            std::vector<int4> it;
            for (const auto& x : items) it.push_back(x.second);
            ctx->c4nitem = (int)it.size();
            ctx->c4nterms = (int)t.terms.size();
            ctx->c4nseg = (int)t.seg_begin.size();
            ctx->c4nlam = o.n_lambda();
            {
                Contract4WArgs c{};
                c.nr = ctx->nr;
                c.nlm = ctx->nlm;
                c.nterms = ctx->c4nterms;
                c.nseg = ctx->c4nseg;
                int dev = 0, optin = 0;
                CU(cudaGetDevice(&dev));
                CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
                ctx->c4g_needed = contract4w_smem_bytes(c) + 1024 > (size_t)optin;
                if (ctx->prec == NPCF_FP32 && ctx->c4g_needed &&
                    contract4g_smem_bytes(ctx->nr, ctx->nlm) + 1024 > (size_t)optin)
                    return fail(ctx, NPCF_EUNSUPPORTED, "4PCF: a tile of %d shells x %d harmonics needs %zu B of "
                                "shared memory (limit %d)", ctx->nr, ctx->nlm,
                                contract4g_smem_bytes(ctx->nr, ctx->nlm), optin);
            }
            if (ctx->prec == NPCF_FP32) {
                ContractTable4G tg = make_contract4g(t);
                std::vector<int4> itg;   // the same items over segment pairs
                for (const int4& x : it) {
                    int a = 0;
                    while (t.lam_seg0[a] != x.x) ++a;
                    itg.push_back(make_int4(tg.lam_pair0[a], tg.lam_pair0[a + 1], x.z, x.w));
                }
                std::vector<float4> cf(tg.tlm.size());
                std::vector<int4> gr(tg.groups.size() / 4), pr(tg.pairs.size() / 4);
                if (!cf.empty()) std::memcpy(cf.data(), tg.coef.data(), cf.size() * sizeof(float4));
                if (!gr.empty()) std::memcpy(gr.data(), tg.groups.data(), gr.size() * sizeof(int4));
                if (!pr.empty()) std::memcpy(pr.data(), tg.pairs.data(), pr.size() * sizeof(int4));
                CU(upload(ctx->c4g_coef, cf));
                CU(upload(ctx->c4g_tlm, tg.tlm));
                CU(upload(ctx->c4g_groups, gr));
                CU(upload(ctx->c4g_pairs, pr));
                CU(upload(ctx->c4g_items, itg));
            }
            CU(upload(ctx->c4terms, t.terms));
            CU(upload(ctx->c4segs, segs));
            CU(upload(ctx->c4items, it));
            CU(upload(ctx->c4lamseg0, t.lam_seg0));
            ctx->off4 = off;
            ctx->nb4 = nb;
            if (ctx->prec == NPCF_SPLIT_BF16) {
                npcf_status st = setup_tc_tables(ctx, o, t);
                if (st != NPCF_OK) return st;
            }
        } else if (o.N == 5) {
            npcf_status st = setup_c5_tables(ctx, o, off);
            if (st != NPCF_OK) return st;
        } else if (o.N == 6) {
            npcf_status st = setup_c6_tables(ctx, o, off);
            if (st != NPCF_OK) return st;
        }
    }
    return NPCF_OK;
}

npcf_status check_ctx(npcf_ctx* ctx) {
    if (!ctx) return NPCF_EINVAL;
    return NPCF_OK;
}

// Grid and neighbour rows for the current geometry.
// Cells per r_max when tuning key 0 is 0, from the mean number of neighbours within r_max
// of a primary, nbar 4/3 pi r_max^3 (nbar: points per catalog / volume). Coarse cells mean
// fewer neighbour rows per primary, which is what a sparse catalog pays for; finer ones cut
// the rows to the x-window more tightly. Measured on the pair kernel: 2 was best below ~600
// neighbours, 3 at ~3,400 (2 to 5 within 5 % there).
int auto_cells_per_rmax(double points, double volume, double rmax) {
    if (!(volume > 0) || !(points > 0)) return 5;
    const double nb = points / volume * (4.0 / 3.0) * M_PI * rmax * rmax * rmax;
    return nb < 630.0 ? 2 : 3;
}

npcf_status setup_grid(npcf_ctx* ctx, const float* d_pos, int n, int ncat, cudaStream_t s,
                       const float* d_pos2 = nullptr, int n2 = 0) {
    const double rmax = ctx->edges[ctx->nr];
    const double per_cat = (double)(n + (d_pos2 ? n2 : 0)) / std::max(ncat, 1);
    GridInfo g{};
    std::vector<int> rows;
    if (ctx->box > 0) {
        const int k = ctx->cells_per_rmax > 0 ? ctx->cells_per_rmax
                                              : auto_cells_per_rmax(per_cat, ctx->box * ctx->box * ctx->box, rmax);
        if (!plan_periodic_grid(ctx->box, rmax, k, 1 << 27, &g, &rows))
            return fail(ctx, NPCF_EINVAL, "box %.6g too small for r_max %.6g", ctx->box, rmax);
    } else {
        // bounding box of the catalog (one stream synchronisation)
        // (a second list of points, if given, is bounded together with the first)
        const int nb = d_pos2 && n2 > 0 ? 512 : 256;
        CU(ctx->bbox.ensure(nb * 6));
        launch_bbox(d_pos, n, ctx->bbox.p, 256, s);
        if (nb > 256) launch_bbox(d_pos2, n2, ctx->bbox.p + 256 * 6, 256, s);
        CU(cudaGetLastError());
        std::vector<float> part(nb * 6);
        CU(cudaMemcpyAsync(part.data(), ctx->bbox.p, nb * 6 * sizeof(float), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) {
            mn[a] = part[a];
            mx[a] = part[3 + a];
            for (int b = 1; b < nb; ++b) {
                mn[a] = std::min(mn[a], part[b * 6 + a]);
                mx[a] = std::max(mx[a], part[b * 6 + 3 + a]);
            }
            if (!std::isfinite(mn[a]) || !std::isfinite(mx[a]))
                return fail(ctx, NPCF_EINVAL, "non-finite positions");
        }
        double vol = 1.0;   // the bounding box (at least r_max on a side)
        for (int a = 0; a < 3; ++a) vol *= std::max((double)mx[a] - (double)mn[a], rmax);
        const int k = ctx->cells_per_rmax > 0 ? ctx->cells_per_rmax : auto_cells_per_rmax(per_cat, vol, rmax);
        plan_open_grid(mn, mx, rmax, k, 1 << 24, &g, &rows);
    }
    if (rows != ctx->rows_host) {
        ctx->rows_host = rows;
        std::vector<int4> r4;
        for (size_t i = 0; i < rows.size(); i += 4)
            r4.push_back(make_int4(rows[i], rows[i + 1], rows[i + 2], rows[i + 3]));
        CU(upload(ctx->rows, r4));
    }
    ctx->grid = g;
    return NPCF_OK;
}

// Host plan of one accumulate call: a single catalog is a batch of one.
struct Plan {
    int n = 0, ncat = 0, nchunk = 0, nchunk4 = 0;
    PairArgs pa{};
};

template <typename T>
bool same_table(const DevBuf<T>& b, const std::vector<T>& host, const std::vector<T>& v) {
    return b.p && host.size() == v.size() && std::memcmp(host.data(), v.data(), v.size() * sizeof(T)) == 0;
}

// Contraction chunks of a batch (primary ranges that never cross a catalog), the catalog
// offsets and the chunk rows of the FP64 partial sums.
npcf_status plan_chunks(npcf_ctx* ctx, const std::vector<long long>& off, Plan& P) {
    const long long n64 = off.back();
    const int ncat = (int)off.size() - 1;
    // contraction chunks of the 3PCF and 5PCF kernels: ranges of about n / (4 x SMs)
    // primaries (a multiple of 64), never crossing a catalog
    const int waves = 4;
    long long C = ctx->chunk_target > 0 ? ctx->chunk_target : (n64 + (long long)waves * ctx->nsm - 1) /
                                                                   ((long long)waves * ctx->nsm);
    C = std::max(64LL, (C + 63) / 64 * 64);
    std::vector<int2> chunks;
    std::vector<int> cbeg(1, 0);
    for (int k = 0; k < ncat; ++k) {
        for (long long p = off[k]; p < off[k + 1]; p += C)
            chunks.push_back(make_int2((int)p, (int)std::min(off[k + 1], p + C)));
        cbeg.push_back((int)chunks.size());
    }
    P.nchunk = (int)chunks.size();
    // the 4PCF kernels take a coarser table (about one chunk per SM and catalog, whole
    // 64-primary tiles): the FP32 kernel takes chunks dynamically and writes one FP64 row
    // per chunk, the tensor-core kernel keeps its accumulators for a whole chunk
    const long long C4 = ctx->chunk_target > 0 ? C : std::max(64LL, ((n64 + ctx->nsm - 1) / ctx->nsm + 63) / 64 * 64);
    std::vector<int2> chunks4;
    std::vector<int> cbeg4(1, 0);
    for (int k = 0; k < ncat; ++k) {
        for (long long p = off[k]; p < off[k + 1]; p += C4)
            chunks4.push_back(make_int2((int)p, (int)std::min(off[k + 1], p + C4)));
        cbeg4.push_back((int)chunks4.size());
    }
    P.nchunk4 = (int)chunks4.size();
    if (!same_table(ctx->chunks4, ctx->h_chunks4, chunks4)) {
        CU(upload(ctx->chunks4, chunks4));
        ctx->h_chunks4 = chunks4;
    }
    if (!same_table(ctx->cbeg4, ctx->h_cbeg4, cbeg4)) {
        CU(upload(ctx->cbeg4, cbeg4));
        ctx->h_cbeg4 = cbeg4;
    }
    if (!same_table(ctx->d_off, ctx->h_off, off)) {
        CU(upload(ctx->d_off, off));
        ctx->h_off = off;
    }
    if (!same_table(ctx->chunks, ctx->h_chunks, chunks)) {
        CU(upload(ctx->chunks, chunks));
        ctx->h_chunks = chunks;
    }
    if (!same_table(ctx->cbeg, ctx->h_cbeg, cbeg)) {
        CU(upload(ctx->cbeg, cbeg));
        ctx->h_cbeg = cbeg;
    }
    CU(ctx->partial.ensure((size_t)std::max({P.nchunk, P.nchunk4, 1}) * std::max(ctx->total, 1)));

    return NPCF_OK;
}

// Host part of an accumulate call: validation, grid, buffers and the tables of this batch
// (catalog offsets, contraction chunks). Uploads happen only when a table changes, so a
// repeated call with the same shapes does no synchronous work here.
npcf_status prepare(npcf_ctx* ctx, const float* d_pos, const float* d_w, const std::vector<long long>& off,
                    cudaStream_t s, Plan& P, const float* d_pos2 = nullptr, int n2 = 0) {
    const long long n64 = off.back();
    const int ncat = (int)off.size() - 1;
    if (n64 < 0 || n64 >= (int64_t(1) << 31)) return fail(ctx, NPCF_EINVAL, "n = %lld out of range", n64);
    if (n64 >= (int64_t(1) << 26))
        return fail(ctx, NPCF_EUNSUPPORTED, "n = %lld: the pair kernel indexes at most 2^26 points per call", n64);
    if (!d_pos || !d_w) return fail(ctx, NPCF_EINVAL, "null position or weight pointer");
    if (ctx->ncat != 0 && ctx->ncat != ncat)
        return fail(ctx, NPCF_EINVAL, "the accumulators hold %d catalogs, this call has %d (npcf_reset first)",
                    ctx->ncat, ncat);
    const int n = (int)n64;
    P.n = n;
    P.ncat = ncat;
    if (ctx->ncat == 0) {
        // the first call fixes how many catalogs the accumulators hold
        CU(ctx->zeta.ensure((size_t)ncat * std::max(ctx->total, 1)));
        CU(ctx->counts.ensure((size_t)ncat * ctx->nr));
        CU(ctx->sumw.ensure(ncat));
        if (ctx->total > 0) CU(cudaMemset(ctx->zeta.p, 0, (size_t)ncat * ctx->total * sizeof(double)));
        CU(cudaMemset(ctx->counts.p, 0, (size_t)ncat * ctx->nr * sizeof(unsigned long long)));
        CU(cudaMemset(ctx->sumw.p, 0, ncat * sizeof(double)));
        ctx->ncat = ncat;
    }
    npcf_status st = setup_grid(ctx, d_pos, d_pos2 ? n - n2 : n, ncat, s, d_pos2, n2);
    if (st != NPCF_OK) return st;
    const GridInfo& g = ctx->grid;
    const size_t cells = (size_t)g.ncell * ncat;
    if (cells >= (size_t)1 << 31) return fail(ctx, NPCF_EUNSUPPORTED, "%zu cells in the batch's grids", cells);

    CU(ctx->pts.ensure(n));
    CU(ctx->wp.ensure(n));
    CU(ctx->idx.ensure(n));
    CU(ctx->cell_of.ensure(n));
    CU(ctx->cid.ensure(n));
    CU(ctx->alm.ensure((size_t)n * ctx->nr * ctx->nlm));
    CU(ctx->cnt.ensure((size_t)n * ctx->nr));
    CU(ctx->count.ensure(cells));
    CU(ctx->start.ensure(cells + 1));
    CU(ctx->cursor.ensure(cells));
    CU(ctx->work.ensure(4));

    npcf_status cst = plan_chunks(ctx, off, P);
    if (cst != NPCF_OK) return cst;

    PairArgs& pa = P.pa;
    pa = PairArgs{};
    pa.pts = ctx->pts.p;
    pa.wp = ctx->wp.p;
    pa.cell_of = ctx->cell_of.p;
    pa.ppts = ctx->pts.p;
    pa.pwp = ctx->wp.p;
    pa.pcell = ctx->cell_of.p;
    pa.np = n;
    pa.add = 0;
    pa.cell_start = ctx->start.p;
    pa.rows = ctx->rows.p;
    pa.nrows = (int)(ctx->rows_host.size() / 4);
    pa.g = g;
    for (int i = 0; i <= ctx->nr; ++i) pa.e2[i] = ctx->e2[i];
    pa.nr = ctx->nr;
    pa.lmax = ctx->lmax;
    pa.kmat = ctx->kmat.p;
    pa.alm = ctx->alm.p;
    pa.cnt = ctx->cnt.p;
    pa.counts = ctx->counts.p;
    pa.ncat = ncat;
    pa.n = n;
    pa.work = ctx->work.p;
    pa.err = ctx->errflag.p;
    {
        // buckets: every shell at least kPairBucketMin entries (twice what one scan step
        // can add), the rest shared in proportion to the shell volumes (the expected share
        // of pairs of an unclustered catalog)
        const int nr = ctx->nr, C = std::max(ctx->pair_cap, kPairBucketMin * nr);
        const double e0 = ctx->edges[0], en = ctx->edges[nr];
        const double vtot = en * en * en - e0 * e0 * e0;
        const int spare = C - kPairBucketMin * nr;
        pa.boff[0] = 0;
        for (int t = 0; t < nr; ++t) {
            const double lo = ctx->edges[t], hi = ctx->edges[t + 1];
            const double f = (hi * hi * hi - lo * lo * lo) / vtot;
            pa.boff[t + 1] = pa.boff[t] + kPairBucketMin + (int)std::floor(f * spare);
        }
        CU(ctx->bucket.ensure((size_t)ctx->nsm * kPairWarps * pa.boff[nr]));
        pa.bucket = ctx->bucket.p;
    }
    {
        pa.chunk = ctx->pair_chunk;
        // linear shell edges allow a direct shell estimate (corrected exactly on the device)
        // (shells narrower than 1e-3 r_max take the binary search)
        const double r0 = ctx->edges[0], w = (ctx->edges[ctx->nr] - r0) / ctx->nr;
        bool lin = w >= 1e-3 * ctx->edges[ctx->nr];
        for (int i = 0; i <= ctx->nr && lin; ++i)
            lin = std::fabs(ctx->edges[i] - (r0 + i * w)) <= 1e-9 * ctx->edges[ctx->nr];
        pa.linear = lin ? 1 : 0;
        pa.lin_r0 = (float)r0;
        pa.lin_inv_w = lin ? (float)(1.0 / w) : 0.f;
        if (!ctx->stab.p && !ctx->stab_ok) {
            std::vector<int4> tab;
            float scale = 0.f;
            if (build_shell_table(ctx->e2, ctx->nr, kPairShellTab, &tab, &scale)) {
                CU(upload(ctx->stab, tab));
                ctx->stab_ok = 1;
                ctx->stab_n = (int)tab.size();
                ctx->stab_scale = scale;
            }
        }
        pa.tab_ok = ctx->stab_ok && ctx->use_stab;
        pa.tab_n = ctx->stab_n;
        pa.tab_scale = ctx->stab_scale;
        pa.tab = ctx->stab.p;
        // x-window cut of the staged rows: row cells are packed in 13 bits per axis
        const double cell = 1.0 / (double)g.inv_cell;
        double M = 0.0;
        const double o[3] = {g.ox, g.oy, g.oz};
        const int dims[3] = {g.gx, g.gy, g.gz};
        for (int q = 0; q < 3; ++q) M = std::max({M, std::fabs(o[q]), std::fabs(o[q] + dims[q] * cell)});
        pa.cell = (float)cell;
        pa.trim_margin = (float)std::max(cell * 1e-3, M * 4e-6);
        pa.trim = (ctx->trim && g.gy < 8192 && g.gz < 8192) ? 1 : 0;
    }
    {
        int dev = 0, optin = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const size_t need = pair_static_smem(ctx->lmax) + pair_dynamic_smem(pa);
        if (need > (size_t)optin)
            return fail(ctx, NPCF_EUNSUPPORTED, "pair kernel: %d neighbour rows need %zu B of shared memory "
                        "(limit %d B)", pa.nrows, need, optin);
    }
    if (ctx->prec == NPCF_SPLIT_BF16) {
        int dev = 0, optin = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        Contract4TCArgs c{};
        c.nr = ctx->nr;
        c.nlm = ctx->nlm;
        c.nterms = ctx->c4nterms;
        c.nseg = ctx->c4nseg;
        c.nlam = ctx->c4nlam;
        c.ncombo = ctx->tc_ncombo;
        c.maxcomp = ctx->tc_maxcomp;
        if (ctx->c4nitem > 0 && contract4_tc_smem_bytes(c) + 1024 > (size_t)optin)
            return fail(ctx, NPCF_EUNSUPPORTED, "split-bf16 4PCF: operands need %zu B of shared memory",
                        contract4_tc_smem_bytes(c));
    }
    ctx->last_n = n;
    return NPCF_OK;
}

npcf_status enqueue_contract(npcf_ctx* ctx, const Plan& P, cudaStream_t s, bool timed);

// Device part of an accumulate call: memsets and kernels only, all on stream s, so that a
// batch can be captured into a CUDA graph and replayed. Stage events only when timed.
npcf_status enqueue(npcf_ctx* ctx, const float* d_pos, const float* d_w, const float* d_wprim, const Plan& P,
                    cudaStream_t s, bool timed) {
    const GridInfo& g = ctx->grid;
    const int n = P.n, ncat = P.ncat;
    const size_t cells = (size_t)g.ncell * ncat;
    if (timed) CU(cudaEventRecord(ctx->ev[0], s));
    CU(cudaMemsetAsync(ctx->count.p, 0, cells * sizeof(uint32_t), s));
    CU(cudaMemsetAsync(ctx->work.p, 0, 4 * sizeof(int), s));
    launch_sumw(d_w, ctx->d_off.p, ncat, ctx->sumw.p, s);

    BinArgs b{};
    b.pos = d_pos;
    b.w = d_w;
    b.wprim = d_wprim;
    b.n = n;
    b.g = g;
    b.cid = ctx->cid.p;
    b.count = ctx->count.p;
    b.start = ctx->start.p;
    b.cursor = ctx->cursor.p;
    b.pts = ctx->pts.p;
    b.wp = ctx->wp.p;
    b.idx = ctx->idx.p;
    b.cell_of = ctx->cell_of.p;
    b.err = ctx->errflag.p;
    b.off = ctx->d_off.p;
    b.ncat = ncat;
    launch_bin(b, s);
    CU(cudaGetLastError());
    if (timed) CU(cudaEventRecord(ctx->ev[1], s));

    PairArgs pa = P.pa;
    pa.skip_zero = d_wprim != nullptr;
    launch_pair(pa, ctx->nsm, s);   // persistent: one block per SM, work units taken dynamically
    CU(cudaGetLastError());
    if (timed) CU(cudaEventRecord(ctx->ev[2], s));
    return enqueue_contract(ctx, P, s, timed);
}

// The contractions over the primaries of a plan (a4 to a6): every order's kernel into the
// chunk rows, then the FP64 reduction of each catalog's rows into its accumulators.
npcf_status enqueue_contract(npcf_ctx* ctx, const Plan& P, cudaStream_t s, bool timed) {
    const int n = P.n, ncat = P.ncat;
    for (size_t k = 0; k < ctx->orders.size(); ++k) {
        const OrderTable& o = ctx->orders[k];
        if (o.N == 3) {
            if (ctx->c3nitem == 0) continue;
            Contract3Args c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.lmax = ctx->lmax;
            c.chunks = ctx->chunks.p;
            c.nchunk = P.nchunk;
            c.items = ctx->c3items.p;
            c.nitem = ctx->c3nitem;
            c.coef = ctx->c3coef.p;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.out_off = ctx->order_off[k];
            c.nout = (ctx->lmax + 1) * o.n_bins();
            launch_contract3(c, s);
        } else if (o.N == 4 && ctx->prec == NPCF_SPLIT_BF16) {
            if (ctx->c4nitem == 0) continue;
            Contract4TCArgs c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.chunks = ctx->chunks4.p;
            c.terms = ctx->c4terms.p;
            c.nterms = ctx->c4nterms;
            c.segs = ctx->c4segs.p;
            c.nseg = ctx->c4nseg;
            c.lam_seg0 = ctx->c4lamseg0.p;
            c.nlam = ctx->c4nlam;
            c.groups = ctx->tc_groups.p;
            c.group_lams = ctx->tc_group_lams.p;
            c.ngroup = ctx->tc_ngroup;
            c.tiles = ctx->tc_tiles.p;
            c.ntile = ctx->tc_ntile;
            c.runs = ctx->tc_runs.p;
            c.tile_run0 = ctx->tc_tile_run0.p;
            c.combos = ctx->tc_combos.p;
            c.combo_bin = ctx->tc_combo_bin.p;
            c.ncombo = ctx->tc_ncombo;
            c.group_bslab = ctx->tc_group_bslab.p;
            c.nbslab = ctx->tc_nbslab;
            c.maxcomp = ctx->tc_maxcomp;
            c.off4 = ctx->off4;
            c.nb4 = ctx->nb4;
            c.drain_steps = ctx->drain_steps;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.err = ctx->errflag.p;
            launch_contract4_tc(c, P.nchunk4, s);
        } else if (o.N == 4 && (ctx->c4g_needed || ctx->c4g_force)) {
            if (ctx->c4nitem == 0) continue;
            Contract4GArgs c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.coef = ctx->c4g_coef.p;
            c.tlm = ctx->c4g_tlm.p;
            c.groups = ctx->c4g_groups.p;
            c.pairs = ctx->c4g_pairs.p;
            c.items = ctx->c4g_items.p;
            c.nitem = ctx->c4nitem;
            c.chunks = ctx->chunks4.p;
            c.nchunk = P.nchunk4;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.out_off = ctx->order_off[k];
            c.nout = o.n_lambda() * o.n_bins();
            c.chunk_counter = ctx->work.p + 1;
            launch_contract4g(c, contract4w_blocks(ctx->nsm, P.nchunk4), s);
        } else if (o.N == 4) {
            if (ctx->c4nitem == 0) continue;
            Contract4WArgs c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.terms = ctx->c4terms.p;
            c.nterms = ctx->c4nterms;
            c.segs = ctx->c4segs.p;
            c.nseg = ctx->c4nseg;
            c.items = ctx->c4items.p;
            c.nitem = ctx->c4nitem;
            c.chunks = ctx->chunks4.p;
            c.nchunk = P.nchunk4;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.out_off = ctx->order_off[k];
            c.nout = o.n_lambda() * o.n_bins();
            c.chunk_counter = ctx->work.p + 1;
            launch_contract4w(c, contract4w_blocks(ctx->nsm, P.nchunk4), s);
        } else if (o.N == 5) {
            if (ctx->c5nitem == 0) continue;
            const bool tabs = ctx->c5c_tabs_fit && (ctx->c5_mode == 0 || ctx->c5_mode == 3);
            const bool cached = ctx->c5_mode == 0 || ctx->c5_mode == 2 || (ctx->c5_mode == 3 && tabs);
            if (ctx->c5c_ok && cached) {
                Contract5CArgs c{};
                c.alm = ctx->alm.p;
                c.wp = ctx->wp.p;
                c.n = n;
                c.nr = ctx->nr;
                c.nlm = ctx->nlm;
                c.c12 = ctx->c5c12.p;
                c.o12 = ctx->c5i12.p;
                c.c34 = ctx->c5c34.p;
                c.o34 = ctx->c5i34.p;
                c.segs12 = ctx->c5segs12.p;
                c.segs34 = ctx->c5segs34.p;
                c.binq = ctx->c5binq.p;
                c.work = ctx->c5c_work.p;
                c.phase_begin = ctx->c5c_phase.p;
                c.partners = ctx->c5c_partners.p;
                c.nphase = ctx->c5c_nphase;
                c.slot_entries = ctx->c5c_slot;
                c.blocks_per_sm = ctx->c5c_bps;
                c.tables_smem = tabs ? 1 : 0;
                c.nterms12 = ctx->c5nterms12;
                c.nterms34 = ctx->c5nterms34;
                c.nseg12 = ctx->c5nseg12;
                c.nseg34 = ctx->c5nseg34;
                c.chunks = ctx->chunks.p;
                c.nchunk = P.nchunk;
                c.partial = ctx->partial.p;
                c.total = ctx->total;
                c.out_off = ctx->order_off[k];
                c.nout = o.n_lambda() * o.n_bins();
                c.chunk_counter = ctx->work.p + 2;
                launch_contract5c(c, std::max(1, std::min((tabs ? 1 : ctx->c5c_bps) * ctx->nsm, P.nchunk)), s);
                continue;
            }
            Contract5WArgs c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.c12 = ctx->c5c12.p;
            c.o12 = ctx->c5i12.p;
            c.c34 = ctx->c5c34.p;
            c.o34 = ctx->c5i34.p;
            c.segs12 = ctx->c5segs12.p;
            c.segs34 = ctx->c5segs34.p;
            c.nterms12 = ctx->c5nterms12;
            c.nterms34 = ctx->c5nterms34;
            c.nseg12 = ctx->c5nseg12;
            c.nseg34 = ctx->c5nseg34;
            c.binq = ctx->c5binq.p;
            c.items = ctx->c5items.p;
            c.nitem = ctx->c5nitem;
            c.partners = ctx->c5parts.p;
            c.npartner = ctx->c5npart;
            c.chunks = ctx->chunks.p;
            c.nchunk = P.nchunk;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.out_off = ctx->order_off[k];
            c.nout = o.n_lambda() * o.n_bins();
            c.chunk_counter = ctx->work.p + 2;
            launch_contract5w(c, std::max(1, std::min(2 * ctx->nsm, P.nchunk)), s);
        } else if (o.N == 6) {
            if (ctx->c6nitem == 0) continue;
            Contract6Args c{};
            c.alm = ctx->alm.p;
            c.wp = ctx->wp.p;
            c.n = n;
            c.nr = ctx->nr;
            c.nlm = ctx->nlm;
            c.lmax = ctx->lmax;
            c.lam = ctx->c6lam.p;
            c.lam2 = ctx->c6lam2.p;
            c.seg1 = ctx->c6seg1.p;
            c.terms1 = ctx->c6terms1.p;
            c.seg2 = ctx->c6seg2.p;
            c.terms2 = ctx->c6terms2.p;
            c.seg3 = ctx->c6seg3.p;
            c.terms3 = ctx->c6terms3.p;
            c.binq = ctx->c6binq.p;
            c.items = ctx->c6items.p;
            c.nitem = ctx->c6nitem;
            c.chunks = ctx->chunks.p;
            c.nchunk = P.nchunk;
            c.partial = ctx->partial.p;
            c.total = ctx->total;
            c.out_off = ctx->order_off[k];
            c.nout = o.n_lambda() * o.n_bins();
            c.chunk_counter = ctx->work.p + 3;
            launch_contract6(c, std::max(1, std::min(2 * ctx->nsm, P.nchunk)), s);
        }
        CU(cudaGetLastError());
    }
    if (timed) CU(cudaEventRecord(ctx->ev[3], s));
    for (size_t k = 0; k < ctx->orders.size(); ++k) {
        const OrderTable& o = ctx->orders[k];
        const bool coarse = o.N == 4;   // both 4PCF kernels use the coarse chunk table
        launch_reduce(ctx->partial.p, coarse ? ctx->cbeg4.p : ctx->cbeg.p, ncat, ctx->total, ctx->order_off[k],
                      o.n_lambda() * o.n_bins(), ctx->zscale.p, ctx->zeta.p, s);
    }
    CU(cudaGetLastError());
    if (timed) CU(cudaEventRecord(ctx->ev[4], s));
    return NPCF_OK;
}

npcf_status run_accumulate(npcf_ctx* ctx, const float* d_pos, const float* d_w, const float* d_wprim,
                           int64_t n64, cudaStream_t s) {
    if (n64 < 0 || n64 >= (int64_t(1) << 31)) return fail(ctx, NPCF_EINVAL, "n = %lld out of range", (long long)n64);
    if (n64 == 0) return NPCF_OK;
    Plan P;
    npcf_status st = prepare(ctx, d_pos, d_w, std::vector<long long>{0, (long long)n64}, s, P);
    if (st != NPCF_OK) return st;
    return enqueue(ctx, d_pos, d_w, d_wprim, P, s, ctx->timed);
}

// Batch: catalog k holds points off[k] .. off[k+1] of d_pos / d_w. The device work is
// captured into a CUDA graph on the first call with a given shape; later calls with the
// same pointers, offsets, tuning and context buffers replay the graph (one launch). The
// legacy default stream cannot be captured: there the work is enqueued directly.
npcf_status run_batch(npcf_ctx* ctx, const float* d_pos, const float* d_w, const float* d_wprim,
                      const std::vector<long long>& off, cudaStream_t s) {
    if (!(ctx->box > 0))
        return fail(ctx, NPCF_EUNSUPPORTED, "batches take periodic boxes (one grid shape for every catalog)");
    for (size_t k = 0; k + 1 < off.size(); ++k)
        if (off[k + 1] < off[k]) return fail(ctx, NPCF_EINVAL, "batch offsets must not decrease");
    if (off.front() != 0) return fail(ctx, NPCF_EINVAL, "batch offsets must start at 0");
    Plan P;
    npcf_status st = prepare(ctx, d_pos, d_w, off, s, P);
    if (st != NPCF_OK) return st;
    if (P.n == 0) return NPCF_OK;
    if (s == 0 || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return enqueue(ctx, d_pos, d_w, d_wprim, P, s, false);
    // everything the captured work depends on
    std::vector<uintptr_t> sig = {
        (uintptr_t)d_pos, (uintptr_t)d_w, (uintptr_t)d_wprim, (uintptr_t)ctx->pts.p, (uintptr_t)ctx->wp.p, (uintptr_t)ctx->idx.p,
        (uintptr_t)ctx->cell_of.p, (uintptr_t)ctx->cid.p, (uintptr_t)ctx->alm.p, (uintptr_t)ctx->cnt.p,
        (uintptr_t)ctx->count.p, (uintptr_t)ctx->start.p, (uintptr_t)ctx->cursor.p, (uintptr_t)ctx->work.p,
        (uintptr_t)ctx->partial.p, (uintptr_t)ctx->zeta.p, (uintptr_t)ctx->counts.p, (uintptr_t)ctx->sumw.p,
        (uintptr_t)ctx->d_off.p, (uintptr_t)ctx->chunks.p, (uintptr_t)ctx->cbeg.p, (uintptr_t)ctx->rows.p,
        (uintptr_t)ctx->chunks4.p, (uintptr_t)ctx->cbeg4.p, (uintptr_t)P.nchunk4,
        (uintptr_t)P.n, (uintptr_t)P.ncat, (uintptr_t)P.nchunk, (uintptr_t)P.pa.chunk, (uintptr_t)P.pa.bucket, (uintptr_t)P.pa.boff[ctx->nr],
        (uintptr_t)P.pa.trim, (uintptr_t)P.pa.tab_ok, (uintptr_t)ctx->cells_per_rmax, (uintptr_t)ctx->drain_steps,
        (uintptr_t)ctx->c4g_force, (uintptr_t)ctx->c5_mode};
    for (long long v : off) sig.push_back((uintptr_t)v);
    if (ctx->gexec && sig == ctx->gsig) {
        CU(cudaGraphLaunch(ctx->gexec, s));
        ++ctx->graph_launches;
        return NPCF_OK;
    }
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        ctx->gsig.clear();
    }
    CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    st = enqueue(ctx, d_pos, d_w, d_wprim, P, s, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != NPCF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    CU(e);
    const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    CU(ei);
    ctx->gsig = sig;
    CU(cudaGraphLaunch(ctx->gexec, s));
    ++ctx->graph_launches;
    return NPCF_OK;
}

// One list of points binned into a region of the context's buffers: sorted points, weights,
// input index and cell from first; cell counts, starts and cursors from cell0 (ncell + 1
// starts per list).
void bin_list(npcf_ctx* ctx, const float* pos, const float* w, int n, int first, size_t cell0,
              const long long* d_off, cudaStream_t s) {
    BinArgs b{};
    b.pos = pos;
    b.w = w;
    b.wprim = nullptr;
    b.n = n;
    b.g = ctx->grid;
    b.cid = ctx->cid.p + first;
    b.count = ctx->count.p + cell0;
    b.start = ctx->start.p + cell0 + cell0 / ctx->grid.ncell;   // ncell + 1 starts per list
    b.cursor = ctx->cursor.p + cell0;
    b.pts = ctx->pts.p + first;
    b.wp = ctx->wp.p + first;
    b.idx = ctx->idx.p + first;
    b.cell_of = ctx->cell_of.p + first;
    b.err = ctx->errflag.p;
    b.off = d_off;
    b.ncat = 1;
    launch_bin(b, s);
}

// Data-minus-randoms split with the data harmonics kept from npcf_cache_data (Sec. 4.2):
// the data (n_d points, cached) and this split's randoms (n_r) are binned as two lists on one
// grid; a_lm of the data primaries = cached data part + the randoms as secondaries; a_lm of the
// random primaries = the data as secondaries + the randoms as secondaries; then the usual
// contractions over all n_d + n_r primaries.
npcf_status run_split(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n_r, cudaStream_t s) {
    if (ctx->sd_n <= 0) return fail(ctx, NPCF_EINVAL, "no cached data: call npcf_cache_data first");
    if (n_r < 0) return fail(ctx, NPCF_EINVAL, "negative number of randoms");
    if (n_r > 0 && (!d_pos || !d_w)) return fail(ctx, NPCF_EINVAL, "null position or weight pointer");
    if (ctx->ncat > 1) return fail(ctx, NPCF_EINVAL, "the accumulators hold a batch (npcf_reset first)");
    const int n_d = (int)ctx->sd_n;
    const long long N = (long long)n_d + n_r;
    Plan P;
    npcf_status st = prepare(ctx, ctx->sd_pos.p, ctx->sd_w.p, std::vector<long long>{0, N}, s, P,
                             n_r > 0 ? d_pos : nullptr, (int)n_r);
    if (st != NPCF_OK) return st;
    const size_t cells = (size_t)ctx->grid.ncell;
    CU(ctx->count.ensure(2 * cells));
    CU(ctx->start.ensure(2 * cells + 2));
    CU(ctx->cursor.ensure(2 * cells));
    const bool timed = ctx->timed;
    if (timed) CU(cudaEventRecord(ctx->ev[0], s));
    launch_set4(ctx->sd_off.p, 0, n_d, 0, n_r, s);   // the two lists' ranges
    CU(cudaMemsetAsync(ctx->count.p, 0, 2 * cells * sizeof(uint32_t), s));
    CU(cudaMemsetAsync(ctx->work.p, 0, 4 * sizeof(int), s));
    launch_sumw(ctx->sd_w.p, ctx->sd_off.p, 1, ctx->sumw.p, s);
    if (n_r > 0) launch_sumw(d_w, ctx->sd_off.p + 2, 1, ctx->sumw.p, s);
    bin_list(ctx, ctx->sd_pos.p, ctx->sd_w.p, n_d, 0, 0, ctx->sd_off.p, s);
    bin_list(ctx, d_pos, d_w, (int)n_r, n_d, cells, ctx->sd_off.p + 2, s);
    CU(cudaGetLastError());
    if (timed) CU(cudaEventRecord(ctx->ev[1], s));
    const int row = ctx->nr * ctx->nlm;
    launch_alm_from_input(ctx->sd_alm.p, ctx->sd_cnt.p, ctx->idx.p, n_d, row, ctx->nr, ctx->alm.p, ctx->cnt.p, s);
    // the three passes: (data, randoms) added to the cached part, (randoms, data), (randoms, randoms) added
    const uint32_t* start_d = ctx->start.p;
    const uint32_t* start_r = ctx->start.p + cells + 1;
    struct Pass { int prim0, np, sec0, nsec; const uint32_t* start; int add; };
    const Pass passes[3] = {{0, n_d, n_d, (int)n_r, start_r, 1},
                            {n_d, (int)n_r, 0, n_d, start_d, 0},
                            {n_d, (int)n_r, n_d, (int)n_r, start_r, 1}};
    for (const Pass& q : passes) {
        if (q.np == 0 || q.nsec == 0) continue;
        CU(cudaMemsetAsync(ctx->work.p, 0, sizeof(int), s));
        PairArgs pa = P.pa;
        pa.ppts = ctx->pts.p + q.prim0;
        pa.pwp = ctx->wp.p + q.prim0;
        pa.pcell = ctx->cell_of.p + q.prim0;
        pa.np = q.np;
        pa.pts = ctx->pts.p + q.sec0;
        pa.wp = ctx->wp.p + q.sec0;
        pa.cell_of = ctx->cell_of.p + q.sec0;
        pa.cell_start = q.start;
        pa.alm = ctx->alm.p + (size_t)q.prim0 * row;
        pa.cnt = ctx->cnt.p + (size_t)q.prim0 * ctx->nr;
        pa.add = q.add;
        pa.skip_zero = 0;
        launch_pair(pa, ctx->nsm, s);
        CU(cudaGetLastError());
    }
    launch_add_counts(ctx->counts.p, ctx->sd_counts.p, ctx->nr, s);
    if (timed) CU(cudaEventRecord(ctx->ev[2], s));
    return enqueue_contract(ctx, P, s, timed);
}

}  // namespace

extern "C" {

npcf_status npcf_create(npcf_ctx** out, int lmax, unsigned order_mask, int nr, const double* edges,
                        double box, int prec, int allparity) {
    if (!out) return NPCF_EINVAL;
    *out = nullptr;
    npcf_ctx* ctx = new (std::nothrow) npcf_ctx();
    if (!ctx) return NPCF_ENOMEM;
    auto bad = [&](npcf_status s) {
        // the message stays readable through npcf_last_error(NULL)
        g_create_error = ctx->err;
        delete ctx;
        return s;
    };
    if (lmax < 0 || lmax > kMaxL) return bad(fail(ctx, NPCF_EINVAL, "lmax %d outside [0, %d]", lmax, kMaxL));
    if (nr < 1 || nr > kMaxNr) return bad(fail(ctx, NPCF_EINVAL, "nr %d outside [1, %d]", nr, kMaxNr));
    if (!edges) return bad(fail(ctx, NPCF_EINVAL, "edges is null"));
    if ((order_mask & ~((1u << 3) | (1u << 4) | (1u << 5) | (1u << 6))) || order_mask == 0)
        return bad(fail(ctx, NPCF_EINVAL, "order_mask 0x%x must select orders among 3, 4, 5, 6", order_mask));
    if (prec != NPCF_FP32 && prec != NPCF_SPLIT_BF16)
        return bad(fail(ctx, NPCF_EINVAL, "unknown precision %d", prec));
    for (int i = 0; i <= nr; ++i)
        if (!std::isfinite(edges[i]) || edges[i] < 0 || (i > 0 && !(edges[i] > edges[i - 1])))
            return bad(fail(ctx, NPCF_EINVAL, "edges must be finite, >= 0 and strictly increasing"));
    if (!(box >= 0) || !std::isfinite(box)) return bad(fail(ctx, NPCF_EINVAL, "box must be >= 0"));
    if (box > 0 && !(edges[nr] * 3.0 < box))
        return bad(fail(ctx, NPCF_EINVAL, "periodic box %.6g must exceed 3 r_max (%.6g)", box, edges[nr]));
    ctx->lmax = lmax;
    ctx->nr = nr;
    ctx->mask = order_mask;
    ctx->box = box;
    ctx->prec = prec;
    ctx->allparity = allparity ? 1 : 0;
    ctx->edges.assign(edges, edges + nr + 1);
    for (int i = 0; i <= nr; ++i) ctx->e2[i] = (float)(edges[i] * edges[i]);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bad(fail(ctx, NPCF_ECUDA, "no CUDA device"));
    npcf_status st = setup_tables(ctx);
    if (st != NPCF_OK) return bad(st);
    if (ctx->zeta.ensure(ctx->total) != cudaSuccess || ctx->counts.ensure(nr) != cudaSuccess ||
        ctx->errflag.ensure(1) != cudaSuccess || ctx->sumw.ensure(1) != cudaSuccess)
        return bad(fail(ctx, NPCF_ENOMEM, "device allocation failed"));
    for (auto& e : ctx->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bad(fail(ctx, NPCF_ECUDA, "event creation failed"));
    ctx->timed = true;
    st = npcf_reset(ctx);
    if (st != NPCF_OK) return bad(st);
    *out = ctx;
    return NPCF_OK;
}

npcf_status npcf_reset(npcf_ctx* ctx) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    const size_t k = (size_t)std::max(ctx->ncat, 1);
    if (ctx->total > 0) CU(cudaMemset(ctx->zeta.p, 0, k * ctx->total * sizeof(double)));
    CU(cudaMemset(ctx->counts.p, 0, k * ctx->nr * sizeof(unsigned long long)));
    CU(cudaMemset(ctx->errflag.p, 0, sizeof(int)));
    CU(cudaMemset(ctx->sumw.p, 0, k * sizeof(double)));
    ctx->ncat = 0;   // the next accumulate call fixes the number of catalogs again
    return NPCF_OK;
}

npcf_status npcf_accumulate(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    return run_accumulate(ctx, d_pos, d_w, nullptr, n, (cudaStream_t)stream);
}

npcf_status npcf_accumulate_ex(npcf_ctx* ctx, const float* d_pos, const float* d_w, const float* d_wprim,
                               int64_t n, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    return run_accumulate(ctx, d_pos, d_w, d_wprim, n, (cudaStream_t)stream);
}

npcf_status npcf_accumulate_host(npcf_ctx* ctx, const float* h_pos, const float* h_w, int64_t n,
                                 void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(ctx, NPCF_EINVAL, "n out of range");
    if (n == 0) return NPCF_OK;
    if (!h_pos || !h_w) return fail(ctx, NPCF_EINVAL, "null host pointer");
    cudaStream_t s = (cudaStream_t)stream;
    CU(ctx->hpos_stage.ensure((size_t)n * 3));
    CU(ctx->hw_stage.ensure((size_t)n));
    CU(cudaMemcpyAsync(ctx->hpos_stage.p, h_pos, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->hw_stage.p, h_w, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
    npcf_status st = run_accumulate(ctx, ctx->hpos_stage.p, ctx->hw_stage.p, nullptr, n, s);
    if (st != NPCF_OK) return st;
    CU(cudaStreamSynchronize(s));
    return NPCF_OK;
}

npcf_status npcf_cache_data(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (n <= 0 || n >= (int64_t(1) << 26)) return fail(ctx, NPCF_EINVAL, "n = %lld outside [1, 2^26)", (long long)n);
    if (!d_pos || !d_w) return fail(ctx, NPCF_EINVAL, "null position or weight pointer");
    if (ctx->ncat > 1) return fail(ctx, NPCF_EINVAL, "the accumulators hold a batch (npcf_reset first)");
    cudaStream_t s = (cudaStream_t)stream;
    CU(ctx->sd_pos.ensure((size_t)3 * n));
    CU(ctx->sd_w.ensure((size_t)n));
    CU(cudaMemcpyAsync(ctx->sd_pos.p, d_pos, (size_t)3 * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(ctx->sd_w.p, d_w, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    Plan P;
    npcf_status st = prepare(ctx, ctx->sd_pos.p, ctx->sd_w.p, std::vector<long long>{0, n}, s, P);
    if (st != NPCF_OK) return st;
    const int row = ctx->nr * ctx->nlm;
    CU(ctx->sd_alm.ensure((size_t)n * row));
    CU(ctx->sd_cnt.ensure((size_t)n * ctx->nr));
    CU(ctx->sd_counts.ensure(ctx->nr));
    CU(ctx->sd_off.ensure(4));
    launch_set4(ctx->sd_off.p, 0, n, 0, 0, s);
    const size_t cells = (size_t)ctx->grid.ncell;
    CU(cudaMemsetAsync(ctx->count.p, 0, cells * sizeof(uint32_t), s));
    CU(cudaMemsetAsync(ctx->work.p, 0, 4 * sizeof(int), s));
    CU(cudaMemsetAsync(ctx->sd_counts.p, 0, ctx->nr * sizeof(unsigned long long), s));
    bin_list(ctx, ctx->sd_pos.p, ctx->sd_w.p, (int)n, 0, 0, ctx->sd_off.p, s);
    PairArgs pa = P.pa;
    pa.counts = ctx->sd_counts.p;   // the data-data counts are added by every split
    pa.skip_zero = 0;
    launch_pair(pa, ctx->nsm, s);
    launch_alm_to_input(ctx->alm.p, ctx->cnt.p, ctx->idx.p, (int)n, row, ctx->nr, ctx->sd_alm.p, ctx->sd_cnt.p, s);
    CU(cudaGetLastError());
    ctx->sd_n = n;
    return NPCF_OK;
}

npcf_status npcf_accumulate_split(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    return run_split(ctx, d_pos, d_w, n, (cudaStream_t)stream);
}

npcf_status npcf_accumulate_grid(npcf_ctx* ctx, const float* d_delta, int ngrid, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (!(ctx->box > 0)) return fail(ctx, NPCF_EUNSUPPORTED, "gridded fields need a periodic box");
    if (ngrid < 1 || ngrid > 406) return fail(ctx, NPCF_EINVAL, "ngrid %d outside [1, 406]", ngrid);
    if (!d_delta) return fail(ctx, NPCF_EINVAL, "null field pointer");
    if (ctx->ncat > 1) return fail(ctx, NPCF_EINVAL, "the accumulators hold a batch (npcf_reset first)");
    cudaStream_t s = (cudaStream_t)stream;
    const long long cells = (long long)ngrid * ngrid * ngrid;
    if (ctx->ncat == 0) {
        CU(ctx->zeta.ensure(std::max(ctx->total, 1)));
        CU(ctx->counts.ensure(ctx->nr));
        CU(ctx->sumw.ensure(1));
        if (ctx->total > 0) CU(cudaMemset(ctx->zeta.p, 0, (size_t)ctx->total * sizeof(double)));
        CU(cudaMemset(ctx->counts.p, 0, (size_t)ctx->nr * sizeof(unsigned long long)));
        CU(cudaMemset(ctx->sumw.p, 0, sizeof(double)));
        ctx->ncat = 1;
    }
    Plan P;
    P.n = (int)cells;
    P.ncat = 1;
    npcf_status st = plan_chunks(ctx, std::vector<long long>{0, cells}, P);
    if (st != NPCF_OK) return st;
    CU(ctx->alm.ensure((size_t)cells * ctx->nr * ctx->nlm));
    CU(ctx->wp.ensure((size_t)cells));
    CU(ctx->work.ensure(4));
    if (!ctx->gfft) ctx->gfft = gridfft_create();
    GridFFTArgs ga{};
    for (int i = 0; i <= ctx->nr; ++i) ga.e2[i] = ctx->e2[i];
    ga.nr = ctx->nr;
    ga.lmax = ctx->lmax;
    const bool timed = ctx->timed;
    if (timed) CU(cudaEventRecord(ctx->ev[0], s));
    if (timed) CU(cudaEventRecord(ctx->ev[1], s));
    CU(cudaMemsetAsync(ctx->work.p, 0, 4 * sizeof(int), s));
    char msg[256] = {};
    const int rc = gridfft_alm(ctx->gfft, d_delta, ngrid, (float)ctx->box, ga, ctx->alm.p, ctx->wp.p, s, msg, sizeof(msg));
    if (rc != 0) return fail(ctx, rc == 2 ? NPCF_ENOMEM : NPCF_ECUDA, "gridded a_lm: %s", msg);
    ctx->last_n = 0;   // the a_lm of this call are cells', not particles' (no npcf_debug_alm)
    if (timed) CU(cudaEventRecord(ctx->ev[2], s));
    return enqueue_contract(ctx, P, s, timed);
}

npcf_status npcf_output_size(const npcf_ctx* ctx, size_t* len) {
    if (!ctx || !len) return NPCF_EINVAL;
    *len = (size_t)ctx->total;
    return NPCF_OK;
}

npcf_status npcf_truncate(const npcf_ctx* ctx, const double* in, size_t in_len, int lmax_out, double* out,
                          size_t* out_len) {
    if (!ctx || !out_len) return NPCF_EINVAL;
    if (lmax_out < 0 || lmax_out > ctx->lmax) return NPCF_EINVAL;
    // the multiplets an lmax_out context holds are those of this one whose l's fit
    auto keep = [&](const OrderTable& o, int a) {
        const int* L = &o.lam[(size_t)a * o.width];
        for (int k = 0; k < o.width; ++k) {
            // l12 and l123 couple two l's
            const int cap = ((o.N == 5 && k == 2) || (o.N == 6 && (k == 2 || k == 4))) ? 2 * lmax_out : lmax_out;
            if (L[k] > cap) return false;
        }
        return true;
    };
    size_t need = 0;
    for (const OrderTable& o : ctx->orders)
        for (int a = 0; a < o.n_lambda(); ++a)
            if (keep(o, a)) need += (size_t)o.n_bins();
    if (!out) {
        *out_len = need;
        return NPCF_OK;
    }
    if (!in || in_len != (size_t)ctx->total || *out_len != need) return NPCF_EINVAL;
    size_t src = 0, dst = 0;
    for (const OrderTable& o : ctx->orders) {
        const size_t nb = (size_t)o.n_bins();
        for (int a = 0; a < o.n_lambda(); ++a, src += nb)
            if (keep(o, a)) {
                std::memcpy(out + dst, in + src, nb * sizeof(double));
                dst += nb;
            }
    }
    return NPCF_OK;
}

npcf_status npcf_layout(const npcf_ctx* ctx, int order, int* n_lambda, int* n_bins, int* lambdas, int* bins) {
    if (!ctx) return NPCF_EINVAL;
    for (const OrderTable& o : ctx->orders) {
        if (o.N != order) continue;
        if (n_lambda) *n_lambda = o.n_lambda();
        if (n_bins) *n_bins = o.n_bins();
        if (lambdas) std::memcpy(lambdas, o.lam.data(), o.lam.size() * sizeof(int));
        if (bins) std::memcpy(bins, o.bins.data(), o.bins.size() * sizeof(int));
        return NPCF_OK;
    }
    return NPCF_EINVAL;
}

}  // extern "C"

namespace {

// Copy ncopy catalogs' multiplets (synchronises); normalise catalog k with its own sum of
// weights when asked.
npcf_status finalize_catalogs(npcf_ctx* ctx, double* out, int ncopy, int normalize) {
    CU(cudaDeviceSynchronize());
    int errbits = 0;
    CU(cudaMemcpy(&errbits, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (errbits & 1) return fail(ctx, NPCF_EINVAL, "positions outside [0, box) or not finite");
    if (errbits & 2) return fail(ctx, NPCF_ETIMEOUT, "a bounded device wait gave up; results are incomplete");
    if (ctx->total == 0 || ncopy == 0) return NPCF_OK;
    if (ctx->ncat == 0) {
        std::memset(out, 0, (size_t)ncopy * ctx->total * sizeof(double));
        return NPCF_OK;
    }
    CU(cudaMemcpy(out, ctx->zeta.p, (size_t)ncopy * ctx->total * sizeof(double), cudaMemcpyDeviceToHost));
    if (!normalize) return NPCF_OK;
    if (!(ctx->box > 0)) return fail(ctx, NPCF_EUNSUPPORTED, "normalisation needs a periodic box");
    std::vector<double> sumw(ncopy);
    CU(cudaMemcpy(sumw.data(), ctx->sumw.p, ncopy * sizeof(double), cudaMemcpyDeviceToHost));
    const double V = ctx->box * ctx->box * ctx->box;
    const double fourpi = 4.0 * M_PI;
    std::vector<double> vb(ctx->nr);
    for (int b = 0; b < ctx->nr; ++b)
        vb[b] = fourpi / 3.0 * (std::pow(ctx->edges[b + 1], 3) - std::pow(ctx->edges[b], 3));
    for (int c = 0; c < ncopy; ++c) {
        const double nbar = sumw[c] / V;
        double* oc = out + (size_t)c * ctx->total;
        for (size_t k = 0; k < ctx->orders.size(); ++k) {
            const OrderTable& o = ctx->orders[k];
            const int N = o.N, nb = o.n_bins();
            const double R0 = std::pow(fourpi, -(N - 1) / 2.0) * std::pow(nbar, N);
            for (int a = 0; a < o.n_lambda(); ++a)
                for (int b = 0; b < nb; ++b) {
                    double vB = V;
                    for (int q = 0; q < N - 1; ++q) vB *= vb[o.bins[(size_t)b * (N - 1) + q]];
                    oc[ctx->order_off[k] + a * nb + b] /= vB * R0;
                }
        }
    }
    return NPCF_OK;
}

}  // namespace

extern "C" {

npcf_status npcf_finalize(npcf_ctx* ctx, double* out, size_t out_len, int normalize) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if ((!out && ctx->total > 0) || out_len < (size_t)ctx->total)
        return fail(ctx, NPCF_EINVAL, "output buffer too small");
    if (ctx->ncat > 1) return fail(ctx, NPCF_EINVAL, "the context holds a batch: use npcf_finalize_batch");
    return finalize_catalogs(ctx, out, 1, normalize);
}

npcf_status npcf_finalize_batch(npcf_ctx* ctx, double* out, size_t out_len, int normalize) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    const int k = std::max(ctx->ncat, 1);
    if ((!out && ctx->total > 0) || out_len < (size_t)k * ctx->total)
        return fail(ctx, NPCF_EINVAL, "output buffer too small (%d catalogs x %d)", k, ctx->total);
    return finalize_catalogs(ctx, out, k, normalize);
}

npcf_status npcf_accumulate_batch(npcf_ctx* ctx, const float* d_pos, const float* d_w, const int64_t* offsets,
                                  int ncat, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (ncat < 1 || ncat > 65535 || !offsets) return fail(ctx, NPCF_EINVAL, "ncat must be in [1, 65535]");
    std::vector<long long> off(offsets, offsets + ncat + 1);
    return run_batch(ctx, d_pos, d_w, nullptr, off, (cudaStream_t)stream);
}

npcf_status npcf_accumulate_batch_ex(npcf_ctx* ctx, const float* d_pos, const float* d_w, const float* d_wprim,
                                     const int64_t* offsets, int ncat, void* stream) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (ncat < 1 || ncat > 65535 || !offsets) return fail(ctx, NPCF_EINVAL, "ncat must be in [1, 65535]");
    std::vector<long long> off(offsets, offsets + ncat + 1);
    return run_batch(ctx, d_pos, d_w, d_wprim, off, (cudaStream_t)stream);
}

npcf_status npcf_autotune(npcf_ctx* ctx, const float* d_pos, const float* d_w, int64_t n, void* stream,
                          int* chosen) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (ctx->ncat != 0) return fail(ctx, NPCF_EINVAL, "autotune needs empty accumulators (npcf_reset first)");
    if (n <= 0 || !d_pos || !d_w) return fail(ctx, NPCF_EINVAL, "autotune needs a non-empty catalog");
    cudaStream_t s = (cudaStream_t)stream;
    const bool was_timed = ctx->timed;
    ctx->timed = true;
    // median of three timed runs of one stage (after one warm-up run)
    auto stage_ms = [&](int stage, float* ms) -> npcf_status {
        float t[3];
        for (int r = 0; r < 4; ++r) {
            npcf_status st = run_accumulate(ctx, d_pos, d_w, nullptr, n, s);
            if (st != NPCF_OK) return st;
            CU(cudaEventSynchronize(ctx->ev[stage + 1]));
            if (r > 0) CU(cudaEventElapsedTime(&t[r - 1], ctx->ev[stage], ctx->ev[stage + 1]));
        }
        std::sort(t, t + 3);
        *ms = t[1];
        return NPCF_OK;
    };
    const int keep[4] = {ctx->cells_per_rmax, ctx->pair_chunk, ctx->pair_cap, ctx->chunk_target};
    int best[4] = {keep[0], keep[1], keep[2], keep[3]};
    float best_ms = 1e30f;
    // pair kernel: grid cell size, primaries per chunk, bucket entries per warp
    for (int k : {2, 3, 4, 5, 6})
        for (int run : {8, 16, 32, 64})
            for (int cap : {4096, 8192}) {
                ctx->cells_per_rmax = k;
                ctx->pair_chunk = run;
                ctx->pair_cap = cap;
                float ms = 0.f;
                if (stage_ms(1, &ms) != NPCF_OK) continue;   // e.g. no room to stage: skip
                if (ms < best_ms) {
                    best_ms = ms;
                    best[0] = k;
                    best[1] = run;
                    best[2] = cap;
                }
            }
    ctx->cells_per_rmax = best[0];
    ctx->pair_chunk = best[1];
    ctx->pair_cap = best[2];
    // contractions: primaries per chunk (waves of chunks over the SMs)
    best_ms = 1e30f;
    for (int waves : {1, 2, 4, 8}) {
        ctx->chunk_target = (int)std::max<int64_t>(64, (n + (int64_t)waves * ctx->nsm - 1) / ((int64_t)waves * ctx->nsm));
        float ms = 0.f;
        if (stage_ms(2, &ms) != NPCF_OK) continue;
        if (ms < best_ms) {
            best_ms = ms;
            best[3] = ctx->chunk_target;
        }
    }
    ctx->chunk_target = best[3];
    ctx->timed = was_timed;
    npcf_status st = npcf_reset(ctx);
    if (st != NPCF_OK) return st;
    if (best_ms >= 1e30f) {
        ctx->cells_per_rmax = keep[0];
        ctx->pair_chunk = keep[1];
        ctx->pair_cap = keep[2];
        ctx->chunk_target = keep[3];
        return fail(ctx, NPCF_EINVAL, "autotune: no candidate setting ran");
    }
    if (chosen)
        for (int i = 0; i < 4; ++i) chosen[i] = best[i];
    return NPCF_OK;
}

npcf_status npcf_batch_info(const npcf_ctx* ctx, int* ncat, int64_t* graph_launches) {
    if (!ctx) return NPCF_EINVAL;
    if (ncat) *ncat = ctx->ncat;
    if (graph_launches) *graph_launches = ctx->graph_launches;
    return NPCF_OK;
}

npcf_status npcf_pair_counts_batch(npcf_ctx* ctx, uint64_t* out, size_t out_len) {
    if (check_ctx(ctx) != NPCF_OK || !out) return NPCF_EINVAL;
    const int k = std::max(ctx->ncat, 1);
    if (out_len < (size_t)k * ctx->nr) return fail(ctx, NPCF_EINVAL, "output buffer too small");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(out, ctx->counts.p, (size_t)k * ctx->nr * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return NPCF_OK;
}

npcf_status npcf_pair_counts(npcf_ctx* ctx, uint64_t* out) {
    if (check_ctx(ctx) != NPCF_OK || !out) return NPCF_EINVAL;
    if (ctx->ncat > 1) return fail(ctx, NPCF_EINVAL, "the context holds a batch: use npcf_pair_counts_batch");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(out, ctx->counts.p, ctx->nr * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return NPCF_OK;
}

npcf_status npcf_gaunt(int N, const int* L1, const int* L2, const int* L3, double* out) {
    if (N < 3 || N > 5 || !L1 || !L2 || !L3 || !out) return NPCF_EINVAL;
    const int width = N == 3 ? 2 : (N == 4 ? 3 : 5);
    for (int i = 0; i < width; ++i)
        if (L1[i] < 0 || L2[i] < 0 || L3[i] < 0 || L1[i] > 4 * kMaxL || L2[i] > 4 * kMaxL || L3[i] > 4 * kMaxL)
            return NPCF_EINVAL;
    *out = generalized_gaunt(N, L1, L2, L3);
    return NPCF_OK;
}

npcf_status npcf_multiplets(int N, int lmax, int allparity, int* count, int* out) {
    if (N < 3 || N > 6 || lmax < 0 || lmax > kMaxL || !count) return NPCF_EINVAL;
    const OrderTable o = make_order(N, lmax, N - 1, allparity != 0);
    *count = o.n_lambda();
    if (out) std::memcpy(out, o.lam.data(), o.lam.size() * sizeof(int));
    return NPCF_OK;
}

npcf_status npcf_coupling(int N, const int* L, const int* M, double* out) {
    if (N < 3 || N > 6 || !L || !M || !out) return NPCF_EINVAL;
    const int width = N == 3 ? 2 : (N == 4 ? 3 : (N == 5 ? 5 : 7));
    for (int i = 0; i < width; ++i)
        if (L[i] < 0 || L[i] > 4 * kMaxL) return NPCF_EINVAL;
    for (int i = 0; i < N - 1; ++i)
        if (M[i] < -4 * kMaxL || M[i] > 4 * kMaxL) return NPCF_EINVAL;
    *out = coupling(N, L, M);
    return NPCF_OK;
}

npcf_status npcf_edge_correct(npcf_ctx* nctx, npcf_ctx* rctx, double* out) {
    if (check_ctx(nctx) != NPCF_OK || check_ctx(rctx) != NPCF_OK) return NPCF_EINVAL;
    npcf_ctx* ctx = nctx;   // CUDA failures are reported on the data context
    if (!out && nctx->total > 0) return fail(nctx, NPCF_EINVAL, "output buffer is null");
    if (nctx->lmax != rctx->lmax || nctx->mask != rctx->mask || nctx->nr != rctx->nr ||
        nctx->box != rctx->box || nctx->allparity != rctx->allparity || nctx->edges != rctx->edges)
        return fail(nctx, NPCF_EINVAL, "the two contexts differ in lmax, orders, shells or box");
    if (nctx->allparity) return fail(nctx, NPCF_EUNSUPPORTED, "edge correction takes parity-even multiplets");
    if (nctx->ncat > 1 || rctx->ncat > 1) return fail(nctx, NPCF_EINVAL, "edge correction takes single catalogs");
    for (const OrderTable& o : nctx->orders)
        if (o.N >= 5) return fail(nctx, NPCF_EUNSUPPORTED, "edge correction is built for orders 3 and 4");
    CU(cudaDeviceSynchronize());
    int errbits = 0, rerr = 0;
    CU(cudaMemcpy(&errbits, nctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&rerr, rctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if ((errbits | rerr) & 3) return fail(nctx, NPCF_EINVAL, "an accumulate call of either context failed");
    if (!nctx->edge_ready) {
        for (size_t k = 0; k < nctx->orders.size(); ++k) {
            const OrderTable& o = nctx->orders[k];
            const int nl = o.n_lambda(), w = o.width;
            // G is symmetric in its three multiplets: evaluate a <= b <= c once
            std::vector<double> G((size_t)nl * nl * nl, 0.0);
            for (int a = 0; a < nl; ++a)
                for (int b = a; b < nl; ++b)
                    for (int c = b; c < nl; ++c) {
                        const double g = generalized_gaunt(o.N, &o.lam[(size_t)a * w], &o.lam[(size_t)b * w],
                                                           &o.lam[(size_t)c * w]);
                        const int p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
                        for (const auto& q : p) G[((size_t)q[0] * nl + q[1]) * nl + q[2]] = g;
                    }
            // entry M[L''][L] collects (L', G^{L L' L''}) over L'
            std::vector<int> tptr(1, 0), tlp;
            std::vector<double> tg;
            for (int c = 0; c < nl; ++c)
                for (int a = 0; a < nl; ++a) {
                    for (int b = 0; b < nl; ++b) {
                        const double g = G[((size_t)a * nl + b) * nl + c];
                        if (std::fabs(g) > 1e-15) { tlp.push_back(b); tg.push_back(g); }
                    }
                    tptr.push_back((int)tlp.size());
                }
            CU(upload(nctx->e_tptr[k], tptr));
            CU(upload(nctx->e_tlp[k], tlp));
            CU(upload(nctx->e_tg[k], tg));
        }
        nctx->edge_ready = true;
    }
    if (nctx->total == 0) return NPCF_OK;
    CU(nctx->e_out.ensure(nctx->total));
    CU(cudaMemset(nctx->errflag.p, 0, sizeof(int)));
    int dev = 0, optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (size_t k = 0; k < nctx->orders.size(); ++k) {
        const OrderTable& o = nctx->orders[k];
        if (o.n_bins() == 0) continue;
        if (edge_smem_bytes(o.n_lambda()) > (size_t)optin)
            return fail(nctx, NPCF_EUNSUPPORTED, "edge correction: %d multiplets exceed shared memory",
                        o.n_lambda());
        EdgeArgs e{};
        e.nraw = nctx->zeta.p + nctx->order_off[k];
        e.rraw = rctx->zeta.p + rctx->order_off[k];
        e.nl = o.n_lambda();
        e.nb = o.n_bins();
        e.tptr = nctx->e_tptr[k].p;
        e.tlp = nctx->e_tlp[k].p;
        e.tg = nctx->e_tg[k].p;
        e.out = nctx->e_out.p + nctx->order_off[k];
        e.err = nctx->errflag.p;
        launch_edge_solve(e, 0);
        CU(cudaGetLastError());
    }
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(out, nctx->e_out.p, nctx->total * sizeof(double), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&errbits, nctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemset(nctx->errflag.p, 0, sizeof(int)));
    if (errbits & 4) return fail(nctx, NPCF_EINVAL, "edge correction: singular system (R_0 = 0?) for some bins");
    return NPCF_OK;
}

npcf_status npcf_debug_alm(npcf_ctx* ctx, const int64_t* idx, int64_t k, float* alm, uint32_t* counts) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    if (k < 0 || (k > 0 && (!idx || !alm))) return fail(ctx, NPCF_EINVAL, "bad arguments");
    if (k == 0) return NPCF_OK;
    const int n = (int)ctx->last_n;
    if (n == 0) return fail(ctx, NPCF_EINVAL, "no accumulate call yet");
    CU(cudaDeviceSynchronize());
    std::vector<uint32_t> sidx(n);
    CU(cudaMemcpy(sidx.data(), ctx->idx.p, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    std::vector<int> inv(n, -1);
    for (int q = 0; q < n; ++q) inv[sidx[q]] = q;
    const int per = ctx->nr * ctx->nlm;
    for (int64_t q = 0; q < k; ++q) {
        if (idx[q] < 0 || idx[q] >= n) return fail(ctx, NPCF_EINVAL, "index out of range");
        const int sp = inv[idx[q]];
        float* dst = alm + q * per * 2;
        CU(cudaMemcpy(dst, ctx->alm.p + (size_t)sp * per, per * sizeof(float2), cudaMemcpyDeviceToHost));
        // the device holds reduced harmonics: restore sqrt((2l+1)/(4 pi))
        for (int b = 0; b < ctx->nr; ++b)
            for (int l = 0; l <= ctx->lmax; ++l)
                for (int m = 0; m <= l; ++m) {
                    const size_t e = 2 * ((size_t)b * ctx->nlm + lm_index(l, m));
                    dst[e] = (float)(dst[e] * ylm_l_norm(l));
                    dst[e + 1] = (float)(dst[e + 1] * ylm_l_norm(l));
                }
        if (counts)
            CU(cudaMemcpy(counts + q * ctx->nr, ctx->cnt.p + (size_t)sp * ctx->nr, ctx->nr * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost));
    }
    return NPCF_OK;
}

npcf_status npcf_set_tuning(npcf_ctx* ctx, int key, int value) {
    if (check_ctx(ctx) != NPCF_OK) return NPCF_EINVAL;
    switch (key) {
        case 0:
            if (value < 0 || value > 8)
                return fail(ctx, NPCF_EINVAL, "cells per r_max in [1, 8], or 0 for the density rule");
            ctx->cells_per_rmax = value;
            return NPCF_OK;
        case 2:
            if (value < 0) return fail(ctx, NPCF_EINVAL, "chunk must be >= 0");
            ctx->chunk_target = value;
            return NPCF_OK;
        case 3:
            // every shell's bucket gets at least kPairBucketMin = 512 entries (a scan step
            // appends at most 256 per shell, and a bucket with less room is summed first)
            if (value < 1024 || value > 65536 || (value % 256) || value < kPairBucketMin * ctx->nr)
                return fail(ctx, NPCF_EINVAL, "pair bucket entries per warp must be a multiple of 256 in "
                            "[max(1024, %d x shells), 65536]", kPairBucketMin);
            ctx->pair_cap = value;
            return NPCF_OK;
        case 4:
            if (value != 0 && value != 1) return fail(ctx, NPCF_EINVAL, "high-lmax 4PCF contraction is 0 or 1");
            ctx->c4g_force = value;
            return NPCF_OK;
        case 9:
            if (value < 0 || value > 3) return fail(ctx, NPCF_EINVAL, "5PCF contraction mode in [0, 3]");
            ctx->c5_mode = value;
            return NPCF_OK;
        case 5:
            if (value < 1 || value > 1024) return fail(ctx, NPCF_EINVAL, "primaries per chunk in [1, 1024]");
            ctx->pair_chunk = value;
            return NPCF_OK;
        case 6:
            if (value < 1) return fail(ctx, NPCF_EINVAL, "drain interval must be >= 1");
            ctx->drain_steps = value;
            return NPCF_OK;
        case 7:
            if (value != 0 && value != 1) return fail(ctx, NPCF_EINVAL, "x-window cut is 0 or 1");
            ctx->trim = value;
            return NPCF_OK;
        case 8:
            if (value != 0 && value != 1) return fail(ctx, NPCF_EINVAL, "shell table is 0 or 1");
            ctx->use_stab = value;
            return NPCF_OK;
        default:
            return fail(ctx, NPCF_EINVAL, "unknown tuning key %d", key);
    }
}

npcf_status npcf_get_timings(npcf_ctx* ctx, float* ms4) {
    if (check_ctx(ctx) != NPCF_OK || !ms4) return NPCF_EINVAL;
    for (int i = 0; i < 4; ++i) {
        ms4[i] = 0.f;
        CU(cudaEventSynchronize(ctx->ev[i + 1]));
        CU(cudaEventElapsedTime(&ms4[i], ctx->ev[i], ctx->ev[i + 1]));
    }
    return NPCF_OK;
}

const char* npcf_last_error(const npcf_ctx* ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

void npcf_destroy(npcf_ctx* ctx) {
    if (!ctx) return;
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gfft) gridfft_destroy(ctx->gfft);
    delete ctx;  // device buffers are released by their destructors
}

}  // extern "C"
