// Host-side planning of the neighbour-search grid, shared by every entry point.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "npcf_device.h"

namespace npcf {

std::vector<int> neighbour_rows(float cell, double rmax, int* reach) {
    // rows (dy, dz, dx_lo, dx_hi) of cells that may hold a point within rmax of some point
    // of the centre cell; cell-box gaps get a small slack so that points put in a
    // neighbouring cell by rounding are never missed
    const double slack = 1e-3 * cell;
    const double r2 = rmax * (1.0 + 1e-6) * rmax * (1.0 + 1e-6);
    const int R = (int)std::ceil(rmax / cell) + 1;
    auto gap = [&](int d) {
        double gg = (std::abs(d) - 1) * (double)cell - slack;
        return gg > 0 ? gg : 0.0;
    };
    std::vector<int> out;
    int rmaxd = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy) {
            const double gyz = gap(dy) * gap(dy) + gap(dz) * gap(dz);
            if (gyz > r2) continue;
            int X = 0;
            while (X + 1 <= R && gyz + gap(X + 1) * gap(X + 1) <= r2) ++X;
            out.insert(out.end(), {dy, dz, -X, X});
            rmaxd = std::max(rmaxd, std::max(X, std::max(std::abs(dy), std::abs(dz))));
        }
    *reach = rmaxd;
    return out;
}

bool plan_periodic_grid(double L, double rmax, int cells_per_rmax, int max_cells, GridInfo* g,
                        std::vector<int>* rows) {
    // the preferred cells per r_max first, then finer, then coarser grids; a grid is valid
    // when no neighbour offset reaches the same cell twice (2 reach + 1 <= cells per side)
    std::vector<int> order;
    for (int q = cells_per_rmax; q <= 16; ++q) order.push_back(q);
    for (int q = cells_per_rmax - 1; q >= 1; --q) order.push_back(q);
    for (int q : order) {
        // 0.999: r_max / cell is never an integer, so rows at exactly r_max drop out
        int gg = (int)std::floor(L * q / rmax * 0.999);
        gg = std::max(1, std::min(gg, 1024));
        if ((double)gg * gg * gg > (double)max_cells) continue;
        const float cell = (float)(L / gg);
        int reach = 0;
        std::vector<int> r = neighbour_rows(cell, rmax, &reach);
        if (2 * reach + 1 > gg) continue;
        g->gx = g->gy = g->gz = gg;
        g->ox = g->oy = g->oz = 0.f;
        g->inv_cell = (float)(gg / L);
        g->periodic = 1;
        g->L = (float)L;
        g->hL = (float)(0.5 * L);
        g->ncell = gg * gg * gg;
        *rows = r;
        return true;
    }
    return false;
}

void plan_open_grid(const float mn[3], const float mx[3], double rmax, int cells_per_rmax,
                    int max_cells, GridInfo* g, std::vector<int>* rows) {
    float cell = (float)(rmax / cells_per_rmax * 1.001);
    int dims[3];
    for (;;) {
        double ncell = 1;
        for (int a = 0; a < 3; ++a) {
            dims[a] = std::max(1, (int)std::floor((mx[a] - mn[a]) / cell) + 1);
            ncell *= dims[a];
        }
        if (ncell <= max_cells) break;
        cell *= 1.25f;  // keep the grid bounded for sparse, extended catalogs
    }
    g->gx = dims[0];
    g->gy = dims[1];
    g->gz = dims[2];
    g->ox = mn[0];
    g->oy = mn[1];
    g->oz = mn[2];
    g->inv_cell = 1.0f / cell;
    g->periodic = 0;
    g->L = 0.f;
    g->hL = 0.f;
    g->ncell = g->gx * g->gy * g->gz;
    int reach = 0;
    *rows = neighbour_rows(cell, rmax, &reach);
}

// Shell of the FP32 neighbour rule as a function of r2 alone: -1 for r2 == 0 (coincident
// points), below e2[0] or at/above e2[nr]; b for e2[b] <= r2 < e2[b+1]. Same comparisons as
// the device rule (float operands).
static int rule_shell(float r2, const float* e2, int nr) {
    if (!(r2 > 0.f) || !(r2 >= e2[0]) || !(r2 < e2[nr])) return -1;
    int b = 0;
    while (b + 1 < nr && r2 >= e2[b + 1]) ++b;
    return b;
}

bool build_shell_table(const float* e2, int nr, int max_bins, std::vector<int4>* tab, float* scale) {
    // bins of width 2^-k over [0, e2[nr]], as many as fit: k the largest integer with
    // floor(e2[nr] 2^k) + 1 <= max_bins; then r2 * 2^k is exact in FP32 and so is its floor
    const double top = e2[nr];
    if (!(top > 0.0) || !std::isfinite(top)) return false;
    int k = (int)std::floor(std::log2((max_bins - 1) / top));
    while (std::floor(top * std::ldexp(1.0, k)) + 1 > max_bins) --k;
    while (std::floor(top * std::ldexp(1.0, k + 1)) + 1 <= max_bins) ++k;
    if (k < -120 || k > 120) return false;
    const int nb = (int)std::floor(top * std::ldexp(1.0, k)) + 1;
    // the points where the rule's shell changes: just above 0, and every edge
    std::vector<float> brk;
    brk.push_back(std::numeric_limits<float>::denorm_min());
    for (int b = 0; b <= nr; ++b)
        if (e2[b] > 0.f) brk.push_back(e2[b]);
    std::sort(brk.begin(), brk.end());
    brk.erase(std::unique(brk.begin(), brk.end()), brk.end());
    tab->assign(nb, make_int4(0, 0, 0, 0));
    size_t q = 0;
    for (int i = 0; i < nb; ++i) {
        const double lo = std::ldexp((double)i, -k), hi = std::ldexp((double)(i + 1), -k);
        while (q < brk.size() && (double)brk[q] <= lo) ++q;   // already in force at the bin start
        const float flo = (float)lo;                            // exact: lo has few significant bits
        const int below = rule_shell(flo, e2, nr);
        int above = below;
        float edge = std::numeric_limits<float>::infinity();
        size_t inside = 0;
        while (q + inside < brk.size() && (double)brk[q + inside] < hi) ++inside;
        if (inside > 1) return false;   // two changes in one bin: no table
        if (inside == 1) {
            edge = brk[q];
            above = rule_shell(edge, e2, nr);
        }
        int bits;
        std::memcpy(&bits, &edge, 4);
        (*tab)[i] = make_int4(below, above, bits, 0);
    }
    *scale = (float)std::ldexp(1.0, k);
    return true;
}

}  // namespace npcf
