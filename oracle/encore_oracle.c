/*
 * encore_oracle.c -- plain FP64 CPU oracle for the isotropic NPCF estimator
 * (Philcox, Slepian, Hou, Warner, Cahn, Eisenstein, arXiv:2105.08722).
 *
 * TEST INFRASTRUCTURE: slow and obviously correct on purpose. Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg load it.
 * It shares no code with the GPU library.
 *
 * What it follows (paper sections / equations):
 *   orc_wigner3j    Racah's closed form of the Wigner 3-j symbol (DLMF 34.2.4),
 *                   the building block of Eq. (basis-coupling).
 *   orc_ylm         Condon-Shortley spherical harmonics (Sec. 2.1) from the
 *                   associated-Legendre three-term recurrence in cos(theta) and
 *                   e^{i m phi} from atan2 -- the textbook route.
 *   orc_multiplets  the multiplets L of orders 3 to 6 (Sec. 2.2: triangle conditions
 *                   of the 3-j symbols, parity-even unless allparity), lexicographic
 *                   with the last entry fastest (the order of the edge-correction
 *                   matrices of the mock-catalog figures, Sec. 5.4); orc_multiplets_cap bounds
 *                   the intermediate l's.
 *   orc_coupling    C^L_M: Eq. (N=3-coeff), Eq. (N=4-coeff) and, for N=5 and N=6,
 *                   the general Eq. (basis-coupling) with its sqrt(2 l12 + 1) (and
 *                   sqrt(2 l123 + 1)) factors.
 *   orc_alm         a^b_lm(s_i) = sum_j w_j Y_lm(unit(r_j - s_i)) Theta^b,
 *                   Eq. (binned-discrete-alm) without 1/v_b.
 *   orc_npcf        zeta^B_L = sum_i u_i sum_M E(L) C^L_M prod_k a^{b_k}_{l_k m_k},
 *                   Eq. (NPCF-mult-discrete-binned-estimator) without 1/V, summed
 *                   over the FULL M range (no m >= 0 halving), OpenMP over
 *                   primaries with per-thread accumulators merged in thread order
 *                   (the paper's CPU strategy, Sec. 4.1.2).
 *   orc_gaunt       Eq. (generalized-gaunt-def) evaluated from its definition:
 *                   sum over M, M', M'' of C C' C'' times products of ordinary
 *                   Gaunt integrals (DLMF 34.3.22).
 *   orc_edge_correct Eqs. (edge-correction-matrix) and (edge-corrected-NPCF):
 *                   M_{L L''} = sum_L' f_L' E(L'') G^{L L' L''}, f = R_L / R_0,
 *                   then solve sum_L zeta_L M_{L L''} = N_{L''} / R_0 for each
 *                   bin tuple (Gaussian elimination, partial pivoting).
 */
#include "encore_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static long double fact(int n) {
    long double f = 1.0L;
    for (int k = 2; k <= n; ++k) f *= (long double)k;
    return f;
}

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }
static int parity_sign(int k) { return (k % 2 == 0) ? 1 : -1; }

double orc_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    long double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) /
                      fact(j1 + j2 + j3 + 1);
    long double pre = sqrtl(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) *
                            fact(j2 - m2) * fact(j3 + m3) * fact(j3 - m3));
    int kmin = imax(0, imax(j2 - j3 - m1, j1 - j3 + m2));
    int kmax = imin(j1 + j2 - j3, imin(j1 - m1, j2 + m2));
    long double s = 0.0L;
    for (int k = kmin; k <= kmax; ++k) {
        long double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2) *
                          fact(j1 + j2 - j3 - k) * fact(j1 - k - m1) * fact(j2 - k + m2);
        s += (long double)parity_sign(k) / den;
    }
    return (double)(parity_sign(j1 - j2 - m3) * pre * s);
}

void orc_ylm(int lmax, double x, double y, double z, double* re, double* im) {
    double r = sqrt(x * x + y * y + z * z);
    double ct = z / r;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double st = sqrt(x * x + y * y) / r;
    double phi = atan2(y, x);
    double* P = (double*)malloc(sizeof(double) * (size_t)(lmax + 1));
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m = (-1)^m (2m-1)!! sin^m(theta), then the upward recurrence in l. */
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= -(double)(2 * i - 1) * st;
        P[m] = pmm;
        if (m + 1 <= lmax) P[m + 1] = ct * (double)(2 * m + 1) * pmm;
        for (int l = m + 2; l <= lmax; ++l)
            P[l] = ((double)(2 * l - 1) * ct * P[l - 1] - (double)(l + m - 1) * P[l - 2]) /
                   (double)(l - m);
        for (int l = m; l <= lmax; ++l) {
            double norm = sqrt((double)(2 * l + 1) / (4.0 * ORC_PI) *
                               (double)(fact(l - m) / fact(l + m)));
            double yr = norm * P[l] * cos(m * phi);
            double yi = norm * P[l] * sin(m * phi);
            re[l * l + l + m] = yr;
            im[l * l + l + m] = yi;
            if (m > 0) { /* Y_{l,-m} = (-1)^m conj(Y_{l m}) */
                double s = (double)parity_sign(m);
                re[l * l + l - m] = s * yr;
                im[l * l + l - m] = -s * yi;
            }
        }
    }
    free(P);
}

static int n_ell(int N) { return N == 3 ? 2 : (N == 4 ? 3 : (N == 5 ? 5 : 7)); }

/* Multiplets in lexicographic order, the last entry fastest (Sec. 5.4). icap bounds
 * the intermediate l's (l12, l123); their natural range (triangle conditions with every
 * principal l <= lmax) is 2 lmax, which orc_multiplets uses. */
int orc_multiplets_cap(int N, int lmax, int icap, int allparity, int* out) {
    int c = 0;
    if (N == 3) {
        for (int l = 0; l <= lmax; ++l) {
            if (out) { out[2 * c] = l; out[2 * c + 1] = l; }
            ++c;
        }
    } else if (N == 4) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l3 = abs(l1 - l2); l3 <= imin(l1 + l2, lmax); ++l3) {
                    if (!allparity && ((l1 + l2 + l3) & 1)) continue;
                    if (out) { out[3 * c] = l1; out[3 * c + 1] = l2; out[3 * c + 2] = l3; }
                    ++c;
                }
    } else if (N == 5) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l12 = abs(l1 - l2); l12 <= imin(l1 + l2, icap); ++l12)
                    for (int l3 = 0; l3 <= lmax; ++l3)
                        for (int l4 = abs(l12 - l3); l4 <= imin(l12 + l3, lmax); ++l4) {
                            if (!allparity && ((l1 + l2 + l3 + l4) & 1)) continue;
                            if (out) {
                                out[5 * c] = l1; out[5 * c + 1] = l2; out[5 * c + 2] = l12;
                                out[5 * c + 3] = l3; out[5 * c + 4] = l4;
                            }
                            ++c;
                        }
    } else if (N == 6) {
        /* L = (l1, l2, (l12), l3, (l123), l4, l5): Eq. (basis-coupling) with two
         * intermediates, each bounded by the triangle conditions of its 3-j symbols */
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l12 = abs(l1 - l2); l12 <= imin(l1 + l2, icap); ++l12)
                    for (int l3 = 0; l3 <= lmax; ++l3)
                        for (int l123 = abs(l12 - l3); l123 <= imin(l12 + l3, icap); ++l123)
                            for (int l4 = 0; l4 <= lmax; ++l4)
                                for (int l5 = abs(l123 - l4); l5 <= imin(l123 + l4, lmax); ++l5) {
                                    if (!allparity && ((l1 + l2 + l3 + l4 + l5) & 1)) continue;
                                    if (out) {
                                        int* o = out + 7 * c;
                                        o[0] = l1; o[1] = l2; o[2] = l12; o[3] = l3;
                                        o[4] = l123; o[5] = l4; o[6] = l5;
                                    }
                                    ++c;
                                }
    } else {
        return -1;
    }
    return c;
}

int orc_multiplets(int N, int lmax, int allparity, int* out) {
    return orc_multiplets_cap(N, lmax, 2 * lmax, allparity, out);
}

int orc_bins(int N, int nr, int* out) {
    int k = N - 1, c = 0;
    int b[8];
    if (k < 1 || k > 8 || nr < k) return 0;
    for (int i = 0; i < k; ++i) b[i] = i;
    for (;;) {
        if (out) for (int i = 0; i < k; ++i) out[k * c + i] = b[i];
        ++c;
        int i = k - 1;
        while (i >= 0 && b[i] == nr - k + i) --i;
        if (i < 0) break;
        ++b[i];
        for (int j = i + 1; j < k; ++j) b[j] = b[j - 1] + 1;
    }
    return c;
}

double orc_coupling(int N, const int* L, const int* M) {
    if (N == 3) {
        /* Eq. (N=3-coeff): (-1)^{l-m1} / sqrt(2l+1) delta_{l1 l2} delta_{m1,-m2}. */
        if (L[0] != L[1] || M[0] != -M[1] || abs(M[0]) > L[0]) return 0.0;
        return parity_sign(L[0] - M[0]) / sqrt(2.0 * L[0] + 1.0);
    }
    if (N == 4) {
        /* Eq. (N=4-coeff): (-1)^{l1+l2+l3} (l1 l2 l3; m1 m2 m3). */
        return parity_sign(L[0] + L[1] + L[2]) *
               orc_wigner3j(L[0], L[1], L[2], M[0], M[1], M[2]);
    }
    if (N == 5) {
        /* Eq. (basis-coupling) at N=5: E sqrt(2 l12 + 1) sum_{m12} (-1)^{l12-m12}
         * (l1 l2 l12; m1 m2 -m12)(l12 l3 l4; m12 m3 m4). The 3-j symbols force
         * m12 = m1 + m2, so the sum has one term. */
        int l1 = L[0], l2 = L[1], l12 = L[2], l3 = L[3], l4 = L[4];
        int m12 = M[0] + M[1];
        if (abs(m12) > l12) return 0.0;
        double v = orc_wigner3j(l1, l2, l12, M[0], M[1], -m12) *
                   orc_wigner3j(l12, l3, l4, m12, M[2], M[3]);
        return parity_sign(l1 + l2 + l3 + l4) * sqrt(2.0 * l12 + 1.0) *
               parity_sign(l12 - m12) * v;
    }
    if (N == 6) {
        /* Eq. (basis-coupling) at N=6: E sqrt(2 l12 + 1) sqrt(2 l123 + 1)
         * sum_{m12, m123} (-1)^{l12-m12+l123-m123} (l1 l2 l12; m1 m2 -m12)
         * (l12 l3 l123; m12 m3 -m123)(l123 l4 l5; m123 m4 m5); the 3-j symbols force
         * m12 = m1 + m2 and m123 = m12 + m3. */
        int l1 = L[0], l2 = L[1], l12 = L[2], l3 = L[3], l123 = L[4], l4 = L[5], l5 = L[6];
        int m12 = M[0] + M[1], m123 = m12 + M[2];
        if (abs(m12) > l12 || abs(m123) > l123) return 0.0;
        double v = orc_wigner3j(l1, l2, l12, M[0], M[1], -m12) *
                   orc_wigner3j(l12, l3, l123, m12, M[2], -m123) *
                   orc_wigner3j(l123, l4, l5, m123, M[3], M[4]);
        return parity_sign(l1 + l2 + l3 + l4 + l5) * sqrt(2.0 * l12 + 1.0) * sqrt(2.0 * l123 + 1.0) *
               parity_sign(l12 - m12 + l123 - m123) * v;
    }
    return 0.0;
}

/* Principal angular momenta of a multiplet (the l's that index Y's). */
static void principal(int N, const int* L, int* ell) {
    if (N == 3) { ell[0] = L[0]; ell[1] = L[1]; }
    else if (N == 4) { ell[0] = L[0]; ell[1] = L[1]; ell[2] = L[2]; }
    else if (N == 5) { ell[0] = L[0]; ell[1] = L[1]; ell[2] = L[3]; ell[3] = L[4]; }
    else { ell[0] = L[0]; ell[1] = L[1]; ell[2] = L[3]; ell[3] = L[5]; ell[4] = L[6]; }
}

/* Terms of one multiplet: every M over the full range with C^L_M != 0. */
typedef struct {
    int nterm;
    int* m;        /* nterm x (N-1) */
    double* coef;  /* E(L) C^L_M */
} term_list;

static void build_terms(int N, const int* L, term_list* t) {
    int ell[5];
    int k = N - 1;
    principal(N, L, ell);
    int sumell = 0;
    for (int i = 0; i < k; ++i) sumell += ell[i];
    int E = parity_sign(sumell);
    int cap = 1;
    for (int i = 0; i < k - 1; ++i) cap *= 2 * ell[i] + 1;
    t->m = (int*)malloc(sizeof(int) * (size_t)(cap * k));
    t->coef = (double*)malloc(sizeof(double) * (size_t)cap);
    t->nterm = 0;
    int M[5];
    for (int idx = 0; idx < cap; ++idx) {
        int r = idx, s = 0;
        for (int i = 0; i < k - 1; ++i) {
            M[i] = r % (2 * ell[i] + 1) - ell[i];
            r /= 2 * ell[i] + 1;
            s += M[i];
        }
        M[k - 1] = -s;
        if (abs(M[k - 1]) > ell[k - 1]) continue;
        double c = orc_coupling(N, L, M);
        if (fabs(c) < 1e-14) continue;
        for (int i = 0; i < k; ++i) t->m[t->nterm * k + i] = M[i];
        t->coef[t->nterm] = E * c;
        ++t->nterm;
    }
}

static void free_terms(term_list* t) { free(t->m); free(t->coef); }

int64_t orc_count_terms(int N, int lmax, int allparity) {
    int nl = orc_multiplets(N, lmax, allparity, NULL);
    if (nl <= 0) return -1;
    int nL = n_ell(N);
    int* lam = (int*)malloc(sizeof(int) * (size_t)(nl * nL));
    orc_multiplets(N, lmax, allparity, lam);
    int64_t total = 0;
    for (int a = 0; a < nl; ++a) {
        term_list t;
        build_terms(N, lam + a * nL, &t);
        for (int q = 0; q < t.nterm; ++q) {
            int mlast = t.m[q * (N - 1) + (N - 2)];
            if (mlast >= 0) ++total;
        }
        free_terms(&t);
    }
    free(lam);
    return total;
}

/* The neighbour / shell rule, in float arithmetic (built with -ffp-contract=off).
 * Writes the float separation into d (nullable). */
static int shell_rule(const float* pi, const float* pj, double box, const float* e2, int nr,
                      float* d_out) {
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = pj[a] - pi[a];
    if (box > 0.0) {
        float L = (float)box;
        float h = (float)(0.5 * box);
        for (int a = 0; a < 3; ++a) {
            if (d[a] > h) d[a] = d[a] - L;
            else if (d[a] < -h) d[a] = d[a] + L;
        }
    }
    float xx = d[0] * d[0];
    float yy = d[1] * d[1];
    float zz = d[2] * d[2];
    float r2 = xx + yy;
    r2 = r2 + zz;
    if (d_out) { d_out[0] = d[0]; d_out[1] = d[1]; d_out[2] = d[2]; }
    if (!(r2 > 0.0f)) return -1;
    if (r2 < e2[0] || !(r2 < e2[nr])) return -1;
    for (int b = 0; b < nr; ++b)
        if (r2 < e2[b + 1]) return b;
    return -1;
}

int orc_shell(const float* pi, const float* pj, double box, const float* e2, int nr) {
    return shell_rule(pi, pj, box, e2, nr, NULL);
}

static float* make_e2(int nr, const double* edges) {
    float* e2 = (float*)malloc(sizeof(float) * (size_t)(nr + 1));
    for (int k = 0; k <= nr; ++k) e2[k] = (float)(edges[k] * edges[k]);
    return e2;
}

int orc_pair_counts(int64_t n, const float* pos, const int64_t* prim, int64_t n_prim, int nr,
                    const double* edges, double box, int nthreads, uint64_t* counts) {
    float* e2 = make_e2(nr, edges);
    int64_t np = prim ? n_prim : n;
    memset(counts, 0, sizeof(uint64_t) * (size_t)nr);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        uint64_t* loc = (uint64_t*)calloc((size_t)nr, sizeof(uint64_t));
#pragma omp for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
            int64_t i = prim ? prim[q] : q;
            for (int64_t j = 0; j < n; ++j) {
                int b = shell_rule(pos + 3 * i, pos + 3 * j, box, e2, nr, NULL);
                if (b >= 0) ++loc[b];
            }
        }
#pragma omp critical
        for (int b = 0; b < nr; ++b) counts[b] += loc[b];
        free(loc);
    }
    free(e2);
    return 0;
}

/* a^b_lm of one primary for every l <= lmax and -l <= m <= l. */
static void alm_one(int64_t n, const float* pos, const float* w, int64_t i, int lmax, int nr,
                    const float* e2, double box, double* are, double* aim, uint32_t* cnt,
                    double* yre, double* yim) {
    int nlm = (lmax + 1) * (lmax + 1);
    memset(are, 0, sizeof(double) * (size_t)(nr * nlm));
    memset(aim, 0, sizeof(double) * (size_t)(nr * nlm));
    if (cnt) memset(cnt, 0, sizeof(uint32_t) * (size_t)nr);
    float d[3];
    for (int64_t j = 0; j < n; ++j) {
        int b = shell_rule(pos + 3 * i, pos + 3 * j, box, e2, nr, d);
        if (b < 0) continue;
        if (cnt) ++cnt[b];
        orc_ylm(lmax, (double)d[0], (double)d[1], (double)d[2], yre, yim);
        double wj = (double)w[j];
        for (int q = 0; q < nlm; ++q) {
            are[b * nlm + q] += wj * yre[q];
            aim[b * nlm + q] += wj * yim[q];
        }
    }
}

int orc_alm(int64_t n, const float* pos, const float* w, const int64_t* prim, int64_t n_prim,
            int lmax, int nr, const double* edges, double box, double* alm_re, double* alm_im,
            uint32_t* counts) {
    float* e2 = make_e2(nr, edges);
    int nlm = (lmax + 1) * (lmax + 1);
#pragma omp parallel
    {
        double* yre = (double*)malloc(sizeof(double) * (size_t)nlm);
        double* yim = (double*)malloc(sizeof(double) * (size_t)nlm);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < n_prim; ++q)
            alm_one(n, pos, w, prim[q], lmax, nr, e2, box, alm_re + q * nr * nlm,
                    alm_im + q * nr * nlm, counts ? counts + q * nr : NULL, yre, yim);
        free(yre);
        free(yim);
    }
    free(e2);
    return 0;
}

typedef struct {
    int N, nl, nb, nL;
    int* lam;
    int* bins;
    int* odd;       /* per multiplet: 1 if parity-odd */
    term_list* terms;
} order_tab;

static void build_order(int N, int lmax, int nr, int allparity, order_tab* o) {
    o->N = N;
    o->nL = n_ell(N);
    o->nl = orc_multiplets(N, lmax, allparity, NULL);
    o->lam = (int*)malloc(sizeof(int) * (size_t)(o->nl * o->nL));
    orc_multiplets(N, lmax, allparity, o->lam);
    o->nb = orc_bins(N, nr, NULL);
    o->bins = (int*)malloc(sizeof(int) * (size_t)(o->nb * (N - 1)) + 1);
    orc_bins(N, nr, o->bins);
    o->terms = (term_list*)malloc(sizeof(term_list) * (size_t)o->nl);
    o->odd = (int*)malloc(sizeof(int) * (size_t)o->nl);
    for (int a = 0; a < o->nl; ++a) {
        int ell[5], s = 0;
        principal(N, o->lam + a * o->nL, ell);
        for (int i = 0; i < N - 1; ++i) s += ell[i];
        o->odd[a] = s & 1;
        build_terms(N, o->lam + a * o->nL, &o->terms[a]);
    }
}

static void free_order(order_tab* o) {
    for (int a = 0; a < o->nl; ++a) free_terms(&o->terms[a]);
    free(o->terms); free(o->lam); free(o->bins); free(o->odd);
}

/* Add u * sum_M E C prod_k a^{b_k}_{l_k m_k} for every (L, B) of one order. */
static void add_primary(const order_tab* o, int lmax, const double* are, const double* aim,
                        double u, double* zre, double* zim) {
    int nlm = (lmax + 1) * (lmax + 1);
    int k = o->N - 1;
    for (int a = 0; a < o->nl; ++a) {
        int ell[5];
        principal(o->N, o->lam + a * o->nL, ell);
        const term_list* t = &o->terms[a];
        for (int bb = 0; bb < o->nb; ++bb) {
            const int* B = o->bins + bb * k;
            double sr = 0.0, si = 0.0;
            for (int q = 0; q < t->nterm; ++q) {
                double pr = t->coef[q], pi = 0.0;
                for (int i = 0; i < k; ++i) {
                    int m = t->m[q * k + i];
                    int idx = B[i] * nlm + ell[i] * ell[i] + ell[i] + m;
                    double xr = are[idx], xi = aim[idx];
                    double nr_ = pr * xr - pi * xi;
                    double ni_ = pr * xi + pi * xr;
                    pr = nr_;
                    pi = ni_;
                }
                sr += pr;
                si += pi;
            }
            zre[a * o->nb + bb] += u * sr;
            zim[a * o->nb + bb] += u * si;
        }
    }
}

int orc_npcf(int64_t n, const float* pos, const float* w, const float* wprim, const int64_t* prim,
             int64_t n_prim, int orders_mask, int lmax, int nr, const double* edges, double box,
             int allparity, int nthreads, double* zeta, double* resid, uint64_t* counts) {
    order_tab ord[4];
    int nord = 0;
    for (int N = 3; N <= 6; ++N)
        if (orders_mask & (1 << N)) build_order(N, lmax, nr, allparity, &ord[nord++]);
    size_t total = 0;
    for (int o = 0; o < nord; ++o) total += (size_t)ord[o].nl * (size_t)ord[o].nb;
    float* e2 = make_e2(nr, edges);
    int nlm = (lmax + 1) * (lmax + 1);
    int64_t np = prim ? n_prim : n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    int nt = omp_get_max_threads();
#else
    int nt = 1;
#endif
    double* zr_all = (double*)calloc(total * (size_t)nt, sizeof(double));
    double* zi_all = (double*)calloc(total * (size_t)nt, sizeof(double));
    uint64_t* c_all = (uint64_t*)calloc((size_t)nr * (size_t)nt, sizeof(uint64_t));
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double* zr = zr_all + (size_t)tid * total;
        double* zi = zi_all + (size_t)tid * total;
        uint64_t* cc = c_all + (size_t)tid * nr;
        double* are = (double*)malloc(sizeof(double) * (size_t)(nr * nlm));
        double* aim = (double*)malloc(sizeof(double) * (size_t)(nr * nlm));
        uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nr);
        double* yre = (double*)malloc(sizeof(double) * (size_t)nlm);
        double* yim = (double*)malloc(sizeof(double) * (size_t)nlm);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < np; ++q) {
            int64_t i = prim ? prim[q] : q;
            alm_one(n, pos, w, i, lmax, nr, e2, box, are, aim, cnt, yre, yim);
            for (int b = 0; b < nr; ++b) cc[b] += cnt[b];
            double u = (double)(wprim ? wprim[i] : w[i]);
            size_t off = 0;
            for (int o = 0; o < nord; ++o) {
                add_primary(&ord[o], lmax, are, aim, u, zr + off, zi + off);
                off += (size_t)ord[o].nl * (size_t)ord[o].nb;
            }
        }
        free(are); free(aim); free(cnt); free(yre); free(yim);
    }
    /* ordered merge of the per-thread accumulators */
    size_t off = 0;
    for (int o = 0; o < nord; ++o) {
        for (int a = 0; a < ord[o].nl; ++a)
            for (int bb = 0; bb < ord[o].nb; ++bb) {
                size_t e = off + (size_t)a * ord[o].nb + bb;
                double sr = 0.0, si = 0.0;
                for (int t = 0; t < nt; ++t) {
                    sr += zr_all[(size_t)t * total + e];
                    si += zi_all[(size_t)t * total + e];
                }
                /* even multiplets are real, odd ones purely imaginary (Sec. 2.2) */
                zeta[e] = ord[o].odd[a] ? si : sr;
                if (resid) resid[e] = ord[o].odd[a] ? sr : si;
            }
        off += (size_t)ord[o].nl * (size_t)ord[o].nb;
    }
    if (counts) {
        memset(counts, 0, sizeof(uint64_t) * (size_t)nr);
        for (int t = 0; t < nt; ++t)
            for (int b = 0; b < nr; ++b) counts[b] += c_all[(size_t)t * nr + b];
    }
    free(zr_all); free(zi_all); free(c_all); free(e2);
    for (int o = 0; o < nord; ++o) free_order(&ord[o]);
    return 0;
}

/* Ordinary Gaunt integral int Y_{l1m1} Y_{l2m2} Y_{l3m3} dOmega (DLMF 34.3.22). */
static double gaunt3(int l1, int l2, int l3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (((l1 + l2 + l3) & 1) || l3 < abs(l1 - l2) || l3 > l1 + l2) return 0.0;
    return sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * ORC_PI)) *
           orc_wigner3j(l1, l2, l3, 0, 0, 0) * orc_wigner3j(l1, l2, l3, m1, m2, m3);
}

/* C^L_M of one multiplet on a dense grid over (m_1, ..., m_{N-1}). */
typedef struct {
    int k;
    int ell[5];
    double* c;
} dense_coupling;

static void build_dense(int N, const int* L, dense_coupling* d) {
    d->k = N - 1;
    principal(N, L, d->ell);
    int size = 1;
    for (int i = 0; i < d->k; ++i) size *= 2 * d->ell[i] + 1;
    d->c = (double*)calloc((size_t)size, sizeof(double));
    int M[5];
    for (int idx = 0; idx < size; ++idx) {
        int r = idx;
        for (int i = d->k - 1; i >= 0; --i) {
            M[i] = r % (2 * d->ell[i] + 1) - d->ell[i];
            r /= 2 * d->ell[i] + 1;
        }
        d->c[idx] = orc_coupling(N, L, M);
    }
}

static double dense_at(const dense_coupling* d, const int* M) {
    int idx = 0;
    for (int i = 0; i < d->k; ++i) {
        if (abs(M[i]) > d->ell[i]) return 0.0;
        idx = idx * (2 * d->ell[i] + 1) + M[i] + d->ell[i];
    }
    return d->c[idx];
}

/* G^{L1 L2 L3} = sum_{M1,M2,M3} C C C prod_i gaunt3, with M3 = -M1 - M2 forced by
 * the ordinary Gaunt integrals. */
static double gaunt_dense(const dense_coupling* d1, const dense_coupling* d2,
                          const dense_coupling* d3) {
    int k = d1->k;
    for (int i = 0; i < k; ++i) {
        int a = d1->ell[i], b = d2->ell[i], c = d3->ell[i];
        if (((a + b + c) & 1) || c < abs(a - b) || c > a + b) return 0.0;
    }
    int s1 = 1, s2 = 1;
    for (int i = 0; i < k; ++i) { s1 *= 2 * d1->ell[i] + 1; s2 *= 2 * d2->ell[i] + 1; }
    double total = 0.0;
    int M1[5], M2[5], M3[5];
    for (int p = 0; p < s1; ++p) {
        if (d1->c[p] == 0.0) continue;
        int r = p;
        for (int i = k - 1; i >= 0; --i) {
            M1[i] = r % (2 * d1->ell[i] + 1) - d1->ell[i];
            r /= 2 * d1->ell[i] + 1;
        }
        for (int q = 0; q < s2; ++q) {
            if (d2->c[q] == 0.0) continue;
            int r2 = q;
            for (int i = k - 1; i >= 0; --i) {
                M2[i] = r2 % (2 * d2->ell[i] + 1) - d2->ell[i];
                r2 /= 2 * d2->ell[i] + 1;
            }
            for (int i = 0; i < k; ++i) M3[i] = -M1[i] - M2[i];
            double c3 = dense_at(d3, M3);
            if (c3 == 0.0) continue;
            double g = 1.0;
            for (int i = 0; i < k && g != 0.0; ++i)
                g *= gaunt3(d1->ell[i], d2->ell[i], d3->ell[i], M1[i], M2[i], M3[i]);
            total += d1->c[p] * d2->c[q] * c3 * g;
        }
    }
    return total;
}

double orc_gaunt(int N, const int* L1, const int* L2, const int* L3) {
    dense_coupling d1, d2, d3;
    build_dense(N, L1, &d1);
    build_dense(N, L2, &d2);
    build_dense(N, L3, &d3);
    double g = gaunt_dense(&d1, &d2, &d3);
    free(d1.c); free(d2.c); free(d3.c);
    return g;
}

/* Solve A x = b (n x n, row-major, destroyed) by Gaussian elimination with
 * partial pivoting. Returns 0 on success, -1 if singular. */
static int gauss_solve(int n, double* A, double* b) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (fabs(A[p * n + c]) == 0.0) return -1;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

int orc_edge_correct(int N, int lmax, int nr, int allparity, const double* nraw,
                     const double* rraw, double* zeta) {
    if (allparity) return -2; /* parity-even multiplets only: every quantity is real */
    int nl = orc_multiplets(N, lmax, 0, NULL);
    int nL = n_ell(N);
    int nb = orc_bins(N, nr, NULL);
    int* lam = (int*)malloc(sizeof(int) * (size_t)(nl * nL));
    orc_multiplets(N, lmax, 0, lam);
    dense_coupling* dc = (dense_coupling*)malloc(sizeof(dense_coupling) * (size_t)nl);
    for (int a = 0; a < nl; ++a) build_dense(N, lam + a * nL, &dc[a]);
    double* G = (double*)malloc(sizeof(double) * (size_t)nl * nl * nl);
    for (int a = 0; a < nl; ++a)
        for (int b = 0; b < nl; ++b)
            for (int c = 0; c < nl; ++c)
                G[((size_t)a * nl + b) * nl + c] = gaunt_dense(&dc[a], &dc[b], &dc[c]);
    for (int a = 0; a < nl; ++a) free(dc[a].c);
    free(dc);
    double* A = (double*)malloc(sizeof(double) * (size_t)nl * nl);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)nl);
    int rc = 0;
    for (int bb = 0; bb < nb; ++bb) {
        double R0 = rraw[0 * nb + bb]; /* multiplet 0 is L = (0,...,0) */
        /* A[L''][L] = M_{L L''} = sum_L' f_L' E(L'') G^{L L' L''}; E(L'') = +1 here. */
        for (int l2 = 0; l2 < nl; ++l2) {
            for (int l0 = 0; l0 < nl; ++l0) {
                double s = 0.0;
                for (int l1 = 0; l1 < nl; ++l1)
                    s += (rraw[(size_t)l1 * nb + bb] / R0) * G[((size_t)l0 * nl + l1) * nl + l2];
                A[l2 * nl + l0] = s;
            }
            rhs[l2] = nraw[(size_t)l2 * nb + bb] / R0;
        }
        if (gauss_solve(nl, A, rhs) != 0) rc = -1;
        for (int l0 = 0; l0 < nl; ++l0) zeta[(size_t)l0 * nb + bb] = rhs[l0];
    }
    free(A); free(rhs); free(G); free(lam);
    return rc;
}
