// Host-side tables of libencore_gpu (see npcf_tables.h).
#include "npcf_tables.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace npcf {

namespace {

// n! for n < 160 in long double (exact to 25! and within a few ulp beyond).
struct FactTable {
    long double f[160];
    FactTable() {
        f[0] = 1.0L;
        for (int i = 1; i < 160; ++i) f[i] = f[i - 1] * (long double)i;
    }
};
const FactTable& facts() {
    static FactTable t;
    return t;
}

inline int neg1pow(int k) { return (k & 1) ? -1 : 1; }

}  // namespace

double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
    if (j3 > j1 + j2 || j3 < std::abs(j1 - j2)) return 0.0;
    const long double* f = facts().f;
    // triangle coefficient and the m-dependent square root, then the alternating sum
    long double delta = f[j1 + j2 - j3] * f[j1 - j2 + j3] * f[-j1 + j2 + j3] / f[j1 + j2 + j3 + 1];
    long double root = std::sqrt(delta * f[j1 + m1] * f[j1 - m1] * f[j2 + m2] * f[j2 - m2] *
                                 f[j3 + m3] * f[j3 - m3]);
    int lo = 0;
    if (j2 - j3 - m1 > lo) lo = j2 - j3 - m1;
    if (j1 - j3 + m2 > lo) lo = j1 - j3 + m2;
    int hi = j1 + j2 - j3;
    if (j1 - m1 < hi) hi = j1 - m1;
    if (j2 + m2 < hi) hi = j2 + m2;
    long double sum = 0.0L;
    for (int t = lo; t <= hi; ++t) {
        long double d = f[t] * f[j3 - j2 + t + m1] * f[j3 - j1 + t - m2] * f[j1 + j2 - j3 - t] *
                        f[j1 - t - m1] * f[j2 - t + m2];
        sum += neg1pow(t) / d;
    }
    return (double)(neg1pow(j1 - j2 - m3) * root * sum);
}

namespace {

bool triangle(int a, int b, int c) { return c <= a + b && c >= std::abs(a - b); }

// sqrt of the triangle coefficient (a+b-c)! (a-b+c)! (-a+b+c)! / (a+b+c+1)!
long double tri_root(int a, int b, int c) {
    const long double* f = facts().f;
    return std::sqrt(f[a + b - c] * f[a - b + c] * f[-a + b + c] / f[a + b + c + 1]);
}

}  // namespace

double wigner6j(int j1, int j2, int j3, int j4, int j5, int j6) {
    if (!triangle(j1, j2, j3) || !triangle(j1, j5, j6) || !triangle(j4, j2, j6) || !triangle(j4, j5, j3))
        return 0.0;
    const long double* f = facts().f;
    const int a1 = j1 + j2 + j3, a2 = j1 + j5 + j6, a3 = j4 + j2 + j6, a4 = j4 + j5 + j3;
    const int b1 = j1 + j2 + j4 + j5, b2 = j2 + j3 + j5 + j6, b3 = j3 + j1 + j6 + j4;
    const int lo = std::max({a1, a2, a3, a4}), hi = std::min({b1, b2, b3});
    long double sum = 0.0L;
    for (int t = lo; t <= hi; ++t)
        sum += neg1pow(t) * f[t + 1] /
               (f[t - a1] * f[t - a2] * f[t - a3] * f[t - a4] * f[b1 - t] * f[b2 - t] * f[b3 - t]);
    return (double)(tri_root(j1, j2, j3) * tri_root(j1, j5, j6) * tri_root(j4, j2, j6) * tri_root(j4, j5, j3) *
                    sum);
}

double wigner9j(int j1, int j2, int j3, int j4, int j5, int j6, int j7, int j8, int j9) {
    // sum over x of (2x+1) {j1 j4 j7; j8 j9 x} {j2 j5 j8; j4 x j6} {j3 j6 j9; x j1 j2}
    const int lo = std::max({std::abs(j1 - j9), std::abs(j4 - j8), std::abs(j2 - j6)});
    const int hi = std::min({j1 + j9, j4 + j8, j2 + j6});
    double sum = 0.0;
    for (int x = lo; x <= hi; ++x)
        sum += (2.0 * x + 1.0) * wigner6j(j1, j4, j7, j8, j9, x) * wigner6j(j2, j5, j8, j4, x, j6) *
               wigner6j(j3, j6, j9, x, j1, j2);
    return sum;
}

double generalized_gaunt(int N, const int* L1, const int* L2, const int* L3) {
    const double fourpi = 4.0 * 3.14159265358979323846;
    // one factor per principal angular momentum: sqrt((2l+1)(2l'+1)(2l''+1)) (l l' l''; 0 0 0)
    auto leg = [](int a, int b, int c) {
        return std::sqrt((2.0 * a + 1.0) * (2.0 * b + 1.0) * (2.0 * c + 1.0)) * wigner3j(a, b, c, 0, 0, 0);
    };
    if (N == 3) {
        const double t = wigner3j(L1[0], L2[0], L3[0], 0, 0, 0);
        return std::sqrt((2.0 * L1[0] + 1.0) * (2.0 * L2[0] + 1.0) * (2.0 * L3[0] + 1.0)) * t * t / fourpi;
    }
    if (N == 4) {
        double p = 1.0;
        for (int i = 0; i < 3; ++i) p *= leg(L1[i], L2[i], L3[i]);
        if (p == 0.0) return 0.0;
        return p * std::pow(fourpi, -1.5) *
               wigner9j(L1[0], L2[0], L3[0], L1[1], L2[1], L3[1], L1[2], L2[2], L3[2]);
    }
    if (N == 5) {
        // multiplets (l1, l2, l12, l3, l4)
        double p = 1.0;
        for (int i : {0, 1, 3, 4}) p *= leg(L1[i], L2[i], L3[i]);
        if (p == 0.0) return 0.0;
        p *= std::sqrt((2.0 * L1[2] + 1.0) * (2.0 * L2[2] + 1.0) * (2.0 * L3[2] + 1.0));
        return p / (fourpi * fourpi) *
               wigner9j(L1[0], L1[1], L1[2], L2[0], L2[1], L2[2], L3[0], L3[1], L3[2]) *
               wigner9j(L1[2], L1[3], L1[4], L2[2], L2[3], L2[4], L3[2], L3[3], L3[4]);
    }
    return 0.0;
}

bool OrderTable::odd(int a) const {
    const int* L = &lam[(size_t)a * width];
    int s = (N == 6)   ? L[0] + L[1] + L[3] + L[5] + L[6]
            : (N == 5) ? L[0] + L[1] + L[3] + L[4]
                       : (N == 4 ? L[0] + L[1] + L[2] : 2 * L[0]);
    return (s & 1) != 0;
}

double coupling(int N, const int* L, const int* M) {
    if (N == 3) {
        // Eq. (N=3-coeff): (-1)^{l - m} / sqrt(2 l + 1) for l1 = l2 = l, m2 = -m1
        if (L[0] != L[1] || M[0] + M[1] != 0 || std::abs(M[0]) > L[0]) return 0.0;
        return neg1pow(L[0] - M[0]) / std::sqrt(2.0 * L[0] + 1.0);
    }
    if (N == 4) return neg1pow(L[0] + L[1] + L[2]) * wigner3j(L[0], L[1], L[2], M[0], M[1], M[2]);
    if (N == 5) {
        // Eq. (basis-coupling) with one intermediate: m12 = m1 + m2 by the first 3-j symbol
        const int m12 = M[0] + M[1];
        if (std::abs(m12) > L[2]) return 0.0;
        return neg1pow(L[0] + L[1] + L[3] + L[4]) * std::sqrt(2.0 * L[2] + 1.0) * neg1pow(L[2] - m12) *
               wigner3j(L[0], L[1], L[2], M[0], M[1], -m12) * wigner3j(L[2], L[3], L[4], m12, M[2], M[3]);
    }
    if (N == 6) {
        // two intermediates: L = (l1, l2, (l12), l3, (l123), l4, l5), m12 = m1 + m2 and
        // m123 = m12 + m3 by the 3-j symbols
        const int m12 = M[0] + M[1], m123 = m12 + M[2];
        if (std::abs(m12) > L[2] || std::abs(m123) > L[4]) return 0.0;
        return neg1pow(L[0] + L[1] + L[3] + L[5] + L[6]) * std::sqrt((2.0 * L[2] + 1.0) * (2.0 * L[4] + 1.0)) *
               neg1pow(L[2] - m12 + L[4] - m123) * wigner3j(L[0], L[1], L[2], M[0], M[1], -m12) *
               wigner3j(L[2], L[3], L[4], m12, M[2], -m123) * wigner3j(L[4], L[5], L[6], m123, M[3], M[4]);
    }
    return 0.0;
}

OrderTable make_order(int N, int lmax, int nr, bool allparity) {
    OrderTable o;
    o.N = N;
    o.width = (N == 3) ? 2 : (N == 4 ? 3 : (N == 5 ? 5 : 7));
    if (N == 3) {
        for (int l = 0; l <= lmax; ++l) { o.lam.push_back(l); o.lam.push_back(l); }
    } else if (N == 4) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2) {
                int top = l1 + l2 < lmax ? l1 + l2 : lmax;
                for (int l3 = std::abs(l1 - l2); l3 <= top; ++l3) {
                    if (!allparity && ((l1 + l2 + l3) & 1)) continue;
                    o.lam.insert(o.lam.end(), {l1, l2, l3});
                }
            }
    } else if (N == 5) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l12 = std::abs(l1 - l2); l12 <= l1 + l2; ++l12)
                    for (int l3 = 0; l3 <= lmax; ++l3) {
                        int top = l12 + l3 < lmax ? l12 + l3 : lmax;
                        for (int l4 = std::abs(l12 - l3); l4 <= top; ++l4) {
                            if (!allparity && ((l1 + l2 + l3 + l4) & 1)) continue;
                            o.lam.insert(o.lam.end(), {l1, l2, l12, l3, l4});
                        }
                    }
    } else if (N == 6) {
        // intermediates l12 and l123 over their triangle ranges (at most 2 lmax)
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l12 = std::abs(l1 - l2); l12 <= l1 + l2; ++l12)
                    for (int l3 = 0; l3 <= lmax; ++l3)
                        for (int l123 = std::abs(l12 - l3); l123 <= std::min(l12 + l3, 2 * lmax); ++l123)
                            for (int l4 = 0; l4 <= lmax; ++l4) {
                                const int top = std::min(l123 + l4, lmax);
                                for (int l5 = std::abs(l123 - l4); l5 <= top; ++l5) {
                                    if (!allparity && ((l1 + l2 + l3 + l4 + l5) & 1)) continue;
                                    o.lam.insert(o.lam.end(), {l1, l2, l12, l3, l123, l4, l5});
                                }
                            }
    }
    // strictly increasing bin tuples, lexicographic, last index fastest
    int k = N - 1;
    std::vector<int> b(k);
    if (nr >= k) {
        for (int i = 0; i < k; ++i) b[i] = i;
        while (true) {
            o.bins.insert(o.bins.end(), b.begin(), b.end());
            int i = k - 1;
            while (i >= 0 && b[i] == nr - k + i) --i;
            if (i < 0) break;
            ++b[i];
            for (int j = i + 1; j < k; ++j) b[j] = b[j - 1] + 1;
        }
    }
    return o;
}

double ylm_l_norm(int l) {
    const long double pi = 3.141592653589793238462643383279502884L;
    return (double)std::sqrt((2.0L * l + 1.0L) / (4.0L * pi));
}

std::vector<double> ylm_chebyshev_matrix(int lmax) {
    const long double* f = facts().f;
    // power-series coefficients of the Chebyshev polynomials T_k, k <= lmax
    std::vector<std::vector<long double>> T(lmax + 1, std::vector<long double>(lmax + 1, 0.0L));
    T[0][0] = 1.0L;
    if (lmax >= 1) T[1][1] = 1.0L;
    for (int k = 2; k <= lmax; ++k)
        for (int n = 0; n <= k; ++n)
            T[k][n] = (n > 0 ? 2.0L * T[k - 1][n - 1] : 0.0L) - T[k - 2][n];
    std::vector<double> K((size_t)nlm(lmax) * (lmax + 1), 0.0);
    for (int l = 0; l <= lmax; ++l) {
        // power-series coefficients of P_l: c[n] z^n, n = l - 2j
        std::vector<long double> c(l + 1, 0.0L);
        for (int j = 0; 2 * j <= l; ++j)
            c[l - 2 * j] = neg1pow(j) * f[2 * l - 2 * j] /
                           (std::pow(2.0L, l) * f[j] * f[l - j] * f[l - 2 * j]);
        for (int m = 0; m <= l; ++m) {
            // reduced harmonic: the factor sqrt((2l+1)/(4 pi)) is left out here and
            // applied once per multiplet in FP64 (ylm_l_norm)
            long double norm = std::sqrt(f[l - m] / f[l + m]);
            // q(z) = N_lm (-1)^m d^m P_l / dz^m in powers of z
            std::vector<long double> q(l - m + 1, 0.0L);
            for (int kk = 0; kk + m <= l; ++kk) q[kk] = norm * neg1pow(m) * c[kk + m] * f[kk + m] / f[kk];
            // rewrite q in the Chebyshev basis, highest degree first
            for (int d = l - m; d >= 0; --d) {
                long double coef = q[d] / T[d][d];
                K[(size_t)lm_index(l, m) * (lmax + 1) + d] = (double)coef;
                for (int n = 0; n <= d; ++n) q[n] -= coef * T[d][n];
            }
        }
    }
    return K;
}

PairTerm make_pair_term(double c, int l1, int m1, int l2, int m2) {
    double s1 = (m1 < 0) ? neg1pow(m1) : 1.0, g1 = (m1 < 0) ? -1.0 : 1.0;
    double s2 = (m2 < 0) ? neg1pow(m2) : 1.0, g2 = (m2 < 0) ? -1.0 : 1.0;
    double cc = c * s1 * s2;
    PairTerm t;
    t.cA = (float)cc;
    t.cB = (float)(-cc * g1 * g2);
    t.cC = (float)(cc * g1);
    t.cD = (float)(cc * g2);
    t.lm1 = (uint16_t)lm_index(l1, std::abs(m1));
    t.lm2 = (uint16_t)lm_index(l2, std::abs(m2));
    return t;
}

ContractTable4 make_contract4(const OrderTable& o) {
    ContractTable4 t;
    int na = o.n_lambda();
    for (int a = 0; a < na; ++a) {
        const int* L = &o.lam[(size_t)a * 3];
        int l1 = L[0], l2 = L[1], l3 = L[2];
        int E = neg1pow(l1 + l2 + l3);
        t.lam_seg0.push_back((int)t.seg_begin.size());
        for (int m3 = 0; m3 <= l3; ++m3) {
            t.seg_begin.push_back((int)t.terms.size());
            for (int m1 = -l1; m1 <= l1; ++m1) {
                int m2 = -m1 - m3;
                if (std::abs(m2) > l2) continue;
                // E(L) C^L_M with C^L_M = E(L) (l1 l2 l3; m1 m2 m3)  (Eq. N=4-coeff)
                double c = E * (E * wigner3j(l1, l2, l3, m1, m2, m3));
                if (std::fabs(c) < 1e-14) continue;
                t.terms.push_back(make_pair_term(c, l1, m1, l2, m2));
            }
            t.seg_end.push_back((int)t.terms.size());
            t.seg_lm3.push_back(lm_index(l3, m3));
            t.seg_factor.push_back(m3 == 0 ? 1.0f : 2.0f);
        }
    }
    t.lam_seg0.push_back((int)t.seg_begin.size());
    return t;
}

ContractTable4G make_contract4g(const ContractTable4& t) {
    ContractTable4G p;
    auto bits = [](float f) {
        int b;
        std::memcpy(&b, &f, 4);
        return b;
    };
    const int na = (int)t.lam_seg0.size() - 1;
    for (int a = 0; a < na; ++a) {
        p.lam_pair0.push_back((int)(p.pairs.size() / 8));
        const int s0 = t.lam_seg0[a], s1 = t.lam_seg0[a + 1];
        for (int sa = s0; sa < s1; sa += 2) {
            const int sb = sa + 1 < s1 ? sa + 1 : -1;
            const bool m0 = t.seg_factor[sa] == 1.0f;   // m3 = 0: a_{l3 0} is real
            p.pairs.push_back((int)(p.groups.size() / 4));
            // distinct lm2 of the two segments, ascending
            std::vector<int> lm2s;
            for (int sg : {sa, sb}) {
                if (sg < 0) continue;
                for (int i = t.seg_begin[sg]; i < t.seg_end[sg]; ++i) lm2s.push_back(t.terms[i].lm2);
            }
            std::sort(lm2s.begin(), lm2s.end());
            lm2s.erase(std::unique(lm2s.begin(), lm2s.end()), lm2s.end());
            for (int lm2 : lm2s) {
                for (int sg : {sa, sb}) {
                    p.groups.push_back((int)p.tlm.size());
                    if (sg < 0) continue;
                    for (int i = t.seg_begin[sg]; i < t.seg_end[sg]; ++i) {
                        const PairTerm& q = t.terms[i];
                        if (q.lm2 != lm2) continue;
                        p.coef.insert(p.coef.end(), {q.cA, q.cB, q.cC, q.cD});
                        p.tlm.push_back((int)q.lm1);
                    }
                }
                p.groups.push_back((int)p.tlm.size());
                p.groups.push_back(lm2);
            }
            p.pairs.push_back((int)(p.groups.size() / 4));
            p.pairs.push_back(t.seg_lm3[sa]);
            p.pairs.push_back(sb >= 0 ? t.seg_lm3[sb] : -1);
            p.pairs.push_back(bits(t.seg_factor[sa]));
            p.pairs.push_back(sb >= 0 ? bits(t.seg_factor[sb]) : 0);
            p.pairs.push_back(m0 ? 1 : 0);
            p.pairs.push_back(0);
        }
    }
    p.lam_pair0.push_back((int)(p.pairs.size() / 8));
    return p;
}

ContractTable5 make_contract5(const OrderTable& o) {
    ContractTable5 t;
    std::vector<std::array<int, 3>> k12, k34;
    auto find_or_add = [](std::vector<std::array<int, 3>>& v, std::array<int, 3> key) {
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i] == key) return (int)i;
        v.push_back(key);
        return (int)v.size() - 1;
    };
    for (int a = 0; a < o.n_lambda(); ++a) {
        const int* L = &o.lam[(size_t)a * 5];
        t.lam_t12.push_back(find_or_add(k12, {L[0], L[1], L[2]}));
        t.lam_t34.push_back(find_or_add(k34, {L[2], L[3], L[4]}));
        t.l12max = std::max(t.l12max, L[2]);
    }
    for (const auto& k : k12) {
        const int l1 = k[0], l2 = k[1], l12 = k[2];
        t.t12_seg0.push_back((int)t.seg12_begin.size());
        for (int m12 = 0; m12 <= l12; ++m12) {
            t.seg12_begin.push_back((int)t.terms12.size());
            for (int m1 = -l1; m1 <= l1; ++m1) {
                const int m2 = m12 - m1;
                if (std::abs(m2) > l2) continue;
                const double c = wigner3j(l1, l2, l12, m1, m2, -m12);
                if (std::fabs(c) < 1e-14) continue;
                t.terms12.push_back(make_pair_term(c, l1, m1, l2, m2));
            }
            t.seg12_end.push_back((int)t.terms12.size());
        }
    }
    t.t12_seg0.push_back((int)t.seg12_begin.size());
    for (const auto& k : k34) {
        const int l12 = k[0], l3 = k[1], l4 = k[2];
        t.t34_seg0.push_back((int)t.seg34_begin.size());
        t.t34_l12.push_back(l12);
        for (int m12 = 0; m12 <= l12; ++m12) {
            t.seg34_begin.push_back((int)t.terms34.size());
            for (int m3 = -l3; m3 <= l3; ++m3) {
                const int m4 = -m12 - m3;
                if (std::abs(m4) > l4) continue;
                const double c = wigner3j(l12, l3, l4, m12, m3, m4);
                if (std::fabs(c) < 1e-14) continue;
                t.terms34.push_back(make_pair_term(c, l3, m3, l4, m4));
            }
            t.seg34_end.push_back((int)t.terms34.size());
        }
    }
    t.t34_seg0.push_back((int)t.seg34_begin.size());
    return t;
}

}  // namespace npcf
