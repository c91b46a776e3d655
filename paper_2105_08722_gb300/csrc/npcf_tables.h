// Host-side tables of libencore_gpu: multiplet and bin enumerations, coupling
// coefficients and the spherical-harmonic conversion matrix. Built once per
// context and uploaded to the device.
#pragma once

#include <cstdint>
#include <vector>

namespace npcf {

constexpr int kMaxL = 10;    // largest lmax of the pair kernel
constexpr int kMaxNr = 16;   // largest number of radial shells

// Wigner 3-j symbol (Racah's closed form, DLMF 34.2.4).
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);

// Wigner 6-j symbol (Racah's single-sum form, DLMF 34.4.3) and 9-j symbol (sum over
// products of three 6-j symbols, DLMF 34.6.2), integer arguments.
double wigner6j(int j1, int j2, int j3, int j4, int j5, int j6);
double wigner9j(int j1, int j2, int j3, int j4, int j5, int j6, int j7, int j8, int j9);

// Generalized Gaunt integral G^{L L' L''} = int dR P_L P_L' P_L'' of Eq. (generalized-
// gaunt-def), from the closed forms of App. A for N = 3, 4, 5 (multiplets laid out as in
// OrderTable: (l, l), (l1, l2, l3), (l1, l2, l12, l3, l4)); 0 for other N.
double generalized_gaunt(int N, const int* L1, const int* L2, const int* L3);

// Coupling coefficient C^L_M of Eq. (basis-coupling) (Eq. (N=3-coeff) and Eq. (N=4-coeff)
// for N = 3, 4; one intermediate for N = 5, two for N = 6), multiplets laid out as in
// OrderTable, M = (m_1, ..., m_{N-1}); 0 where the 3-j symbols vanish.
double coupling(int N, const int* L, const int* M);

// Number of complex slots per shell in the a_lm layout: l <= lmax, 0 <= m <= l.
inline int nlm(int lmax) { return (lmax + 1) * (lmax + 2) / 2; }
inline int lm_index(int l, int m) { return l * (l + 1) / 2 + m; }

// One order N of the statistic: its multiplets L and bin tuples B.
struct OrderTable {
    int N = 0;
    int width = 0;                  // ints per multiplet: 2 (N=3), 3 (N=4), 5 (N=5), 7 (N=6)
    std::vector<int> lam;           // n_lambda x width
    std::vector<int> bins;          // n_bins x (N-1)
    int n_lambda() const { return width ? (int)lam.size() / width : 0; }
    int n_bins() const { return N > 1 ? (int)bins.size() / (N - 1) : 0; }
    bool odd(int a) const;          // parity-odd multiplet (odd sum of principal l)
};

OrderTable make_order(int N, int lmax, int nr, bool allparity);

// a_lm from the sums S_{m,k} = sum_j w_j (x + i y)^m T_k(z) over unit separations,
// m + k <= lmax, T_k the Chebyshev polynomials: a_lm = sum_k K[lm_index(l,m)][k] S_{m,k}.
// Derived from Y_lm = N_lm (-1)^m (x+iy)^m d^m P_l(z)/dz^m (Condon-Shortley phase,
// unit vectors): the polynomial factor is rewritten in the Chebyshev basis, whose
// coefficients stay O(1) where the plain powers z^k would alternate in sign and grow,
// so the FP32 sums lose little to cancellation.
//
// The matrix yields the reduced coefficients a_lm / sqrt((2l+1)/(4 pi)): with that
// factor gone the l = 0 row is exactly 1 and every m = 0 row is a dyadic rational, so
// the FP32 sums carry no rounded normalisation. A rounded Y_00 = 1/(2 sqrt(pi)) would
// otherwise bias every coefficient of order N by (N-1) times its relative rounding
// (2e-7 for the 5PCF), far above the random rounding of the sums. The product of the
// factors of a multiplet's N-1 harmonics is applied in FP64 after the reduction.
std::vector<double> ylm_chebyshev_matrix(int lmax);
double ylm_l_norm(int l);   // sqrt((2l+1)/(4 pi))

// One product term c * a^{b1}_{l1 m1} * a^{b2}_{l2 m2} with m1, m2 of either sign,
// written on the stored m >= 0 coefficients (x1 + i y1), (x2 + i y2) using
// a_{l,-m} = (-1)^m conj(a_{l m}):
//   re += cA x1 x2 + cB y1 y2 ;  im += cC y1 x2 + cD x1 y2.
struct PairTerm {
    float cA, cB, cC, cD;
    uint16_t lm1, lm2;
};

PairTerm make_pair_term(double c, int l1, int m1, int l2, int m2);

// 4PCF contraction table (Eq. simple-NPCF-summation at N=4): for multiplet a and
// m3 = 0..l3 one segment of terms over m1, with m2 = -m1 - m3,
//   P^{a,m3}(b1,b2) = sum_{m1} E(L) C^L_{m1 m2 m3} a^{b1}_{l1 m1} a^{b2}_{l2 m2},
// and zeta += u * 2 S(m3) * Q_L[P^{a,m3} a^{b3}_{l3 m3}].
struct ContractTable4 {
    std::vector<PairTerm> terms;
    std::vector<int> seg_begin;     // per segment: [begin, end) into terms
    std::vector<int> seg_end;
    std::vector<int> seg_lm3;       // lm index of a_{l3 m3}
    std::vector<float> seg_factor;  // 2 S(m3)
    std::vector<int> lam_seg0;      // first segment of multiplet a (n_lambda + 1 entries)
};

ContractTable4 make_contract4(const OrderTable& o);

// The same terms regrouped for the high-lmax kernel, which holds two segments of one
// multiplet at a time: segments m3 = 0..l3 are taken in pairs (0,1), (2,3), ..., and within
// a pair the terms are grouped by the stored harmonic a^{b2}_{l2 |m2|} they read (the
// first segment's terms, then the second's), so each a^{b2} value is loaded once per group.
// A pair whose first segment has m3 = 0 needs one part of that segment's P only.
struct ContractTable4G {
    std::vector<float> coef;        // 4 per term (cA, cB, cC, cD)
    std::vector<int> tlm;           // lm1 per term
    std::vector<int> groups;        // 4 per group: first term of segment 0, of segment 1, end, lm2
    std::vector<int> pairs;         // 8 per pair: first group, end, lm3 of segment 0, of segment 1
                                    //   (-1 if none), 2 S(m3) bits of both, m3 == 0 of segment 0, 0
    std::vector<int> lam_pair0;     // first pair of multiplet a (n_lambda + 1 entries)
};

ContractTable4G make_contract4g(const ContractTable4& t);

// 5PCF coupling tables: the distinct (l1 l2 l12) and (l12 l3 l4) triples of the order's
// multiplets, each with one term segment per m12 = 0..l12:
//   P12: terms over m1 with m2 = m12 - m1, coefficient (l1 l2 l12; m1, m2, -m12);
//   P34: terms over m3 with m4 = -m12 - m3, coefficient (l12 l3 l4; m12, m3, m4).
struct ContractTable5 {
    std::vector<PairTerm> terms12, terms34;
    std::vector<int> seg12_begin, seg12_end, t12_seg0;   // t12_seg0: n_t12 + 1 entries
    std::vector<int> seg34_begin, seg34_end, t34_seg0;
    std::vector<int> t34_l12;
    std::vector<int> lam_t12, lam_t34;                  // triple ids of each multiplet
    int l12max = 0;
};

ContractTable5 make_contract5(const OrderTable& o);

}  // namespace npcf
