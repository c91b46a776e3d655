/*
 * encore_oracle.h -- plain FP64 CPU oracle for the isotropic N-point
 * correlation function (NPCF) estimator of Philcox et al. (arXiv:2105.08722).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference leg load this library. The GPU library
 * shares no code, header, table or helper with it.
 *
 * Conventions (readings of the paper, all stated once here):
 *  - Spherical harmonics Y_lm are orthonormal, Condon-Shortley phase (Sec. 2.1).
 *  - Separation vector of a pair is r_j - s_i (Eq. binned-discrete-alm), and
 *    a^b_lm(s_i) = sum_j w_j Y_lm(unit(r_j - s_i)) over j in shell b of i.
 *  - Raw multiplets: zeta^B_L = sum_i u_i sum_M E(L) C^L_M prod_k a^{b_k}_{l_k m_k}
 *    (Eq. NPCF-mult-discrete-binned-estimator without 1/V and 1/v_b), with
 *    u_i the primary weight (u = w unless a separate primary weight is given).
 *    Parity-even multiplets are real; parity-odd ones are purely imaginary and
 *    their imaginary part is stored.
 *  - Neighbour/shell rule (IEEE FP32, round-to-nearest, no fused multiply-add):
 *      d = p_j - p_i per axis; if periodic (L > 0): d > L/2 -> d - L,
 *      d < -L/2 -> d + L (L/2 and L rounded to float);
 *      r2 = (dx*dx + dy*dy) + dz*dz;  e2[k] = float(double(edge_k)^2);
 *      accepted iff r2 > 0 and e2[0] <= r2 < e2[nr]; shell b: e2[b] <= r2 < e2[b+1].
 *  - Bins are strictly ordered b1 < b2 < ... (Sec. 3.2.1).
 *  - Multiplet order: l1 outer, then l2, [l12], l3, [l4]; the last index varies
 *    fastest. 3PCF multiplets are written (l, l).
 */
#ifndef ENCORE_ORACLE_H
#define ENCORE_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

double orc_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);
/* All Y_lm for l <= lmax at the direction (x,y,z) (normalised inside);
 * index l*l + l + m. */
void orc_ylm(int lmax, double x, double y, double z, double* re, double* im);
/* Number of multiplets of order N (3,4,5); lambdas (nullable) receives
 * 2, 3 or 5 ints per multiplet. */
int orc_multiplets(int N, int lmax, int allparity, int* lambdas);
int orc_bins(int N, int nr, int* bins);
/* Coupling C^L_M (real). N=3: L=(l,l), M=(m1,m2). N=4: L=(l1,l2,l3).
 * N=5: L=(l1,l2,l12,l3,l4), M=(m1,m2,m3,m4). */
double orc_coupling(int N, const int* L, const int* M);
/* Count of (L, M) with C^L_M != 0 and 0 <= m_{N-1} <= l_{N-1}. */
int64_t orc_count_terms(int N, int lmax, int allparity);
/* Shell of the pair (i, j) by the rule above, or -1. */
int orc_shell(const float* pi, const float* pj, double box, const float* e2, int nr);
int orc_pair_counts(int64_t n, const float* pos, const int64_t* prim, int64_t n_prim,
                    int nr, const double* edges, double box, int nthreads, uint64_t* counts);
int orc_alm(int64_t n, const float* pos, const float* w, const int64_t* prim, int64_t n_prim,
            int lmax, int nr, const double* edges, double box,
            double* alm_re, double* alm_im, uint32_t* counts);
int orc_npcf(int64_t n, const float* pos, const float* w, const float* wprim,
             const int64_t* prim, int64_t n_prim, int orders_mask, int lmax, int nr,
             const double* edges, double box, int allparity, int nthreads,
             double* zeta, double* resid, uint64_t* counts);
/* Generalised Gaunt integral int dR P_L P_L' P_L'' (Eq. generalized-gaunt-def). */
double orc_gaunt(int N, const int* L1, const int* L2, const int* L3);
int orc_edge_correct(int N, int lmax, int nr, int allparity,
                     const double* nraw, const double* rraw, double* zeta);

#ifdef __cplusplus
}
#endif
#endif
