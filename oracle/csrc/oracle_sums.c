/*
 * CTR-IBIM oracle -- plain FP64 loops (test infrastructure only).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline arm use
 * this file.  It shares nothing with the CUDA path.  Every function is a
 * direct transcription of a definition in the paper; there is no blocking,
 * no reordering and no approximation beyond IEEE FP64 rounding.  It must be
 * compiled with -ffp-contract=off so that no multiply-add is fused.
 *
 * Parity status: pinned through the operator (the double-layer identity,
 * the sphere kernel integrals in closed form, the exact sphere solution
 * satisfying the discrete equations to the method's order, planted mistakes
 * that the consistency test must catch).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } acc_t;
static inline void acc_add(acc_t* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double acc_get(const acc_t* a) { return a->s + a->c; }

/*
 * The four Poisson-Boltzmann kernels of Eq. (1.4)-(1.5) at (x, n_x; y, n_y):
 *   K11 = dG0/dn_y - (eps_E/eps_I) dGk/dn_y
 *   K12 = G0 - Gk
 *   K21 = d2G0/dn_x dn_y - d2Gk/dn_x dn_y
 *   K22 = dG0/dn_x - (eps_I/eps_E) dGk/dn_x
 * with G0 = 1/(4 pi r), Gk = exp(-kappa r)/(4 pi r), r = |x - y|.
 * Derivatives written out from those definitions (d = x - y):
 *   dG/dn_y  = -G'(r) (d.n_y)/r,          dG/dn_x = G'(r) (d.n_x)/r,
 *   d2G/dn_x dn_y = F(r) (n_x.n_y) + F'(r)/r (d.n_x)(d.n_y),  F = -G'/r.
 */
static void pb_kernels(const double x[3], const double nxv[3], const double y[3], const double nyv[3],
                       double kappa, double ratio_EI, double K[4]) {
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double E = exp(-kappa * r);
    double fourpi = 4.0 * M_PI;
    /* G and G' */
    double G0 = 1.0 / (fourpi * r);
    double Gk = E / (fourpi * r);
    double dG0 = -1.0 / (fourpi * r2);                       /* d/dr of 1/(4 pi r) */
    double dGk = -E * (1.0 + kappa * r) / (fourpi * r2);     /* d/dr of e^{-kr}/(4 pi r) */
    /* F = -G'/r and F'/r */
    double F0 = -dG0 / r;
    double Fk = -dGk / r;
    double F0p_r = -3.0 / (fourpi * r2 * r2 * r);
    double Fkp_r = -E * (3.0 + 3.0 * kappa * r + kappa * kappa * r2) / (fourpi * r2 * r2 * r);
    double dny = d[0] * nyv[0] + d[1] * nyv[1] + d[2] * nyv[2];
    double dnx = d[0] * nxv[0] + d[1] * nxv[1] + d[2] * nxv[2];
    double nn = nxv[0] * nyv[0] + nxv[1] * nyv[1] + nxv[2] * nyv[2];
    double dG0_dny = -dG0 * dny / r;
    double dGk_dny = -dGk * dny / r;
    double dG0_dnx = dG0 * dnx / r;
    double dGk_dnx = dGk * dnx / r;
    double d2G0 = F0 * nn + F0p_r * dnx * dny;
    double d2Gk = Fk * nn + Fkp_r * dnx * dny;
    K[0] = dG0_dny - ratio_EI * dGk_dny;
    K[1] = G0 - Gk;
    K[2] = d2G0 - d2Gk;
    K[3] = dG0_dnx - (1.0 / ratio_EI) * dGk_dnx;
}

/*
 * Punctured Riemann sum of the linear system, Eqs. (2.14)-(2.15):
 *   out1[i] = h^3 sum_{j not in N(i)} W_j (K11 rho1_j - K12 rho2_j)
 *   out2[i] = h^3 sum_{j not in N(i)} W_j (K21 rho1_j - K22 rho2_j)
 * kernels evaluated at (P_i, n_i; P_j, n_j).  N(i) is given in CSR form
 * (excl_ptr, excl_idx) with sorted indices.  Only rows[0..n_rows) are
 * computed; out is indexed by position in `rows`.
 */
void oracle_punctured_sum(int64_t M, const double* P, const double* N, const double* W,
                          const double* rho1, const double* rho2, double h, double kappa,
                          double ratio_EI, const int64_t* excl_ptr, const int64_t* excl_idx,
                          const int64_t* rows, int64_t n_rows, double* out1, double* out2) {
    double h3 = h * h * h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_rows; ++t) {
        int64_t i = rows[t];
        acc_t a1 = {0, 0}, a2 = {0, 0};
        int64_t e = excl_ptr[i], e_end = excl_ptr[i + 1];
        for (int64_t j = 0; j < M; ++j) {
            while (e < e_end && excl_idx[e] < j) ++e;
            if (e < e_end && excl_idx[e] == j) continue;
            double K[4];
            pb_kernels(P + 3 * i, N + 3 * i, P + 3 * j, N + 3 * j, kappa, ratio_EI, K);
            double w = h3 * W[j];
            acc_add(&a1, w * (K[0] * rho1[j] - K[1] * rho2[j]));
            acc_add(&a2, w * (K[2] * rho1[j] - K[3] * rho2[j]));
        }
        out1[t] = acc_get(&a1);
        out2[t] = acc_get(&a2);
    }
}

/*
 * Reaction potential by the standard trapezoidal rule on the tube, Eq. (2.31):
 *   psi_rxn(z) = sum_j h^3 W_j [ ((eps_E/eps_I) dGk/dn_y - dG0/dn_y)(z, P_j) psi_j
 *                                + (G0 - Gk)(z, P_j) dpsi_j ]
 */
void oracle_reaction_potential(int64_t M, const double* P, const double* N, const double* W,
                               const double* psi, const double* dpsi, double h, double kappa,
                               double ratio_EI, int64_t n_z, const double* z, double* out) {
    double h3 = h * h * h;
    double fourpi = 4.0 * M_PI;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_z; ++k) {
        acc_t a = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            double d[3] = {z[3 * k] - P[3 * j], z[3 * k + 1] - P[3 * j + 1], z[3 * k + 2] - P[3 * j + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double E = exp(-kappa * r);
            double dny = d[0] * N[3 * j] + d[1] * N[3 * j + 1] + d[2] * N[3 * j + 2];
            double dG0_dny = dny / (fourpi * r2 * r);
            double dGk_dny = E * (1.0 + kappa * r) * dny / (fourpi * r2 * r);
            double G0 = 1.0 / (fourpi * r);
            double Gk = E / (fourpi * r);
            double f = (ratio_EI * dGk_dny - dG0_dny) * psi[j] + (G0 - Gk) * dpsi[j];
            acc_add(&a, h3 * W[j] * f);
        }
        out[k] = acc_get(&a);
    }
}

/*
 * Flat-top radial cutoff g for the weight limit, Eq. (2.29): g = 1 on
 * |x| <= r0, a C-infinity transition S(t) = e^{-1/(1-t)} / (e^{-1/t} + e^{-1/(1-t)})
 * on r0 < |x| < 1 (t = (|x| - r0)/(1 - r0)), and 0 for |x| >= 1.
 */
double oracle_cutoff_g(double r, double r0) {
    if (r <= r0) return 1.0;
    if (r >= 1.0) return 0.0;
    double t = (r - r0) / (1.0 - r0);
    double A = exp(-1.0 / (1.0 - t));
    double B = exp(-1.0 / t);
    return A / (A + B);
}

/*
 * Punctured trapezoidal sum T^0_h of Eq. (2.29) for the harmonics
 * k = 0, kstep, 2 kstep, ..., kmax at once:
 *   re[k/kstep] + i im[k/kstep] = h^2 sum_{n in Z^2, n != 0} s_k(x_n) g(x_n),
 *   x_n = h n - h (alpha, beta),   s_k(x) = |x|^{-1} (cos k psi(x) + i sin k psi(x)).
 * Compensated sums: omega_h divides the small difference (int s g - T0_h) by h.
 */
void oracle_punctured_lattice(double alpha, double beta, double h, double r0, int kmax, int kstep,
                              double* re, double* im) {
    int64_t R = (int64_t)ceil(1.0 / h) + 2;
    int nk = kmax / kstep + 1;
    acc_t* ar = (acc_t*)calloc((size_t)nk, sizeof(acc_t));
    acc_t* ai = (acc_t*)calloc((size_t)nk, sizeof(acc_t));
    for (int64_t n2 = -R; n2 <= R; ++n2) {
        for (int64_t n1 = -R; n1 <= R; ++n1) {
            if (n1 == 0 && n2 == 0) continue;
            double x1 = h * (double)n1 - h * alpha;
            double x2 = h * (double)n2 - h * beta;
            double r = sqrt(x1 * x1 + x2 * x2);
            double g = oracle_cutoff_g(r, r0);
            if (g == 0.0) continue;
            double c = x1 / r, s = x2 / r;        /* e^{i psi} */
            double sr = 1.0, si = 0.0;            /* e^{i kstep psi} by repeated product */
            for (int q = 0; q < kstep; ++q) {
                double nr = sr * c - si * s;
                double ni = sr * s + si * c;
                sr = nr; si = ni;
            }
            double pr = 1.0, pi = 0.0;            /* e^{i k psi}, k = 0 */
            double base = h * h * g / r;
            for (int q = 0; q < nk; ++q) {
                acc_add(&ar[q], base * pr);
                acc_add(&ai[q], base * pi);
                double nr = pr * sr - pi * si;
                double ni = pr * si + pi * sr;
                pr = nr; pi = ni;
            }
        }
    }
    for (int q = 0; q < nk; ++q) { re[q] = acc_get(&ar[q]); im[q] = acc_get(&ai[q]); }
    free(ar); free(ai);
}

/* Many (alpha, beta) points at one h, in parallel. re/im are [n_pts][kmax/kstep+1]. */
void oracle_punctured_lattice_many(int64_t n_pts, const double* alpha, const double* beta, double h,
                                   double r0, int kmax, int kstep, double* re, double* im) {
    int nk = kmax / kstep + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n_pts; ++p)
        oracle_punctured_lattice(alpha[p], beta[p], h, r0, kmax, kstep, re + p * nk, im + p * nk);
}

/*
 * Far-field acceleration of the punctured sum (the fast summation of K v inside
 * GMRES, Sec. 2.5), evaluation loops of oracle/treecode.py.  Tree positions
 * p = 0..M-1 hold node perm[p]; target block I is the positions
 * [I*BS, min(M, (I+1)*BS)).
 *
 * Near field: for target i in block I, the punctured sum of Eqs. (2.14)-(2.15)
 * over the sources at the positions of the block's near ranges
 * [near_rng[2r], near_rng[2r+1]), r in [near_ptr[I], near_ptr[I+1]).
 * Results go to out1/out2 at the original index i (overwritten).
 */
void oracle_tree_near(int64_t M, const double* P, const double* N, const double* W,
                      const double* rho1, const double* rho2, double h, double kappa, double ratio_EI,
                      const int64_t* excl_ptr, const int64_t* excl_idx, const int64_t* perm, int64_t BS,
                      const int64_t* near_ptr, const int64_t* near_rng, double* out1, double* out2) {
    double h3 = h * h * h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < M; ++p) {
        int64_t i = perm[p], I = p / BS;
        acc_t a1 = {0, 0}, a2 = {0, 0};
        for (int64_t r = near_ptr[I]; r < near_ptr[I + 1]; ++r) {
            for (int64_t q = near_rng[2 * r]; q < near_rng[2 * r + 1]; ++q) {
                int64_t j = perm[q];
                int skip = 0;
                for (int64_t e = excl_ptr[i]; e < excl_ptr[i + 1]; ++e)
                    if (excl_idx[e] == j) skip = 1;
                if (skip) continue;
                double K[4];
                pb_kernels(P + 3 * i, N + 3 * i, P + 3 * j, N + 3 * j, kappa, ratio_EI, K);
                double w = h3 * W[j];
                acc_add(&a1, w * (K[0] * rho1[j] - K[1] * rho2[j]));
                acc_add(&a2, w * (K[2] * rho1[j] - K[3] * rho2[j]));
            }
        }
        out1[i] = acc_get(&a1);
        out2[i] = acc_get(&a2);
    }
}

/*
 * Far field: for target i in block I and every cluster c = far_cl[r],
 * r in [far_ptr[I], far_ptr[I+1]), the sum over the cluster's proxy points
 * s_k = (sx[c][0][k1], sx[c][1][k2], sx[c][2][k3]), k = (k3 n1 + k2) n1 + k1, of
 *   out1 += G0(P_i, s_k) Q[c][0][k] + Gk(P_i, s_k) Q[c][1][k]
 *   out2 += dG0/dn_x(P_i, s_k) Q[c][0][k] + dGk/dn_x(P_i, s_k) Q[c][2][k]
 * with G0 = 1/(4 pi r), Gk = e^{-kappa r}/(4 pi r), d/dn_x = n_i . grad_x.
 * sx is [n_far][3][n1], Q is [n_far][3][n1^3].  Results are added to out1/out2
 * at the original index i.
 */
void oracle_tree_far(int64_t M, const double* P, const double* N, double kappa, const int64_t* perm,
                     int64_t BS, const int64_t* far_ptr, const int64_t* far_cl, int64_t n1, const double* sx,
                     const double* Q, double* out1, double* out2) {
    double fourpi = 4.0 * M_PI;
    int64_t np = n1 * n1 * n1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < M; ++p) {
        int64_t i = perm[p], I = p / BS;
        const double* x = P + 3 * i;
        const double* nx = N + 3 * i;
        acc_t a1 = {0, 0}, a2 = {0, 0};
        for (int64_t r = far_ptr[I]; r < far_ptr[I + 1]; ++r) {
            int64_t c = far_cl[r];
            const double* s = sx + c * 3 * n1;
            const double* q = Q + c * 3 * np;
            for (int64_t k3 = 0; k3 < n1; ++k3)
                for (int64_t k2 = 0; k2 < n1; ++k2)
                    for (int64_t k1 = 0; k1 < n1; ++k1) {
                        int64_t k = (k3 * n1 + k2) * n1 + k1;
                        double d[3] = {x[0] - s[k1], x[1] - s[n1 + k2], x[2] - s[2 * n1 + k3]};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        double rr = sqrt(r2);
                        double E = exp(-kappa * rr);
                        double dnx = d[0] * nx[0] + d[1] * nx[1] + d[2] * nx[2];
                        double G0 = 1.0 / (fourpi * rr);
                        double Gk = E / (fourpi * rr);
                        double dG0_dnx = -dnx / (fourpi * r2 * rr);
                        double dGk_dnx = -E * (1.0 + kappa * rr) * dnx / (fourpi * r2 * rr);
                        acc_add(&a1, G0 * q[k] + Gk * q[np + k]);
                        acc_add(&a2, dG0_dnx * q[k] + dGk_dnx * q[2 * np + k]);
                    }
        }
        out1[i] += acc_get(&a1);
        out2[i] += acc_get(&a2);
    }
}

#ifdef _OPENMP
#include <omp.h>
void oracle_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int oracle_max_threads(void) { return omp_get_max_threads(); }
#else
void oracle_set_threads(int n) { (void)n; }
int oracle_max_threads(void) { return 1; }
#endif
