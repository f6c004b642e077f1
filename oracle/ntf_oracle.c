/*
 * ntf_oracle.c -- plain, slow FP64 CPU oracle for the unfolding-free beta-divergence
 * majorization-minimization updates of nonnegative CP and Tucker decompositions
 * (Leplat, arXiv 2602.14683).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every function follows the paper's definitions literally, in FP64, with plain nested
 * loops over multi-indices (row-major, last mode fastest).  Intermediate tensors (the
 * reconstruction, P, Q, the Tucker partial tensor) are materialised exactly as the
 * algorithms state them; no blocking, fusion or reordering is applied beyond the one
 * parallel loop over independent output rows that some functions carry.
 *
 * Readings where the paper is silent:
 *   - eps (parameter floor) and the clip max(Xhat, eps) inside the powers are caller
 *     arguments; the objective uses the same clipped reconstruction.
 *   - eps_x: at beta = 0 the data are floored, X <- max(X, eps_x) (Remark "The case
 *     beta = 0"), in both the powers and the objective.
 *   - Tucker sweep order: core first, then modes 1..N.
 *   - Sparse objective: zero entries contribute d_1(0|Xhat) = Xhat, summed in closed form
 *     as prod_n colsum(A^(n)) (no clip on entries that are not stored).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NTFO_MAXN 8

/* ----------------------------------------------------------------------------------
 * Scalars
 * ---------------------------------------------------------------------------------- */

/* Exponent gamma(beta): 1/(2-beta) for 0 <= beta < 1, 1 for 1 <= beta < 2
 * (Section 4.1, Remark "Exponent gamma(beta)"). */
double ntfo_gamma(double beta) { return beta < 1.0 ? 1.0 / (2.0 - beta) : 1.0; }

/* Scalar beta-divergence d_beta(x|y), x >= 0, y > 0 (Section 3.2, Definition
 * "beta-divergence"); KL at beta = 1 with 0 log 0 = 0, Itakura-Saito at beta = 0. */
double ntfo_dbeta(double x, double y, double beta) {
    if (beta == 1.0) return (x > 0.0 ? x * log(x / y) : 0.0) - x + y;
    if (beta == 0.0) return x / y - log(x / y) - 1.0;
    return (pow(x, beta) + (beta - 1.0) * pow(y, beta) - beta * x * pow(y, beta - 1.0)) /
           (beta * (beta - 1.0));
}

/* Multiplicative update with the epsilon-constrained minimiser (Theorem "CP block
 * multiplicative update"; Remark "eps-constrained updates"):
 *   out = max(pre * (num / den)^gamma(beta), eps), entrywise. */
void ntfo_mu_apply(int64_t count, const double *pre, const double *num, const double *den,
                   double beta, double eps, double *out) {
    double g = ntfo_gamma(beta);
    for (int64_t t = 0; t < count; ++t) {
        double cand = pre[t] * pow(num[t] / den[t], g);
        out[t] = cand > eps ? cand : eps;
    }
}

/* Transforms of Section 5.3 ("Two transforms"):
 *   chi1(Z, Zt) = Zt^(2-beta) * Z^(beta-1)
 *   chi2(Z, Zt) = Z                          (beta < 1)
 *               = Z^beta * Zt^(-(beta-1))    (1 <= beta < 2) */
void ntfo_chi1(int64_t count, const double *Z, const double *Zt, double beta, double *out) {
    for (int64_t t = 0; t < count; ++t) out[t] = pow(Zt[t], 2.0 - beta) * pow(Z[t], beta - 1.0);
}
void ntfo_chi2(int64_t count, const double *Z, const double *Zt, double beta, double *out) {
    for (int64_t t = 0; t < count; ++t)
        out[t] = beta < 1.0 ? Z[t] : pow(Z[t], beta) * pow(Zt[t], -(beta - 1.0));
}

/* ----------------------------------------------------------------------------------
 * Multi-index helpers (row-major, last mode fastest)
 * ---------------------------------------------------------------------------------- */

static int64_t numel(int N, const int64_t *dims) {
    int64_t n = 1;
    for (int m = 0; m < N; ++m) n *= dims[m];
    return n;
}

static int64_t linear(int N, const int64_t *dims, const int64_t *idx) {
    int64_t l = 0;
    for (int m = 0; m < N; ++m) l = l * dims[m] + idx[m];
    return l;
}

/* Advance idx over every mode except `skip` (skip < 0: all modes).  Returns 0 after
 * the last multi-index (idx wraps to all zeros on the free modes). */
static int next_index(int N, const int64_t *dims, int skip, int64_t *idx) {
    for (int m = N - 1; m >= 0; --m) {
        if (m == skip) continue;
        if (++idx[m] < dims[m]) return 1;
        idx[m] = 0;
    }
    return 0;
}

/* P = X' * max(Xhat, eps)^(beta-2), Q = max(Xhat, eps)^(beta-1), with X' = max(X, eps_x)
 * at beta = 0 and X' = X otherwise (Section 4.1 "Weights"; Assumption "Positivity
 * safeguard"; Remark "The case beta = 0"). */
static void powers(int64_t count, const double *X, const double *Xhat, double beta, double eps,
                   double eps_x, double *P, double *Q) {
    for (int64_t t = 0; t < count; ++t) {
        double y = Xhat[t] > eps ? Xhat[t] : eps;
        double x = (beta == 0.0 && X[t] < eps_x) ? eps_x : X[t];
        P[t] = x * pow(y, beta - 2.0);
        Q[t] = pow(y, beta - 1.0);
    }
}

/* D_beta(X, max(Xhat, eps)) = sum_i d_beta(X_i | .) (Section 3.2). */
static double objective_from_full(int64_t count, const double *X, const double *Xhat, double beta,
                                  double eps, double eps_x) {
    double s = 0.0;
    for (int64_t t = 0; t < count; ++t) {
        double y = Xhat[t] > eps ? Xhat[t] : eps;
        double x = (beta == 0.0 && X[t] < eps_x) ? eps_x : X[t];
        s += ntfo_dbeta(x, y, beta);
    }
    return s;
}

/* ----------------------------------------------------------------------------------
 * CP model (Section 3.3, "Nonnegative CP")
 * ---------------------------------------------------------------------------------- */

/* Xhat_i = sum_r prod_n A^(n)_{i_n r}.  A[n] is I_n x R row-major. */
double ntfo_cp_entry(int N, int R, const double *const *A, const int64_t *idx) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = 1.0;
        for (int n = 0; n < N; ++n) p *= A[n][idx[n] * R + r];
        s += p;
    }
    return s;
}

void ntfo_cp_full(int N, const int64_t *dims, int R, const double *const *A, double *Xhat) {
    int64_t idx[NTFO_MAXN] = {0};
    int64_t t = 0;
    do {
        Xhat[t++] = ntfo_cp_entry(N, R, A, idx);
    } while (next_index(N, dims, -1, idx));
}

double ntfo_cp_objective(int N, const int64_t *dims, const double *X, int R,
                         const double *const *A, double beta, double eps, double eps_x) {
    int64_t cnt = numel(N, dims);
    double *Xhat = (double *)malloc(sizeof(double) * cnt);
    ntfo_cp_full(N, dims, R, A, Xhat);
    double f = objective_from_full(cnt, X, Xhat, beta, eps, eps_x);
    free(Xhat);
    return f;
}

/* CPContr^(n)(T; {B^(m)}_{m != n})_{i_n r} = sum_{i_-n} T_i prod_{m != n} B^(m)_{i_m r}
 * (Section 6.1, "Contraction operators").  B[n] is ignored. out is I_n x R. */
void ntfo_cp_contr(int N, const int64_t *dims, const double *T, int R, const double *const *B,
                   int n, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t in = 0; in < dims[n]; ++in) {
        double *o = out + in * R;
        for (int r = 0; r < R; ++r) o[r] = 0.0;
        int64_t idx[NTFO_MAXN] = {0};
        idx[n] = in;
        do {
            double t = T[linear(N, dims, idx)];
            for (int r = 0; r < R; ++r) {
                double s = t;
                for (int m = 0; m < N; ++m)
                    if (m != n) s *= B[m][idx[m] * R + r];
                o[r] += s;
            }
        } while (next_index(N, dims, n, idx));
    }
}

/* One block of Algorithm 1 (B-CoMM) for mode n, i.e. Theorem "CP block multiplicative
 * update": rebuild Xhat from the current factors, form P and Q, contract, update, clip.
 * num/den (I_n x R, may be NULL) receive Num^(n) and Den^(n). */
void ntfo_cp_block_update(int N, const int64_t *dims, const double *X, int R, double *const *A,
                          int n, double beta, double eps, double eps_x, double *num_out,
                          double *den_out) {
    int64_t cnt = numel(N, dims);
    double *Xhat = (double *)malloc(sizeof(double) * cnt);
    double *P = (double *)malloc(sizeof(double) * cnt);
    double *Q = (double *)malloc(sizeof(double) * cnt);
    double *num = (double *)malloc(sizeof(double) * dims[n] * R);
    double *den = (double *)malloc(sizeof(double) * dims[n] * R);
    ntfo_cp_full(N, dims, R, (const double *const *)A, Xhat);
    powers(cnt, X, Xhat, beta, eps, eps_x, P, Q);
    ntfo_cp_contr(N, dims, P, R, (const double *const *)A, n, num);
    ntfo_cp_contr(N, dims, Q, R, (const double *const *)A, n, den);
    ntfo_mu_apply(dims[n] * R, A[n], num, den, beta, eps, A[n]);
    if (num_out) memcpy(num_out, num, sizeof(double) * dims[n] * R);
    if (den_out) memcpy(den_out, den, sizeof(double) * dims[n] * R);
    free(Xhat); free(P); free(Q); free(num); free(den);
}

/* One outer iteration of Algorithm 1 (B-CoMM): modes n = 1..N in order.  F_in (may be
 * NULL) receives the objective of the incoming iterate. */
void ntfo_cp_mu_sweep(int N, const int64_t *dims, const double *X, int R, double *const *A,
                      double beta, double eps, double eps_x, double *F_in) {
    if (F_in) *F_in = ntfo_cp_objective(N, dims, X, R, (const double *const *)A, beta, eps, eps_x);
    for (int n = 0; n < N; ++n)
        ntfo_cp_block_update(N, dims, X, R, A, n, beta, eps, eps_x, NULL, NULL);
}

/* One extrapolated B-CoMM outer iteration for CP (Section "Going beyond: Majorization-
 * Minimization with Extrapolation", item (i)).  A holds the current iterate A^t and becomes
 * A^(t+1); Aprev holds the previous outer iterate A^(t-1) and becomes A^t.  For n = 1..N:
 *   D = [A^(n) - Aprev^(n)]_+ (componentwise positive part, A^(n) not yet updated),
 *   alpha_n = min(alpha_nes, cap / (||D||_F + delta)),
 *   Ahat = max(A^(n) + alpha_n D, eps),
 * then the block update of Theorem "CP block multiplicative update" with Xhat rebuilt from
 * Ahat in mode n and the current other blocks, and Ahat as the multiplicative pre-factor.
 * F_in (may be NULL) receives the objective of the incoming iterate A^t.  Readings: the
 * previous iterate kept for the next call is the incoming one (so that the next
 * displacement is A^(t+1) - A^t); the cap is applied per block. */
void ntfo_cp_mu_sweep_extrap(int N, const int64_t *dims, const double *X, int R, double *const *A,
                             double *const *Aprev, double beta, double eps, double eps_x, double alpha_nes,
                             double cap, double delta, double *F_in) {
    if (F_in) *F_in = ntfo_cp_objective(N, dims, X, R, (const double *const *)A, beta, eps, eps_x);
    double *saved[8];
    for (int n = 0; n < N; ++n) {
        saved[n] = (double *)malloc(sizeof(double) * dims[n] * R);
        memcpy(saved[n], A[n], sizeof(double) * dims[n] * R);
    }
    for (int n = 0; n < N; ++n) {
        const int64_t cnt = dims[n] * R;
        double nrm2 = 0.0;
        for (int64_t e = 0; e < cnt; ++e) {
            const double d = A[n][e] - Aprev[n][e];
            if (d > 0.0) nrm2 += d * d;
        }
        double alpha = cap / (sqrt(nrm2) + delta);
        if (alpha_nes < alpha) alpha = alpha_nes;
        for (int64_t e = 0; e < cnt; ++e) {
            const double d = A[n][e] - Aprev[n][e];
            const double v = A[n][e] + alpha * (d > 0.0 ? d : 0.0);
            A[n][e] = v > eps ? v : eps;
        }
        /* block n now holds Ahat: the block update rebuilds Xhat from it and uses it as the
         * pre-factor */
        ntfo_cp_block_update(N, dims, X, R, A, n, beta, eps, eps_x, NULL, NULL);
    }
    for (int n = 0; n < N; ++n) {
        memcpy(Aprev[n], saved[n], sizeof(double) * dims[n] * R);
        free(saved[n]);
    }
}

/* One outer iteration of Algorithm 2 (J-CoMM) for CP with L inner sweeps (Section 5.3,
 * "CP inner update"): the reference is the incoming iterate; Ptilde/Qtilde are formed
 * once; each inner block update uses chi1 of the other current blocks for the numerator,
 * chi2 for the denominator, the reference block as pre-factor, then the eps clip.
 * F_ref (may be NULL) receives D_beta at the reference.  max_blocks >= 0 stops after that
 * many block updates (tests use it to inspect the state after each block). */
void ntfo_cp_jcomm_outer(int N, const int64_t *dims, const double *X, int R, double *const *A,
                         double beta, double eps, double eps_x, int L, int max_blocks,
                         double *F_ref) {
    int64_t cnt = numel(N, dims);
    double *At[NTFO_MAXN] = {0}, *C1[NTFO_MAXN] = {0}, *C2[NTFO_MAXN] = {0};
    for (int m = 0; m < N; ++m) {
        At[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        C1[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        C2[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        memcpy(At[m], A[m], sizeof(double) * dims[m] * R);
    }
    double *Xt = (double *)malloc(sizeof(double) * cnt);
    double *Pt = (double *)malloc(sizeof(double) * cnt);
    double *Qt = (double *)malloc(sizeof(double) * cnt);
    ntfo_cp_full(N, dims, R, (const double *const *)At, Xt);
    if (F_ref) *F_ref = objective_from_full(cnt, X, Xt, beta, eps, eps_x);
    powers(cnt, X, Xt, beta, eps, eps_x, Pt, Qt);
    int done = 0;
    for (int l = 0; l < L; ++l) {
        for (int n = 0; n < N; ++n) {
            if (max_blocks >= 0 && done++ >= max_blocks) break;
            for (int m = 0; m < N; ++m) {
                ntfo_chi1(dims[m] * R, A[m], At[m], beta, C1[m]);
                ntfo_chi2(dims[m] * R, A[m], At[m], beta, C2[m]);
            }
            double *num = (double *)malloc(sizeof(double) * dims[n] * R);
            double *den = (double *)malloc(sizeof(double) * dims[n] * R);
            ntfo_cp_contr(N, dims, Pt, R, (const double *const *)C1, n, num);
            ntfo_cp_contr(N, dims, Qt, R, (const double *const *)C2, n, den);
            ntfo_mu_apply(dims[n] * R, At[n], num, den, beta, eps, A[n]);
            free(num); free(den);
        }
    }
    for (int m = 0; m < N; ++m) { free(At[m]); free(C1[m]); free(C2[m]); }
    free(Xt); free(Pt); free(Qt);
}

/* One J-CoMM outer iteration from an extrapolated outer reference (Section "Going beyond:
 * Majorization-Minimization with Extrapolation", item (iii)).  A holds A^t (becomes the new
 * iterate), Aprev holds A^(t-1) (becomes A^t).  Every block is first moved to
 *   At^(n) = max(A^(n) + alpha_n [A^(n) - Aprev^(n)]_+, eps),
 *   alpha_n = min(alpha_nes, cap / (||[A^(n) - Aprev^(n)]_+||_F + delta)),
 * and the outer iteration of Algorithm 2 then runs with that point as its reference (and as
 * the inner iterations' starting point).  F_in (may be NULL) receives the objective of the
 * incoming iterate A^t.  Readings as for ntfo_cp_mu_sweep_extrap. */
void ntfo_cp_jcomm_outer_extrap(int N, const int64_t *dims, const double *X, int R, double *const *A,
                                double *const *Aprev, double beta, double eps, double eps_x, int L,
                                double alpha_nes, double cap, double delta, double *F_in) {
    if (F_in) *F_in = ntfo_cp_objective(N, dims, X, R, (const double *const *)A, beta, eps, eps_x);
    for (int n = 0; n < N; ++n) {
        const int64_t cnt = dims[n] * R;
        double nrm2 = 0.0;
        for (int64_t e = 0; e < cnt; ++e) {
            const double d = A[n][e] - Aprev[n][e];
            if (d > 0.0) nrm2 += d * d;
        }
        double alpha = cap / (sqrt(nrm2) + delta);
        if (alpha_nes < alpha) alpha = alpha_nes;
        for (int64_t e = 0; e < cnt; ++e) {
            const double a = A[n][e], d = a - Aprev[n][e];
            const double v = a + alpha * (d > 0.0 ? d : 0.0);
            Aprev[n][e] = a;
            A[n][e] = v > eps ? v : eps;
        }
    }
    ntfo_cp_jcomm_outer(N, dims, X, R, A, beta, eps, eps_x, L, -1, NULL);
}

/* Num^(n)/Den^(n) rows of one block update, for a few selected rows i_n only, with P and
 * Q evaluated entry by entry from the factors given (recon factors Ar for Xhat, Bn for the
 * numerator contraction, Bd for the denominator contraction).  Used to check single rows
 * of large problems that the full-tensor functions above cannot hold in memory. */
void ntfo_cp_numden_rows(int N, const int64_t *dims, const double *X, int R,
                         const double *const *Ar, const double *const *Bn,
                         const double *const *Bd, int n, double beta, double eps, double eps_x,
                         int nrows, const int64_t *rows, double *num, double *den) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nrows; ++q) {
        double *on = num + (int64_t)q * R, *od = den + (int64_t)q * R;
        for (int r = 0; r < R; ++r) on[r] = od[r] = 0.0;
        int64_t idx[NTFO_MAXN] = {0};
        idx[n] = rows[q];
        do {
            int64_t li = linear(N, dims, idx);
            double xh = ntfo_cp_entry(N, R, Ar, idx);
            double p, qq;
            powers(1, X + li, &xh, beta, eps, eps_x, &p, &qq);
            for (int r = 0; r < R; ++r) {
                double sn = p, sd = qq;
                for (int m = 0; m < N; ++m)
                    if (m != n) { sn *= Bn[m][idx[m] * R + r]; sd *= Bd[m][idx[m] * R + r]; }
                on[r] += sn;
                od[r] += sd;
            }
        } while (next_index(N, dims, n, idx));
    }
}

/* ----------------------------------------------------------------------------------
 * Tucker model (Section 3.3 "Nonnegative Tucker"; Appendix C, eq. (tucker_entry))
 * ---------------------------------------------------------------------------------- */

/* Xhat_i = sum_j G_j prod_n A^(n)_{i_n j_n}.  G is J_1 x ... x J_N row-major, A[n] is
 * I_n x J_n row-major. */
double ntfo_tucker_entry(int N, const int64_t *J, const double *G, const double *const *A,
                         const int64_t *idx) {
    int64_t j[NTFO_MAXN] = {0};
    double s = 0.0;
    int64_t t = 0;
    do {
        double p = G[t++];
        for (int n = 0; n < N; ++n) p *= A[n][idx[n] * J[n] + j[n]];
        s += p;
    } while (next_index(N, J, -1, j));
    return s;
}

void ntfo_tucker_full(int N, const int64_t *dims, const int64_t *J, const double *G,
                      const double *const *A, double *Xhat) {
    int64_t cnt = numel(N, dims);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t idx[NTFO_MAXN], rem = t;
        for (int m = N - 1; m >= 0; --m) { idx[m] = rem % dims[m]; rem /= dims[m]; }
        Xhat[t] = ntfo_tucker_entry(N, J, G, A, idx);
    }
}

double ntfo_tucker_objective(int N, const int64_t *dims, const double *X, const int64_t *J,
                             const double *G, const double *const *A, double beta, double eps,
                             double eps_x) {
    int64_t cnt = numel(N, dims);
    double *Xhat = (double *)malloc(sizeof(double) * cnt);
    ntfo_tucker_full(N, dims, J, G, A, Xhat);
    double f = objective_from_full(cnt, X, Xhat, beta, eps, eps_x);
    free(Xhat);
    return f;
}

/* Core contraction T x_1 B^(1)T ... x_N B^(N)T:
 *   out_j = sum_i T_i prod_n B^(n)_{i_n j_n}   (Appendix C, eq. (block_core_num_den)). */
void ntfo_tucker_core_contr(int N, const int64_t *dims, const double *T, const int64_t *J,
                            const double *const *B, double *out) {
    int64_t cj = numel(N, J);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t tj = 0; tj < cj; ++tj) {
        int64_t j[NTFO_MAXN], rem = tj;
        for (int m = N - 1; m >= 0; --m) { j[m] = rem % J[m]; rem /= J[m]; }
        int64_t idx[NTFO_MAXN] = {0};
        double s = 0.0;
        int64_t t = 0;
        do {
            double p = T[t++];
            for (int n = 0; n < N; ++n) p *= B[n][idx[n] * J[n] + j[n]];
            s += p;
        } while (next_index(N, dims, -1, idx));
        out[tj] = s;
    }
}

/* Partial tensor B^(n)_{j_n, i_-n} = sum_{j_-n} G_j prod_{m != n} A^(m)_{i_m j_m}
 * (Appendix C, eq. (block_Bn)).  Stored as J_n x prod_{m != n} I_m, i_-n row-major. */
void ntfo_tucker_partial(int N, const int64_t *dims, const int64_t *J, const double *G,
                         const double *const *A, int n, double *Bn) {
    int64_t rest = numel(N, dims) / dims[n];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t jn = 0; jn < J[n]; ++jn) {
        int64_t idx[NTFO_MAXN] = {0};
        int64_t t = 0;
        do {
            int64_t j[NTFO_MAXN] = {0};
            j[n] = jn;
            double s = 0.0;
            do {
                double p = G[linear(N, J, j)];
                for (int m = 0; m < N; ++m)
                    if (m != n) p *= A[m][idx[m] * J[m] + j[m]];
                s += p;
            } while (next_index(N, J, n, j));
            Bn[jn * rest + t++] = s;
        } while (next_index(N, dims, n, idx));
    }
}

/* Factor contraction out_{i_n j_n} = sum_{i_-n} T_i B^(n)_{j_n, i_-n} with B^(n) built
 * from (G, A) (Appendix C, eqs. (block_factor_num)/(block_factor_den); with transformed
 * blocks it is eqs. (jmm_factor_num)/(jmm_factor_den)). out is I_n x J_n. */
void ntfo_tucker_factor_contr(int N, const int64_t *dims, const double *T, const int64_t *J,
                              const double *G, const double *const *A, int n, double *out) {
    int64_t rest = numel(N, dims) / dims[n];
    double *Bn = (double *)malloc(sizeof(double) * J[n] * rest);
    ntfo_tucker_partial(N, dims, J, G, A, n, Bn);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t in = 0; in < dims[n]; ++in) {
        for (int64_t jn = 0; jn < J[n]; ++jn) out[in * J[n] + jn] = 0.0;
        int64_t idx[NTFO_MAXN] = {0};
        idx[n] = in;
        int64_t t = 0;
        do {
            double v = T[linear(N, dims, idx)];
            for (int64_t jn = 0; jn < J[n]; ++jn) out[in * J[n] + jn] += v * Bn[jn * rest + t];
            ++t;
        } while (next_index(N, dims, n, idx));
    }
    free(Bn);
}

/* Tucker block MM sweep (Theorem "Tucker block multiplicative updates"; Appendix C.2):
 * core first, then modes 1..N, each block rebuilding Xhat, P, Q from the current blocks,
 * followed by the eps clip.  F_in (may be NULL) receives the incoming objective.
 * max_blocks >= 0 stops after that many block updates (core = block 1). */
void ntfo_tucker_mu_sweep(int N, const int64_t *dims, const double *X, const int64_t *J,
                          double *G, double *const *A, double beta, double eps, double eps_x,
                          int max_blocks, double *F_in) {
    int64_t cnt = numel(N, dims), cj = numel(N, J);
    double *Xhat = (double *)malloc(sizeof(double) * cnt);
    double *P = (double *)malloc(sizeof(double) * cnt);
    double *Q = (double *)malloc(sizeof(double) * cnt);
    const double *const *Ac = (const double *const *)A;
    ntfo_tucker_full(N, dims, J, G, Ac, Xhat);
    if (F_in) *F_in = objective_from_full(cnt, X, Xhat, beta, eps, eps_x);
    /* core block */
    powers(cnt, X, Xhat, beta, eps, eps_x, P, Q);
    double *pc = (double *)malloc(sizeof(double) * cj), *qc = (double *)malloc(sizeof(double) * cj);
    ntfo_tucker_core_contr(N, dims, P, J, Ac, pc);
    ntfo_tucker_core_contr(N, dims, Q, J, Ac, qc);
    ntfo_mu_apply(cj, G, pc, qc, beta, eps, G);
    free(pc); free(qc);
    /* factor blocks */
    for (int n = 0; n < N; ++n) {
        if (max_blocks >= 0 && n + 1 >= max_blocks) break;
        ntfo_tucker_full(N, dims, J, G, Ac, Xhat);
        powers(cnt, X, Xhat, beta, eps, eps_x, P, Q);
        double *num = (double *)malloc(sizeof(double) * dims[n] * J[n]);
        double *den = (double *)malloc(sizeof(double) * dims[n] * J[n]);
        ntfo_tucker_factor_contr(N, dims, P, J, G, Ac, n, num);
        ntfo_tucker_factor_contr(N, dims, Q, J, G, Ac, n, den);
        ntfo_mu_apply(dims[n] * J[n], A[n], num, den, beta, eps, A[n]);
        free(num); free(den);
    }
    free(Xhat); free(P); free(Q);
}

/* Z <- max(Z + alpha [Z - Zprev]_+, eps) with alpha = min(alpha_nes, cap / (||[Z - Zprev]_+||_F
 * + delta)) (Section "Going beyond: Majorization-Minimization with Extrapolation"). */
static void extrap_block(int64_t cnt, double *Z, const double *Zprev, double alpha_nes, double cap, double delta,
                         double eps) {
    double nrm2 = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        const double d = Z[e] - Zprev[e];
        if (d > 0.0) nrm2 += d * d;
    }
    double alpha = cap / (sqrt(nrm2) + delta);
    if (alpha_nes < alpha) alpha = alpha_nes;
    for (int64_t e = 0; e < cnt; ++e) {
        const double d = Z[e] - Zprev[e];
        const double v = Z[e] + alpha * (d > 0.0 ? d : 0.0);
        Z[e] = v > eps ? v : eps;
    }
}

/* One extrapolated block-MM sweep for Tucker (Section "Going beyond: Majorization-
 * Minimization with Extrapolation", item (ii)): the core, then factors 1..N; before its update
 * each block is moved to its extrapolated point (the displacement from the previous outer
 * iterate, positive part, capped weight), Xhat is rebuilt with that block and the current
 * others, and the extrapolated block is the multiplicative pre-factor (Theorem "Tucker block
 * multiplicative updates", Appendix C.2).  G, A: G^t, A^t in, the new iterate out; Gprev, Aprev:
 * the previous outer iterate in, G^t, A^t out.  F_in (may be NULL): objective of the incoming
 * iterate. */
void ntfo_tucker_mu_sweep_extrap(int N, const int64_t *dims, const double *X, const int64_t *J, double *G,
                                 double *const *A, double *Gprev, double *const *Aprev, double beta, double eps,
                                 double eps_x, double alpha_nes, double cap, double delta, double *F_in) {
    int64_t cnt = numel(N, dims), cj = numel(N, J);
    double *Xhat = (double *)malloc(sizeof(double) * cnt);
    double *P = (double *)malloc(sizeof(double) * cnt);
    double *Q = (double *)malloc(sizeof(double) * cnt);
    const double *const *Ac = (const double *const *)A;
    if (F_in) {
        ntfo_tucker_full(N, dims, J, G, Ac, Xhat);
        *F_in = objective_from_full(cnt, X, Xhat, beta, eps, eps_x);
    }
    double *G0 = (double *)malloc(sizeof(double) * cj), *A0[NTFO_MAXN];
    memcpy(G0, G, sizeof(double) * cj);
    for (int n = 0; n < N; ++n) {
        A0[n] = (double *)malloc(sizeof(double) * dims[n] * J[n]);
        memcpy(A0[n], A[n], sizeof(double) * dims[n] * J[n]);
    }
    /* core block at its extrapolated point */
    extrap_block(cj, G, Gprev, alpha_nes, cap, delta, eps);
    ntfo_tucker_full(N, dims, J, G, Ac, Xhat);
    powers(cnt, X, Xhat, beta, eps, eps_x, P, Q);
    double *pc = (double *)malloc(sizeof(double) * cj), *qc = (double *)malloc(sizeof(double) * cj);
    ntfo_tucker_core_contr(N, dims, P, J, Ac, pc);
    ntfo_tucker_core_contr(N, dims, Q, J, Ac, qc);
    ntfo_mu_apply(cj, G, pc, qc, beta, eps, G);
    free(pc); free(qc);
    /* factor blocks */
    for (int n = 0; n < N; ++n) {
        extrap_block(dims[n] * J[n], A[n], Aprev[n], alpha_nes, cap, delta, eps);
        ntfo_tucker_full(N, dims, J, G, Ac, Xhat);
        powers(cnt, X, Xhat, beta, eps, eps_x, P, Q);
        double *num = (double *)malloc(sizeof(double) * dims[n] * J[n]);
        double *den = (double *)malloc(sizeof(double) * dims[n] * J[n]);
        ntfo_tucker_factor_contr(N, dims, P, J, G, Ac, n, num);
        ntfo_tucker_factor_contr(N, dims, Q, J, G, Ac, n, den);
        ntfo_mu_apply(dims[n] * J[n], A[n], num, den, beta, eps, A[n]);
        free(num); free(den);
    }
    memcpy(Gprev, G0, sizeof(double) * cj);
    free(G0);
    for (int n = 0; n < N; ++n) {
        memcpy(Aprev[n], A0[n], sizeof(double) * dims[n] * J[n]);
        free(A0[n]);
    }
    free(Xhat); free(P); free(Q);
}

/* Tucker J-CoMM outer iteration (Algorithm 2; Appendix C.3): reference tensors once
 * (eq. (ref_PQ)); per inner block the transformed blocks G_(1), G_(2), A_(1), A_(2);
 * core by eqs. (jmm_core_num)/(jmm_core_den), factors by eqs. (jmm_factor_num)/
 * (jmm_factor_den); the reference block is the pre-factor; eps clip after each block.
 * Block order: core, then modes 1..N.  max_blocks >= 0 stops after that many blocks. */
void ntfo_tucker_jcomm_outer(int N, const int64_t *dims, const double *X, const int64_t *J,
                             double *G, double *const *A, double beta, double eps, double eps_x,
                             int L, int max_blocks, double *F_ref) {
    int64_t cnt = numel(N, dims), cj = numel(N, J);
    double *Gt = (double *)malloc(sizeof(double) * cj);
    double *G1 = (double *)malloc(sizeof(double) * cj), *G2 = (double *)malloc(sizeof(double) * cj);
    memcpy(Gt, G, sizeof(double) * cj);
    double *At[NTFO_MAXN], *A1[NTFO_MAXN], *A2[NTFO_MAXN];
    for (int m = 0; m < N; ++m) {
        At[m] = (double *)malloc(sizeof(double) * dims[m] * J[m]);
        A1[m] = (double *)malloc(sizeof(double) * dims[m] * J[m]);
        A2[m] = (double *)malloc(sizeof(double) * dims[m] * J[m]);
        memcpy(At[m], A[m], sizeof(double) * dims[m] * J[m]);
    }
    double *Xt = (double *)malloc(sizeof(double) * cnt);
    double *Pt = (double *)malloc(sizeof(double) * cnt);
    double *Qt = (double *)malloc(sizeof(double) * cnt);
    ntfo_tucker_full(N, dims, J, Gt, (const double *const *)At, Xt);
    if (F_ref) *F_ref = objective_from_full(cnt, X, Xt, beta, eps, eps_x);
    powers(cnt, X, Xt, beta, eps, eps_x, Pt, Qt);
    int done = 0;
    for (int l = 0; l < L; ++l) {
        /* core block */
        if (max_blocks >= 0 && done++ >= max_blocks) break;
        for (int m = 0; m < N; ++m) {
            ntfo_chi1(dims[m] * J[m], A[m], At[m], beta, A1[m]);
            ntfo_chi2(dims[m] * J[m], A[m], At[m], beta, A2[m]);
        }
        double *pc = (double *)malloc(sizeof(double) * cj), *qc = (double *)malloc(sizeof(double) * cj);
        ntfo_tucker_core_contr(N, dims, Pt, J, (const double *const *)A1, pc);
        ntfo_tucker_core_contr(N, dims, Qt, J, (const double *const *)A2, qc);
        ntfo_mu_apply(cj, Gt, pc, qc, beta, eps, G);
        free(pc); free(qc);
        /* factor blocks */
        for (int n = 0; n < N; ++n) {
            if (max_blocks >= 0 && done++ >= max_blocks) break;
            ntfo_chi1(cj, G, Gt, beta, G1);
            ntfo_chi2(cj, G, Gt, beta, G2);
            for (int m = 0; m < N; ++m) {
                ntfo_chi1(dims[m] * J[m], A[m], At[m], beta, A1[m]);
                ntfo_chi2(dims[m] * J[m], A[m], At[m], beta, A2[m]);
            }
            double *num = (double *)malloc(sizeof(double) * dims[n] * J[n]);
            double *den = (double *)malloc(sizeof(double) * dims[n] * J[n]);
            ntfo_tucker_factor_contr(N, dims, Pt, J, G1, (const double *const *)A1, n, num);
            ntfo_tucker_factor_contr(N, dims, Qt, J, G2, (const double *const *)A2, n, den);
            ntfo_mu_apply(dims[n] * J[n], At[n], num, den, beta, eps, A[n]);
            free(num); free(den);
        }
    }
    for (int m = 0; m < N; ++m) { free(At[m]); free(A1[m]); free(A2[m]); }
    free(Gt); free(G1); free(G2); free(Xt); free(Pt); free(Qt);
}

/* Tucker J-CoMM outer iteration from an extrapolated outer reference (Section "Going beyond:
 * Majorization-Minimization with Extrapolation", item (iii)): every block (core and factors)
 * is first moved to its extrapolated point as in ntfo_tucker_mu_sweep_extrap, then the outer
 * iteration of Algorithm 2 runs from that reference.  Gprev / Aprev become the incoming
 * iterate; F_in (may be NULL) receives the objective of the incoming iterate. */
void ntfo_tucker_jcomm_outer_extrap(int N, const int64_t *dims, const double *X, const int64_t *J, double *G,
                                    double *const *A, double *Gprev, double *const *Aprev, double beta, double eps,
                                    double eps_x, int L, double alpha_nes, double cap, double delta, double *F_in) {
    int64_t cnt = numel(N, dims), cj = numel(N, J);
    if (F_in) {
        double *Xhat = (double *)malloc(sizeof(double) * cnt);
        ntfo_tucker_full(N, dims, J, G, (const double *const *)A, Xhat);
        *F_in = objective_from_full(cnt, X, Xhat, beta, eps, eps_x);
        free(Xhat);
    }
    double *G0 = (double *)malloc(sizeof(double) * cj);
    memcpy(G0, G, sizeof(double) * cj);
    extrap_block(cj, G, Gprev, alpha_nes, cap, delta, eps);
    memcpy(Gprev, G0, sizeof(double) * cj);
    free(G0);
    for (int n = 0; n < N; ++n) {
        const int64_t c = dims[n] * J[n];
        double *A0 = (double *)malloc(sizeof(double) * c);
        memcpy(A0, A[n], sizeof(double) * c);
        extrap_block(c, A[n], Aprev[n], alpha_nes, cap, delta, eps);
        memcpy(Aprev[n], A0, sizeof(double) * c);
        free(A0);
    }
    ntfo_tucker_jcomm_outer(N, dims, X, J, G, A, beta, eps, eps_x, L, -1, NULL);
}

/* ----------------------------------------------------------------------------------
 * Sparse COO tensors under KL (beta = 1), Section 6.3 "For sparse tensors"
 * idx is N arrays of nnz int32 coordinates; coordinates are unique.
 * ---------------------------------------------------------------------------------- */

static double coo_entry(int N, int R, const double *const *A, const int32_t *const *idx, int64_t e) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = 1.0;
        for (int n = 0; n < N; ++n) p *= A[n][(int64_t)idx[n][e] * R + r];
        s += p;
    }
    return s;
}

/* sum_i Xhat_i = sum_r prod_n sum_{i_n} A^(n)_{i_n r}. */
static double cp_total(int N, const int64_t *dims, int R, const double *const *A) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = 1.0;
        for (int n = 0; n < N; ++n) {
            double c = 0.0;
            for (int64_t i = 0; i < dims[n]; ++i) c += A[n][i * R + r];
            p *= c;
        }
        s += p;
    }
    return s;
}

/* D_1(X, Xhat) = sum_{stored} [x log(x / y) - x] + sum_{all i} Xhat_i, y = max(Xhat, eps)
 * on stored entries; the all-entries sum in closed form. */
double ntfo_coo_kl_objective(int N, const int64_t *dims, int64_t nnz, const int32_t *const *idx,
                             const double *vals, int R, const double *const *A, double eps) {
    double s = 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        double y = coo_entry(N, R, A, idx, e);
        if (y < eps) y = eps;
        double x = vals[e];
        s += (x > 0.0 ? x * log(x / y) : 0.0) - x;
    }
    return s + cp_total(N, dims, R, A);
}

/* CP J-CoMM outer iteration for a COO tensor at beta = 1: Ptilde = X / Xtilde is
 * nonzero only on stored entries, so each numerator is a loop over the nonzeros; Qtilde
 * is identically 1 and each denominator is Den^(n)_{i r} = prod_{m != n} colsum(chi2(A^(m)))_r
 * with chi2(Z, Zt) = Z at beta = 1. */
void ntfo_coo_kl_jcomm_outer(int N, const int64_t *dims, int64_t nnz, const int32_t *const *idx,
                             const double *vals, int R, double *const *A, double eps, int L,
                             double *F_ref) {
    const double beta = 1.0;
    double *At[NTFO_MAXN], *C1[NTFO_MAXN], *C2[NTFO_MAXN];
    for (int m = 0; m < N; ++m) {
        At[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        C1[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        C2[m] = (double *)malloc(sizeof(double) * dims[m] * R);
        memcpy(At[m], A[m], sizeof(double) * dims[m] * R);
    }
    if (F_ref) *F_ref = ntfo_coo_kl_objective(N, dims, nnz, idx, vals, R, (const double *const *)At, eps);
    double *Pt = (double *)malloc(sizeof(double) * nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        double y = coo_entry(N, R, (const double *const *)At, idx, e);
        if (y < eps) y = eps;
        Pt[e] = vals[e] / y; /* X * y^(beta-2) at beta = 1 */
    }
    for (int l = 0; l < L; ++l) {
        for (int n = 0; n < N; ++n) {
            for (int m = 0; m < N; ++m) {
                ntfo_chi1(dims[m] * R, A[m], At[m], beta, C1[m]);
                ntfo_chi2(dims[m] * R, A[m], At[m], beta, C2[m]);
            }
            double *num = (double *)calloc(dims[n] * R, sizeof(double));
            double *den = (double *)malloc(sizeof(double) * dims[n] * R);
            for (int64_t e = 0; e < nnz; ++e)
                for (int r = 0; r < R; ++r) {
                    double s = Pt[e];
                    for (int m = 0; m < N; ++m)
                        if (m != n) s *= C1[m][(int64_t)idx[m][e] * R + r];
                    num[(int64_t)idx[n][e] * R + r] += s;
                }
            for (int r = 0; r < R; ++r) {
                double p = 1.0;
                for (int m = 0; m < N; ++m) {
                    if (m == n) continue;
                    double c = 0.0;
                    for (int64_t i = 0; i < dims[m]; ++i) c += C2[m][i * R + r];
                    p *= c;
                }
                for (int64_t i = 0; i < dims[n]; ++i) den[i * R + r] = p;
            }
            ntfo_mu_apply(dims[n] * R, At[n], num, den, beta, eps, A[n]);
            free(num); free(den);
        }
    }
    for (int m = 0; m < N; ++m) { free(At[m]); free(C1[m]); free(C2[m]); }
    free(Pt);
}

/* CP block MM (Algorithm 1) on a COO tensor at beta = 1: per mode, Xhat on the stored
 * entries from the current factors, numerator over the nonzeros, closed-form denominator
 * prod_{m != n} colsum(A^(m)). */
void ntfo_coo_kl_mu_sweep(int N, const int64_t *dims, int64_t nnz, const int32_t *const *idx,
                          const double *vals, int R, double *const *A, double eps, double *F_in) {
    if (F_in) *F_in = ntfo_coo_kl_objective(N, dims, nnz, idx, vals, R, (const double *const *)A, eps);
    for (int n = 0; n < N; ++n) {
        double *num = (double *)calloc(dims[n] * R, sizeof(double));
        double *den = (double *)malloc(sizeof(double) * dims[n] * R);
        for (int64_t e = 0; e < nnz; ++e) {
            double y = coo_entry(N, R, (const double *const *)A, idx, e);
            if (y < eps) y = eps;
            double p = vals[e] / y;
            for (int r = 0; r < R; ++r) {
                double s = p;
                for (int m = 0; m < N; ++m)
                    if (m != n) s *= A[m][(int64_t)idx[m][e] * R + r];
                num[(int64_t)idx[n][e] * R + r] += s;
            }
        }
        for (int r = 0; r < R; ++r) {
            double p = 1.0;
            for (int m = 0; m < N; ++m) {
                if (m == n) continue;
                double c = 0.0;
                for (int64_t i = 0; i < dims[m]; ++i) c += A[m][i * R + r];
                p *= c;
            }
            for (int64_t i = 0; i < dims[n]; ++i) den[i * R + r] = p;
        }
        ntfo_mu_apply(dims[n] * R, A[n], num, den, 1.0, eps, A[n]);
        free(num); free(den);
    }
}

/* Stable permutation of 0..nnz-1 by an integer key in [0, K): a counting sort (count,
 * exclusive prefix sum, place in input order), which is stable by construction. */
void ntfo_stable_perm(int64_t nnz, const int32_t *key, int64_t K, int64_t *perm) {
    int64_t *start = (int64_t *)calloc(K + 1, sizeof(int64_t));
    for (int64_t e = 0; e < nnz; ++e) start[key[e] + 1]++;
    for (int64_t k = 0; k < K; ++k) start[k + 1] += start[k];
    for (int64_t e = 0; e < nnz; ++e) perm[start[key[e]]++] = e;
    free(start);
}
