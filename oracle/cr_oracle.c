/*
 * cr_oracle.c -- plain FP64 CPU oracle for the dual smoothing method of
 * Aybat & Wang, "A Parallelizable Dual Smoothing Method for Large Scale Convex
 * Regression Problems" (arXiv 1608.02227), specialised to K = N blocks (every
 * pairwise convexity constraint dualised, so Step 1 of P-APG has a closed form).
 *
 * TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the CPU-baseline leg of the
 * benchmark call this file; the CUDA library never does, and this file shares no
 * code, header or table with it.
 *
 * Conventions (Eq. (2) "original", Definition 1 of A1, A2):
 *   points x_l in R^n, l = 0..N-1, stored row-major X[l*n + k];
 *   the constraint of the ordered pair (i, j), i != j, is
 *       (C eta)_ij = y_j - y_i + xi_i . (x_i - x_j)  >= 0,
 *   and its multiplier theta_ij is stored at th[i*N + j] (diagonal unused, kept 0).
 *   With K = N, C = [A1 A2] (Definition 3: A3 = A1, A4 = A2).
 *
 * Every loop below is the definition written out; OpenMP only splits loops whose
 * iterations write disjoint outputs, so results do not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, N) ((size_t)(i) * (size_t)(N) + (size_t)(j))

/* (C eta)_ij for all ordered pairs (Eq. (2)); out[i*N+i] = 0. */
void cro_c_apply(int N, int n, const double *X, const double *y, const double *xi,
                 double *out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < N; ++j) {
            double v = 0.0;
            if (i != j) {
                double d = 0.0;
                for (int k = 0; k < n; ++k)
                    d += xi[(size_t)i * n + k] * (X[(size_t)i * n + k] - X[(size_t)j * n + k]);
                v = y[j] - y[i] + d;
            }
            out[IDX(i, j, N)] = v;
        }
    }
}

/* C^T theta = (a, b), the transpose of the map above (Definition 1):
 *   a_l = sum_{i != l} theta_il - sum_{j != l} theta_lj      (y-columns of A1)
 *   b_l = sum_{j != l} theta_lj (x_l - x_j)                 (xi-columns of A2)  */
void cro_ct_apply(int N, int n, const double *X, const double *th, double *a, double *b)
{
    /* column sums, each summed in increasing i; threads own disjoint column ranges */
    double *col = (double *)calloc((size_t)N, sizeof(double));
    const int CB = 256;
#pragma omp parallel for schedule(static)
    for (int l0 = 0; l0 < N; l0 += CB) {
        int l1 = l0 + CB < N ? l0 + CB : N;
        for (int i = 0; i < N; ++i)
            for (int l = l0; l < l1; ++l)
                if (l != i) col[l] += th[IDX(i, l, N)];
    }
#pragma omp parallel for schedule(static)
    for (int l = 0; l < N; ++l) {
        double row = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != l) row += th[IDX(l, j, N)];
        a[l] = col[l] - row;
        for (int k = 0; k < n; ++k) b[(size_t)l * n + k] = 0.0;
        for (int j = 0; j < N; ++j) {
            if (j == l) continue;
            double w = th[IDX(l, j, N)];
            for (int k = 0; k < n; ++k)
                b[(size_t)l * n + k] += w * (X[(size_t)l * n + k] - X[(size_t)j * n + k]);
        }
    }
    free(col);
}

/* Step 1 of P-APG with K = N: the unconstrained minimiser of
 *   1/2||y - ybar||^2 + gamma/2 ||xi||^2 - <C^T theta, eta>      (Eq. (g_gamma))
 * is y = ybar + a, xi = b / gamma with (a, b) = C^T theta.                      */
void cro_eta_of_theta(int N, int n, const double *X, const double *ybar, double gamma,
                      const double *th, double *y, double *xi)
{
    double *a = (double *)malloc((size_t)N * sizeof(double));
    double *b = (double *)malloc((size_t)N * n * sizeof(double));
    cro_ct_apply(N, n, X, th, a, b);
    for (int l = 0; l < N; ++l) y[l] = ybar[l] + a[l];
    for (size_t q = 0; q < (size_t)N * n; ++q) xi[q] = b[q] / gamma;
    free(a);
    free(b);
}

/* r_gamma(y, xi) = 1/2||y - ybar||^2 + gamma/2 ||xi||^2  (Eq. (regularize)) */
double cro_primal_obj(int N, int n, const double *ybar, double gamma, const double *y,
                      const double *xi)
{
    double s = 0.0, t = 0.0;
    for (int l = 0; l < N; ++l) s += (y[l] - ybar[l]) * (y[l] - ybar[l]);
    for (size_t q = 0; q < (size_t)N * n; ++q) t += xi[q] * xi[q];
    return 0.5 * s + 0.5 * gamma * t;
}

/* g_gamma(theta) = L_gamma(eta(theta), theta)
 *   = r_gamma(eta(theta)) - <theta, C eta(theta)>     (Eqs. (lagrangian), (g_gamma)).
 * Also returns r_gamma(eta(theta)), <theta, C eta(theta)> and, when y/xi are
 * non-NULL, eta(theta).  cbuf is an N*N scratch array.                          */
double cro_dual_obj(int N, int n, const double *X, const double *ybar, double gamma,
                    const double *th, double *cbuf, double *r_out, double *lg_out,
                    double *y_out, double *xi_out)
{
    double *y = y_out ? y_out : (double *)malloc((size_t)N * sizeof(double));
    double *xi = xi_out ? xi_out : (double *)malloc((size_t)N * n * sizeof(double));
    cro_eta_of_theta(N, n, X, ybar, gamma, th, y, xi);
    cro_c_apply(N, n, X, y, xi, cbuf);
    double *rowdot = (double *)malloc((size_t)N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i) s += th[IDX(i, j, N)] * cbuf[IDX(i, j, N)];
        rowdot[i] = s;
    }
    double lg = 0.0;
    for (int i = 0; i < N; ++i) lg += rowdot[i];
    double r = cro_primal_obj(N, n, ybar, gamma, y, xi);
    free(rowdot);
    if (!y_out) free(y);
    if (!xi_out) free(xi);
    if (r_out) *r_out = r;
    if (lg_out) *lg_out = lg;
    return r - lg;
}

/*
 * P-APG (Figure "papg") with K = N, taking `iters` iterations from the state
 * (theta^{k-1}, theta~^k, t_k).  With accel == 0 the momentum of Step 4 is dropped
 * (plain projected dual gradient ascent, the comparison in Section 5.1).
 *   Step 1  eta^k      = argmin of Eq. (g_gamma) at theta~^k        (closed form)
 *   Step 2  theta^k    = ( theta~^k - (1/L) C eta^k )_+
 *   Step 3  t_{k+1}    = (1 + sqrt(1 + 4 t_k^2)) / 2
 *   Step 4  theta~^{k+1} = theta^k + (t_k - 1)/t_{k+1} (theta^k - theta^{k-1})
 * In/out: th_prev (theta^{k-1} -> theta^{k-1+iters}), th_tilde (theta~^k ->
 * theta~^{k+iters}), *t (t_k -> t_{k+iters}).  All arrays N*N.
 * log_g / log_r / log_lg (length iters, may be NULL): g_gamma(theta^k),
 * r_gamma(eta(theta^k)) and <theta^k, C eta(theta^k)> after each iteration.
 * Returns 0, or -1 on allocation failure.
 */
int cro_papg(int N, int n, const double *X, const double *ybar, double gamma, double L,
             int iters, int accel, double *th_prev, double *th_tilde, double *t,
             double *log_g, double *log_r, double *log_lg)
{
    size_t NN = (size_t)N * N;
    double *y = (double *)malloc((size_t)N * sizeof(double));
    double *xi = (double *)malloc((size_t)N * n * sizeof(double));
    double *ceta = (double *)malloc(NN * sizeof(double));
    double *th_new = (double *)malloc(NN * sizeof(double));
    if (!y || !xi || !ceta || !th_new) {
        free(y); free(xi); free(ceta); free(th_new);
        return -1;
    }
    for (int it = 0; it < iters; ++it) {
        /* Step 1 */
        cro_eta_of_theta(N, n, X, ybar, gamma, th_tilde, y, xi);
        cro_c_apply(N, n, X, y, xi, ceta);
        /* Step 2 */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double v = 0.0;
                if (i != j) {
                    v = th_tilde[IDX(i, j, N)] - ceta[IDX(i, j, N)] / L;
                    if (v < 0.0) v = 0.0;
                }
                th_new[IDX(i, j, N)] = v;
            }
        /* Step 3 */
        double tk = *t;
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
        double beta = accel ? (tk - 1.0) / tn : 0.0;
        /* Step 4 */
#pragma omp parallel for schedule(static)
        for (long long q = 0; q < (long long)NN; ++q) {
            th_tilde[q] = th_new[q] + beta * (th_new[q] - th_prev[q]);
            th_prev[q] = th_new[q];
        }
        *t = tn;
        if (log_g || log_r || log_lg) {
            double r, lg;
            double g = cro_dual_obj(N, n, X, ybar, gamma, th_prev, ceta, &r, &lg, NULL, NULL);
            if (log_g) log_g[it] = g;
            if (log_r) log_r[it] = r;
            if (log_lg) log_lg[it] = lg;
        }
    }
    free(y); free(xi); free(ceta); free(th_new);
    return 0;
}

/*
 * P-APG with the adaptive step size of Section 4 ("Adaptive Step Size Strategy"),
 * taking `iters` iterations from the state (theta^{k-1}, theta~^k, t_k, s_{k-1}):
 * iteration k tries s_k = s_{k-1} * upsilon^(l - 1) for l = 0, 1, 2, ... and keeps the
 * first l for which Eq. (adaptive-check)
 *     g(theta^k) >= g(theta~^k) + <grad g(theta~^k), theta^k - theta~^k>
 *                   - (s_k / 2) ||theta^k - theta~^k||^2
 * holds, where theta^k = (theta~^k - C eta^k / s_k)_+ (Step 2 with 1/s_k for 1/L);
 * s_0 = L_gamma (the caller's initial *s).  Steps 1, 3 and 4 are those of Figure "papg".
 * g_gamma is a concave quadratic (Eq. (g_gamma) at eta(theta) is
 * -1/2||a||^2 - a.ybar - ||b||^2/(2 gamma) with (a, b) = C^T theta), so for D = theta^k - theta~^k
 * the check is exactly
 *     ||da||^2 + ||db||^2 / gamma <= s_k ||D||^2,   (da, db) = C^T D,
 * and s_k never exceeds L: Section 4 allows any s_k <= L_gamma, and at s_k = L (a bound on
 * the curvature of g_gamma) the check holds in exact arithmetic, so that candidate is kept
 * (rounding cannot push the step below the constant one).
 * which is how it is evaluated here (C^T applied to D over all pairs): the literal form
 * subtracts nearly equal objective values once the steps are small.  A test pins the
 * identity against the literal form.
 * In/out: th_prev, th_tilde, *t as in cro_papg; *s: s_{k-1} -> s_{k-1+iters}; *g_prev:
 * g(theta^{k-1}) for the restart test (NaN before the first iteration).
 * trials (length iters, may be NULL): l_k + 1, the candidate steps of each iteration.
 * log_g (may be NULL): g(theta^k).  Returns 0, -1 on allocation failure, -2 when no step
 * passes within 200 trials (non-finite data).
 */
int cro_papg_adaptive(int N, int n, const double *X, const double *ybar, double gamma,
                      double L, double upsilon, int iters, int accel, int restart, double *th_prev,
                      double *th_tilde, double *t, double *s, double *g_prev, int *trials, double *log_g)
{
    size_t NN = (size_t)N * N;
    double *y = (double *)malloc((size_t)N * sizeof(double));
    double *xi = (double *)malloc((size_t)N * n * sizeof(double));
    double *ceta = (double *)malloc(NN * sizeof(double));
    double *th_new = (double *)malloc(NN * sizeof(double));
    double *dif = (double *)malloc(NN * sizeof(double));
    double *da = (double *)malloc((size_t)N * sizeof(double));
    double *db = (double *)malloc((size_t)N * n * sizeof(double));
    if (!y || !xi || !ceta || !th_new || !dif || !da || !db) {
        free(y); free(xi); free(ceta); free(th_new); free(dif); free(da); free(db);
        return -1;
    }
    int rc = 0;
    for (int it = 0; it < iters && rc == 0; ++it) {
        /* Step 1 at theta~^k */
        cro_eta_of_theta(N, n, X, ybar, gamma, th_tilde, y, xi);
        cro_c_apply(N, n, X, y, xi, ceta);
        double sk = *s / upsilon;  /* l = 0 */
        int l = 0;
        for (;;) {
            /* Step 2 with step 1/s_k */
#pragma omp parallel for schedule(static)
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double v = 0.0;
                    if (i != j) {
                        v = th_tilde[IDX(i, j, N)] - ceta[IDX(i, j, N)] / sk;
                        if (v < 0.0) v = 0.0;
                    }
                    th_new[IDX(i, j, N)] = v;
                    dif[IDX(i, j, N)] = v - th_tilde[IDX(i, j, N)];
                }
            /* Eq. (adaptive-check) */
            cro_ct_apply(N, n, X, dif, da, db);
            double lhs = 0.0, nn = 0.0;
            for (int i = 0; i < N; ++i) lhs += da[i] * da[i];
            double bb = 0.0;
            for (size_t q = 0; q < (size_t)N * n; ++q) bb += db[q] * db[q];
            lhs += bb / gamma;
            for (int i = 0; i < N; ++i) {
                double nni = 0.0;
                for (int j = 0; j < N; ++j) nni += dif[IDX(i, j, N)] * dif[IDX(i, j, N)];
                nn += nni;
            }
            if (lhs <= sk * nn || sk >= L) break;  /* s_k = L always qualifies (s_k <= L allowed) */
            if (++l >= 200) {
                rc = -2;
                break;
            }
            sk = sk * upsilon < L ? sk * upsilon : L;
        }
        if (rc) break;
        if (trials) trials[it] = l + 1;
        *s = sk;
        /* Steps 3 and 4; with `restart`, t is reset to 1 (no momentum) when
         * g(theta^k) < g(theta^{k-1}) (function-value restart, not in the paper) */
        int reset = 0;
        if (restart) {
            const double g = cro_dual_obj(N, n, X, ybar, gamma, th_new, ceta, NULL, NULL, NULL, NULL);
            reset = *g_prev == *g_prev && g < *g_prev;  /* g_prev is NaN before the first iteration */
            *g_prev = g;
        }
        const double tk = *t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
        const double beta = (accel && !reset) ? (tk - 1.0) / tn : 0.0;
#pragma omp parallel for schedule(static)
        for (long long q = 0; q < (long long)NN; ++q) {
            th_tilde[q] = th_new[q] + beta * (th_new[q] - th_prev[q]);
            th_prev[q] = th_new[q];
        }
        *t = reset ? 1.0 : tn;
        if (log_g) log_g[it] = cro_dual_obj(N, n, X, ybar, gamma, th_prev, ceta, NULL, NULL, NULL, NULL);
    }
    free(y); free(xi); free(ceta); free(th_new); free(dif); free(da); free(db);
    return rc;
}

/*
 * Certified upper bound on p*_gamma from any (y, xi): the convex piecewise-linear
 * function f(x) = max_i ( y_i + xi_i . (x - x_i) ) is evaluated at every x_j;
 * y_rep_j = f(x_j) and xi_rep_j = xi_{m(j)} for a maximising piece m(j) form a
 * feasible point of Eq. (regularize) (subgradient inequality of a convex
 * function), so r_gamma(y_rep, xi_rep) >= p*_gamma.  Tie-break: m(j) = j when the
 * own piece attains the maximum, else the smallest maximising i.
 * Also returns sum_{i != j} min(0, (C eta)_ij)^2 of the input eta (the squared
 * infeasibility of Section 5.1).  out[0] = r_gamma(y_rep, xi_rep), out[1] = the
 * squared infeasibility.  yrep (N) and m (N) may be NULL.
 */
void cro_certify(int N, int n, const double *X, const double *ybar, double gamma,
                 const double *y, const double *xi, double *yrep, int *m, double *out)
{
    double *yr = (double *)malloc((size_t)N * sizeof(double));
    int *mm = (int *)malloc((size_t)N * sizeof(int));
    double *inf_col = (double *)malloc((size_t)N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j) {
        double best = y[j];
        int arg = j;
        double infs = 0.0;
        for (int i = 0; i < N; ++i) {
            if (i == j) continue;
            double d = 0.0;
            for (int k = 0; k < n; ++k)
                d += xi[(size_t)i * n + k] * (X[(size_t)j * n + k] - X[(size_t)i * n + k]);
            double v = y[i] + d;
            if (v > best) { best = v; arg = i; }
            double c = y[j] - v; /* (C eta)_ij */
            if (c < 0.0) infs += c * c;
        }
        yr[j] = best;
        mm[j] = arg;
        inf_col[j] = infs;
    }
    double s = 0.0, t = 0.0, inf = 0.0;
    for (int j = 0; j < N; ++j) {
        s += (yr[j] - ybar[j]) * (yr[j] - ybar[j]);
        for (int k = 0; k < n; ++k) {
            double v = xi[(size_t)mm[j] * n + k];
            t += v * v;
        }
        inf += inf_col[j];
    }
    out[0] = 0.5 * s + 0.5 * gamma * t;
    out[1] = inf;
    if (yrep) memcpy(yrep, yr, (size_t)N * sizeof(double));
    if (m) memcpy(m, mm, (size_t)N * sizeof(int));
    free(yr); free(mm); free(inf_col);
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int cro_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
