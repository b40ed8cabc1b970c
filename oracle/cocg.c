/*
 * Oracle: plain FP64 shifted COCG for (z S - H) x = e_j on scalar CSR matrices.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the CPU oracle; only tests/,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code with the GPU library.
 *
 * The equation is the generalized shifted linear equation of Eq. 2 (Sec. 3),
 * with A = H and B = S real symmetric, S positive definite (Sec. 2, Eq. 1).
 * The solver named for it in Sec. 3 is the generalized shifted COCG; the paper
 * gives no recurrences, so they are restated here from the shifted-Krylov
 * mathematics, in the order a reader checks them:
 *
 *   S-bilinear form <u,v> = u^T S v (unconjugated).  The seed operator
 *   K_s = z_s I - S^{-1} H is self-adjoint in it, so COCG applies to
 *   K_s x = S^{-1} b.  Write rt = S r for the residual of the original equation.
 *     rt_0 = b, r_0 = S^{-1} rt_0, p_{-1} = 0, beta_{-1} = 0, alpha_{-1} = 1
 *     loop n:
 *       p_n  = r_n + beta_{n-1} p_{n-1}        Sp_n = rt_n + beta_{n-1} Sp_{n-1}
 *       u    = z_s Sp_n - H p_n                (= (z_s S - H) p_n)
 *       alpha_n = rho_n / (p_n^T u),   rho_n = r_n^T rt_n
 *       rt_{n+1} = rt_n - alpha_n u,   r_{n+1} = S^{-1} rt_{n+1}   (inner CG on S)
 *       beta_n = rho_{n+1} / rho_n
 *   Shifted systems K_s + sigma I, sigma = z_m - z_s, have collinear residuals
 *   r^sigma_n = r_n / pi^sigma_n with pi^sigma_n = R_n(-sigma), R_n the seed's
 *   residual polynomial; its three-term recurrence gives
 *       pi_{n+1} = (1 + alpha_n sigma) pi_n + (alpha_n beta_{n-1}/alpha_{n-1})(pi_n - pi_{n-1})
 *       alpha^s_n = alpha_n pi_n / pi_{n+1},  beta^s_{n-1} = (pi_{n-1}/pi_n)^2 beta_{n-1}
 *       p^s_n = r_n / pi_n + beta^s_{n-1} p^s_{n-1},  x^s_{n+1} = x^s_n + alpha^s_n p^s_n
 *   and the original-equation residual of shift m is rt_{n+1} / pi_{n+1}.
 *   A shift is converged (and frozen) when ||rt_{n+1}|| / |pi_{n+1}| <= tol ||b||.
 *   Only the rows I_j of x^s that the caller asks for are kept: every shifted
 *   update is elementwise.
 *
 * S = NULL means S = I (then r = rt and no inner solve is made).  The inner
 * solve is textbook CG with Hermitian inner products from a zero start, to a
 * relative residual inner_tol.
 *
 * Column status: 0 converged, 1 max_iter reached, 2 breakdown (rho or mu is
 * zero), 3 non-finite value.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ST_CONVERGED = 0, ST_MAX_ITER = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3 };

typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *ci;
    const double *v;
} csr_t;

/* y = A x, A real CSR, x complex */
static void csr_mv(const csr_t *A, const cplx *x, cplx *y) {
    for (int64_t i = 0; i < A->n; ++i) {
        cplx s = 0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s += A->v[k] * x[A->ci[k]];
        y[i] = s;
    }
}

/* sum u_i v_i (unconjugated) */
static cplx dot_u(int64_t n, const cplx *u, const cplx *v) {
    cplx s = 0;
    for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

static double norm2(int64_t n, const cplx *u) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += creal(u[i]) * creal(u[i]) + cimag(u[i]) * cimag(u[i]);
    return sqrt(s);
}

/* Solve S y = v by CG (Hermitian forms) from y = 0.  Returns iterations used. */
static int cg_spd(const csr_t *S, const cplx *v, cplx *y, double tol, int max_it, cplx *r, cplx *d,
                  cplx *a) {
    const int64_t n = S->n;
    memset(y, 0, sizeof(cplx) * n);
    memcpy(r, v, sizeof(cplx) * n);
    memcpy(d, v, sizeof(cplx) * n);
    double rr = 0;
    for (int64_t i = 0; i < n; ++i) rr += creal(conj(r[i]) * r[i]);
    const double vnorm = sqrt(rr);
    if (vnorm == 0.0) return 0;
    int it = 0;
    while (it < max_it && sqrt(rr) > tol * vnorm) {
        csr_mv(S, d, a);
        double dad = 0;
        for (int64_t i = 0; i < n; ++i) dad += creal(conj(d[i]) * a[i]);
        const double al = rr / dad;
        double rr_new = 0;
        for (int64_t i = 0; i < n; ++i) {
            y[i] += al * d[i];
            r[i] -= al * a[i];
            rr_new += creal(conj(r[i]) * r[i]);
        }
        const double be = rr_new / rr;
        for (int64_t i = 0; i < n; ++i) d[i] = r[i] + be * d[i];
        rr = rr_new;
        ++it;
    }
    return it;
}

static int finite_c(cplx z) { return isfinite(creal(z)) && isfinite(cimag(z)); }

/*
 * One right-hand side b = e_j.  G_out[k*nz + m] = (x^{sigma_m})_{rows[k]}.
 */
static void solve_column(const csr_t *H, const csr_t *S, int nz, const cplx *z, int seed,
                         int64_t j, int64_t n_out, const int64_t *rows, double tol, int max_iter,
                         double inner_tol, int inner_max, cplx *G_out, double *resid, int *iters,
                         int *status, int *conv_it, cplx *rt_out, cplx *pi_out, int *inner_total) {
    const int64_t n = H->n;
    cplx *r = calloc(n, sizeof(cplx)), *rt = calloc(n, sizeof(cplx));
    cplx *p = calloc(n, sizeof(cplx)), *Sp = calloc(n, sizeof(cplx));
    cplx *q = calloc(n, sizeof(cplx)), *u = calloc(n, sizeof(cplx));
    cplx *w1 = NULL, *w2 = NULL, *w3 = NULL;
    if (S) {
        w1 = calloc(n, sizeof(cplx));
        w2 = calloc(n, sizeof(cplx));
        w3 = calloc(n, sizeof(cplx));
    }
    cplx *pi = malloc(sizeof(cplx) * nz), *pi_prev = malloc(sizeof(cplx) * nz);
    int *active = malloc(sizeof(int) * nz);
    cplx *xs = calloc((size_t)n_out * nz, sizeof(cplx)), *ps = calloc((size_t)n_out * nz, sizeof(cplx));
    int inner = 0;

    const cplx zs = z[seed];
    rt[j] = 1.0;
    const double bnorm = 1.0;
    if (S)
        inner += cg_spd(S, rt, r, inner_tol, inner_max, w1, w2, w3);
    else
        memcpy(r, rt, sizeof(cplx) * n);
    cplx rho = dot_u(n, r, rt);
    cplx beta_prev = 0, alpha_prev = 1;
    for (int m = 0; m < nz; ++m) {
        pi[m] = 1;
        pi_prev[m] = 1;
        active[m] = 1;
        resid[m] = 1.0;
        if (conv_it) conv_it[m] = -1;
    }
    int n_active = nz, it = 0, st = ST_MAX_ITER;
    while (it < max_iter) {
        for (int64_t i = 0; i < n; ++i) {
            p[i] = r[i] + beta_prev * p[i];
            Sp[i] = rt[i] + beta_prev * Sp[i];
        }
        csr_mv(H, p, q);
        for (int64_t i = 0; i < n; ++i) u[i] = zs * Sp[i] - q[i];
        const cplx mu = dot_u(n, p, u);
        if (!finite_c(mu) || !finite_c(rho)) { st = ST_NONFINITE; break; }
        if (mu == 0 || rho == 0) { st = ST_BREAKDOWN; break; }
        const cplx alpha = rho / mu;
        for (int m = 0; m < nz; ++m) {
            if (!active[m]) continue;
            const cplx sig = z[m] - zs;
            const cplx pi_next = (1.0 + alpha * sig) * pi[m] + (alpha * beta_prev / alpha_prev) * (pi[m] - pi_prev[m]);
            const cplx ratio = pi_prev[m] / pi[m];
            const cplx beta_s = ratio * ratio * beta_prev;
            const cplx alpha_s = pi[m] / pi_next * alpha;
            for (int64_t k = 0; k < n_out; ++k) {
                cplx *pk = &ps[k * nz + m];
                *pk = r[rows[k]] / pi[m] + beta_s * (*pk);
                xs[k * nz + m] += alpha_s * (*pk);
            }
            pi_prev[m] = pi[m];
            pi[m] = pi_next;
        }
        for (int64_t i = 0; i < n; ++i) rt[i] -= alpha * u[i];
        if (S)
            inner += cg_spd(S, rt, r, inner_tol, inner_max, w1, w2, w3);
        else
            memcpy(r, rt, sizeof(cplx) * n);
        const cplx rho_next = dot_u(n, r, rt);
        const double rnorm = norm2(n, rt);
        ++it;
        for (int m = 0; m < nz; ++m) {
            if (!active[m]) continue;
            const double res = rnorm / cabs(pi[m]);
            resid[m] = res;
            if (res <= tol * bnorm) {
                active[m] = 0;
                --n_active;
                if (conv_it) conv_it[m] = it;
            }
        }
        beta_prev = rho_next / rho;
        alpha_prev = alpha;
        rho = rho_next;
        if (n_active == 0) { st = ST_CONVERGED; break; }
    }
    memcpy(G_out, xs, sizeof(cplx) * n_out * nz);
    if (rt_out) memcpy(rt_out, rt, sizeof(cplx) * n);
    if (pi_out) memcpy(pi_out, pi, sizeof(cplx) * nz);
    *iters = it;
    *status = st;
    if (inner_total) *inner_total = inner;
    free(r); free(rt); free(p); free(Sp); free(q); free(u);
    free(w1); free(w2); free(w3);
    free(pi); free(pi_prev); free(active); free(xs); free(ps);
}

/*
 * All columns, OpenMP-parallel over columns (each column is an independent
 * solve).  Complex arrays are interleaved (re, im) doubles.
 *   G        [out_ptr[ncols]][nz]   iters, status [ncols]
 *   resid    [ncols][nz]            conv_it [ncols][nz] (optional)
 *   rt_out   [ncols][n] (optional)  pi_out [ncols][nz] (optional)
 */
int oracle_shifted_cocg(int64_t n, const int64_t *h_rp, const int32_t *h_ci, const double *h_v,
                        const int64_t *s_rp, const int32_t *s_ci, const double *s_v, int nz,
                        const double *z_ri, int seed, int64_t ncols, const int64_t *cols,
                        const int64_t *out_ptr, const int64_t *out_rows, double tol, int max_iter,
                        double inner_tol, int inner_max, double *G_ri, int *iters, double *resid,
                        int *status, int *conv_it, double *rt_ri, double *pi_ri, int *inner_its,
                        int nthreads) {
    if (n <= 0 || nz <= 0 || seed < 0 || seed >= nz) return -1;
    csr_t H = {n, h_rp, h_ci, h_v};
    csr_t S = {n, s_rp, s_ci, s_v};
    const csr_t *Sp = s_rp ? &S : NULL;
    const cplx *z = (const cplx *)z_ri;
    int64_t c;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (c = 0; c < ncols; ++c) {
        const int64_t o0 = out_ptr[c], o1 = out_ptr[c + 1];
        solve_column(&H, Sp, nz, z, seed, cols[c], o1 - o0, out_rows + o0, tol, max_iter, inner_tol,
                     inner_max, (cplx *)G_ri + o0 * nz, resid + c * nz, iters + c, status + c,
                     conv_it ? conv_it + c * nz : NULL, rt_ri ? (cplx *)rt_ri + c * n : NULL,
                     pi_ri ? (cplx *)pi_ri + c * nz : NULL, inner_its ? inner_its + c : NULL);
    }
    return 0;
}
