// Kernel templates and graph construction of the panel shifted COCG (see
// cocg_kernels.cuh); instantiated once per precision in inst_*.cu.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "cocg_kernels.cuh"
#include "dispatch.cuh"

namespace tbgf {

constexpr int NT = 256;

// ------------------------------------------------------------------ init
// Column state of a slot that starts column `col` of the queue (or an empty,
// finished slot when the queue has no such column).
template <typename T>
__device__ ColState fresh_column(const Panel<T> &p, int64_t col) {
    ColState C;
    memset(&C, 0, sizeof(C));
    C.alpha = mk(0.0, 0.0);
    C.alpha_prev = mk(1.0, 0.0);
    C.beta_prev = mk(0.0, 0.0);
    C.rho = mk(1.0, 0.0); // S = I: rho_0 = e_j^T e_j; S != I: replaced by the init pass
    C.rn2 = 1.0;
    C.status = TB_COL_MAX_ITER;
    C.n_active = p.nz;
    C.in_done = 1;
    C.zs = p.zs;
    C.chk_n = -1;
    if (col < p.n_cols) {
        C.row = p.col_row[col];
        C.dst = col;
        C.ent0 = p.col_ptr[col];
        C.n_ent = (int32_t)(p.col_ptr[col + 1] - C.ent0);
    } else {
        C.row = C.dst = -1;
        C.done = 1;
        C.n_active = 0;
        C.rho = mk(0.0, 0.0);
        C.rn2 = 0.0;
        C.status = TB_COL_CONVERGED;
    }
    return C;
}

__device__ __forceinline__ ShiftState fresh_shift() {
    ShiftState S;
    S.pi = S.pi_prev = S.pi_next = mk(1.0, 0.0);
    S.alpha_s = mk(0.0, 0.0);
    S.resid = 1.0;
    S.active = 1;
    S.conv_it = -1;
    S.qinv = S.qinv0 = 0.0;
    return S;
}

// A restarting column (a stall restart, or a slot that took the next column of
// the queue) starts its recurrences again with beta = 0: its previous direction
// and the vectors kept by recurrence are cleared, so that nothing of the old
// column (not even an inf or a NaN) survives the multiplication by zero.
template <typename T, int W>
__device__ __forceinline__ void clear_restart_row(const Panel<T> &p, int n, int64_t row, int col) {
    const int64_t o = (row * W + col) * 2;
    T *pp = p.P[n & 1];
    pp[o] = pp[o + 1] = (T)0;
    if (p.SP) p.SP[o] = p.SP[o + 1] = (T)0;
    if (p.HP) p.HP[o] = p.HP[o + 1] = (T)0;
}

template <typename T, int W>
__global__ void k_init_state(Panel<T> p, int has_s) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) p.col[c] = fresh_column(p, c);
    for (int q = threadIdx.x; q < W * p.nz; q += blockDim.x) p.sh[q] = fresh_shift();
    if (threadIdx.x == 0) {
        p.ctl->arrive = 0;
        p.ctl->n = has_s ? 1 : 0;
        p.ctl->k = 0;
        p.ctl->panel_done = 0;
        p.ctl->inner_done = 0;
        p.ctl->iter_ctr = 0;
        p.ctl->in_ctr = 0;
        p.ctl->next_col = p.n_cols < W ? p.n_cols : W;
        p.ctl->inner_total = 0;
        p.ctl->refine_total = 0;
        p.ctl->light_total = 0;
        p.ctl->refine_now = 0;
    }
}

template <typename T, int W>
__global__ void k_init_vec(Panel<T> p, int64_t n_rows, int has_s) {
    const int64_t total = n_rows * W;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t row = t / W;
        const int c = (int)(t % W);
        const int64_t j = p.col[c].row;
        const T one = (j == row) ? (T)1 : (T)0;
        const int64_t o = t * 2;
        p.RT[o] = one, p.RT[o + 1] = 0;
        p.P[0][o] = p.P[0][o + 1] = 0;
        p.P[1][o] = p.P[1][o + 1] = 0;
        p.U[o] = p.U[o + 1] = 0;
        if (has_s) {
            p.R[0][o] = p.R[0][o + 1] = 0;
            p.R[1][o] = one, p.R[1][o + 1] = 0;
            p.SP[o] = p.SP[o + 1] = 0;
            p.Tv[o] = p.Tv[o + 1] = 0;
            p.D[0][o] = p.D[0][o + 1] = 0;
            p.D[1][o] = p.D[1][o + 1] = 0;
            p.Av[o] = p.Av[o + 1] = 0;
        }
        if (p.HP) p.HP[o] = p.HP[o + 1] = 0;
    }
    const int64_t ne = (int64_t)W * p.max_col_ent * p.nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ne; t += stride) {
        p.xs[t] = mk(0.0, 0.0);
        p.ps[t] = mk(0.0, 0.0);
        if (p.xq) p.xq[t] = mk(0.0, 0.0);
    }
}

// ------------------------------------------------------------ shifted steps
// The (slot, shift) pairs are split into contiguous ranges, one per CTA.  Each
// range is processed in chunks: phase 1, one thread per pair, runs the FP64
// shifted recurrence and leaves two coefficients in shared memory; phase 2
// spreads the (pair, kept row) updates over all threads of the CTA, so the
// kept rows of a column are updated in parallel, not one after another.
constexpr int PAIR_CHUNK = 128;

// A refinement pass takes S c in FP32 when every refining column's residual is
// below REFINE_LIGHT times its inner tolerance target: the FP32 product's error
// (about 1e-6 of the correction) then stays below inner_tol ||rt|| / 20.
constexpr double REFINE_LIGHT = 5e4;

// Resident CTAs per SM that IC_A and C are compiled for: four for df
// panels with block edges <= 4 (64 registers suffice), otherwise the three of
// the other kernels (the FP64 and FP32 variants would spill at 64).
template <typename T, int B>
constexpr int ctas_light() {
    return B <= 4 ? (std::is_same<T, df>::value ? 4 : 3) : 1;
}

// A(n): rotate pi, test ||rt_n|| / |pi_n| <= tol, then p^m_n = r_n / pi_n + beta^m_{n-1} p^m_{n-1}.
// gsQMR: the QMR iterate is the COCG one smoothed (Zhou & Walker's QMR smoothing,
// equal in exact arithmetic to QMR on the complex-symmetric Lanczos process of
// the same Krylov space): with omega_n = sqrt|rho_n| / |pi_n| the quasi-norm of
// the shift's COCG residual (rho_n = r_n^T S r_n), 1/tau_n^2 = 1/tau_{n-1}^2 +
// 1/omega_n^2 and xq_n = xq_{n-1} + (tau_n^2 / omega_n^2)(x_n - xq_{n-1}); the shift
// stops when tau_n / tau_0 <= tol.
template <typename T, int W>
__device__ void pair_step_A(const Panel<T> &p, const T *__restrict__ Rc, int n) {
    __shared__ c64 s_a[PAIR_CHUNK], s_b[PAIR_CHUNK];
    __shared__ double s_eta[PAIR_CHUNK];
    __shared__ int s_c[PAIR_CHUNK], s_m[PAIR_CHUNK], s_on[PAIR_CHUNK];
    const int P = W * p.nz;
    const int q0 = (int)((int64_t)blockIdx.x * P / gridDim.x), q1 = (int)((int64_t)(blockIdx.x + 1) * P / gridDim.x);
    const int KM = p.max_col_ent;
    for (int base = q0; base < q1; base += PAIR_CHUNK) {
        const int np = min(PAIR_CHUNK, q1 - base);
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            const int q = base + t, c = q / p.nz, m = q % p.nz;
            int on = 0;
            ColState &C = p.col[c];
            ShiftState &S = p.sh[q];
            if (!C.done && S.active) {
                S.pi_prev = S.pi;
                S.pi = S.pi_next;
                double res;
                if (p.qmr) {
                    const double w2inv = cabs2(S.pi) / sqrt(cabs2(C.rho)); // 1 / omega_n^2
                    if (S.qinv == 0.0) S.qinv0 = w2inv;
                    S.qinv += w2inv;
                    s_eta[t] = w2inv / S.qinv;
                    res = sqrt(S.qinv0 / S.qinv);
                    on = 2; // smoothing update of the kept rows
                } else {
                    res = sqrt(C.rn2) / sqrt(cabs2(S.pi));
                }
                S.resid = res;
                if (res <= p.tol) {
                    S.active = 0;
                    S.conv_it = n;
                    atomicSub(&C.n_active, 1);
                } else {
                    const c64 ratio = cdiv(S.pi_prev, S.pi);
                    s_b[t] = (ratio * ratio) * C.beta_prev;
                    s_a[t] = cdiv(mk(1.0, 0.0), S.pi);
                    on |= 1;
                }
            }
            s_on[t] = on;
            s_c[t] = c;
            s_m[t] = m;
            if (p.rowpar) { // k_rows_A applies them
                p.flagA[q] = on;
                if (on & 1) p.coefA[2 * q] = s_a[t], p.coefA[2 * q + 1] = s_b[t];
                if (on & 2) p.etaA[q] = s_eta[t];
            }
        }
        __syncthreads();
        if (p.rowpar) continue;
        // pairs fastest: the pairs of a chunk are consecutive shifts of a column, so
        // consecutive threads touch consecutive entries of a kept row (coalesced)
        for (int64_t i = threadIdx.x; i < (int64_t)np * KM; i += blockDim.x) {
            const int t = (int)(i % np), k = (int)(i / np);
            if (!s_on[t]) continue;
            const int c = s_c[t], m = s_m[t];
            const ColState &C = p.col[c];
            if (k >= C.n_ent) continue;
            const int64_t e = ((int64_t)c * KM + k) * p.nz + m;
            if (s_on[t] & 2) p.xq[e] = p.xq[e] + s_eta[t] * (p.xs[e] - p.xq[e]);
            if (!(s_on[t] & 1)) continue;
            const int64_t row = p.ent_row[C.ent0 + k];
            const T *rp = Rc + (row * W + c) * 2;
            const c64 rv = mk((double)rp[0], (double)rp[1]);
            p.ps[e] = s_a[t] * rv + s_b[t] * p.ps[e];
        }
        __syncthreads();
    }
}

// B(n) / B'(n): pi_{n+1}, alpha^m_n and x^m += alpha^m_n p^m_n on the kept rows.
template <typename T, int W>
__device__ void pair_step_B(const Panel<T> &p) {
    __shared__ c64 s_a[PAIR_CHUNK];
    __shared__ int s_c[PAIR_CHUNK], s_m[PAIR_CHUNK], s_on[PAIR_CHUNK];
    const int P = W * p.nz;
    const int q0 = (int)((int64_t)blockIdx.x * P / gridDim.x), q1 = (int)((int64_t)(blockIdx.x + 1) * P / gridDim.x);
    const int KM = p.max_col_ent;
    for (int base = q0; base < q1; base += PAIR_CHUNK) {
        const int np = min(PAIR_CHUNK, q1 - base);
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            const int q = base + t, c = q / p.nz, m = q % p.nz;
            int on = 0;
            ColState &C = p.col[c];
            ShiftState &S = p.sh[q];
            if (!C.done && S.active) {
                const c64 sig = p.z[m] - C.zs;
                const c64 coef = cdiv(C.alpha * C.beta_prev, C.alpha_prev);
                const c64 pn = (mk(1.0, 0.0) + C.alpha * sig) * S.pi + coef * (S.pi - S.pi_prev);
                const c64 as = cdiv(S.pi, pn) * C.alpha;
                if (!cfinite(pn) || (pn.re == 0.0 && pn.im == 0.0) || !cfinite(as)) {
                    S.active = 0;
                    S.resid = nan("");
                    C.breakdown = 1;
                    atomicSub(&C.n_active, 1);
                } else {
                    S.pi_next = pn;
                    S.alpha_s = as;
                    s_a[t] = as;
                    on = 1;
                }
            }
            s_on[t] = on;
            s_c[t] = c;
            s_m[t] = m;
            if (p.rowpar) { // k_rows_B applies it
                p.flagB[q] = on;
                if (on) p.coefB[q] = s_a[t];
            }
        }
        __syncthreads();
        if (p.rowpar) continue;
        // pairs fastest: the pairs of a chunk are consecutive shifts of a column, so
        // consecutive threads touch consecutive entries of a kept row (coalesced)
        for (int64_t i = threadIdx.x; i < (int64_t)np * KM; i += blockDim.x) {
            const int t = (int)(i % np), k = (int)(i / np);
            if (!s_on[t]) continue;
            const int c = s_c[t], m = s_m[t];
            if (k >= p.col[c].n_ent) continue;
            const int64_t e = ((int64_t)c * KM + k) * p.nz + m;
            p.xs[e] = p.xs[e] + s_a[t] * p.ps[e];
        }
        __syncthreads();
    }
}

// ----------------------------------------------- row-parallel kept-row updates
// With many kept rows per column (full-vector shifted solutions) the pair steps
// only compute the per-pair coefficients; these kernels apply them to every
// (column, kept row, shift), shifts fastest, so the FP64 complex arrays stream
// at full width.  A column that restarts in this iteration (a stall restart or a
// slot that took the next column) is skipped: A has already cleared its arrays.
// k_rows_A (after A): p^m_n = r_n / pi_n + beta^m_{n-1} p^m_{n-1}; gsQMR smoothing.
// Index of work item t: column c, kept row k, shift m (32-bit division when the
// work fits, the common case).
__device__ __forceinline__ void rows_index(int64_t t, int64_t per, int nz, bool small, int &c, int64_t &k, int &m) {
    if (small) {
        const uint32_t tt = (uint32_t)t, pp = (uint32_t)per, cc = tt / pp, r = tt - cc * pp, kk = r / (uint32_t)nz;
        c = (int)cc, k = kk, m = (int)(r - kk * (uint32_t)nz);
    } else {
        c = (int)(t / per);
        const int64_t r = t - (int64_t)c * per;
        k = r / nz;
        m = (int)(r - k * nz);
    }
}

template <typename T, int W>
__global__ void k_rows_A(Panel<T> p, int has_s) {
    const int n = p.ctl->n;
    const T *Rc = has_s ? p.R[n & 1] : p.RT;
    const int64_t KM = p.max_col_ent, per = KM * p.nz;
    const bool small = W * per < (int64_t)UINT32_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < W * per; t += stride) {
        int c, m;
        int64_t k;
        rows_index(t, per, p.nz, small, c, k, m);
        const ColState &C = p.col[c];
        if (k >= C.n_ent || C.restart) continue;
        const int64_t q = (int64_t)c * p.nz + m;
        const int on = p.flagA[q];
        if (!on) continue;
        if (on & 2) p.xq[t] = p.xq[t] + p.etaA[q] * (p.xs[t] - p.xq[t]);
        if (on & 1) {
            const int64_t row = p.ent_row[C.ent0 + k];
            const T *rp = Rc + (row * W + c) * 2;
            p.ps[t] = p.coefA[2 * q] * mk((double)rp[0], (double)rp[1]) + p.coefA[2 * q + 1] * p.ps[t];
        }
    }
}

// k_rows_B (after B / B'): x^m += alpha^m_n p^m_n.
template <typename T, int W>
__global__ void k_rows_B(Panel<T> p) {
    const int64_t KM = p.max_col_ent, per = KM * p.nz;
    const bool small = W * per < (int64_t)UINT32_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < W * per; t += stride) {
        int c, m;
        int64_t k;
        rows_index(t, per, p.nz, small, c, k, m);
        if (k >= p.col[c].n_ent) continue;
        const int64_t q = (int64_t)c * p.nz + m;
        if (p.flagB[q]) p.xs[t] = p.xs[t] + p.coefB[q] * p.ps[t];
    }
}

// -------------------------------------------------------------- kernel A
template <typename T, int B, int W, bool HAS_S>
__global__ void __launch_bounds__(NT, (B <= 4 ? 3 : 1)) k_outer(Panel<T> p) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    // H p_n: with FP64 and df panels, H r_n + beta_{n-1} (H p_{n-1}) (one
    // product of the finished r_n, H p kept by this recurrence, so the product
    // reads plain neighbour rows); with FP32 panels, the product of p_n formed
    // on the fly from r_n and p_{n-1}.
    constexpr bool HP_REC = !std::is_same<T, float>::value;
    const int n = p.ctl->n;
    const T *Rc = HAS_S ? p.R[n & 1] : p.RT;
    T *Pnew = p.P[n & 1];
    LdAxpy<T, W> ld; // p_n = r_n + beta_{n-1} p_{n-1}
    ld.a = Rc;
    ld.b = p.P[(n + 1) & 1];
    ld.lane = lane;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const ColState &C = p.col[lane * CPT + cc];
        ld.s[cc] = C.done ? mk<T>(0, 0) : cvt<T>(C.beta_prev);
    }
    LdAxpy<T, W> lr = ld; // r_n
    lr.b = nullptr;
    cpx<T> zs[CPT]; // each column's seed shift
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) zs[cc] = cvt<T>(p.col[lane * CPT + cc].zs);
    Acc<T> acc[CPT][2];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero(), acc[cc][1].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
        cpx<T> y[B][CPT];
        if constexpr (HP_REC)
            bsr_row_product<T, B>(p.h_rp, p.h_ci, p.h_val, br, lr, y);
        else
            bsr_row_product<T, B>(p.h_rp, p.h_ci, p.h_val, br, ld, y);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int64_t row = br * B + i;
            cpx<T> pv[CPT], u[CPT];
            ld(row, pv);
            st_row<T, W>(Pnew, row, lane, pv);
            if constexpr (HP_REC) {
                cpx<T> hp[CPT];
                ld_row<T, W>(p.HP, row, lane, hp);
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) y[i][cc] = y[i][cc] + ld.s[cc] * hp[cc];
                st_row<T, W>(p.HP, row, lane, y[i]);
            }
            if constexpr (HAS_S) {
                cpx<T> rt[CPT], sp[CPT];
                ld_row<T, W>(p.RT, row, lane, rt);
                ld_row<T, W>(p.SP, row, lane, sp);
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    sp[cc] = rt[cc] + ld.s[cc] * sp[cc];
                    u[cc] = zs[cc] * sp[cc] - y[i][cc];
                }
                st_row<T, W>(p.SP, row, lane, sp);
            } else {
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) u[cc] = zs[cc] * pv[cc] - y[i][cc];
            }
            st_row<T, W>(p.U, row, lane, u);
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                acc[cc][0].add(pv[cc].re * u[cc].re);
                acc[cc][0].add(-(pv[cc].im * u[cc].im));
                acc[cc][1].add(pv[cc].re * u[cc].im);
                acc[cc][1].add(pv[cc].im * u[cc].re);
            }
        }
    }
    cta_partials<T, W, NT, 2>(acc, p.part);
    pair_step_A<T, W>(p, Rc, n);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    // ---- last CTA: alpha_n = rho_n / mu_n; column completion, retire and refill
    __shared__ double red[W * 2];
    __shared__ int fin[W], n_fin; // slots whose column finished in this iteration
    if (threadIdx.x == 0) n_fin = 0;
    reduce_partials<T, W, NT, 2>(p.part, red);
    for (int c = threadIdx.x; c < W; c += NT) {
        ColState &C = p.col[c];
        if (C.done) continue;
        const c64 mu = mk(red[2 * c], red[2 * c + 1]);
        const int n_active = atomicAdd(&C.n_active, 0);
        int st = -1;
        if (C.s_bad)
            st = TB_COL_BREAKDOWN; // S is not positive definite on an inner CG direction
        else if (n_active <= 0)
            st = C.breakdown ? TB_COL_BREAKDOWN : TB_COL_CONVERGED;
        else if (!cfinite(mu) || !cfinite(C.rho))
            st = TB_COL_NONFINITE;
        else if ((mu.re == 0.0 && mu.im == 0.0) || (C.rho.re == 0.0 && C.rho.im == 0.0))
            st = TB_COL_BREAKDOWN;
        else if (C.iters >= p.max_iter)
            st = TB_COL_MAX_ITER;
        c64 a = mk(0.0, 0.0);
        if (st < 0) {
            a = cdiv(C.rho, mu);
            if (!cfinite(a)) st = TB_COL_NONFINITE;
        }
        if (st >= 0) {
            C.done = 1;
            C.status = st;
            C.alpha = mk(0.0, 0.0);
            fin[atomicAdd(&n_fin, 1)] = c;
        } else {
            C.alpha = a;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) // slots take the queue's columns in slot order (deterministic)
        for (int f = 1; f < n_fin; ++f)
            for (int g = f; g > 0 && fin[g - 1] > fin[g]; --g) {
                const int x = fin[g];
                fin[g] = fin[g - 1];
                fin[g - 1] = x;
            }
    __syncthreads();
    if (n_fin > 0) {
        // retire: the finished columns' results go out now, so that their slots
        // can take the next columns of the queue in this same iteration
        const int KM = p.max_col_ent;
        for (int f = 0; f < n_fin; ++f) {
            const ColState &C = p.col[fin[f]];
            const int64_t base = (int64_t)fin[f] * KM * p.nz, ne = (int64_t)C.n_ent * p.nz;
            const c64 *xo = p.qmr ? p.xq : p.xs;
            for (int64_t t = threadIdx.x; t < ne; t += NT) {
                c64 v = xo[base + t];
                if (p.rowpar && p.qmr) { // this iteration's smoothing step is still pending (k_rows_A)
                    const int64_t q = (int64_t)fin[f] * p.nz + t % p.nz;
                    if (p.flagA[q] & 2) v = v + p.etaA[q] * (p.xs[base + t] - v);
                }
                p.G[C.ent0 * p.nz + t] = v;
            }
            for (int m = threadIdx.x; m < p.nz; m += NT)
                p.resid[C.dst * p.nz + m] = p.sh[(int64_t)fin[f] * p.nz + m].resid;
        }
        __syncthreads();
        // refill: the next column starts through the restart path (alpha = 0 this
        // iteration, B / B' set its rt to e_j and clear its old directions, C
        // starts its recurrences); the restart iteration is not counted
        for (int f = threadIdx.x; f < n_fin; f += NT) {
            ColState &C = p.col[fin[f]];
            p.iters[C.dst] = C.iters;
            p.status[C.dst] = C.status;
            const int64_t next = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&p.ctl->next_col), 1ull);
            ColState N = fresh_column(p, next);
            if (N.dst >= 0) {
                N.restart = 1;
                N.fresh = 1;
                N.iters = -1;
            }
            C = N;
        }
        __syncthreads();
        for (int f = 0; f < n_fin; ++f) {
            const int c = fin[f];
            if (p.col[c].dst < 0) continue; // the queue is empty: the slot stays idle
            for (int m = threadIdx.x; m < p.nz; m += NT) p.sh[(int64_t)c * p.nz + m] = fresh_shift();
            const int64_t base = (int64_t)c * KM * p.nz;
            for (int64_t t = threadIdx.x; t < (int64_t)KM * p.nz; t += NT) {
                p.xs[base + t] = mk(0.0, 0.0);
                p.ps[base + t] = mk(0.0, 0.0);
                if (p.xq) p.xq[base + t] = mk(0.0, 0.0);
            }
        }
        __syncthreads();
    }
    // Restart (df panels): a shift's residual is the seed's divided by |pi|, so
    // a shift much harder than the seed needs the seed residual below what df
    // carries (about 1e-10).  Once a column's seed residual is below that, its
    // worst active shift is checked every 512 iterations; if it improved by
    // less than 1 % the column restarts with that shift as its seed: alpha = 0
    // this iteration, B / B' reset rt to e_j, C restarts the recurrences;
    // converged shifts keep their solutions, active ones start from zero.
    if (p.stall2 > 0.0) {
        const int KM = p.max_col_ent;
        for (int c = threadIdx.x; c < W; c += NT) {
            ColState &C = p.col[c];
            if (C.done || !(C.rn2 < p.stall2) || C.restarts >= 2) continue;
            if (C.chk_n >= 0 && C.iters - C.chk_n < 512) continue;
            double rw = -1.0;
            int mw = -1;
            for (int m = 0; m < p.nz; ++m) {
                const ShiftState &S = p.sh[(int64_t)c * p.nz + m];
                if (S.active && S.resid > rw) rw = S.resid, mw = m;
            }
            if (mw < 0) continue;
            if (C.chk_n < 0 || rw < 0.99 * C.chk_w) {
                C.chk_n = C.iters;
                C.chk_w = rw;
                continue;
            }
            C.zs = p.z[mw];
            C.restart = 1;
            C.restarts += 1;
            C.chk_n = -1;
            C.alpha = mk(0.0, 0.0);
            for (int m = 0; m < p.nz; ++m) {
                ShiftState &S = p.sh[(int64_t)c * p.nz + m];
                if (!S.active) continue;
                S.pi = S.pi_prev = S.pi_next = mk(1.0, 0.0);
                S.resid = 1.0;
                for (int k = 0; k < C.n_ent; ++k) {
                    p.xs[((int64_t)c * KM + k) * p.nz + m] = mk(0.0, 0.0);
                    p.ps[((int64_t)c * KM + k) * p.nz + m] = mk(0.0, 0.0);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < W; ++c) all &= (p.col[c].done != 0);
        p.ctl->panel_done = all;
    }
}

// Common end of an outer iteration (last CTA): beta_n, rotation, loop condition.
template <typename T, int W>
__device__ void finish_outer(const Panel<T> &p, const double *rho_next, int init) {
    for (int c = threadIdx.x; c < W; c += NT) {
        ColState &C = p.col[c];
        if (C.done) continue;
        const c64 rn = mk(rho_next[2 * c], rho_next[2 * c + 1]);
        if (init) {
            C.rho = rn;
            continue;
        }
        if (C.restart) { // first iteration of the new seed follows
            C.beta_prev = mk(0.0, 0.0);
            C.alpha_prev = mk(1.0, 0.0);
            C.rho = rn;
            C.restart = 0;
            C.fresh = 0;
            C.iters += 1;
            continue;
        }
        C.beta_prev = cdiv(rn, C.rho);
        C.alpha_prev = C.alpha;
        C.rho = rn;
        C.iters += 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (init) {
            p.ctl->n = 0;
        } else {
            p.ctl->n += 1;
            p.ctl->iter_ctr += 1;
            const int cont = (!p.ctl->panel_done) && (p.ctl->iter_ctr < p.outer_cap);
            if (p.in_graph) cudaGraphSetConditional(p.h_outer, cont ? 1u : 0u);
        }
    }
}

// -------------------------------------------------------------- kernel B (S = I)
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, (B <= 4 ? 3 : 1)) k_update_sI(Panel<T> p) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    cpx<T> a[CPT];
    unsigned rst = 0; // bit cc: column lane*CPT+cc restarts now (its rt becomes e_j)
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const ColState &C = p.col[lane * CPT + cc];
        a[cc] = cvt<T>(C.alpha);
        rst |= (C.restart ? 1u : 0u) << cc;
    }
    Acc<T> acc[CPT][3];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero(), acc[cc][1].zero(), acc[cc][2].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int64_t row = br * B + i;
            cpx<T> rt[CPT], u[CPT];
            ld_row<T, W>(p.RT, row, lane, rt);
            ld_row<T, W>(p.U, row, lane, u);
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                if (rst >> cc & 1u) {
                    rt[cc] = mk<T>(row == p.col[lane * CPT + cc].row ? (T)1 : (T)0, 0);
                    clear_restart_row<T, W>(p, p.ctl->n, row, lane * CPT + cc);
                } else {
                    rt[cc] = rt[cc] - a[cc] * u[cc];
                }
                const T rr = rt[cc].re * rt[cc].re, ii = rt[cc].im * rt[cc].im;
                acc[cc][0].add(rr);
                acc[cc][0].add(-ii);
                acc[cc][1].add((T)2 * rt[cc].re * rt[cc].im);
                acc[cc][2].add(rr);
                acc[cc][2].add(ii);
            }
            st_row<T, W>(p.RT, row, lane, rt);
        }
    }
    cta_partials<T, W, NT, 3>(acc, p.part);
    pair_step_B<T, W>(p);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    __shared__ double red[W * 3];
    reduce_partials<T, W, NT, 3>(p.part, red);
    __shared__ double rho_next[W * 2];
    for (int c = threadIdx.x; c < W; c += NT) {
        rho_next[2 * c] = red[3 * c];
        rho_next[2 * c + 1] = red[3 * c + 1];
        if (!p.col[c].done) p.col[c].rn2 = red[3 * c + 2];
    }
    __syncthreads();
    finish_outer<T, W>(p, rho_next, 0);
}

// -------------------------------------------------------------- kernel B' (S != I)
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, (B <= 4 ? 3 : 1)) k_update_S(Panel<T> p) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    typedef typename DirOf<T>::type X;
    const int n = p.ctl->n;
    const T *Rc = p.R[n & 1];
    T *Rn = p.R[(n + 1) & 1];
    LdGuess<T, W> ld; // y_0 = r_n - alpha_n u
    ld.r = Rc;
    ld.u = p.U;
    ld.lane = lane;
    cpx<T> a[CPT];
    unsigned rst = 0; // bit cc: column lane*CPT+cc restarts now (its rt becomes e_j)
    // refinement: the first FP32 sweep sees t_0 / ||rt_n|| (no FP32 underflow however
    // small the residuals of a tight solve become); a restarting column's residual
    // becomes e_j, of norm one, so its scale is one
    float inv_sig = 1.f;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const ColState &C = p.col[lane * CPT + cc];
        const c64 al = C.alpha;
        a[cc] = cvt<T>(al);
        ld.s[cc] = mk((X)(-al.re), (X)(-al.im));
        ld.fresh_row[cc] = C.fresh ? C.row : -1;
        rst |= (C.restart ? 1u : 0u) << cc;
        if (cc == 0) inv_sig = (float)(1.0 / (C.restart ? 1.0 : safe_scale(C.rn2)));
    }
    Acc<T> acc[CPT][2];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero(), acc[cc][1].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
        cpx<T> sy[B][CPT];
        bsr_row_product<T, B, X>(p.s_rp, p.s_ci, p.s_val, br, ld, sy, p.s_unit ? br : -1);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int64_t row = br * B + i;
            cpx<T> rt[CPT], u[CPT], y0[CPT], t[CPT];
            cpx<X> g[CPT];
            ld_row<T, W>(p.RT, row, lane, rt);
            ld_row<T, W>(p.U, row, lane, u);
            ld(row, g);
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                y0[cc] = mk((T)g[cc].re, (T)g[cc].im);
                if (rst >> cc & 1u) {
                    rt[cc] = mk<T>(row == p.col[lane * CPT + cc].row ? (T)1 : (T)0, 0);
                    clear_restart_row<T, W>(p, n, row, lane * CPT + cc);
                } else {
                    rt[cc] = rt[cc] - a[cc] * u[cc];
                }
                t[cc] = rt[cc] - sy[i][cc];
                acc[cc][0].add(rt[cc].re * rt[cc].re);
                acc[cc][0].add(rt[cc].im * rt[cc].im);
                acc[cc][1].add(t[cc].re * t[cc].re);
                acc[cc][1].add(t[cc].im * t[cc].im);
            }
            st_row<T, W>(p.RT, row, lane, rt);
            st_row<T, W>(Rn, row, lane, y0);
            st_row<T, W>(p.Tv, row, lane, t);
            if constexpr (std::is_same<T, df>::value) {
                if (p.ir) { // the first FP32 sweep solves S c' = t_0 / ||rt_n||
                    const int64_t o = (row * W + lane) * 2;
                    *reinterpret_cast<float2 *>(p.T32 + o) = make_float2(t[0].re.hi * inv_sig, t[0].im.hi * inv_sig);
                }
            }
        }
    }
    cta_partials<T, W, NT, 2>(acc, p.part);
    pair_step_B<T, W>(p);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    __shared__ double red[W * 2];
    reduce_partials<T, W, NT, 2>(p.part, red);
    __shared__ int all_done;
    if (threadIdx.x == 0) all_done = 1;
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += NT) {
        ColState &C = p.col[c];
        C.in_alpha = 0.0;
        C.in_beta = 0.0;
        if (C.done) {
            C.in_done = 1;
            C.in_sweep = 0;
            continue;
        }
        const double sig = C.restart ? 1.0 : safe_scale(C.rn2); // the scale the rows used
        C.rn2 = red[2 * c];
        C.in_rr = red[2 * c + 1];
        if (p.ir) {
            // refinement: the column sweeps until its true residual t = rt - S y is
            // below inner_tol ||rt||; each FP32 sweep works on t / in_sig and
            // reduces its own residual by sweep_red (or to half the final target)
            const double eta2 = p.inner_tol * p.inner_tol * C.rn2;
            C.in_t2 = C.in_rr;
            C.in_sig = sig;
            C.in_rr = C.in_t2 / (sig * sig);
            C.in_refines = 0;
            C.in_conv = !(C.in_t2 > eta2) || !isfinite(C.in_t2);
            C.in_sweep = !C.in_conv;
            C.in_done = C.in_conv;
            C.in_tol2 = fmax(p.sweep_red * p.sweep_red * C.in_rr, 0.25 * eta2 / (sig * sig));
        } else {
            C.in_tol2 = p.inner_tol * p.inner_tol * C.rn2;
            C.in_done = (C.in_rr <= C.in_tol2) ? 1 : 0;
        }
        if (!C.in_done) atomicAnd(&all_done, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctl->k = 0;
        p.ctl->in_ctr = 0;
        p.ctl->refine_now = 0;
        p.ctl->inner_done = all_done;
        if (p.in_graph) cudaGraphSetConditional(p.h_inner, (!all_done && p.inner_max > 0) ? 1u : 0u);
    }
}

// ------------------------------------------------------- inner CG on S: IC_A
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, ctas_light<T, B>()) k_inner_a(Panel<T> p) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    typedef typename DirOf<T>::type X;
    const int k = p.ctl->k;
    X *Dn = p.D[k & 1];
    LdDir<T, W> ld; // d_k = t_k + beta d_{k-1}, beta real
    ld.t = p.Tv;
    ld.d = (k == 0) ? nullptr : p.D[(k + 1) & 1];
    ld.lane = lane;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) ld.s[cc] = (X)p.col[lane * CPT + cc].in_beta;
    // neighbour blocks per trip: one for FP32 vectors, whose operand (t + beta d)
    // takes two loads per neighbour row (measured faster than two blocks per trip)
    constexpr int UNR = std::is_same<T, float>::value ? 1 : 2;
    Acc<T> acc[CPT][1];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
        cpx<T> sd[B][CPT];
        bsr_row_product<T, B, X, UNR>(p.s_rp, p.s_ci, p.s_val, br, ld, sd, p.s_unit ? br : -1);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int64_t row = br * B + i;
            cpx<X> d[CPT];
            ld(row, d);
            st_dir<T, W>(Dn, row, lane, d);
            st_row<T, W>(p.Av, row, lane, sd[i]);
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                acc[cc][0].add(mul_x(sd[i][cc].re, d[cc].re));
                acc[cc][0].add(mul_x(sd[i][cc].im, d[cc].im));
            }
        }
    }
    cta_partials<T, W, NT, 1>(acc, p.part);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    __shared__ double red[W];
    reduce_partials<T, W, NT, 1>(p.part, red);
    for (int c = threadIdx.x; c < W; c += NT) {
        ColState &C = p.col[c];
        if (C.in_done) {
            C.in_alpha = 0.0;
            continue;
        }
        const double dad = red[c];
        if (!(dad > 0.0) || !isfinite(dad)) { // S not positive definite on this direction
            C.in_done = 1;
            C.in_alpha = 0.0;
            if (C.in_rr > 1e-30) C.s_bad = 1;
            continue;
        }
        C.in_alpha = C.in_rr / dad;
    }
}

// ------------------------------------------------------- inner CG on S: IC_B
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, (B <= 4 ? 3 : 1)) k_inner_b(Panel<T> p) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    typedef typename DirOf<T>::type X;
    const int k = p.ctl->k;
    const X *D = p.D[k & 1];
    T *Y = p.R[(p.ctl->n + 1) & 1];
    // the first step of an FP32 sweep of the refinement starts its correction
    // from zero (written here, not by the refinement pass: that pass still reads
    // the previous correction of neighbouring rows while it runs)
    const bool fresh = p.ir && k == 0;
    T a[CPT]; // inner CG step length (real)
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) a[cc] = (T)p.col[lane * CPT + cc].in_alpha;
    Acc<T> acc[CPT][1];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
        // all loads of the block row first: 4B independent loads in flight
        cpx<T> y[B][CPT], t[B][CPT], av[B][CPT];
        cpx<X> d[B][CPT];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (fresh) {
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) y[i][cc] = mk<T>(0, 0);
            } else {
                ld_row<T, W>(Y, br * B + i, lane, y[i]);
            }
            ld_dir<T, W>(D, br * B + i, lane, d[i]);
            ld_row<T, W>(p.Tv, br * B + i, lane, t[i]);
            ld_row<T, W>(p.Av, br * B + i, lane, av[i]);
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                y[i][cc].re = fma_x(a[cc], d[i][cc].re, y[i][cc].re);
                y[i][cc].im = fma_x(a[cc], d[i][cc].im, y[i][cc].im);
                t[i][cc].re = fma_x(-a[cc], av[i][cc].re, t[i][cc].re);
                t[i][cc].im = fma_x(-a[cc], av[i][cc].im, t[i][cc].im);
                acc[cc][0].add(t[i][cc].re * t[i][cc].re);
                acc[cc][0].add(t[i][cc].im * t[i][cc].im);
            }
            st_row<T, W>(Y, br * B + i, lane, y[i]);
            st_row<T, W>(p.Tv, br * B + i, lane, t[i]);
        }
    }
    cta_partials<T, W, NT, 1>(acc, p.part);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    __shared__ double red[W];
    reduce_partials<T, W, NT, 1>(p.part, red);
    __shared__ int all_done;
    if (threadIdx.x == 0) all_done = 1;
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += NT) {
        ColState &C = p.col[c];
        if (!C.in_done) {
            const double tt = red[c];
            C.in_beta = tt / C.in_rr;
            C.in_rr = tt;
            if (tt <= C.in_tol2 || !isfinite(tt)) C.in_done = 1;
        }
        if (!C.in_done) atomicAnd(&all_done, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctl->k += 1;
        p.ctl->in_ctr += 1;
        p.ctl->inner_total += 1;
        p.ctl->inner_done = all_done;
        const int cont = (!all_done) && (p.ctl->in_ctr < p.inner_max);
        if (p.ir) {
            // an FP32 sweep of the refinement: when it ends, the refinement kernel
            // that follows in the loop body applies it (the loop condition is its).
            // When every refining column's correction is small (its residual below
            // REFINE_LIGHT inner_tol ||rt||), the pass takes S c in FP32
            // (refine_now = 2); otherwise in df (refine_now = 1).
            if (!cont) {
                int light = 1;
                for (int c = 0; c < W; ++c) {
                    const ColState &C = p.col[c];
                    if (C.done || !C.in_sweep) continue;
                    const double lim = REFINE_LIGHT * p.inner_tol;
                    if (!(C.in_t2 <= lim * lim * C.rn2)) light = 0;
                }
                p.ctl->refine_now = light ? 2 : 1;
            }
        } else if (p.in_graph) {
            cudaGraphSetConditional(p.h_inner, cont ? 1u : 0u);
        }
    }
}

// ------------------------------------------ inner solve by refinement (df): R
// After an FP32 sweep has solved S c = t (from c = 0, to its own tolerance):
// y += c, t -= S c (a df product with the FP32 operand c, so t stays the true
// residual rt - S y to df rounding) and the next sweep's FP32 residual t32 = t.
// c is read here as a neighbour operand by every CTA, so this pass leaves it
// as it is; the next sweep's first step overwrites it.  The last CTA ends the inner solve of every column whose ||t|| is below
// inner_tol ||rt|| (or that reached refine_max refinements) and sets the loop
// condition; the kernel returns at once in the loop iterations in which the
// sweep goes on (refine_now == 0).
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, (B <= 4 ? 3 : 1)) k_refine(Panel<T> p) {
    if constexpr (std::is_same<T, df>::value) {
        const int mode = p.ctl->refine_now; // 0: the sweep goes on; 1: df product; 2: FP32 product
        if (!mode) return;
        using TM = Teams<df, W, NT>;
        const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
        df *Y = p.R[(p.ctl->n + 1) & 1];
        LdF32<W> ld{p.C32, lane};
        // the sweep solved S c' = t / sig: c = sig c'; the next sweep sees t / ||t_old||
        const ColState &Cl = p.col[lane];
        const df sig = df(Cl.in_sig);
        const float inv_new = (float)(1.0 / safe_scale(Cl.in_t2));
        Acc<df> acc[1][1];
        acc[0][0].zero();
        const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
        for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
            cpx<df> sc[B][1];
            if (mode == 1) {
                bsr_row_product<df, B, float>(p.s_rp, p.s_ci, p.s_val, br, ld, sc, p.s_unit ? br : -1);
            } else { // a small correction: FP32 values of S, FP32 accumulation
                float sr[B], si[B];
#pragma unroll
                for (int i = 0; i < B; ++i) sr[i] = si[i] = 0.f;
                const int64_t k1 = p.s_rp[br + 1];
                for (int64_t k = p.s_rp[br]; k < k1; ++k) {
                    const int64_t col = p.s_ci[k];
                    cpx<float> x[B][1];
#pragma unroll
                    for (int j = 0; j < B; ++j) ld(col * B + j, x[j]);
                    if (p.s_unit && col == br) {
#pragma unroll
                        for (int i = 0; i < B; ++i) sr[i] += x[i][0].re, si[i] += x[i][0].im;
                    } else {
                        float a[B * B];
                        ld_block<float, B>(p.s_val32 + k * (B * B), a);
#pragma unroll
                        for (int i = 0; i < B; ++i)
#pragma unroll
                            for (int j = 0; j < B; ++j) {
                                sr[i] = fmaf(a[i * B + j], x[j][0].re, sr[i]);
                                si[i] = fmaf(a[i * B + j], x[j][0].im, si[i]);
                            }
                    }
                }
#pragma unroll
                for (int i = 0; i < B; ++i) sc[i][0] = mk(df(sr[i]), df(si[i]));
            }
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const int64_t row = br * B + i;
                cpx<df> y[1], t[1];
                cpx<float> c[1];
                ld_row<df, W>(Y, row, lane, y);
                ld_row<df, W>(p.Tv, row, lane, t);
                ld(row, c);
                y[0] = mk(fma_f(sig, c[0].re, y[0].re), fma_f(sig, c[0].im, y[0].im));
                t[0] = mk(t[0].re - sig * sc[i][0].re, t[0].im - sig * sc[i][0].im);
                acc[0][0].add(t[0].re * t[0].re);
                acc[0][0].add(t[0].im * t[0].im);
                st_row<df, W>(Y, row, lane, y);
                st_row<df, W>(p.Tv, row, lane, t);
                const int64_t o = (row * W + lane) * 2;
                *reinterpret_cast<float2 *>(p.T32 + o) = make_float2(t[0].re.hi * inv_new, t[0].im.hi * inv_new);
            }
        }
        cta_partials<df, W, NT, 1>(acc, p.part);
        if (!last_cta_arrival(&p.ctl->arrive)) return;
        __shared__ double red[W];
        reduce_partials<df, W, NT, 1>(p.part, red);
        __shared__ int any;
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += NT) {
            ColState &C = p.col[c];
            if (C.done || !C.in_sweep) continue;
            const double t2 = red[c];
            const double eta2 = p.inner_tol * p.inner_tol * C.rn2;
            const double sig = safe_scale(C.in_t2); // the scale the rows used for the next sweep
            C.in_refines += 1;
            C.in_t2 = t2;
            if (!(t2 > eta2) || !isfinite(t2) || C.in_refines >= p.refine_max || C.s_bad) {
                C.in_sweep = 0;
                C.in_conv = 1;
                C.in_done = 1;
                continue;
            }
            C.in_sig = sig;
            C.in_rr = t2 / (sig * sig);
            C.in_alpha = 0.0;
            C.in_beta = 0.0;
            C.in_tol2 = fmax(p.sweep_red * p.sweep_red * C.in_rr, 0.25 * eta2 / (sig * sig));
            C.in_done = 0;
            atomicOr(&any, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            p.ctl->k = 0;
            p.ctl->in_ctr = 0;
            p.ctl->refine_now = 0;
            p.ctl->refine_total += 1;
            p.ctl->light_total += (mode == 2);
            if (p.in_graph) cudaGraphSetConditional(p.h_inner, any ? 1u : 0u);
        }
    }
}

// -------------------------------------------------------------- kernel C (S != I)
template <typename T, int B, int W>
__global__ void __launch_bounds__(NT, ctas_light<T, B>()) k_rho(Panel<T> p, int init) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    const int n = p.ctl->n;
    const T *Rn = p.R[(n + 1) & 1];
    Acc<T> acc[CPT][2];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[cc][0].zero(), acc[cc][1].zero();
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < p.n_brows; br += br_step) {
        cpx<T> rb[B][CPT], rtb[B][CPT];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            ld_row<T, W>(Rn, br * B + i, lane, rb[i]);
            ld_row<T, W>(p.RT, br * B + i, lane, rtb[i]);
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const cpx<T>(&r)[CPT] = rb[i];
            const cpx<T>(&rt)[CPT] = rtb[i];
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                acc[cc][0].add(r[cc].re * rt[cc].re);
                acc[cc][0].add(-(r[cc].im * rt[cc].im));
                acc[cc][1].add(r[cc].re * rt[cc].im);
                acc[cc][1].add(r[cc].im * rt[cc].re);
            }
        }
    }
    cta_partials<T, W, NT, 2>(acc, p.part);
    if (!last_cta_arrival(&p.ctl->arrive)) return;
    __shared__ double red[W * 2];
    reduce_partials<T, W, NT, 2>(p.part, red);
    finish_outer<T, W>(p, red, init);
}

// -------------------------------------------------------------- write-out
// Results of the columns still in their slots when the loop ends (columns that
// finished earlier were written when they retired).
template <typename T, int W>
__global__ void k_writeout(Panel<T> p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per_slot = (int64_t)p.max_col_ent * p.nz;
    for (int64_t t = tid; t < W * per_slot; t += stride) {
        const ColState &C = p.col[t / per_slot];
        const int64_t r = t % per_slot;
        if (C.dst < 0 || r >= (int64_t)C.n_ent * p.nz) continue;
        p.G[C.ent0 * p.nz + r] = p.qmr ? p.xq[t] : p.xs[t];
    }
    for (int64_t q = tid; q < (int64_t)W * p.nz; q += stride) {
        const int64_t dst = p.col[q / p.nz].dst;
        if (dst >= 0) p.resid[dst * p.nz + q % p.nz] = p.sh[q].resid;
    }
    if (tid < W) {
        const ColState &C = p.col[tid];
        if (C.dst >= 0) {
            p.iters[C.dst] = C.iters;
            p.status[C.dst] = C.done ? C.status : TB_COL_MAX_ITER;
        }
    }
    if (last_cta_arrival(&p.ctl->arrive) && threadIdx.x == 0 && p.stats) {
        p.stats[0] = p.ctl->iter_ctr;
        p.stats[1] = p.ctl->inner_total;
        p.stats[2] = p.ctl->refine_total;
        p.stats[3] = p.ctl->light_total;
    }
}

// ================================================================== host side
struct GraphBuilder {
    tb_ctx *ctx;
    int rc = TB_OK;
    cudaGraphNode_t add_kernel(cudaGraph_t g, const void *fn, dim3 grid, dim3 block, void **args,
                               const cudaGraphNode_t *deps, int ndeps) {
        if (rc) return nullptr;
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof(kp));
        kp.func = const_cast<void *>(fn);
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t node = nullptr;
        cudaError_t e = cudaGraphAddKernelNode(&node, g, deps, ndeps, &kp);
        if (e != cudaSuccess) rc = set_error(ctx, TB_ERR_CUDA, "cudaGraphAddKernelNode: %s", cudaGetErrorString(e));
        return node;
    }
    cudaGraphNode_t add_while(cudaGraph_t g, cudaGraphConditionalHandle h, const cudaGraphNode_t *deps, int ndeps,
                              cudaGraph_t *body) {
        if (rc) return nullptr;
        // the parameter union has no default constructor: use zeroed raw storage
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        std::memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams *np = reinterpret_cast<cudaGraphNodeParams *>(raw);
        np->type = cudaGraphNodeTypeConditional;
        np->conditional.handle = h;
        np->conditional.type = cudaGraphCondTypeWhile;
        np->conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        cudaError_t e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, np);
        if (e != cudaSuccess) {
            rc = set_error(ctx, TB_ERR_CUDA, "conditional node: %s", cudaGetErrorString(e));
            return nullptr;
        }
        *body = np->conditional.phGraph_out[0];
        return node;
    }
    cudaGraphConditionalHandle handle(cudaGraph_t g, unsigned def, unsigned flags) {
        cudaGraphConditionalHandle h = 0;
        if (rc) return h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, def, flags);
        if (e != cudaSuccess) rc = set_error(ctx, TB_ERR_CUDA, "conditional handle: %s", cudaGetErrorString(e));
        return h;
    }
};

struct SolveLaunch {
    tb_ctx *ctx;
    bool has_s;
    int ncta;
    int64_t n_rows;
    cudaStream_t stream;
    int profile_reps; // > 0: time the kernels of the first panel instead of solving
    double *ms_out;   // [8] average ms per launch (profile)
    Panel<double> pd; // type-erased panel (all T-dependent members are pointers)
    int ncta_a = 0;   // grid of IC_A and C (0: ncta): they fit one more CTA per SM than the others
    int ncta_f = 0;   // grid of the FP32 sweep kernels of the refinement (df panels with S)
    int ncta_fb = 0;  // grid of the FP32 sweep update IC_B (0: ncta_f)
    int rc = TB_OK;

    int vec_grid(int W) const {
        return (int)std::min<int64_t>(std::max<int64_t>((n_rows * W + NT - 1) / NT, 1), 152 * 8);
    }
    // the row-parallel kept-row kernels: one thread per (column, kept row, shift)
    template <typename T>
    static int rows_grid(const Panel<T> &p, int W) {
        const int64_t work = (int64_t)W * p.max_col_ent * p.nz;
        return (int)std::min<int64_t>(std::max<int64_t>((work + NT - 1) / NT, 1), 152 * 8);
    }

    template <typename T, int B, int W>
    void run() {
        Panel<T> p;
        static_assert(sizeof(Panel<T>) == sizeof(Panel<double>), "panel layout");
        std::memcpy(&p, &pd, sizeof(p));
        if (profile_reps > 0)
            profile<T, B, W>(p);
        else
            solve_graph<T, B, W>(p);
    }

    // The FP32 sweeps of the refinement run the FP32 inner CG kernels on this
    // view of a df panel: their solution is the sweep correction c, their
    // residual the FP32 sweep residual, their product a = S d with S's FP32
    // values; the column states are the df panel's own.
    template <typename T>
    static Panel<float> fp32_view(const Panel<T> &p) {
        Panel<float> f;
        std::memcpy(&f, &p, sizeof(f));
        f.h_val = nullptr;
        f.s_val = p.s_val32;
        f.R[0] = f.R[1] = p.C32;
        f.Tv = p.T32;
        f.Av = p.A32;
        f.RT = f.P[0] = f.P[1] = f.SP = f.U = f.HP = nullptr;
        for (int k = 0; k < 2; ++k) f.D[k] = reinterpret_cast<float *>(p.D[k]);
        return f;
    }

    template <typename T, int B, int W>
    void profile(Panel<T> p) {
        p.in_graph = 0;
        const dim3 grid(ncta), block(NT), grid_a(ncta_a > 0 ? ncta_a : ncta), grid_f(ncta_f > 0 ? ncta_f : ncta),
                   grid_fb(ncta_fb > 0 ? ncta_fb : (ncta_f > 0 ? ncta_f : ncta));
        const int has_s_i = has_s ? 1 : 0;
        const bool ir = p.ir != 0;
        Panel<float> pf = fp32_view(p);
        // one inner iteration: the df inner CG pair, or an FP32 sweep step of the refinement
        auto inner_a = [&]() {
            if constexpr (std::is_same<T, df>::value)
                if (ir) return (void)k_inner_a<float, B, W><<<grid_f, block, 0, stream>>>(pf);
            k_inner_a<T, B, W><<<grid_a, block, 0, stream>>>(p);
        };
        auto inner_b = [&]() {
            if constexpr (std::is_same<T, df>::value)
                if (ir) return (void)k_inner_b<float, B, W><<<grid_fb, block, 0, stream>>>(pf);
            k_inner_b<T, B, W><<<grid, block, 0, stream>>>(p);
        };
        // a refinement pass with its work done (outside the graph nothing sets
        // refine_now): mode 1 takes S c in df, mode 2 in FP32
        auto refine = [&](int mode) {
            cudaMemsetAsync(&p.ctl->refine_now, mode, 1, stream);
            k_refine<T, B, W><<<grid, block, 0, stream>>>(p);
        };
        k_init_state<T, W><<<1, NT, 0, stream>>>(p, has_s_i);
        k_init_vec<T, W><<<vec_grid(W), NT, 0, stream>>>(p, n_rows, has_s_i);
        if (has_s) {
            k_update_S<T, B, W><<<grid, block, 0, stream>>>(p);
            inner_a();
            inner_b();
            if (ir) refine(1);
            k_rho<T, B, W><<<grid_a, block, 0, stream>>>(p, 1);
        }
        // events: [0] A [1] B [2] (untimed first inner pair) [3] IC_A [4] IC_B [5] R [6] C [7]
        //         R in FP32 between [8] and [9]
        cudaEvent_t ev[10];
        for (auto &e : ev) cudaEventCreate(&e);
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int r = 0; r < profile_reps && !rc; ++r) {
            cudaEventRecord(ev[0], stream);
            if (has_s)
                k_outer<T, B, W, true><<<grid, block, 0, stream>>>(p);
            else
                k_outer<T, B, W, false><<<grid, block, 0, stream>>>(p);
            if (p.rowpar) k_rows_A<T, W><<<rows_grid(p, W), block, 0, stream>>>(p, has_s_i);
            cudaEventRecord(ev[1], stream);
            if (has_s)
                k_update_S<T, B, W><<<grid, block, 0, stream>>>(p);
            else
                k_update_sI<T, B, W><<<grid, block, 0, stream>>>(p);
            if (p.rowpar) k_rows_B<T, W><<<rows_grid(p, W), block, 0, stream>>>(p);
            cudaEventRecord(ev[2], stream);
            int last = 2;
            if (has_s) {
                // first inner iteration (no previous direction) untimed; time a
                // steady-state one (k = 1), as most inner iterations of a solve are
                inner_a();
                inner_b();
                cudaEventRecord(ev[3], stream);
                inner_a();
                cudaEventRecord(ev[4], stream);
                inner_b();
                cudaEventRecord(ev[5], stream);
                if (ir) refine(1);
                cudaEventRecord(ev[6], stream);
                k_rho<T, B, W><<<grid_a, block, 0, stream>>>(p, 0);
                cudaEventRecord(ev[7], stream);
                last = 7;
                if (ir) {
                    cudaEventRecord(ev[8], stream);
                    refine(2);
                    cudaEventRecord(ev[9], stream);
                    last = 9;
                }
            }
            cudaError_t e = cudaEventSynchronize(ev[last]);
            if (e != cudaSuccess) {
                rc = set_error(ctx, TB_ERR_CUDA, "profile: %s", cudaGetErrorString(e));
                break;
            }
            // (kernel slot, start event, end event)
            const int spans[7][3] = {{0, 0, 1}, {1, 1, 2}, {2, 3, 4}, {3, 4, 5}, {4, 6, 7}, {5, 5, 6}, {6, 8, 9}};
            for (int q = 0; q < (has_s ? (ir ? 7 : 6) : 2); ++q) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[spans[q][1]], ev[spans[q][2]]);
                acc[spans[q][0]] += ms;
            }
        }
        for (auto &e : ev) cudaEventDestroy(e);
        for (int k = 0; k < 8; ++k) ms_out[k] = 0.0;
        for (int k = 0; k < 7; ++k) ms_out[k] = acc[k] / profile_reps;
        if (!has_s) ms_out[2] = ms_out[3] = ms_out[4] = 0.0;
        if (!ir) ms_out[5] = ms_out[6] = 0.0;
    }

    template <typename T, int B, int W>
    void solve_graph(Panel<T> p) {
        p.in_graph = 1;
        GraphBuilder gb{ctx};
        cudaGraph_t g = nullptr;
        if (cudaGraphCreate(&g, 0) != cudaSuccess) {
            rc = set_error(ctx, TB_ERR_CUDA, "cudaGraphCreate");
            return;
        }
        p.h_outer = gb.handle(g, 1u, cudaGraphCondAssignDefault);
        cudaGraphConditionalHandle h_inner_init = has_s ? gb.handle(g, 0u, 0u) : 0;
        const dim3 grid(ncta), block(NT), grid_a(ncta_a > 0 ? ncta_a : ncta), grid_f(ncta_f > 0 ? ncta_f : ncta),
                   grid_fb(ncta_fb > 0 ? ncta_fb : (ncta_f > 0 ? ncta_f : ncta));
        const bool ir = p.ir != 0;
        int has_s_i = has_s ? 1 : 0;
        int init1 = 1, init0 = 0;
        int64_t nr = n_rows;
        // kernel arguments are copied when each node is added
        Panel<T> p_init = p;
        p_init.h_inner = h_inner_init;
        Panel<float> pf_init = fp32_view(p_init);
        void *a_state[] = {&p, &has_s_i};
        void *a_vec[] = {&p, &nr, &has_s_i};
        cudaGraphNode_t n_state = gb.add_kernel(g, (const void *)k_init_state<T, W>, dim3(1), block, a_state, nullptr, 0);
        cudaGraphNode_t last = gb.add_kernel(g, (const void *)k_init_vec<T, W>, dim3(vec_grid(W)), block, a_vec, &n_state, 1);
        void *a_pinit[] = {&p_init};
        void *a_finit[] = {&pf_init};
        void *a_pinit_rho[] = {&p_init, &init1};
        // body of an inner loop: the df inner CG pair, or an FP32 sweep step and
        // the refinement pass that applies a finished sweep
        auto inner_body = [&](cudaGraph_t ib, void **a_t, void **a_f) {
            if constexpr (std::is_same<T, df>::value) {
                if (ir) {
                    cudaGraphNode_t y = gb.add_kernel(ib, (const void *)k_inner_a<float, B, W>, grid_f, block, a_f, nullptr, 0);
                    y = gb.add_kernel(ib, (const void *)k_inner_b<float, B, W>, grid_fb, block, a_f, &y, 1);
                    gb.add_kernel(ib, (const void *)k_refine<T, B, W>, grid, block, a_t, &y, 1);
                    return;
                }
            }
            (void)a_f;
            cudaGraphNode_t y = gb.add_kernel(ib, (const void *)k_inner_a<T, B, W>, grid_a, block, a_t, nullptr, 0);
            gb.add_kernel(ib, (const void *)k_inner_b<T, B, W>, grid, block, a_t, &y, 1);
        };
        if (has_s) {
            last = gb.add_kernel(g, (const void *)k_update_S<T, B, W>, grid, block, a_pinit, &last, 1);
            cudaGraph_t ib = nullptr;
            last = gb.add_while(g, h_inner_init, &last, 1, &ib);
            if (!gb.rc) inner_body(ib, a_pinit, a_finit);
            last = gb.add_kernel(g, (const void *)k_rho<T, B, W>, grid_a, block, a_pinit_rho, &last, 1);
        }
        cudaGraph_t ob = nullptr;
        cudaGraphNode_t outer = gb.add_while(g, p.h_outer, &last, 1, &ob);
        Panel<T> p_body = p;
        Panel<float> pf_body;
        void *a_body[] = {&p_body};
        void *a_fbody[] = {&pf_body};
        void *a_body_rho[] = {&p_body, &init0};
        void *a_rows_a[] = {&p_body, &has_s_i};
        const dim3 rgrid(rows_grid(p, W));
        if (!gb.rc) {
            if (has_s) {
                p_body.h_inner = gb.handle(ob, 0u, 0u);
                pf_body = fp32_view(p_body);
                cudaGraphNode_t x = gb.add_kernel(ob, (const void *)k_outer<T, B, W, true>, grid, block, a_body, nullptr, 0);
                if (p.rowpar) x = gb.add_kernel(ob, (const void *)k_rows_A<T, W>, rgrid, block, a_rows_a, &x, 1);
                x = gb.add_kernel(ob, (const void *)k_update_S<T, B, W>, grid, block, a_body, &x, 1);
                if (p.rowpar) x = gb.add_kernel(ob, (const void *)k_rows_B<T, W>, rgrid, block, a_body, &x, 1);
                cudaGraph_t ib = nullptr;
                x = gb.add_while(ob, p_body.h_inner, &x, 1, &ib);
                if (!gb.rc) inner_body(ib, a_body, a_fbody);
                gb.add_kernel(ob, (const void *)k_rho<T, B, W>, grid_a, block, a_body_rho, &x, 1);
            } else {
                cudaGraphNode_t x = gb.add_kernel(ob, (const void *)k_outer<T, B, W, false>, grid, block, a_body, nullptr, 0);
                if (p.rowpar) x = gb.add_kernel(ob, (const void *)k_rows_A<T, W>, rgrid, block, a_rows_a, &x, 1);
                x = gb.add_kernel(ob, (const void *)k_update_sI<T, B, W>, grid, block, a_body, &x, 1);
                if (p.rowpar) gb.add_kernel(ob, (const void *)k_rows_B<T, W>, rgrid, block, a_body, &x, 1);
            }
        }
        void *a_out[] = {&p};
        gb.add_kernel(g, (const void *)k_writeout<T, W>, dim3(152 * 2), block, a_out, &outer, 1);
        if (gb.rc) {
            rc = gb.rc;
            cudaGraphDestroy(g);
            return;
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
        if (e != cudaSuccess) {
            rc = set_error(ctx, TB_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            cudaGraphDestroy(g);
            return;
        }
        e = cudaGraphLaunch(exec, stream);
        if (e != cudaSuccess) rc = set_error(ctx, TB_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess && !rc) rc = set_error(ctx, TB_ERR_CUDA, "solve: %s", cudaGetErrorString(e));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
    }
};

// one per precision (inst_f64.cu, inst_f32.cu, inst_df.cu)
bool launch_panel_f64(SolveLaunch &L, int b, int W);
bool launch_panel_f32(SolveLaunch &L, int b, int W);
bool launch_panel_df(SolveLaunch &L, int b, int W);

} // namespace tbgf
