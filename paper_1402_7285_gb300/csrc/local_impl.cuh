// shifted_cocg_solve_local: shifted COCG of every column on its own hop-shell
// subspace, one CTA per column, persistent over a device work queue.
//
// Column c solves the truncated problem (z_m S_OO - H_OO) x = e_j on the
// principal submatrices over the subspace O_c (Sec. 2 locality; Eq. 2 with
// b = e_j) by the same generalized shifted COCG as the panel solver: the
// S-bilinear seed recurrence (FP64 scalars), the shifted systems through
// collinear residuals, an inner CG on S_OO when S != I.  The subspace's
// vectors, its local block structure and the per-shift state live in shared
// memory; the block values are read from global memory (L2) each product.
// Columns converge after very different numbers of iterations (the subspace
// sizes differ); each CTA takes the next column from an atomic queue as soon
// as its column is done, so no CTA waits for another.  The queue order is the
// caller's (e.g. longest predicted first).  Every loop is bounded (max_iter,
// inner_max).
#pragma once

#include <algorithm>
#include <vector>

#include "cocg_kernels.cuh"
#include "dispatch.cuh"

namespace tbgf {

constexpr int LNT = 512;

template <typename T>
struct LocalArgs {
    const int64_t *h_rp;
    const int32_t *h_ci;
    const T *h_val;
    const T *s_val; // S values on H's block pattern (nullptr: S = I)
    int64_t n_brows;
    const c64 *z;
    int32_t nz;
    c64 zs;
    const int64_t *rhs;
    const int64_t *sub_ptr;
    const int32_t *sub_atoms;
    const int64_t *optr;
    const int64_t *orows;
    const int64_t *order;
    int64_t n;
    int32_t maxa, dmax, max_kept;
    c64 *scratch; // [gridDim.x][2][max_kept][nz]
    void *gvec;   // null: vectors in shared memory; else [gridDim.x][NV][maxa*B] cpx<T> in global memory
    unsigned long long *queue;
    unsigned long long *stat; // [2]: outer, inner iterations
    double tol, inner_tol;
    double stall2; // restart threshold on ||rt||^2 (see the restart below); 0 = never
    int32_t max_iter, inner_max;
    c64 *G;
    int32_t *iters;
    double *resid;
    int32_t *status;
};

struct ShiftL {
    c64 pi, pi_prev, pi_next;
    double resid;
    int32_t active, conv_it;
};

__device__ __forceinline__ int bsearch_atom(const int32_t *atoms, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int64_t v = atoms[mid];
        if (v == g) return mid;
        if (v < g) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// CTA-wide sum of K accumulators; every thread gets the FP64 results in out[].
template <typename T, int K>
__device__ __forceinline__ void cta_sum(Acc<T> (&acc)[K], double *out) {
    typedef typename Acc<T>::P P;
    __shared__ P wpart[LNT / 32][4];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        warp_reduce(acc[k]);
        if (lane == 0) wpart[warp][k] = acc[k].pack();
    }
    __syncthreads();
    if (threadIdx.x < K) {
        Acc<T> s;
        s.zero();
        for (int w = 0; w < LNT / 32; ++w) s.add(Acc<T>::unpack(wpart[w][threadIdx.x]));
        out[threadIdx.x] = s.value();
    }
    __syncthreads();
}

// y[l] = sum over in-subspace blocks of A(l, .) x  for every local row l
template <typename T, int B>
__device__ __forceinline__ cpx<T> local_row_product(int l, const T *__restrict__ val, const int32_t *nbk,
                                                    const int16_t *nbl, const int16_t *cnt, int dmax,
                                                    const cpx<T> *x) {
    const int la = l / B, i = l % B;
    cpx<T> y = mk<T>(0, 0);
    const int nc = cnt[la];
    for (int s = 0; s < nc; ++s) {
        const int64_t kb = nbk[la * dmax + s];
        const int lc = nbl[la * dmax + s];
        const T *row = val + kb * (B * B) + i * B;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const T v = ldg_val(row + j);
            const cpx<T> xv = x[lc * B + j];
            y.re = fma(v, xv.re, y.re);
            y.im = fma(v, xv.im, y.im);
        }
    }
    return y;
}

template <typename T, int B, bool HAS_S>
__global__ void __launch_bounds__(LNT) k_local(LocalArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NV = HAS_S ? 8 : 3;
    const int maxr = a.maxa * B;
    // the subspace vectors live in shared memory, or (subspaces too large for
    // it) in this CTA's slice of a global array, which stays in L2
    cpx<T> *vec = a.gvec ? reinterpret_cast<cpx<T> *>(a.gvec) + (int64_t)blockIdx.x * NV * maxr
                         : reinterpret_cast<cpx<T> *>(smem);
    cpx<T> *RT = vec;               // rt (= r when S = I)
    cpx<T> *P = vec + maxr;
    cpx<T> *U = vec + 2 * maxr;
    cpx<T> *R = HAS_S ? vec + 3 * maxr : RT;
    cpx<T> *SP = vec + 4 * maxr, *Tv = vec + 5 * maxr, *D = vec + 6 * maxr, *Av = vec + 7 * maxr;
    ShiftL *shs = a.gvec ? reinterpret_cast<ShiftL *>(smem) : reinterpret_cast<ShiftL *>(vec + NV * maxr);
    int32_t *atoms = reinterpret_cast<int32_t *>(shs + a.nz);
    int32_t *nbk = atoms + a.maxa;
    int32_t *kept = nbk + a.maxa * a.dmax;
    int16_t *nbl = reinterpret_cast<int16_t *>(kept + a.max_kept);
    int16_t *cnt = nbl + a.maxa * a.dmax;

    __shared__ double red[4];
    __shared__ int s_col, s_nat, s_jloc, s_nkept, s_nact;
    __shared__ c64 s_rho, s_alpha, s_alpha_prev, s_beta_prev;
    __shared__ double s_rn2, s_in_rr, s_in_alpha, s_in_beta, s_in_tol2;
    __shared__ int s_status, s_stop, s_in_stop, s_restarts, s_restart, s_chk_n;
    __shared__ double s_chk_w;
    __shared__ c64 s_zs; // this column's seed shift

    const int tid = threadIdx.x;
    c64 *xs = a.scratch + (int64_t)blockIdx.x * 2 * a.max_kept * a.nz;
    c64 *ps = xs + (int64_t)a.max_kept * a.nz;

    for (;;) {
        if (tid == 0) s_col = (int)atomicAdd(a.queue, 1ull);
        __syncthreads();
        const int64_t qi = s_col;
        if (qi >= a.n) break;
        const int64_t col = a.order ? a.order[qi] : qi;
        // ---- local structure
        const int64_t a0 = a.sub_ptr[col];
        const int nat = (int)(a.sub_ptr[col + 1] - a0);
        for (int l = tid; l < nat; l += LNT) atoms[l] = a.sub_atoms[a0 + l];
        __syncthreads();
        for (int l = tid; l < nat; l += LNT) {
            const int64_t g = atoms[l];
            int c = 0;
            for (int64_t k = a.h_rp[g]; k < a.h_rp[g + 1] && c < a.dmax; ++k) {
                const int lc = bsearch_atom(atoms, nat, a.h_ci[k]);
                if (lc >= 0) {
                    nbl[l * a.dmax + c] = (int16_t)lc;
                    nbk[l * a.dmax + c] = (int32_t)k;
                    ++c;
                }
            }
            cnt[l] = (int16_t)c;
        }
        const int64_t j = a.rhs[col];
        const int64_t k0 = a.optr[col];
        const int nkept = (int)(a.optr[col + 1] - k0);
        if (tid == 0) {
            s_nat = nat;
            const int la = bsearch_atom(atoms, nat, j / B);
            s_jloc = la >= 0 ? la * B + (int)(j % B) : -1;
            s_nkept = nkept;
        }
        for (int k = tid; k < nkept; k += LNT) {
            const int64_t row = a.orows[k0 + k];
            const int la = bsearch_atom(atoms, nat, row / B);
            kept[k] = la >= 0 ? la * B + (int)(row % B) : -1;
        }
        __syncthreads();
        const int nrows = nat * B;
        const int jloc = s_jloc;
        // ---- initial state
        for (int l = tid; l < nrows; l += LNT) {
            const cpx<T> e = mk<T>(l == jloc ? (T)1 : (T)0, 0);
            RT[l] = e;
            P[l] = mk<T>(0, 0);
            U[l] = mk<T>(0, 0);
            if constexpr (HAS_S) {
                R[l] = e; // inner CG start
                SP[l] = mk<T>(0, 0);
            }
        }
        for (int q = tid; q < nkept * a.nz; q += LNT) xs[q] = ps[q] = mk(0.0, 0.0);
        for (int m = tid; m < a.nz; m += LNT) {
            ShiftL s;
            s.pi = s.pi_prev = s.pi_next = mk(1.0, 0.0);
            s.resid = 1.0;
            s.active = 1;
            s.conv_it = -1;
            shs[m] = s;
        }
        if (tid == 0) {
            s_rho = mk(1.0, 0.0);
            s_alpha = mk(0.0, 0.0);
            s_alpha_prev = mk(1.0, 0.0);
            s_beta_prev = mk(0.0, 0.0);
            s_rn2 = 1.0;
            s_status = TB_COL_MAX_ITER;
            s_stop = (jloc < 0);
            if (jloc < 0) s_status = TB_COL_BREAKDOWN;
            s_zs = a.zs;
            s_restarts = 0;
            s_restart = 0;
            s_chk_n = -1;
            s_chk_w = 0.0;
        }
        __syncthreads();

        // inner CG: R <- S^{-1} RT starting from R (Hermitian CG), bounded
        auto inner_solve = [&]() -> int {
            int it = 0;
            if constexpr (HAS_S) {
                Acc<T> acc[2];
                acc[0].zero(), acc[1].zero();
                for (int l = tid; l < nrows; l += LNT) {
                    const cpx<T> sy = local_row_product<T, B>(l, a.s_val, nbk, nbl, cnt, a.dmax, R);
                    const cpx<T> t = RT[l] - sy;
                    Tv[l] = t;
                    D[l] = t;
                    acc[0].add(t.re * t.re);
                    acc[0].add(t.im * t.im);
                    acc[1].add(RT[l].re * RT[l].re);
                    acc[1].add(RT[l].im * RT[l].im);
                }
                cta_sum<T, 2>(acc, red);
                if (tid == 0) {
                    s_in_rr = red[0];
                    s_in_tol2 = a.inner_tol * a.inner_tol * red[1];
                    s_in_stop = !(s_in_rr > s_in_tol2);
                }
                __syncthreads();
                while (!s_in_stop && it < a.inner_max) {
                    Acc<T> ad[1];
                    ad[0].zero();
                    for (int l = tid; l < nrows; l += LNT) {
                        const cpx<T> sd = local_row_product<T, B>(l, a.s_val, nbk, nbl, cnt, a.dmax, D);
                        Av[l] = sd;
                        ad[0].add(D[l].re * sd.re);
                        ad[0].add(D[l].im * sd.im);
                    }
                    cta_sum<T, 1>(ad, red);
                    if (tid == 0) {
                        if (!(red[0] > 0.0) || !isfinite(red[0])) {
                            s_in_stop = 1;
                            s_in_alpha = 0.0;
                        } else {
                            s_in_alpha = s_in_rr / red[0];
                        }
                    }
                    __syncthreads();
                    if (s_in_stop) break;
                    const T al = (T)s_in_alpha;
                    Acc<T> tt[1];
                    tt[0].zero();
                    for (int l = tid; l < nrows; l += LNT) {
                        R[l] = R[l] + mk<T>(al, 0) * D[l];
                        const cpx<T> t = Tv[l] - mk<T>(al, 0) * Av[l];
                        Tv[l] = t;
                        tt[0].add(t.re * t.re);
                        tt[0].add(t.im * t.im);
                    }
                    cta_sum<T, 1>(tt, red);
                    if (tid == 0) {
                        s_in_beta = red[0] / s_in_rr;
                        s_in_rr = red[0];
                        s_in_stop = !(red[0] > s_in_tol2) || !isfinite(red[0]);
                    }
                    __syncthreads();
                    ++it;
                    if (s_in_stop) break;
                    const T be = (T)s_in_beta;
                    for (int l = tid; l < nrows; l += LNT) D[l] = Tv[l] + mk<T>(be, 0) * D[l];
                    __syncthreads();
                }
            }
            return it;
        };

        int64_t inner_total = 0;
        // r_0 = S^{-1} e_j and rho_0 = r_0^T rt_0 (S != I; rho_0 = 1 when S = I)
        auto seed_start = [&]() {
            if constexpr (HAS_S) {
                inner_total += inner_solve();
                Acc<T> rr[2];
                rr[0].zero(), rr[1].zero();
                for (int l = tid; l < nrows; l += LNT) {
                    rr[0].add(R[l].re * RT[l].re);
                    rr[0].add(-(R[l].im * RT[l].im));
                    rr[1].add(R[l].re * RT[l].im);
                    rr[1].add(R[l].im * RT[l].re);
                }
                cta_sum<T, 2>(rr, red);
                if (tid == 0) s_rho = mk(red[0], red[1]);
                __syncthreads();
            }
        };
        seed_start();

        int n = 0;
        for (;; ++n) {
            // ---- shifted step A: rotate pi, residual test, p^m on kept rows
            if (tid == 0) s_nact = 0;
            __syncthreads();
            int my_act = 0;
            for (int m = tid; m < a.nz; m += LNT) {
                ShiftL &s = shs[m];
                if (!s.active) continue;
                s.pi_prev = s.pi;
                s.pi = s.pi_next;
                const double pi2 = cabs2(s.pi);
                s.resid = sqrt(s_rn2 / pi2);
                if (s_rn2 <= a.tol * a.tol * pi2) {
                    s.active = 0;
                    s.conv_it = n;
                    continue;
                }
                ++my_act;
                const c64 ratio = cdiv(s.pi_prev, s.pi);
                const c64 bs = (ratio * ratio) * s_beta_prev;
                const c64 ipi = cdiv(mk(1.0, 0.0), s.pi);
                for (int k = 0; k < s_nkept; ++k) {
                    const int lr = kept[k];
                    if (lr < 0) continue;
                    const c64 rv = to64(R[lr]);
                    c64 &pk = ps[(int64_t)k * a.nz + m];
                    pk = ipi * rv + bs * pk;
                }
            }
            if (my_act) atomicAdd(&s_nact, my_act);
            __syncthreads();
            // Restart with a new seed.  Every shift's residual is the seed's
            // divided by |pi|: a shift much harder than the seed needs the seed
            // residual far below the tolerance, below what the working
            // precision carries (df: near 1e-10 relative).  Once the seed
            // residual is below that level, the worst active shift is checked
            // every 256 iterations; if it improved by less than 10 % the column
            // restarts with that shift as its seed: converged shifts keep their
            // solutions, active ones start again from zero.
            if (tid == 0) {
                s_restart = 0;
                if (s_nact > 0 && !s_stop && s_rn2 < a.stall2 && s_restarts < 2 &&
                    (s_chk_n < 0 || n - s_chk_n >= 256)) {
                    int mw = -1;
                    double rw = -1.0;
                    for (int m = 0; m < a.nz; ++m)
                        if (shs[m].active && shs[m].resid > rw) rw = shs[m].resid, mw = m;
                    if (s_chk_n >= 0 && mw >= 0 && rw > 0.9 * s_chk_w) {
                        s_zs = a.z[mw];
                        s_restart = 1;
                        s_restarts += 1;
                        s_chk_n = -1;
                    } else {
                        s_chk_n = n;
                        s_chk_w = rw;
                    }
                }
            }
            __syncthreads();
            if (s_restart) {
                for (int m = tid; m < a.nz; m += LNT) {
                    ShiftL &sm = shs[m];
                    if (!sm.active) continue;
                    sm.pi = sm.pi_prev = sm.pi_next = mk(1.0, 0.0);
                    sm.resid = 1.0;
                    for (int k = 0; k < s_nkept; ++k) {
                        xs[(int64_t)k * a.nz + m] = mk(0.0, 0.0);
                        ps[(int64_t)k * a.nz + m] = mk(0.0, 0.0);
                    }
                }
                for (int l = tid; l < nrows; l += LNT) {
                    const cpx<T> e = mk<T>(l == jloc ? (T)1 : (T)0, 0);
                    RT[l] = e;
                    P[l] = mk<T>(0, 0);
                    U[l] = mk<T>(0, 0);
                    if constexpr (HAS_S) {
                        R[l] = e;
                        SP[l] = mk<T>(0, 0);
                    }
                }
                if (tid == 0) {
                    s_rho = mk(1.0, 0.0);
                    s_alpha = mk(0.0, 0.0);
                    s_alpha_prev = mk(1.0, 0.0);
                    s_beta_prev = mk(0.0, 0.0);
                    s_rn2 = 1.0;
                }
                __syncthreads();
                seed_start();
                continue; // the next iteration tests the restarted shifts again
            }
            if (tid == 0) {
                if (s_nact == 0 && !s_stop) {
                    s_stop = 1;
                    s_status = TB_COL_CONVERGED;
                } else if (n >= a.max_iter && !s_stop) {
                    s_stop = 1;
                    s_status = TB_COL_MAX_ITER;
                }
            }
            __syncthreads();
            if (s_stop) break;
            // ---- seed step: p, Sp, u = z_s Sp - H p, mu = p^T u
            const cpx<T> beta = cvt<T>(s_beta_prev);
            const cpx<T> zs = cvt<T>(s_zs);
            for (int l = tid; l < nrows; l += LNT) {
                P[l] = R[l] + beta * P[l];
                if constexpr (HAS_S) SP[l] = RT[l] + beta * SP[l];
            }
            __syncthreads();
            Acc<T> mu[2];
            mu[0].zero(), mu[1].zero();
            for (int l = tid; l < nrows; l += LNT) {
                const cpx<T> hp = local_row_product<T, B>(l, a.h_val, nbk, nbl, cnt, a.dmax, P);
                const cpx<T> pv = P[l];
                const cpx<T> u = zs * (HAS_S ? SP[l] : pv) - hp;
                U[l] = u;
                mu[0].add(pv.re * u.re);
                mu[0].add(-(pv.im * u.im));
                mu[1].add(pv.re * u.im);
                mu[1].add(pv.im * u.re);
            }
            cta_sum<T, 2>(mu, red);
            if (tid == 0) {
                const c64 m = mk(red[0], red[1]);
                if (!cfinite(m) || !cfinite(s_rho)) {
                    s_stop = 1;
                    s_status = TB_COL_NONFINITE;
                } else if ((m.re == 0.0 && m.im == 0.0) || (s_rho.re == 0.0 && s_rho.im == 0.0)) {
                    s_stop = 1;
                    s_status = TB_COL_BREAKDOWN;
                } else {
                    s_alpha = cdiv(s_rho, m);
                    if (!cfinite(s_alpha)) {
                        s_stop = 1;
                        s_status = TB_COL_NONFINITE;
                    }
                }
            }
            __syncthreads();
            if (s_stop) break;
            // ---- shifted step B: pi_{n+1}, alpha^m, x^m += alpha^m p^m
            const c64 al64 = s_alpha;
            for (int m = tid; m < a.nz; m += LNT) {
                ShiftL &s = shs[m];
                if (!s.active) continue;
                const c64 sig = a.z[m] - s_zs;
                const c64 coef = cdiv(al64 * s_beta_prev, s_alpha_prev);
                const c64 pn = (mk(1.0, 0.0) + al64 * sig) * s.pi + coef * (s.pi - s.pi_prev);
                const c64 as = cdiv(s.pi, pn) * al64;
                if (!cfinite(pn) || (pn.re == 0.0 && pn.im == 0.0) || !cfinite(as)) {
                    s.active = 0;
                    s.resid = nan("");
                    continue;
                }
                s.pi_next = pn;
                for (int k = 0; k < s_nkept; ++k) {
                    c64 &xk = xs[(int64_t)k * a.nz + m];
                    xk = xk + as * ps[(int64_t)k * a.nz + m];
                }
            }
            // ---- residual update (and inner solve when S != I)
            const cpx<T> alpha = cvt<T>(al64);
            if constexpr (HAS_S) {
                for (int l = tid; l < nrows; l += LNT) {
                    RT[l] = RT[l] - alpha * U[l];
                    R[l] = R[l] - alpha * U[l]; // inner start y_0 = r_n - alpha u
                }
                __syncthreads();
                inner_total += inner_solve();
                Acc<T> rr[3];
                rr[0].zero(), rr[1].zero(), rr[2].zero();
                for (int l = tid; l < nrows; l += LNT) {
                    const cpx<T> r = R[l], rt = RT[l];
                    rr[0].add(r.re * rt.re);
                    rr[0].add(-(r.im * rt.im));
                    rr[1].add(r.re * rt.im);
                    rr[1].add(r.im * rt.re);
                    rr[2].add(rt.re * rt.re);
                    rr[2].add(rt.im * rt.im);
                }
                cta_sum<T, 3>(rr, red);
            } else {
                Acc<T> rr[3];
                rr[0].zero(), rr[1].zero(), rr[2].zero();
                for (int l = tid; l < nrows; l += LNT) {
                    const cpx<T> rt = RT[l] - alpha * U[l];
                    RT[l] = rt;
                    const T x2 = rt.re * rt.re, y2 = rt.im * rt.im;
                    rr[0].add(x2);
                    rr[0].add(-y2);
                    rr[1].add((T)2 * rt.re * rt.im);
                    rr[2].add(x2);
                    rr[2].add(y2);
                }
                cta_sum<T, 3>(rr, red);
            }
            if (tid == 0) {
                const c64 rn = mk(red[0], red[1]);
                s_beta_prev = cdiv(rn, s_rho);
                s_alpha_prev = s_alpha;
                s_rho = rn;
                s_rn2 = red[2];
            }
            __syncthreads();
        }
        // ---- outputs
        for (int q = tid; q < s_nkept * a.nz; q += LNT) a.G[(k0 + q / a.nz) * a.nz + q % a.nz] = xs[q];
        for (int m = tid; m < a.nz; m += LNT) a.resid[col * a.nz + m] = shs[m].resid;
        if (tid == 0) {
            a.iters[col] = n;
            a.status[col] = s_status;
            atomicAdd(&a.stat[0], (unsigned long long)n);
            atomicAdd(&a.stat[1], (unsigned long long)inner_total);
        }
        __syncthreads();
    }
}

// Shared memory of k_local: the subspace vectors (unless they are placed in
// global memory), the per-shift states and the local block structure.
inline size_t local_vec_bytes(int maxa, int b, size_t cpx_size, bool has_s) {
    return (size_t)(has_s ? 8 : 3) * maxa * b * cpx_size;
}
inline size_t local_smem(int maxa, int dmax, int max_kept, int nz, bool has_s, int b, size_t cpx_size,
                         bool vectors) {
    return (vectors ? local_vec_bytes(maxa, b, cpx_size, has_s) : 0) + (size_t)nz * sizeof(ShiftL) +
           (size_t)maxa * 4 + (size_t)maxa * dmax * 4 + (size_t)max_kept * 4 + (size_t)maxa * dmax * 2 +
           (size_t)maxa * 2 + 16;
}

struct LocalLaunch {
    tb_ctx *ctx;
    LocalArgs<double> args; // type-erased (T-dependent members are pointers)
    bool has_s;
    int grid;
    cudaStream_t stream;
    int rc = TB_OK;
    template <typename T, int B, int W>
    void run() {
        if (W != 8) return; // W is not used by the local solver; dispatch once
        LocalArgs<T> a;
        static_assert(sizeof(LocalArgs<T>) == sizeof(LocalArgs<double>), "layout");
        std::memcpy(&a, &args, sizeof(a));
        const size_t sm = local_smem(a.maxa, a.dmax, a.max_kept, a.nz, has_s, B, sizeof(cpx<T>), a.gvec == nullptr);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (sm > (size_t)optin) {
            rc = set_error(ctx, TB_ERR_SIZE, "local subspace needs %zu bytes of shared memory (limit %d)", sm, optin);
            return;
        }
        const void *fn = has_s ? (const void *)k_local<T, B, true> : (const void *)k_local<T, B, false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) {
            rc = set_error(ctx, TB_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            return;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LNT, sm);
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int g = std::max(1, std::min<int>(grid, sms * std::max(per_sm, 1)));
        if (has_s)
            k_local<T, B, true><<<g, LNT, sm, stream>>>(a);
        else
            k_local<T, B, false><<<g, LNT, sm, stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(ctx, TB_ERR_CUDA, "k_local launch: %s", cudaGetErrorString(e));
    }
};

bool launch_local_f64(LocalLaunch &L, int b);
bool launch_local_f32(LocalLaunch &L, int b);
bool launch_local_df(LocalLaunch &L, int b);

} // namespace tbgf
