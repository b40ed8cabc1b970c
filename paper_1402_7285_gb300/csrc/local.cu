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
    unsigned long long *queue;
    unsigned long long *stat; // [2]: outer, inner iterations
    double tol, inner_tol;
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
            const T v = __ldg(row + j);
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
    cpx<T> *vec = reinterpret_cast<cpx<T> *>(smem);
    cpx<T> *RT = vec;               // rt (= r when S = I)
    cpx<T> *P = vec + maxr;
    cpx<T> *U = vec + 2 * maxr;
    cpx<T> *R = HAS_S ? vec + 3 * maxr : RT;
    cpx<T> *SP = vec + 4 * maxr, *Tv = vec + 5 * maxr, *D = vec + 6 * maxr, *Av = vec + 7 * maxr;
    ShiftL *shs = reinterpret_cast<ShiftL *>(vec + NV * maxr);
    int32_t *atoms = reinterpret_cast<int32_t *>(shs + a.nz);
    int32_t *nbk = atoms + a.maxa;
    int32_t *kept = nbk + a.maxa * a.dmax;
    int16_t *nbl = reinterpret_cast<int16_t *>(kept + a.max_kept);
    int16_t *cnt = nbl + a.maxa * a.dmax;

    __shared__ double red[4];
    __shared__ int s_col, s_nat, s_jloc, s_nkept, s_nact;
    __shared__ c64 s_rho, s_alpha, s_alpha_prev, s_beta_prev;
    __shared__ double s_rn2, s_in_rr, s_in_alpha, s_in_beta, s_in_tol2;
    __shared__ int s_status, s_stop, s_in_stop;

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
            const cpx<T> zs = cvt<T>(a.zs);
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
                const c64 sig = a.z[m] - a.zs;
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

template <typename T, int B>
size_t local_smem(int maxa, int dmax, int max_kept, int nz, bool has_s) {
    const int NV = has_s ? 8 : 3;
    return (size_t)NV * maxa * B * sizeof(cpx<T>) + (size_t)nz * sizeof(ShiftL) + (size_t)maxa * 4 +
           (size_t)maxa * dmax * 4 + (size_t)max_kept * 4 + (size_t)maxa * dmax * 2 + (size_t)maxa * 2 + 16;
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
        const size_t sm = local_smem<T, B>(a.maxa, a.dmax, a.max_kept, a.nz, has_s);
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
        args.scratch = args.scratch; // sized by the caller for `grid` CTAs
        if (has_s)
            k_local<T, B, true><<<g, LNT, sm, stream>>>(a);
        else
            k_local<T, B, false><<<g, LNT, sm, stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(ctx, TB_ERR_CUDA, "k_local launch: %s", cudaGetErrorString(e));
    }
};

__global__ void k_copy_z_local(const double *z, c64 *zc, int nz) {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) zc[i] = mk(z[2 * i], z[2 * i + 1]);
}

__global__ void k_same_pattern(const int64_t *a_rp, const int32_t *a_ci, const int64_t *b_rp, const int32_t *b_ci,
                               int64_t n, int64_t nnzb, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += stride)
        if (a_rp[i] != b_rp[i]) atomicOr(bad, 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnzb; i += stride)
        if (a_ci[i] != b_ci[i]) atomicOr(bad, 1);
}

} // namespace tbgf

using namespace tbgf;

namespace {
template <typename X>
int fetch_host_l(tb_ctx *ctx, const X *p, size_t n, std::vector<X> &out) {
    out.resize(n);
    if (n == 0) return TB_OK;
    if (is_device_ptr(p)) {
        TB_CUDA_TRY(ctx, cudaMemcpy(out.data(), p, n * sizeof(X), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), p, n * sizeof(X));
    }
    return TB_OK;
}
} // namespace

extern "C" int shifted_cocg_solve_local(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
                                        const int64_t *rhs_rows, int64_t n_rhs, const int64_t *sub_ptr,
                                        const int32_t *sub_atoms, const int64_t *out_row_ptr, const int64_t *out_rows,
                                        const int64_t *order, const tb_solve_opts *opts_in, double *G, int32_t *iters,
                                        double *resid, int32_t *status) {
    if (!ctx) return TB_ERR_ARG;
    tb_solve_opts opts;
    if (opts_in)
        opts = *opts_in;
    else
        tb_solve_opts_default(&opts);
    TB_CHECK(ctx, H && H->row_ptr && H->col_idx && H->val && H->n_brows > 0, TB_ERR_ARG, "H is incomplete");
    TB_CHECK(ctx, supported_bdim(H->bdim), TB_ERR_UNSUPPORTED, "bdim %d has no compiled kernels", H->bdim);
    TB_CHECK(ctx, !S || (S->row_ptr && S->col_idx && S->val && S->n_brows == H->n_brows && S->bdim == H->bdim &&
                         S->nnzb == H->nnzb),
             TB_ERR_ARG, "S must have H's block pattern");
    TB_CHECK(ctx, z && n_z >= 1 && n_z <= 1024, TB_ERR_ARG, "n_z must be 1..1024 for the local solver");
    TB_CHECK(ctx, n_rhs >= 0 && (n_rhs == 0 || (rhs_rows && sub_ptr && sub_atoms && out_row_ptr)), TB_ERR_ARG,
             "rhs / subspace arrays missing");
    TB_CHECK(ctx, opts.precision == TB_PREC_FP64 || opts.precision == TB_PREC_MIXED, TB_ERR_ARG, "bad precision");
    TB_CHECK(ctx, opts.tol > 0.0 && opts.max_iter >= 0, TB_ERR_ARG, "tol must be > 0 and max_iter >= 0");
    if (opts.stats) opts.stats[0] = opts.stats[1] = 0;
    if (n_rhs == 0) return TB_OK;
    cudaStream_t stream = (cudaStream_t)opts.stream;
    const bool mixed = opts.precision == TB_PREC_MIXED;
    const bool has_s = S != nullptr;
    const int b = H->bdim;
    const int64_t n_rows = H->n_brows * b;
    const int64_t bb = (int64_t)b * b;
    // ---- host-side checks of the index arrays
    std::vector<int64_t> h_rhs, h_sptr, h_optr, h_orows, h_order, h_hrp;
    std::vector<int32_t> h_atoms;
    std::vector<double> h_z;
    int rc = fetch_host_l(ctx, rhs_rows, n_rhs, h_rhs);
    if (!rc) rc = fetch_host_l(ctx, sub_ptr, n_rhs + 1, h_sptr);
    if (!rc) rc = fetch_host_l(ctx, out_row_ptr, n_rhs + 1, h_optr);
    if (!rc) rc = fetch_host_l(ctx, z, 2 * (size_t)n_z, h_z);
    if (!rc) rc = fetch_host_l(ctx, H->row_ptr, H->n_brows + 1, h_hrp);
    if (rc) return rc;
    TB_CHECK(ctx, h_sptr[0] == 0 && h_optr[0] == 0, TB_ERR_ARG, "sub_ptr and out_row_ptr must start at 0");
    const int64_t n_sub = h_sptr[n_rhs], n_out = h_optr[n_rhs];
    rc = fetch_host_l(ctx, sub_atoms, n_sub, h_atoms);
    if (!rc) rc = fetch_host_l(ctx, out_rows, n_out, h_orows);
    if (!rc && order) rc = fetch_host_l(ctx, order, n_rhs, h_order);
    if (rc) return rc;
    int maxa = 1, max_kept = 1, dmax = 1;
    for (int64_t a = 0; a < H->n_brows; ++a) dmax = std::max<int64_t>(dmax, h_hrp[a + 1] - h_hrp[a]);
    for (int64_t c = 0; c < n_rhs; ++c) {
        const int64_t na = h_sptr[c + 1] - h_sptr[c];
        TB_CHECK(ctx, na >= 1 && na <= 32767, TB_ERR_ARG, "subspace %lld has %lld atoms (1..32767)", (long long)c,
                 (long long)na);
        TB_CHECK(ctx, h_rhs[c] >= 0 && h_rhs[c] < n_rows, TB_ERR_ARG, "rhs row out of range");
        bool has_j = false;
        for (int64_t i = h_sptr[c]; i < h_sptr[c + 1]; ++i) {
            TB_CHECK(ctx, h_atoms[i] >= 0 && h_atoms[i] < H->n_brows, TB_ERR_ARG, "subspace atom out of range");
            TB_CHECK(ctx, i == h_sptr[c] || h_atoms[i] > h_atoms[i - 1], TB_ERR_ARG, "subspace atoms must ascend");
            has_j |= (h_atoms[i] == h_rhs[c] / b);
        }
        TB_CHECK(ctx, has_j, TB_ERR_ARG, "subspace %lld does not contain its right-hand side", (long long)c);
        TB_CHECK(ctx, h_optr[c + 1] >= h_optr[c], TB_ERR_ARG, "out_row_ptr not monotone");
        maxa = std::max<int64_t>(maxa, na);
        max_kept = std::max<int64_t>(max_kept, h_optr[c + 1] - h_optr[c]);
    }
    for (int64_t e = 0; e < n_out; ++e) TB_CHECK(ctx, h_orows[e] >= 0 && h_orows[e] < n_rows, TB_ERR_ARG, "out row");
    if (order) {
        std::vector<char> seen(n_rhs, 0);
        for (int64_t i = 0; i < n_rhs; ++i) {
            TB_CHECK(ctx, h_order[i] >= 0 && h_order[i] < n_rhs && !seen[h_order[i]], TB_ERR_ARG,
                     "order must be a permutation");
            seen[h_order[i]] = 1;
        }
    }
    // ---- stage
    Stager stg(ctx, WS_STAGE_IN, stream);
    void *d_hrp, *d_hci, *d_hval, *d_srp = nullptr, *d_sci = nullptr, *d_sval = nullptr, *d_z, *d_rhs, *d_sptr,
                                  *d_atoms, *d_optr, *d_orows = nullptr, *d_order = nullptr;
    void *d_G, *d_iters, *d_resid, *d_status;
    stg.add(H->row_ptr, sizeof(int64_t) * (H->n_brows + 1), true, false, &d_hrp);
    stg.add(H->col_idx, sizeof(int32_t) * H->nnzb, true, false, &d_hci);
    stg.add(H->val, sizeof(double) * H->nnzb * bb, true, false, &d_hval);
    if (has_s) {
        stg.add(S->row_ptr, sizeof(int64_t) * (S->n_brows + 1), true, false, &d_srp);
        stg.add(S->col_idx, sizeof(int32_t) * S->nnzb, true, false, &d_sci);
        stg.add(S->val, sizeof(double) * S->nnzb * bb, true, false, &d_sval);
    }
    stg.add(z, sizeof(double) * 2 * n_z, true, false, &d_z);
    stg.add(rhs_rows, sizeof(int64_t) * n_rhs, true, false, &d_rhs);
    stg.add(sub_ptr, sizeof(int64_t) * (n_rhs + 1), true, false, &d_sptr);
    stg.add(sub_atoms, sizeof(int32_t) * n_sub, true, false, &d_atoms);
    stg.add(out_row_ptr, sizeof(int64_t) * (n_rhs + 1), true, false, &d_optr);
    if (n_out) stg.add(out_rows, sizeof(int64_t) * n_out, true, false, &d_orows);
    if (order) stg.add(order, sizeof(int64_t) * n_rhs, true, false, &d_order);
    stg.add(G, sizeof(double) * 2 * n_out * n_z, false, true, &d_G);
    stg.add(iters, sizeof(int32_t) * n_rhs, false, true, &d_iters);
    stg.add(resid, sizeof(double) * n_rhs * n_z, false, true, &d_resid);
    stg.add(status, sizeof(int32_t) * n_rhs, false, true, &d_status);
    rc = stg.commit();
    if (rc) return rc;
    rc = validate_bsr(ctx, (const int64_t *)d_hrp, (const int32_t *)d_hci, d_hval, H->n_brows, H->nnzb, stream, "H");
    if (rc) return rc;
    // ---- workspace: per-CTA kept-row states, z, FP32 matrix copies, queue, pattern check
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_scr = take(sizeof(c64) * 2 * (size_t)max_kept * n_z * grid);
    const size_t o_zc = take(sizeof(c64) * n_z);
    const size_t o_q = take(sizeof(unsigned long long) * 4);
    const size_t o_h32 = mixed ? take(sizeof(float) * H->nnzb * bb) : 0;
    const size_t o_s32 = (mixed && has_s) ? take(sizeof(float) * S->nnzb * bb) : 0;
    void *wsp = nullptr;
    rc = ws_get(ctx, WS_SOLVE_SMALL, off, &wsp);
    if (rc) return rc;
    char *ws = (char *)wsp;
    TB_CUDA_TRY(ctx, cudaMemsetAsync(ws + o_q, 0, sizeof(unsigned long long) * 4, stream));
    if (has_s) {
        int *flag = (int *)(ws + o_q) + 6;
        k_same_pattern<<<152 * 4, 256, 0, stream>>>((const int64_t *)d_hrp, (const int32_t *)d_hci,
                                                     (const int64_t *)d_srp, (const int32_t *)d_sci, H->n_brows,
                                                     H->nnzb, flag);
        int h = 0;
        TB_CUDA_TRY(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        TB_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        TB_CHECK(ctx, h == 0, TB_ERR_ARG, "S must have H's block pattern");
    }
    k_copy_z_local<<<1, 256, 0, stream>>>((const double *)d_z, (c64 *)(ws + o_zc), n_z);
    const void *hval = d_hval, *sval = d_sval;
    if (mixed) {
        launch_to_float((const double *)d_hval, (float *)(ws + o_h32), H->nnzb * bb, stream);
        hval = ws + o_h32;
        if (has_s) {
            launch_to_float((const double *)d_sval, (float *)(ws + o_s32), S->nnzb * bb, stream);
            sval = ws + o_s32;
        }
    }
    // seed shift: median real part
    std::vector<int> idx(n_z);
    for (int i = 0; i < n_z; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return h_z[2 * x] < h_z[2 * y]; });
    const int seed = opts.seed_shift >= 0 ? opts.seed_shift : idx[n_z / 2];
    LocalArgs<double> la;
    std::memset(&la, 0, sizeof(la));
    la.h_rp = (const int64_t *)d_hrp;
    la.h_ci = (const int32_t *)d_hci;
    la.h_val = (const double *)hval;
    la.s_val = has_s ? (const double *)sval : nullptr;
    la.n_brows = H->n_brows;
    la.z = (const c64 *)(ws + o_zc);
    la.nz = n_z;
    la.zs = mk(h_z[2 * seed], h_z[2 * seed + 1]);
    la.rhs = (const int64_t *)d_rhs;
    la.sub_ptr = (const int64_t *)d_sptr;
    la.sub_atoms = (const int32_t *)d_atoms;
    la.optr = (const int64_t *)d_optr;
    la.orows = (const int64_t *)d_orows;
    la.order = (const int64_t *)d_order;
    la.n = n_rhs;
    la.maxa = maxa;
    la.dmax = dmax;
    la.max_kept = max_kept;
    la.scratch = (c64 *)(ws + o_scr);
    la.queue = (unsigned long long *)(ws + o_q);
    la.stat = (unsigned long long *)(ws + o_q) + 1;
    la.tol = opts.tol;
    la.inner_tol = opts.inner_tol > 0.0 ? opts.inner_tol : (mixed ? 1e-7 : 1e-13);
    la.max_iter = opts.max_iter;
    la.inner_max = opts.inner_max > 0 ? opts.inner_max : 40;
    la.G = (c64 *)d_G;
    la.iters = (int32_t *)d_iters;
    la.resid = (double *)d_resid;
    la.status = (int32_t *)d_status;
    LocalLaunch L{ctx, la, has_s, grid, stream};
    if (!dispatch_tbw(L, mixed, b, 8)) return set_error(ctx, TB_ERR_UNSUPPORTED, "no local solver variant");
    if (L.rc) return L.rc;
    TB_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    if (opts.stats) {
        unsigned long long st2[2];
        TB_CUDA_TRY(ctx, cudaMemcpy(st2, la.stat, sizeof(st2), cudaMemcpyDeviceToHost));
        opts.stats[0] = (int64_t)st2[0];
        opts.stats[1] = (int64_t)st2[1];
    }
    std::vector<int32_t> stv(n_rhs);
    TB_CUDA_TRY(ctx, cudaMemcpy(stv.data(), d_status, sizeof(int32_t) * n_rhs, cudaMemcpyDeviceToHost));
    rc = stg.finish();
    if (rc) return rc;
    int warn = 0;
    for (int32_t s : stv) {
        if (s == TB_COL_MAX_ITER) warn |= TB_WARN_MAX_ITER;
        if (s == TB_COL_BREAKDOWN) warn |= TB_WARN_BREAKDOWN;
        if (s == TB_COL_NONFINITE) warn |= TB_WARN_NONFINITE;
    }
    return warn;
}
