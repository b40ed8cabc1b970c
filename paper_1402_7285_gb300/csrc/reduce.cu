// gf_reduce_ldos_dm: Green's-function entries -> LDOS and density-matrix elements.
//
// Sec. 2 takes the density of states and a Green's-function population analysis
// from G; the standard formulas are used (FP64 throughout):
//   ldos_j(E_m) = -(1/pi) Im sum_k G_{i_k j}(z_m) S_{i_k j}   (S = I: -(1/pi) Im G_jj)
//   rho_{i j}   = -(1/pi) Im sum_m w_m f(E_m) G_{i j}(z_m)
// with f the Fermi-Dirac occupation (kT = 0: step, f(mu) = 1/2).
#include "common.cuh"

namespace {

constexpr double INV_PI = 0.318309886183790671537767526745028724;

__device__ __forceinline__ double fermi(double e, double mu, double kT) {
    if (kT == 0.0) return e < mu ? 1.0 : (e > mu ? 0.0 : 0.5);
    const double x = (e - mu) / kT;
    if (x > 0.0) {
        const double ex = exp(-x);
        return ex / (1.0 + ex);
    }
    return 1.0 / (1.0 + exp(x));
}

// weight of each kept entry in the LDOS sum: S_{i j} (or [i == j] when S = I)
__global__ void k_entry_weight(const int64_t *rhs, int64_t n_rhs, const int64_t *optr, const int64_t *orows,
                               const int64_t *s_rp, const int32_t *s_ci, const double *s_val, int bdim,
                               double *wt, int *missing) {
    const int64_t n_out = optr[n_rhs];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_out; e += (int64_t)gridDim.x * blockDim.x) {
        // column owning entry e: binary search in optr
        int64_t lo = 0, hi = n_rhs;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            if (optr[mid] <= e) lo = mid; else hi = mid;
        }
        const int64_t j = rhs[lo], i = orows[e];
        if (!s_rp) {
            wt[e] = (i == j) ? 1.0 : 0.0;
            continue;
        }
        const int64_t ai = i / bdim, aj = j / bdim;
        int64_t k0 = s_rp[ai], k1 = s_rp[ai + 1];
        double v = 0.0;
        while (k0 < k1) { // col_idx ascending within the block row
            const int64_t mid = (k0 + k1) / 2;
            const int64_t cm = s_ci[mid];
            if (cm == aj) {
                v = s_val[mid * bdim * bdim + (i % bdim) * bdim + (j % bdim)];
                break;
            }
            if (cm < aj) k0 = mid + 1; else k1 = mid;
        }
        wt[e] = v;
    }
    (void)missing;
}

__global__ void k_has_diag(const int64_t *rhs, int64_t n_rhs, const int64_t *optr, const int64_t *orows, int *missing) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_rhs; c += (int64_t)gridDim.x * blockDim.x) {
        bool found = false;
        for (int64_t e = optr[c]; e < optr[c + 1] && !found; ++e) found = (orows[e] == rhs[c]);
        if (!found) atomicAdd(missing, 1);
    }
}

__global__ void k_ldos(const double *G, int nz, const int64_t *optr, int64_t n_rhs, const double *wt, double *ldos) {
    const int64_t total = n_rhs * nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / nz;
        const int m = (int)(t % nz);
        double s = 0.0;
        for (int64_t e = optr[c]; e < optr[c + 1]; ++e) s += G[(e * nz + m) * 2 + 1] * wt[e];
        ldos[t] = -INV_PI * s;
    }
}

__global__ void k_dm(const double *G, int nz, const double *z, const double *w, double mu, double kT, int64_t n_out,
                     double *dm) {
    extern __shared__ double occ[];
    for (int m = threadIdx.x; m < nz; m += blockDim.x) occ[m] = w[m] * fermi(z[2 * m], mu, kT);
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_out; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int m = 0; m < nz; ++m) s += occ[m] * G[(e * nz + m) * 2 + 1];
        dm[e] = -INV_PI * s;
    }
}

} // namespace

extern "C" int gf_reduce_ldos_dm(tb_ctx *ctx, const double *G, int32_t n_z, const double *z, const double *w,
                                 double mu, double kT, const int64_t *rhs_rows, int64_t n_rhs,
                                 const int64_t *out_row_ptr, const int64_t *out_rows, const tb_bsr *S, double *ldos,
                                 double *dm, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, n_z >= 1 && n_rhs >= 0 && G && z && rhs_rows && out_row_ptr, TB_ERR_ARG, "gf_reduce_ldos_dm: bad arguments");
    TB_CHECK(ctx, kT >= 0.0, TB_ERR_ARG, "kT must be >= 0");
    TB_CHECK(ctx, !dm || w, TB_ERR_ARG, "quadrature weights required for the density matrix");
    TB_CHECK(ctx, !S || (S->row_ptr && S->col_idx && S->val), TB_ERR_ARG, "S is incomplete");
    if (n_rhs == 0) return TB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n_out = 0;
    if (is_device_ptr(out_row_ptr)) {
        TB_CUDA_TRY(ctx, cudaMemcpy(&n_out, out_row_ptr + n_rhs, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
        n_out = out_row_ptr[n_rhs];
    }
    TB_CHECK(ctx, n_out >= 0 && (n_out == 0 || out_rows), TB_ERR_ARG, "out_rows missing");
    const int64_t bb = S ? (int64_t)S->bdim * S->bdim : 0;
    Stager st(ctx, WS_REDUCE, s);
    void *dG, *dz, *dw = nullptr, *drhs, *dptr, *drows = nullptr, *dsrp = nullptr, *dsci = nullptr, *dsval = nullptr;
    void *dldos = nullptr, *ddm = nullptr;
    st.add(G, sizeof(double) * 2 * n_out * n_z, true, false, &dG);
    st.add(z, sizeof(double) * 2 * n_z, true, false, &dz);
    if (w) st.add(w, sizeof(double) * n_z, true, false, &dw);
    st.add(rhs_rows, sizeof(int64_t) * n_rhs, true, false, &drhs);
    st.add(out_row_ptr, sizeof(int64_t) * (n_rhs + 1), true, false, &dptr);
    if (n_out) st.add(out_rows, sizeof(int64_t) * n_out, true, false, &drows);
    if (S) {
        st.add(S->row_ptr, sizeof(int64_t) * (S->n_brows + 1), true, false, &dsrp);
        st.add(S->col_idx, sizeof(int32_t) * S->nnzb, true, false, &dsci);
        st.add(S->val, sizeof(double) * S->nnzb * bb, true, false, &dsval);
    }
    if (ldos) st.add(ldos, sizeof(double) * n_rhs * n_z, false, true, &dldos);
    if (dm) st.add(dm, sizeof(double) * n_out, false, true, &ddm);
    int rc = st.commit();
    if (rc) return rc;
    void *wsp = nullptr;
    rc = ws_get(ctx, WS_SPMM_STAGE, sizeof(double) * std::max<int64_t>(n_out, 1) + 256, &wsp);
    if (rc) return rc;
    double *wt = (double *)wsp;
    int *missing = (int *)((char *)wsp + align_up(sizeof(double) * std::max<int64_t>(n_out, 1), 128));
    const int g = 152 * 4;
    if (ldos) {
        if (!S) {
            TB_CUDA_TRY(ctx, cudaMemsetAsync(missing, 0, sizeof(int), s));
            k_has_diag<<<g, 256, 0, s>>>((const int64_t *)drhs, n_rhs, (const int64_t *)dptr, (const int64_t *)drows, missing);
            int h_missing = 0;
            TB_CUDA_TRY(ctx, cudaMemcpyAsync(&h_missing, missing, sizeof(int), cudaMemcpyDeviceToHost, s));
            TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            TB_CHECK(ctx, h_missing == 0, TB_ERR_ARG, "S = I: %d columns do not keep their own row", h_missing);
        }
        k_entry_weight<<<g, 256, 0, s>>>((const int64_t *)drhs, n_rhs, (const int64_t *)dptr, (const int64_t *)drows,
                                         (const int64_t *)dsrp, (const int32_t *)dsci, (const double *)dsval,
                                         S ? S->bdim : 1, wt, missing);
        k_ldos<<<g, 256, 0, s>>>((const double *)dG, n_z, (const int64_t *)dptr, n_rhs, wt, (double *)dldos);
    }
    if (dm && n_out)
        k_dm<<<g, 256, sizeof(double) * n_z, s>>>((const double *)dG, n_z, (const double *)dz, (const double *)dw, mu, kT,
                                                  n_out, (double *)ddm);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}
