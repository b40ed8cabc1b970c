// shifted_cocg_solve_local: host driver (kernels in local_impl.cuh).
#include "local_impl.cuh"

namespace tbgf {

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
    TB_CHECK(ctx, opts.precision == TB_PREC_FP64 || opts.precision == TB_PREC_MIXED || opts.precision == TB_PREC_DF64,
             TB_ERR_ARG, "bad precision");
    TB_CHECK(ctx, opts.tol > 0.0 && opts.max_iter >= 0, TB_ERR_ARG, "tol must be > 0 and max_iter >= 0");
    if (opts.stats) opts.stats[0] = opts.stats[1] = opts.stats[2] = opts.stats[3] = 0;
    TB_CHECK(ctx, opts.solver == TB_SOLVER_COCG, TB_ERR_UNSUPPORTED, "the local solver runs gsCOCG only");
    if (n_rhs == 0) return TB_OK;
    cudaStream_t stream = (cudaStream_t)opts.stream;
    const bool mixed = opts.precision == TB_PREC_MIXED;
    const bool lowp = opts.precision != TB_PREC_FP64; // matrix values converted to FP32 or df
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
    // subspace vectors in global memory when they do not fit in shared memory
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t csz = mixed ? 8 : 16;
    const bool vec_global = local_smem(maxa, dmax, max_kept, n_z, has_s, b, csz, true) > (size_t)optin;
    const size_t o_gvec = vec_global ? take(local_vec_bytes(maxa, b, csz, has_s) * grid) : 0;
    const size_t o_zc = take(sizeof(c64) * n_z);
    const size_t o_q = take(sizeof(unsigned long long) * 4);
    const size_t vsz = mixed ? sizeof(float) : sizeof(double);
    const size_t o_h32 = lowp ? take(vsz * H->nnzb * bb) : 0;
    const size_t o_s32 = (lowp && has_s) ? take(vsz * S->nnzb * bb) : 0;
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
    if (lowp) {
        convert_values(opts.precision, (const double *)d_hval, ws + o_h32, H->nnzb * bb, stream);
        hval = ws + o_h32;
        if (has_s) {
            convert_values(opts.precision, (const double *)d_sval, ws + o_s32, S->nnzb * bb, stream);
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
    la.gvec = vec_global ? (void *)(ws + o_gvec) : nullptr;
    la.queue = (unsigned long long *)(ws + o_q);
    la.stat = (unsigned long long *)(ws + o_q) + 1;
    la.tol = opts.tol;
    la.inner_tol = opts.inner_tol > 0.0 ? opts.inner_tol : std::max(1e-3 * opts.tol, mixed ? 1e-7 : (lowp ? 1e-12 : 1e-13));
    la.max_iter = opts.max_iter;
    la.inner_max = opts.inner_max > 0 ? opts.inner_max : 40;
    // seed residual below which df64 no longer carries the harder shifts
    // (restart with a new seed); FP64 converges without, FP32 never gets there
    la.stall2 = opts.precision == TB_PREC_DF64 ? 1e-20 : 0.0;
    la.G = (c64 *)d_G;
    la.iters = (int32_t *)d_iters;
    la.resid = (double *)d_resid;
    la.status = (int32_t *)d_status;
    LocalLaunch L{ctx, la, has_s, grid, stream};
    const bool launched = opts.precision == TB_PREC_FP64    ? launch_local_f64(L, b)
                          : opts.precision == TB_PREC_MIXED ? launch_local_f32(L, b)
                                                            : launch_local_df(L, b);
    if (!launched) return set_error(ctx, TB_ERR_UNSUPPORTED, "no local solver variant");
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
