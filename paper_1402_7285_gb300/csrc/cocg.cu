// shifted_cocg_solve / shifted_cocg_profile: host driver of the panel shifted COCG.
#include "cocg_impl.cuh"

namespace tbgf {

__global__ void k_copy_z(const double *z, c64 *zc, int nz) {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) zc[i] = mk(z[2 * i], z[2 * i + 1]);
}

// *not_unit = 1 unless every block row holds a diagonal block equal to the
// identity (the overlap of orthonormal orbitals on one site).
__global__ void k_unit_diag(const int64_t *rp, const int32_t *ci, const double *val, int64_t n_brows, int b,
                            int *not_unit) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t br = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; br < n_brows; br += stride) {
        bool ok = false;
        for (int64_t k = rp[br]; k < rp[br + 1]; ++k) {
            if (ci[k] != br) continue;
            ok = true;
            for (int q = 0; q < b * b; ++q)
                if (val[k * b * b + q] != ((q / b == q % b) ? 1.0 : 0.0)) ok = false;
        }
        if (!ok) atomicOr(not_unit, 1);
    }
}

} // namespace tbgf

// =================================================================== entry points
using namespace tbgf;

namespace {

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

int seed_index(const std::vector<double> &zh, int nz, int requested) {
    if (requested >= 0) return requested;
    std::vector<int> idx(nz);
    for (int i = 0; i < nz; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return zh[2 * a] < zh[2 * b]; });
    return idx[nz / 2];
}

template <typename X>
int fetch_host(tb_ctx *ctx, const X *p, size_t n, std::vector<X> &out) {
    out.resize(n);
    if (n == 0) return TB_OK;
    if (is_device_ptr(p)) {
        TB_CUDA_TRY(ctx, cudaMemcpy(out.data(), p, n * sizeof(X), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), p, n * sizeof(X));
    }
    return TB_OK;
}

// Shared by shifted_cocg_solve (profile_reps == 0) and shifted_cocg_profile.
int run_solver(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
               const int64_t *rhs_rows, int64_t n_rhs, const int64_t *out_row_ptr, const int64_t *out_rows,
               const tb_solve_opts *opts_in, double *G, int32_t *iters, double *resid, int32_t *status,
               int profile_reps, double *ms) {
    if (!ctx) return TB_ERR_ARG;
    tb_solve_opts opts;
    if (opts_in)
        opts = *opts_in;
    else
        tb_solve_opts_default(&opts);
    const bool profiling = profile_reps > 0;
    TB_CHECK(ctx, H && H->row_ptr && H->col_idx && H->val && H->n_brows > 0, TB_ERR_ARG, "H is incomplete");
    TB_CHECK(ctx, supported_bdim(H->bdim), TB_ERR_UNSUPPORTED, "bdim %d has no compiled kernels", H->bdim);
    TB_CHECK(ctx, !S || (S->row_ptr && S->col_idx && S->val && S->n_brows == H->n_brows && S->bdim == H->bdim),
             TB_ERR_ARG, "S does not match H");
    TB_CHECK(ctx, z && n_z >= 1 && n_z <= 4096, TB_ERR_ARG, "n_z must be 1..4096");
    TB_CHECK(ctx, n_rhs >= 0 && (n_rhs == 0 || (rhs_rows && out_row_ptr)), TB_ERR_ARG, "rhs arrays missing");
    TB_CHECK(ctx, opts.precision == TB_PREC_FP64 || opts.precision == TB_PREC_MIXED || opts.precision == TB_PREC_DF64,
             TB_ERR_ARG, "bad precision");
    TB_CHECK(ctx, opts.tol > 0.0 && opts.max_iter >= 0, TB_ERR_ARG, "tol must be > 0 and max_iter >= 0");
    TB_CHECK(ctx, opts.panel_w == 0 || opts.panel_w == 8 || opts.panel_w == 16 || opts.panel_w == 32 ||
                      opts.panel_w == 64,
             TB_ERR_ARG, "panel_w must be 0, 8, 16, 32 or 64");
    TB_CHECK(ctx, opts.seed_shift >= -1 && opts.seed_shift < n_z, TB_ERR_ARG, "seed_shift out of range");
    TB_CHECK(ctx, opts.solver == TB_SOLVER_COCG || opts.solver == TB_SOLVER_QMR, TB_ERR_ARG, "bad solver");
    TB_CHECK(ctx, !profiling || (ms && n_rhs > 0), TB_ERR_ARG, "profile needs right-hand sides and ms[]");
    if (opts.stats) opts.stats[0] = opts.stats[1] = opts.stats[2] = opts.stats[3] = 0;
    if (n_rhs == 0) return TB_OK;
    cudaStream_t stream = (cudaStream_t)opts.stream;
    const bool mixed = opts.precision == TB_PREC_MIXED;
    const bool lowp = opts.precision != TB_PREC_FP64; // matrix values converted to FP32 or df
    const bool has_s = S != nullptr;
    const int b = H->bdim;
    const int64_t n_rows = H->n_brows * b;
    const int64_t bb = (int64_t)b * b;

    // ---- host copies of the index arrays (panel descriptors are built on the host)
    std::vector<int64_t> h_rhs, h_optr, h_orows;
    std::vector<double> h_z;
    int rc = fetch_host(ctx, rhs_rows, n_rhs, h_rhs);
    if (!rc) rc = fetch_host(ctx, out_row_ptr, n_rhs + 1, h_optr);
    if (rc) return rc;
    const int64_t n_out = h_optr[n_rhs];
    TB_CHECK(ctx, h_optr[0] == 0 && n_out >= 0 && (n_out == 0 || out_rows), TB_ERR_ARG, "out_row_ptr must start at 0");
    rc = fetch_host(ctx, out_rows, n_out, h_orows);
    if (!rc) rc = fetch_host(ctx, z, 2 * (size_t)n_z, h_z);
    if (rc) return rc;
    for (int64_t c = 0; c < n_rhs; ++c) {
        TB_CHECK(ctx, h_rhs[c] >= 0 && h_rhs[c] < n_rows, TB_ERR_ARG, "rhs row %lld out of range", (long long)h_rhs[c]);
        TB_CHECK(ctx, h_optr[c + 1] >= h_optr[c], TB_ERR_ARG, "out_row_ptr not monotone");
    }
    for (int64_t e = 0; e < n_out; ++e)
        TB_CHECK(ctx, h_orows[e] >= 0 && h_orows[e] < n_rows, TB_ERR_ARG, "out row out of range");

    // ---- one panel of W slots; the columns form a queue in the given order: a
    // slot whose column finishes takes the next column (refill on the device)
    int W = opts.panel_w;
    if (W == 0) W = panel_width_for((int)std::min<int64_t>(n_rhs, mixed ? 64 : 32));
    int64_t max_col_ent = 1;
    for (int64_t c = 0; c < n_rhs; ++c) max_col_ent = std::max<int64_t>(max_col_ent, h_optr[c + 1] - h_optr[c]);
    TB_CHECK(ctx, max_col_ent < (1 << 24), TB_ERR_SIZE, "too many kept rows in one column");

    // ---- stage caller arrays
    Stager stg(ctx, WS_STAGE_IN, stream);
    void *d_hrp, *d_hci, *d_hval, *d_srp = nullptr, *d_sci = nullptr, *d_sval = nullptr, *d_z;
    void *d_G = nullptr, *d_iters = nullptr, *d_resid = nullptr, *d_status = nullptr;
    stg.add(H->row_ptr, sizeof(int64_t) * (H->n_brows + 1), true, false, &d_hrp);
    stg.add(H->col_idx, sizeof(int32_t) * H->nnzb, true, false, &d_hci);
    stg.add(H->val, sizeof(double) * H->nnzb * bb, true, false, &d_hval);
    if (has_s) {
        stg.add(S->row_ptr, sizeof(int64_t) * (S->n_brows + 1), true, false, &d_srp);
        stg.add(S->col_idx, sizeof(int32_t) * S->nnzb, true, false, &d_sci);
        stg.add(S->val, sizeof(double) * S->nnzb * bb, true, false, &d_sval);
    }
    stg.add(z, sizeof(double) * 2 * n_z, true, false, &d_z);
    if (!profiling) {
        stg.add(G, sizeof(double) * 2 * std::max<int64_t>(n_out, 0) * n_z, false, true, &d_G);
        stg.add(iters, sizeof(int32_t) * n_rhs, false, true, &d_iters);
        stg.add(resid, sizeof(double) * n_rhs * n_z, false, true, &d_resid);
        stg.add(status, sizeof(int32_t) * n_rhs, false, true, &d_status);
    }
    rc = stg.commit();
    if (rc) return rc;
    TB_CHECK(ctx, profiling || (d_G && d_iters && d_resid && d_status), TB_ERR_ARG, "output arrays missing");
    rc = validate_bsr(ctx, (const int64_t *)d_hrp, (const int32_t *)d_hci, d_hval, H->n_brows, H->nnzb, stream, "H");
    if (!rc && has_s)
        rc = validate_bsr(ctx, (const int64_t *)d_srp, (const int32_t *)d_sci, d_sval, S->n_brows, S->nnzb, stream, "S");
    if (rc) return rc;
    int s_unit = 0;
    if (has_s) {
        int *flag = nullptr;
        TB_CUDA_TRY(ctx, cudaMallocAsync((void **)&flag, sizeof(int), stream));
        TB_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(int), stream));
        k_unit_diag<<<num_sms() * 4, 256, 0, stream>>>((const int64_t *)d_srp, (const int32_t *)d_sci,
                                                      (const double *)d_sval, S->n_brows, b, flag);
        int h = 1;
        TB_CUDA_TRY(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        TB_CUDA_TRY(ctx, cudaFreeAsync(flag, stream));
        TB_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        s_unit = h == 0;
    }

    // ---- workspace
    const size_t esz = mixed ? 4 : 8;
    const size_t vec_bytes = align_up(esz * 2 * n_rows * W, 256);
    const int n_vec = (has_s ? 11 : 4) + (mixed ? 0 : 1); // + H p (recurrence) unless FP32
    // df panels with S: the inner solve runs as FP32 sweeps with df refinement
    // (FP32 sweep residual, correction and product: three FP32 vectors)
    const bool ir = has_s && opts.precision == TB_PREC_DF64;
    const size_t vec32_bytes = align_up(sizeof(float) * 2 * n_rows * W, 256);
    const int per_cta = NT / (W / (mixed ? 2 : 1));
    TB_CHECK(ctx, opts.ctas_per_sm >= 0 && opts.ctas_per_sm <= 8, TB_ERR_ARG, "ctas_per_sm must be 0..8");
    const int per_sm = opts.ctas_per_sm > 0 ? opts.ctas_per_sm : 3;
    int ncta = (int)std::min<int64_t>((int64_t)per_sm * num_sms(), (H->n_brows + per_cta - 1) / per_cta);
    if (ncta < 1) ncta = 1;
    // IC_A and C are compiled for four resident CTAs per SM (df panels, block edges <= 4): one more
    // than the other kernels
    int ncta_a = ncta;
    // the FP32 sweep kernels of the refinement: FP32 team geometry (two complex per thread)
    const int per_cta_f = NT / (W / 2);
    const int ncta_f = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * num_sms(),
                                                                   (H->n_brows + per_cta_f - 1) / per_cta_f));
    // (with the refinement, df panels use IC_A only in FP32, and C was measured faster on the
    // common grid: 75.0 against 79.9 us on C2 at W = 64)
    if (b <= 4 && opts.precision == TB_PREC_DF64 && per_sm < 4 && !ir)
        ncta_a = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(per_sm + 1) * num_sms(),
                                                             (H->n_brows + per_cta - 1) / per_cta));
    // the FP32 sweep update IC_B streams five vectors: one CTA per SM fewer than the others
    // (measured 70.9 against 72.5 us on C2 at W = 64)
    const int ncta_fb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, per_sm - 1) * num_sms(),
                                                                    (H->n_brows + per_cta_f - 1) / per_cta_f));
    const int ncta_max = std::max(std::max(ncta, ncta_a), ncta_f);
    void *vec_base = nullptr;
    rc = ws_get(ctx, WS_SOLVE_VEC, vec_bytes * n_vec + (ir ? 3 * vec32_bytes : 0), &vec_base);
    if (rc) return rc;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_col = take(sizeof(ColState) * W);
    const size_t o_sh = take(sizeof(ShiftState) * (size_t)W * n_z);
    const size_t o_ctl = take(sizeof(Ctrl));
    const size_t o_part = take(sizeof(double) * (size_t)W * 4 * ncta_max);
    const size_t o_zc = take(sizeof(c64) * n_z);
    const size_t o_crow = take(sizeof(int64_t) * n_rhs);
    const size_t o_cptr = take(sizeof(int64_t) * (n_rhs + 1));
    const size_t o_erow = take(sizeof(int64_t) * std::max<int64_t>(n_out, 1));
    const size_t o_stats = take(sizeof(int64_t) * 4);
    // many kept rows: the shifted steps' kept-row updates run row-parallel (k_rows_A / k_rows_B)
    const bool rowpar = max_col_ent >= 256;
    const size_t o_coefa = rowpar ? take(sizeof(c64) * 2 * W * n_z) : 0;
    const size_t o_coefb = rowpar ? take(sizeof(c64) * W * n_z) : 0;
    const size_t o_eta = rowpar ? take(sizeof(double) * W * n_z) : 0;
    const size_t o_flaga = rowpar ? take(sizeof(int32_t) * W * n_z) : 0;
    const size_t o_flagb = rowpar ? take(sizeof(int32_t) * W * n_z) : 0;
    const size_t vsz = mixed ? sizeof(float) : sizeof(double);
    const size_t o_h32 = lowp ? take(vsz * H->nnzb * bb) : 0;
    const size_t o_s32 = (lowp && has_s) ? take(vsz * S->nnzb * bb) : 0;
    const size_t o_sf32 = ir ? take(sizeof(float) * S->nnzb * bb) : 0; // FP32 S for the sweeps
    void *small_base = nullptr;
    rc = ws_get(ctx, WS_SOLVE_SMALL, off, &small_base);
    if (rc) return rc;
    char *sb = (char *)small_base;
    void *proj_base = nullptr;
    const int64_t proj_entries = (int64_t)W * max_col_ent * n_z; // one region of max_col_ent rows per slot
    const bool qmr = opts.solver == TB_SOLVER_QMR;
    rc = ws_get(ctx, WS_SOLVE_PROJ, sizeof(c64) * (qmr ? 3 : 2) * proj_entries, &proj_base);
    if (rc) return rc;

    TB_CUDA_TRY(ctx, cudaMemsetAsync(sb + o_ctl, 0, sizeof(Ctrl), stream));
    TB_CUDA_TRY(ctx, cudaMemsetAsync(sb + o_stats, 0, sizeof(int64_t) * 4, stream));
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(sb + o_crow, h_rhs.data(), sizeof(int64_t) * n_rhs, cudaMemcpyHostToDevice, stream));
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(sb + o_cptr, h_optr.data(), sizeof(int64_t) * (n_rhs + 1), cudaMemcpyHostToDevice, stream));
    if (n_out > 0)
        TB_CUDA_TRY(ctx, cudaMemcpyAsync(sb + o_erow, h_orows.data(), sizeof(int64_t) * n_out, cudaMemcpyHostToDevice, stream));
    k_copy_z<<<1, 256, 0, stream>>>((const double *)d_z, (c64 *)(sb + o_zc), n_z);
    const void *hval = d_hval, *sval = d_sval;
    if (lowp) {
        convert_values(opts.precision, (const double *)d_hval, sb + o_h32, H->nnzb * bb, stream);
        hval = sb + o_h32;
        if (has_s) {
            convert_values(opts.precision, (const double *)d_sval, sb + o_s32, S->nnzb * bb, stream);
            sval = sb + o_s32;
            if (ir) convert_values(TB_PREC_MIXED, (const double *)d_sval, sb + o_sf32, S->nnzb * bb, stream);
        }
    }
    TB_CUDA_TRY(ctx, cudaGetLastError());

    // ---- panel parameters
    const int seed = seed_index(h_z, n_z, opts.seed_shift);
    Panel<double> p;
    std::memset(&p, 0, sizeof(p));
    p.h_rp = (const int64_t *)d_hrp;
    p.h_ci = (const int32_t *)d_hci;
    p.h_val = (const double *)hval;
    p.s_rp = (const int64_t *)d_srp;
    p.s_ci = (const int32_t *)d_sci;
    p.s_val = (const double *)sval;
    p.s_unit = s_unit;
    p.n_brows = H->n_brows;
    char *vb = (char *)vec_base;
    int vi = 0;
    auto vec = [&]() { return (double *)(vb + vec_bytes * (vi++)); };
    p.RT = vec();
    p.P[0] = vec();
    p.P[1] = vec();
    p.U = vec();
    p.HP = mixed ? nullptr : vec();
    if (has_s) {
        p.R[0] = vec();
        p.R[1] = vec();
        p.SP = vec();
        p.Tv = vec();
        p.D[0] = vec();
        p.D[1] = vec();
        p.Av = vec();
    }
    if (ir) {
        char *v32 = vb + vec_bytes * vi;
        p.T32 = (float *)v32;
        p.C32 = (float *)(v32 + vec32_bytes);
        p.A32 = (float *)(v32 + 2 * vec32_bytes);
        p.s_val32 = (const float *)(sb + o_sf32);
        p.ir = 1;
    }
    p.col = (ColState *)(sb + o_col);
    p.sh = (ShiftState *)(sb + o_sh);
    p.nz = n_z;
    p.seed = seed;
    p.zs = mk(h_z[2 * seed], h_z[2 * seed + 1]);
    p.z = (const c64 *)(sb + o_zc);
    p.max_col_ent = (int32_t)max_col_ent;
    p.xs = (c64 *)proj_base;
    p.ps = (c64 *)proj_base + proj_entries;
    p.xq = qmr ? (c64 *)proj_base + 2 * proj_entries : nullptr;
    p.qmr = qmr ? 1 : 0;
    if (rowpar) {
        p.rowpar = 1;
        p.coefA = (c64 *)(sb + o_coefa);
        p.coefB = (c64 *)(sb + o_coefb);
        p.etaA = (double *)(sb + o_eta);
        p.flagA = (int32_t *)(sb + o_flaga);
        p.flagB = (int32_t *)(sb + o_flagb);
    }
    p.col_row = (const int64_t *)(sb + o_crow);
    p.col_ptr = (const int64_t *)(sb + o_cptr);
    p.ent_row = (const int64_t *)(sb + o_erow);
    p.n_cols = n_rhs;
    p.part = sb + o_part;
    p.ctl = (Ctrl *)(sb + o_ctl);
    p.tol = opts.tol;
    // df64 restarts (see k_outer); not with gsQMR, whose smoothing runs over one seed's iterates
    p.stall2 = (opts.precision == TB_PREC_DF64 && !qmr) ? 1e-20 : 0.0;
    // inner tolerance: FP64 and FP32 panels 1e-3 tol (floors 1e-13, 1e-7); df panels
    // refine to 1e-5 tol (floor 1e-12): the refinement makes the tighter target cheap,
    // and inexact inner solves are what separates the shifted results from the FP64 ones
    p.inner_tol = opts.inner_tol > 0.0 ? opts.inner_tol
                                       : (ir ? std::max(1e-5 * opts.tol, 1e-12)
                                             : std::max(1e-3 * opts.tol, mixed ? 1e-7 : (lowp ? 1e-12 : 1e-13)));
    p.refine_max = 8;
    p.sweep_red = 1e-5;
    p.max_iter = opts.max_iter;
    p.inner_max = opts.inner_max > 0 ? opts.inner_max : 40;
    // loop executions: while the queue is not empty every slot is busy, so at most
    // n_rhs (max_iter + 2) / W of them, then at most max_iter + 2 for the last columns
    p.outer_cap = (n_rhs * ((int64_t)opts.max_iter + 2) + W - 1) / W + opts.max_iter + 2;
    p.G = (c64 *)d_G;
    p.iters = (int32_t *)d_iters;
    p.resid = (double *)d_resid;
    p.status = (int32_t *)d_status;
    p.stats = (int64_t *)(sb + o_stats);

    SolveLaunch L{ctx, has_s, ncta, n_rows, stream, profile_reps, ms};
    L.pd = p;
    L.ncta_a = ncta_a;
    L.ncta_f = ncta_f;
    L.ncta_fb = ncta_fb;
    const bool launched = opts.precision == TB_PREC_FP64    ? launch_panel_f64(L, b, W)
                          : opts.precision == TB_PREC_MIXED ? launch_panel_f32(L, b, W)
                                                            : launch_panel_df(L, b, W);
    if (!launched) return set_error(ctx, TB_ERR_UNSUPPORTED, "no solver variant for W=%d", W);
    if (L.rc) return L.rc;
    TB_CUDA_TRY(ctx, cudaGetLastError());
    if (profiling) return TB_OK;
    if (opts.stats) {
        TB_CUDA_TRY(ctx, cudaMemcpy(opts.stats, sb + o_stats, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost));
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

// Panel width and CTAs per SM for a solve with panel_w == 0: for large solves,
// time one iteration sequence of the solver's own kernels (profile path) for
// each candidate and keep the lowest estimated time per column; results are
// cached in the context per problem shape.  Small solves use the heuristic.
int autotune(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z, const int64_t *rhs_rows,
             int64_t n_rhs, const int64_t *out_row_ptr, const int64_t *out_rows, const tb_solve_opts &opts,
             int *W_out, int *cps_out) {
    const bool mixed = opts.precision == TB_PREC_MIXED;
    *W_out = panel_width_for((int)std::min<int64_t>(n_rhs, mixed ? 64 : 32));
    *cps_out = opts.ctas_per_sm;
    if (n_rhs < 128) return TB_OK; // tuning would cost more than it saves
    tb_tune_key key{H->n_brows, H->nnzb, std::min<int64_t>(n_rhs, 64), H->bdim, S ? 1 : 0, opts.precision, n_z};
    for (auto &kv : ctx->tuned)
        if (kv.first == key) {
            *W_out = kv.second.first;
            *cps_out = kv.second.second;
            return TB_OK;
        }
    double best = 1e300;
    const int widths[4] = {8, 16, 32, 64};
    const int cpss[2] = {2, 3};
    for (int W : widths) {
        if (W > n_rhs) break;
        for (int cps : cpss) {
            tb_solve_opts o = opts;
            o.panel_w = W;
            o.ctas_per_sm = cps;
            o.stats = nullptr;
            double ms[8] = {0};
            int rc = run_solver(ctx, H, S, z, n_z, rhs_rows, W, out_row_ptr, out_rows, &o, nullptr, nullptr, nullptr,
                                nullptr, 2, ms);
            if (rc < 0) return rc;
            const double inner = S ? 8.0 : 0.0;
            const double per_col = (ms[0] + ms[1] + ms[4] + inner * (ms[2] + ms[3])) / W;
            if (per_col < best) {
                best = per_col;
                *W_out = W;
                *cps_out = cps;
            }
        }
    }
    ctx->tuned.push_back({key, {*W_out, *cps_out}});
    return TB_OK;
}

} // namespace

extern "C" int shifted_cocg_solve(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
                                  const int64_t *rhs_rows, int64_t n_rhs, const int64_t *out_row_ptr,
                                  const int64_t *out_rows, const tb_solve_opts *opts, double *G, int32_t *iters,
                                  double *resid, int32_t *status) {
    if (!ctx) return TB_ERR_ARG;
    tb_solve_opts o;
    if (opts)
        o = *opts;
    else
        tb_solve_opts_default(&o);
    if (o.panel_w == 0 && n_rhs > 0 && H && z && rhs_rows && out_row_ptr) {
        int W = 0, cps = 0;
        int rc = autotune(ctx, H, S, z, n_z, rhs_rows, n_rhs, out_row_ptr, out_rows, o, &W, &cps);
        if (rc < 0) return rc;
        o.panel_w = W;
        o.ctas_per_sm = cps;
    }
    return run_solver(ctx, H, S, z, n_z, rhs_rows, n_rhs, out_row_ptr, out_rows, &o, G, iters, resid, status, 0,
                      nullptr);
}

extern "C" int shifted_cocg_profile(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
                                    const int64_t *rhs_rows, int64_t n_rhs, const int64_t *out_row_ptr,
                                    const int64_t *out_rows, const tb_solve_opts *opts, int32_t reps, double *ms) {
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, reps >= 1 && reps <= 100000, TB_ERR_ARG, "reps must be 1..100000");
    return run_solver(ctx, H, S, z, n_z, rhs_rows, n_rhs, out_row_ptr, out_rows, opts, nullptr, nullptr, nullptr,
                      nullptr, reps, ms);
}
