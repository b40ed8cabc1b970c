// tb_bsr_spmm: Y = A X for a real BSR matrix and a complex panel (FP64 or FP32).
#include "spmm.cuh"
#include "dispatch.cuh"

namespace {

template <typename T, int B, int W, int NT>
__device__ __forceinline__ void spmm_rows(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                          const T *__restrict__ val, int64_t n_brows, const T *__restrict__ X,
                                          T *__restrict__ Y) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
    auto ld = [&](int64_t row, cpx<T>(&x)[CPT]) { ld_row<T, W>(X, row, lane, x); };
    const int64_t br_step = (int64_t)gridDim.x * TM::PER_CTA; // groups dealt round-robin
    for (int64_t br = (int64_t)blockIdx.x * TM::PER_CTA + team; br < n_brows; br += br_step) {
        cpx<T> acc[B][CPT];
        bsr_row_product<T, B>(rp, ci, val, br, ld, acc);
#pragma unroll
        for (int i = 0; i < B; ++i) st_row<T, W>(Y, br * B + i, lane, acc[i]);
    }
}

template <typename T, int B, int W, int NT>
__global__ void __launch_bounds__(NT) k_spmm(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                             const T *__restrict__ val, int64_t n_brows, const T *__restrict__ X,
                                             T *__restrict__ Y) {
    spmm_rows<T, B, W, NT>(rp, ci, val, n_brows, X, Y);
}

// FP32 panels: four resident CTAs per SM (64 registers); the product waits on
// L2, so more warps in flight matter more than the few spilled registers.
template <int B, int W, int NT>
__global__ void __launch_bounds__(NT, 4) k_spmm_f32(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                    const float *__restrict__ val, int64_t n_brows,
                                                    const float *__restrict__ X, float *__restrict__ Y) {
    spmm_rows<float, B, W, NT>(rp, ci, val, n_brows, X, Y);
}

// dst[r][0:W] <- src[r][0:ncols] (complex), zero padded; T may be float or double.
template <typename T>
__global__ void k_pad_in(const double *__restrict__ src, int ncols, T *__restrict__ dst, int W, int64_t nrows) {
    const int64_t total = nrows * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / W;
        const int c = (int)(t % W);
        T re = (T)0, im = (T)0;
        if (c < ncols) {
            re = (T)src[(r * ncols + c) * 2];
            im = (T)src[(r * ncols + c) * 2 + 1];
        }
        dst[t * 2] = re;
        dst[t * 2 + 1] = im;
    }
}

template <typename T>
__global__ void k_unpad_out(const T *__restrict__ src, int W, double *__restrict__ dst, int ncols, int64_t nrows) {
    const int64_t total = nrows * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / ncols;
        const int c = (int)(t % ncols);
        dst[t * 2] = (double)src[(r * W + c) * 2];
        dst[t * 2 + 1] = (double)src[(r * W + c) * 2 + 1];
    }
}

__global__ void k_to_float(const double *__restrict__ src, float *__restrict__ dst, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

__global__ void k_to_df(const double *__restrict__ src, df *__restrict__ dst, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = df(src[t]);
}

// x(r, c) = deterministic test values in [-1, 1) (a cheap integer hash)
template <typename T>
__global__ void k_fill_panel(T *__restrict__ x, int64_t n2) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)t * 2654435761u;
        h ^= h >> 15;
        x[t] = (T)((double)(h & 0xffffff) / 8388608.0 - 1.0);
    }
}

struct SpmmLaunch {
    const int64_t *rp;
    const int32_t *ci;
    const void *val;
    int64_t n_brows;
    const void *X;
    void *Y;
    cudaStream_t s;
    int sms;
    template <typename T, int B, int W>
    void run() {
        constexpr int NT = 256;
        using TM = Teams<T, W, NT>;
        int64_t need = (n_brows + TM::PER_CTA - 1) / TM::PER_CTA;
        // FP32: one wave of the four resident CTAs per SM (measured 8 % faster on
        // C2 than two waves); FP64 and df: eight CTAs per SM
        const int64_t grid = (int64_t)sms * (std::is_same<T, float>::value ? 4 : 8);
        int g = (int)(need < grid ? need : grid);
        if (g < 1) g = 1;
        if constexpr (std::is_same<T, float>::value)
            k_spmm_f32<B, W, NT><<<g, NT, 0, s>>>(rp, ci, (const float *)val, n_brows, (const float *)X, (float *)Y);
        else
            k_spmm<T, B, W, NT><<<g, NT, 0, s>>>(rp, ci, (const T *)val, n_brows, (const T *)X, (T *)Y);
    }
};

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

} // namespace

namespace tbgf {
void launch_to_float(const double *src, float *dst, int64_t n, cudaStream_t s) {
    int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (g < 1) g = 1;
    k_to_float<<<g, 256, 0, s>>>(src, dst, n);
}
void launch_to_df(const double *src, void *dst, int64_t n, cudaStream_t s) {
    int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (g < 1) g = 1;
    k_to_df<<<g, 256, 0, s>>>(src, (df *)dst, n);
}
void convert_values(int precision, const double *src, void *dst, int64_t n, cudaStream_t s) {
    if (precision == TB_PREC_MIXED)
        launch_to_float(src, (float *)dst, n, s);
    else if (precision == TB_PREC_DF64)
        launch_to_df(src, dst, n, s);
}
} // namespace tbgf

extern "C" int tb_bsr_spmm(tb_ctx *ctx, const tb_bsr *A, const double *X, int32_t ncols, double *Y,
                           int32_t precision, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, A && A->row_ptr && A->col_idx && A->val, TB_ERR_ARG, "tb_bsr_spmm: matrix arrays missing");
    TB_CHECK(ctx, X && Y && ncols >= 1 && ncols <= 64, TB_ERR_ARG, "tb_bsr_spmm: ncols must be 1..64");
    TB_CHECK(ctx, precision == TB_PREC_FP64 || precision == TB_PREC_MIXED || precision == TB_PREC_DF64, TB_ERR_ARG,
             "bad precision");
    TB_CHECK(ctx, supported_bdim(A->bdim), TB_ERR_UNSUPPORTED, "tb_bsr_spmm: bdim %d not built", A->bdim);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->n_brows * A->bdim;
    const int64_t bb = (int64_t)A->bdim * A->bdim;
    Stager st(ctx, WS_STAGE_IN, s);
    void *rp, *ci, *val, *x, *y;
    st.add(A->row_ptr, sizeof(int64_t) * (A->n_brows + 1), true, false, &rp);
    st.add(A->col_idx, sizeof(int32_t) * A->nnzb, true, false, &ci);
    st.add(A->val, sizeof(double) * A->nnzb * bb, true, false, &val);
    st.add(X, sizeof(double) * 2 * n * ncols, true, false, &x);
    st.add(Y, sizeof(double) * 2 * n * ncols, false, true, &y);
    int rc = st.commit();
    if (rc) return rc;
    rc = validate_bsr(ctx, (const int64_t *)rp, (const int32_t *)ci, val, A->n_brows, A->nnzb, s, "A");
    if (rc) return rc;
    const int W = panel_width_for(ncols);
    const bool f32 = precision == TB_PREC_MIXED, dfp = precision == TB_PREC_DF64;
    const size_t esz = f32 ? 4 : 8;
    size_t off_val = 0, off_x = (f32 || dfp) ? align_up(esz * A->nnzb * bb, 256) : 0;
    size_t off_y = off_x + align_up(esz * 2 * n * W, 256);
    void *wsp;
    rc = ws_get(ctx, WS_SPMM_STAGE, off_y + esz * 2 * n * W, &wsp);
    if (rc) return rc;
    char *ws = (char *)wsp;
    const void *mval = val;
    if (f32 || dfp) {
        convert_values(precision, (const double *)val, ws + off_val, A->nnzb * bb, s);
        mval = ws + off_val;
    }
    int g = (int)std::min<int64_t>((n * W + 255) / 256, 152 * 16);
    if (f32)
        k_pad_in<float><<<g, 256, 0, s>>>((const double *)x, ncols, (float *)(ws + off_x), W, n);
    else if (dfp)
        k_pad_in<df><<<g, 256, 0, s>>>((const double *)x, ncols, (df *)(ws + off_x), W, n);
    else
        k_pad_in<double><<<g, 256, 0, s>>>((const double *)x, ncols, (double *)(ws + off_x), W, n);
    SpmmLaunch L{(const int64_t *)rp, (const int32_t *)ci, mval, A->n_brows, ws + off_x, ws + off_y, s, sm_count()};
    const bool ok = f32 ? dispatch_bw<float>(L, A->bdim, W) : dfp ? dispatch_bw<df>(L, A->bdim, W)
                                                             : dispatch_bw<double>(L, A->bdim, W);
    if (!ok) return set_error(ctx, TB_ERR_UNSUPPORTED, "no SpMM variant");
    if (f32)
        k_unpad_out<float><<<g, 256, 0, s>>>((const float *)(ws + off_y), W, (double *)y, ncols, n);
    else if (dfp)
        k_unpad_out<df><<<g, 256, 0, s>>>((const df *)(ws + off_y), W, (double *)y, ncols, n);
    else
        k_unpad_out<double><<<g, 256, 0, s>>>((const double *)(ws + off_y), W, (double *)y, ncols, n);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}

extern "C" int tb_bsr_spmm_profile(tb_ctx *ctx, const tb_bsr *A, int32_t ncols, int32_t precision, int32_t reps,
                                   void *stream, double *ms_per_launch) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, A && A->row_ptr && A->col_idx && A->val, TB_ERR_ARG, "tb_bsr_spmm_profile: matrix arrays missing");
    TB_CHECK(ctx, ncols >= 1 && ncols <= 64 && reps >= 1 && ms_per_launch, TB_ERR_ARG,
             "tb_bsr_spmm_profile: ncols 1..64, reps >= 1, output required");
    TB_CHECK(ctx, precision == TB_PREC_FP64 || precision == TB_PREC_MIXED || precision == TB_PREC_DF64, TB_ERR_ARG,
             "bad precision");
    TB_CHECK(ctx, supported_bdim(A->bdim), TB_ERR_UNSUPPORTED, "tb_bsr_spmm_profile: bdim %d not built", A->bdim);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->n_brows * A->bdim;
    const int64_t bb = (int64_t)A->bdim * A->bdim;
    Stager st(ctx, WS_STAGE_IN, s);
    void *rp, *ci, *val;
    st.add(A->row_ptr, sizeof(int64_t) * (A->n_brows + 1), true, false, &rp);
    st.add(A->col_idx, sizeof(int32_t) * A->nnzb, true, false, &ci);
    st.add(A->val, sizeof(double) * A->nnzb * bb, true, false, &val);
    int rc = st.commit();
    if (rc) return rc;
    rc = validate_bsr(ctx, (const int64_t *)rp, (const int32_t *)ci, val, A->n_brows, A->nnzb, s, "A");
    if (rc) return rc;
    const int W = panel_width_for(ncols);
    const bool f32 = precision == TB_PREC_MIXED, dfp = precision == TB_PREC_DF64;
    const size_t esz = f32 ? 4 : 8;
    size_t off_val = 0, off_x = (f32 || dfp) ? align_up(esz * A->nnzb * bb, 256) : 0;
    size_t off_y = off_x + align_up(esz * 2 * n * W, 256);
    // a buffer twice the L2 size, written before every timed launch, so no
    // launch finds the previous launch's panel or matrix in L2
    const size_t flush_bytes = (size_t)256 << 20;
    const size_t off_flush = align_up(off_y + esz * 2 * n * W, 256);
    void *wsp;
    rc = ws_get(ctx, WS_SPMM_STAGE, off_flush + flush_bytes, &wsp);
    if (rc) return rc;
    char *ws = (char *)wsp;
    const void *mval = val;
    if (f32 || dfp) {
        convert_values(precision, (const double *)val, ws + off_val, A->nnzb * bb, s);
        mval = ws + off_val;
    }
    const int g = (int)std::min<int64_t>((2 * n * W + 255) / 256, 152 * 16);
    if (f32)
        k_fill_panel<float><<<g, 256, 0, s>>>((float *)(ws + off_x), 2 * n * W);
    else if (dfp)
        k_fill_panel<df><<<g, 256, 0, s>>>((df *)(ws + off_x), 2 * n * W);
    else
        k_fill_panel<double><<<g, 256, 0, s>>>((double *)(ws + off_x), 2 * n * W);
    SpmmLaunch L{(const int64_t *)rp, (const int32_t *)ci, mval, A->n_brows, ws + off_x, ws + off_y, s, sm_count()};
    auto launch = [&]() {
        return f32 ? dispatch_bw<float>(L, A->bdim, W) : dfp ? dispatch_bw<df>(L, A->bdim, W)
                                                         : dispatch_bw<double>(L, A->bdim, W);
    };
    if (!launch()) return set_error(ctx, TB_ERR_UNSUPPORTED, "no SpMM variant");
    cudaEvent_t e0, e1;
    TB_CUDA_TRY(ctx, cudaEventCreate(&e0));
    TB_CUDA_TRY(ctx, cudaEventCreate(&e1));
    double total = 0.0;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaMemsetAsync(ws + off_flush, r & 0xff, flush_bytes, s);
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(ctx, TB_ERR_CUDA, "tb_bsr_spmm_profile: %s", cudaGetErrorString(e));
    *ms_per_launch = total / reps;
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}
