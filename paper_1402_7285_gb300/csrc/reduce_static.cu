// gf_reduce_ldos_dm_static: gf_reduce_ldos_dm for callers that cannot allocate.
//
// Some callers cannot let a library call cudaMalloc / cudaFree: code that
// runs while another component owns every allocation (a custom or
// pre-reserved device-memory arena, a real-time loop that must not hit the
// implicit device synchronisation of cudaFree, an embedding host that forbids
// allocation after start-up).  This entry point does the same reduction as
// gf_reduce_ldos_dm but allocates nothing: its only scratch (one weight per
// kept entry and four check flags) lives in the file-scope array below, which
// every GPU that loads the library holds until the process exits.
//
// Limits and rules:
//  - at most TB_REDUCE_STATIC_MAX_ENTRIES kept entries (n_out); larger calls
//    return TB_ERR_SIZE before any work is queued;
//  - every array must already be in device memory of the current device (no
//    staging copies);
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current, and caches it; make
//    that first call before any stream capture;
//  - all calls on a device share the one array: calls whose work overlaps on
//    the GPU (different streams, or different host threads) race on it.
//    Calls queued on one stream are ordered and safe.  The flags are cleared
//    by each call before they are used; the weights are rewritten by each call;
//  - every call checks its index arrays on the device first (out_row_ptr
//    starts at 0, is monotone and ends at n_out; rows lie inside S; with
//    S = NULL each column keeps its own row) and synchronises its stream once
//    to read the result; only then are the reduction kernels queued, and
//    every loop over kept entries is also bounded by n_out, so no argument
//    makes them write outside the scratch array or the caller's outputs.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

constexpr double INV_PI_S = 0.318309886183790671537767526745028724;
constexpr int64_t MAX_ENTRIES = TB_REDUCE_STATIC_MAX_ENTRIES;

// scratch: [0, MAX_ENTRIES) entry weights, then the check flags (ints in the
// double slots that follow)
static __device__ __align__(256) double g_reduce_scratch[MAX_ENTRIES + 32];

// check flags (int index into the flag area)
enum { F_PTR = 0, F_ROW = 1, F_MISSING = 2, F_STRUCT = 3, F_COUNT = 4 };

std::mutex g_mutex;
double *g_scratch_ptr[128] = {nullptr};

// device or managed memory that the current device can address as its own
bool on_device(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int scratch_for_current_device(tb_ctx *ctx, double **out) {
    int dev = 0;
    TB_CUDA_TRY(ctx, cudaGetDevice(&dev));
    TB_CHECK(ctx, dev >= 0 && dev < 128, TB_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_reduce_scratch);
        if (e != cudaSuccess)
            return tbgf::set_error(ctx, TB_ERR_CUDA, "cudaGetSymbolAddress(reduce scratch): %s",
                                   cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return TB_OK;
}

__device__ __forceinline__ double fermi_s(double e, double mu, double kT) {
    if (kT == 0.0) return e < mu ? 1.0 : (e > mu ? 0.0 : 0.5);
    const double x = (e - mu) / kT;
    if (x > 0.0) {
        const double ex = exp(-x);
        return ex / (1.0 + ex);
    }
    return 1.0 / (1.0 + exp(x));
}

__global__ void k_flag_clear(int *flag) {
    if (threadIdx.x < F_COUNT) flag[threadIdx.x] = 0;
}

// Index checks, one thread per column: out_row_ptr starts at 0, is monotone and
// ends at n_out; with S, every row and every right-hand side lies inside S;
// with S = NULL, each column keeps its own row.  Reads only entries the
// checked pointers allow (every e stays below n_out).
__global__ void k_check_s(const int64_t *rhs, int64_t n_rhs, const int64_t *optr, const int64_t *orows,
                          int64_t n_out, int64_t n_rows, int has_s, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid == 0 && (optr[0] != 0 || optr[n_rhs] != n_out)) atomicOr(flag + F_PTR, 1);
    for (int64_t c = tid; c < n_rhs; c += stride) {
        const int64_t e0 = optr[c], e1 = optr[c + 1], j = rhs[c];
        if (e0 < 0 || e1 < e0 || e1 > n_out) {
            atomicOr(flag + F_PTR, 1);
            continue;
        }
        if (has_s && (j < 0 || j >= n_rows)) atomicOr(flag + F_ROW, 1);
        bool found = false;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t i = orows[e];
            if (has_s && (i < 0 || i >= n_rows)) atomicOr(flag + F_ROW, 1);
            found |= (i == j);
        }
        if (!has_s && !found) atomicAdd(flag + F_MISSING, 1);
    }
}

__global__ void k_weights_s(const int64_t *rhs, int64_t n_rhs, const int64_t *optr, const int64_t *orows,
                            int64_t n_out, const int64_t *s_rp, const int32_t *s_ci, const double *s_val, int bdim,
                            double *wt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t c = tid; c < n_rhs; c += stride) {
        const int64_t j = rhs[c], aj = j / bdim;
        const int64_t e1 = min(optr[c + 1], n_out);
        for (int64_t e = max(optr[c], (int64_t)0); e < e1; ++e) {
            const int64_t i = orows[e];
            if (!s_rp) {
                wt[e] = (i == j) ? 1.0 : 0.0;
                continue;
            }
            const int64_t ai = i / bdim;
            int64_t k0 = s_rp[ai], k1 = s_rp[ai + 1];
            double v = 0.0;
            while (k0 < k1) {
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
    }
}

__global__ void k_ldos_s(const double *G, int nz, const int64_t *optr, int64_t n_rhs, int64_t n_out,
                         const double *wt, double *ldos) {
    const int64_t total = n_rhs * nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / nz;
        const int m = (int)(t % nz);
        const int64_t e1 = min(optr[c + 1], n_out);
        double s = 0.0;
        for (int64_t e = max(optr[c], (int64_t)0); e < e1; ++e) s += G[(e * nz + m) * 2 + 1] * wt[e];
        ldos[t] = -INV_PI_S * s;
    }
}

__global__ void k_dm_s(const double *G, int nz, const double *z, const double *w, double mu, double kT,
                       int64_t n_out, double *dm) {
    extern __shared__ double occ[];
    for (int m = threadIdx.x; m < nz; m += blockDim.x) occ[m] = w[m] * fermi_s(z[2 * m], mu, kT);
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_out; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int m = 0; m < nz; ++m) s += occ[m] * G[(e * nz + m) * 2 + 1];
        dm[e] = -INV_PI_S * s;
    }
}

} // namespace

extern "C" int gf_reduce_ldos_dm_static(tb_ctx *ctx, const double *G, int32_t n_z, const double *z, const double *w,
                                        double mu, double kT, const int64_t *rhs_rows, int64_t n_rhs,
                                        const int64_t *out_row_ptr, int64_t n_out, const int64_t *out_rows,
                                        const tb_bsr *S, double *ldos, double *dm, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, n_z >= 1 && n_z <= 6144 && n_rhs >= 0 && n_out >= 0, TB_ERR_ARG,
             "gf_reduce_ldos_dm_static: bad sizes");
    TB_CHECK(ctx, n_out <= MAX_ENTRIES, TB_ERR_SIZE,
             "gf_reduce_ldos_dm_static: %lld kept entries exceed the static scratch limit of %lld",
             (long long)n_out, (long long)MAX_ENTRIES);
    TB_CHECK(ctx, kT >= 0.0, TB_ERR_ARG, "kT must be >= 0");
    TB_CHECK(ctx, !dm || w, TB_ERR_ARG, "quadrature weights required for the density matrix");
    if (n_rhs == 0) return TB_OK;
    int dev = 0;
    TB_CUDA_TRY(ctx, cudaGetDevice(&dev));
    const void *need[] = {G, z, rhs_rows, out_row_ptr};
    for (const void *p : need)
        TB_CHECK(ctx, on_device(p, dev), TB_ERR_ARG, "all arrays must be device memory of the current device");
    TB_CHECK(ctx, n_out == 0 || on_device(out_rows, dev), TB_ERR_ARG, "out_rows must be device memory");
    TB_CHECK(ctx, !w || on_device(w, dev), TB_ERR_ARG, "w must be device memory");
    TB_CHECK(ctx, !ldos || on_device(ldos, dev), TB_ERR_ARG, "ldos must be device memory");
    TB_CHECK(ctx, !dm || on_device(dm, dev), TB_ERR_ARG, "dm must be device memory");
    TB_CHECK(ctx, !S || (S->n_brows > 0 && S->bdim >= 1 && S->nnzb >= 0 && on_device(S->row_ptr, dev) &&
                         on_device(S->col_idx, dev) && on_device(S->val, dev)),
             TB_ERR_ARG, "S arrays must be device memory");
    double *scratch = nullptr;
    int rc = scratch_for_current_device(ctx, &scratch);
    if (rc) return rc;
    double *wt = scratch;
    int *flag = reinterpret_cast<int *>(scratch + MAX_ENTRIES);
    cudaStream_t s = (cudaStream_t)stream;
    const int g = 152 * 4;
    // ---- checks of the index arrays, read back before any output is written
    k_flag_clear<<<1, 32, 0, s>>>(flag);
    k_check_s<<<g, 256, 0, s>>>(rhs_rows, n_rhs, out_row_ptr, out_rows, n_out, S ? S->n_brows * S->bdim : 0,
                                S ? 1 : 0, flag);
    if (S) {
        const int gv = (int)std::min<int64_t>((S->n_brows + 255) / 256, 152 * 8);
        k_validate_bsr<<<gv < 1 ? 1 : gv, 256, 0, s>>>(S->row_ptr, S->col_idx, S->n_brows, S->nnzb, flag + F_STRUCT);
    }
    int h[F_COUNT] = {0, 0, 0, 0};
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(h, flag, sizeof(h), cudaMemcpyDeviceToHost, s));
    TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    TB_CHECK(ctx, h[F_PTR] == 0, TB_ERR_SIZE,
             "gf_reduce_ldos_dm_static: out_row_ptr must start at 0, be monotone and end at n_out = %lld",
             (long long)n_out);
    TB_CHECK(ctx, h[F_ROW] == 0, TB_ERR_ARG, "gf_reduce_ldos_dm_static: a row index lies outside S");
    TB_CHECK(ctx, h[F_STRUCT] == 0, TB_ERR_STRUCTURE, "gf_reduce_ldos_dm_static: malformed S (code %d)",
             h[F_STRUCT]);
    TB_CHECK(ctx, !ldos || h[F_MISSING] == 0, TB_ERR_ARG, "S = I: %d columns do not keep their own row",
             h[F_MISSING]);
    // ---- the reduction
    if (ldos) {
        k_weights_s<<<g, 256, 0, s>>>(rhs_rows, n_rhs, out_row_ptr, out_rows, n_out, S ? S->row_ptr : nullptr,
                                      S ? S->col_idx : nullptr, S ? S->val : nullptr, S ? S->bdim : 1, wt);
        k_ldos_s<<<g, 256, 0, s>>>(G, n_z, out_row_ptr, n_rhs, n_out, wt, ldos);
    }
    if (dm && n_out) k_dm_s<<<g, 256, sizeof(double) * n_z, s>>>(G, n_z, z, w, mu, kT, n_out, dm);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return TB_OK;
}
