// gf_reduce_ldos_dm_static: gf_reduce_ldos_dm for callers that cannot allocate.
//
// Some callers cannot let a library call cudaMalloc / cudaFree: code that
// runs while another component owns every allocation (a custom or
// pre-reserved device-memory arena, a real-time loop that must not hit the
// implicit device synchronisation of cudaFree, an embedding host that forbids
// allocation after start-up).  This entry point does the same reduction as
// gf_reduce_ldos_dm but allocates nothing: its only scratch (one weight per
// kept entry and one status flag) lives in the file-scope array below, which
// every GPU that loads the library holds until the process exits.
//
// Limits and rules:
//  - at most TB_REDUCE_STATIC_MAX_ENTRIES kept entries (out_row_ptr[n_rhs]);
//    larger calls return TB_ERR_SIZE before any work is queued;
//  - every array must already be in device memory (no staging copies);
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current, and caches it; make
//    that first call before any stream capture;
//  - all calls on a device share the one array: calls whose work overlaps on
//    the GPU (different streams, or different host threads) race on it.
//    Calls queued on one stream are ordered and safe.  The flag is cleared
//    by each call before it is used; the weights are rewritten by each call;
//  - with S = NULL the call synchronises its stream once, to check that every
//    column keeps its own row (as gf_reduce_ldos_dm does).
#include <mutex>

#include "common.cuh"

namespace {

constexpr double INV_PI_S = 0.318309886183790671537767526745028724;
constexpr int64_t MAX_ENTRIES = TB_REDUCE_STATIC_MAX_ENTRIES;

// scratch: [0, MAX_ENTRIES) entry weights, then one int flag (in a double slot)
static __device__ __align__(256) double g_reduce_scratch[MAX_ENTRIES + 32];

std::mutex g_mutex;
double *g_scratch_ptr[128] = {nullptr};

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

__global__ void k_flag_clear(int *flag) { *flag = 0; }

__global__ void k_weights_s(const int64_t *rhs, int64_t n_rhs, const int64_t *optr, const int64_t *orows,
                            const int64_t *s_rp, const int32_t *s_ci, const double *s_val, int bdim, double *wt,
                            int *missing) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (!s_rp) {
        for (int64_t c = tid; c < n_rhs; c += stride) {
            bool found = false;
            for (int64_t e = optr[c]; e < optr[c + 1]; ++e) {
                const bool d = orows[e] == rhs[c];
                wt[e] = d ? 1.0 : 0.0;
                found |= d;
            }
            if (!found) atomicAdd(missing, 1);
        }
        return;
    }
    for (int64_t c = tid; c < n_rhs; c += stride) {
        const int64_t j = rhs[c], aj = j / bdim;
        for (int64_t e = optr[c]; e < optr[c + 1]; ++e) {
            const int64_t i = orows[e], ai = i / bdim;
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

__global__ void k_ldos_s(const double *G, int nz, const int64_t *optr, int64_t n_rhs, const double *wt,
                         double *ldos) {
    const int64_t total = n_rhs * nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / nz;
        const int m = (int)(t % nz);
        double s = 0.0;
        for (int64_t e = optr[c]; e < optr[c + 1]; ++e) s += G[(e * nz + m) * 2 + 1] * wt[e];
        ldos[t] = -INV_PI_S * s;
    }
}

__global__ void k_dm_s(const double *G, int nz, const double *z, const double *w, double mu, double kT,
                       const int64_t *optr, int64_t n_rhs, double *dm) {
    extern __shared__ double occ[];
    for (int m = threadIdx.x; m < nz; m += blockDim.x) occ[m] = w[m] * fermi_s(z[2 * m], mu, kT);
    __syncthreads();
    const int64_t n_out = optr[n_rhs];
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
    const void *need[] = {G, z, rhs_rows, out_row_ptr};
    for (const void *p : need) TB_CHECK(ctx, is_device_ptr(p), TB_ERR_ARG, "all arrays must be device memory");
    TB_CHECK(ctx, n_out == 0 || is_device_ptr(out_rows), TB_ERR_ARG, "out_rows must be device memory");
    TB_CHECK(ctx, !w || is_device_ptr(w), TB_ERR_ARG, "w must be device memory");
    TB_CHECK(ctx, !ldos || is_device_ptr(ldos), TB_ERR_ARG, "ldos must be device memory");
    TB_CHECK(ctx, !dm || is_device_ptr(dm), TB_ERR_ARG, "dm must be device memory");
    TB_CHECK(ctx, !S || (is_device_ptr(S->row_ptr) && is_device_ptr(S->col_idx) && is_device_ptr(S->val)),
             TB_ERR_ARG, "S arrays must be device memory");
    double *scratch = nullptr;
    int rc = scratch_for_current_device(ctx, &scratch);
    if (rc) return rc;
    double *wt = scratch;
    int *missing = reinterpret_cast<int *>(scratch + MAX_ENTRIES);
    cudaStream_t s = (cudaStream_t)stream;
    const int g = 152 * 4;
    if (ldos) {
        k_flag_clear<<<1, 1, 0, s>>>(missing);
        k_weights_s<<<g, 256, 0, s>>>(rhs_rows, n_rhs, out_row_ptr, out_rows, S ? S->row_ptr : nullptr,
                                      S ? S->col_idx : nullptr, S ? S->val : nullptr, S ? S->bdim : 1, wt, missing);
        if (!S) { // S = I: every column must keep its own row (as gf_reduce_ldos_dm checks)
            int h_missing = 0;
            TB_CUDA_TRY(ctx, cudaMemcpyAsync(&h_missing, missing, sizeof(int), cudaMemcpyDeviceToHost, s));
            TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            TB_CHECK(ctx, h_missing == 0, TB_ERR_ARG, "S = I: %d columns do not keep their own row", h_missing);
        }
        k_ldos_s<<<g, 256, 0, s>>>(G, n_z, out_row_ptr, n_rhs, wt, ldos);
    }
    if (dm && n_out)
        k_dm_s<<<g, 256, sizeof(double) * n_z, s>>>(G, n_z, z, w, mu, kT, out_row_ptr, n_rhs, dm);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return TB_OK;
}
