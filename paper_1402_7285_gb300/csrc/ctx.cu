// Context, status strings and host/device staging.
#include <algorithm>
#include <cstdarg>

#include "common.cuh"

namespace tbgf {

int set_error(tb_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

int ws_get(tb_ctx *ctx, int slot, size_t bytes, void **out) {
    if (slot < 0 || slot >= WS_COUNT) return set_error(ctx, TB_ERR_ARG, "bad workspace slot %d", slot);
    if ((int)ctx->ws_ptr.size() < WS_COUNT) {
        ctx->ws_ptr.resize(WS_COUNT, nullptr);
        ctx->ws_size.resize(WS_COUNT, 0);
    }
    bytes = align_up(bytes < 256 ? 256 : bytes, 256);
    if (ctx->ws_size[slot] < bytes) {
        if (ctx->ws_ptr[slot]) {
            // earlier work may still read the old buffer
            cudaDeviceSynchronize();
            cudaFree(ctx->ws_ptr[slot]);
            ctx->ws_ptr[slot] = nullptr;
            ctx->ws_size[slot] = 0;
        }
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, TB_ERR_ALLOC, "cudaMalloc(%zu) for workspace slot %d: %s", bytes, slot,
                             cudaGetErrorString(e));
        }
        ctx->ws_ptr[slot] = p;
        ctx->ws_size[slot] = bytes;
    }
    *out = ctx->ws_ptr[slot];
    return TB_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void Stager::add(const void *p, size_t bytes, bool is_input, bool is_output, void **dev_out) {
    if (!p || bytes == 0 || is_device_ptr(p)) {
        *dev_out = const_cast<void *>(p);
        return;
    }
    any_host_ = true;
    Item it{p, bytes, total_, is_input, is_output, dev_out};
    total_ = align_up(total_ + bytes, 256);
    items_.push_back(it);
}

int Stager::commit() {
    if (items_.empty()) return TB_OK;
    void *base = nullptr;
    int rc = ws_get(ctx_, slot_, total_, &base);
    if (rc != TB_OK) return rc;
    base_ = (char *)base;
    for (auto &it : items_) {
        *it.dev_out = base_ + it.offset;
        if (it.in)
            TB_CUDA_TRY(ctx_, cudaMemcpyAsync(base_ + it.offset, it.host, it.bytes, cudaMemcpyHostToDevice,
                                              stream_));
    }
    return TB_OK;
}

int Stager::finish() {
    bool any_out = false;
    for (auto &it : items_) {
        if (!it.out) continue;
        any_out = true;
        TB_CUDA_TRY(ctx_, cudaMemcpyAsync(const_cast<void *>(it.host), base_ + it.offset, it.bytes,
                                          cudaMemcpyDeviceToHost, stream_));
    }
    if (any_host_) TB_CUDA_TRY(ctx_, cudaStreamSynchronize(stream_));
    (void)any_out;
    return TB_OK;
}

__global__ void k_validate_bsr(const int64_t *rp, const int32_t *ci, int64_t n_brows, int64_t nnzb, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_brows; a += stride) {
        const int64_t k0 = rp[a], k1 = rp[a + 1];
        if (k0 > k1 || k0 < 0 || k1 > nnzb || (a == 0 && k0 != 0) || (a == n_brows - 1 && k1 != nnzb)) {
            atomicOr(bad, 1);
            continue;
        }
        int64_t prev = -1;
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t c = ci[k];
            if (c < 0 || c >= n_brows || c <= prev) {
                atomicOr(bad, 2);
                break;
            }
            prev = c;
        }
    }
}

int validate_bsr(tb_ctx *ctx, const int64_t *row_ptr, const int32_t *col_idx, const void *val, int64_t n_brows,
                 int64_t nnzb, cudaStream_t s, const char *name) {
    if (((uintptr_t)val & 15u) != 0)
        return set_error(ctx, TB_ERR_ARG, "%s values must be 16-byte aligned", name);
    if (n_brows <= 0 || nnzb < 0) return set_error(ctx, TB_ERR_STRUCTURE, "%s: bad sizes", name);
    int *flag = nullptr;
    TB_CUDA_TRY(ctx, cudaMallocAsync((void **)&flag, sizeof(int), s));
    TB_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s));
    const int g = (int)std::min<int64_t>((n_brows + 255) / 256, 152 * 8);
    k_validate_bsr<<<g < 1 ? 1 : g, 256, 0, s>>>(row_ptr, col_idx, n_brows, nnzb, flag);
    int h = 0;
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    TB_CUDA_TRY(ctx, cudaFreeAsync(flag, s));
    TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h) return set_error(ctx, TB_ERR_STRUCTURE, "%s: malformed BSR structure (code %d)", name, h);
    return TB_OK;
}

} // namespace tbgf

extern "C" {

int tb_ctx_create(tb_ctx **out) {
    if (!out) return TB_ERR_ARG;
    *out = nullptr;
    tb_ctx *c = new (std::nothrow) tb_ctx();
    if (!c) return TB_ERR_ALLOC;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TB_ERR_CUDA;
    }
    c->ws_ptr.assign(tbgf::WS_COUNT, nullptr);
    c->ws_size.assign(tbgf::WS_COUNT, 0);
    *out = c;
    return TB_OK;
}

int tb_ctx_destroy(tb_ctx *ctx) {
    if (!ctx) return TB_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != ctx->device) cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (void *p : ctx->ws_ptr)
        if (p) cudaFree(p);
    if (dev >= 0 && dev != ctx->device) cudaSetDevice(dev);
    delete ctx;
    return TB_OK;
}

const char *tb_status_string(int status) {
    switch (status) {
    case TB_OK: return "ok";
    case TB_ERR_ARG: return "invalid argument";
    case TB_ERR_CUDA: return "CUDA error";
    case TB_ERR_ALLOC: return "allocation failed";
    case TB_ERR_UNSUPPORTED: return "unsupported request";
    case TB_ERR_SIZE: return "size exceeds a limit";
    case TB_ERR_STRUCTURE: return "malformed matrix structure";
    default: break;
    }
    if (status > 0) return "some columns did not converge (see per-column status)";
    return "unknown status";
}

const char *tb_last_error(const tb_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int tb_version(void) { return 10100; }

void tb_solve_opts_default(tb_solve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->max_iter = 100000;
    o->precision = TB_PREC_FP64;
    o->panel_w = 0;
    o->seed_shift = -1;
    o->inner_tol = 0.0;
    o->inner_max = 0;
    o->stream = nullptr;
}

} // extern "C"
