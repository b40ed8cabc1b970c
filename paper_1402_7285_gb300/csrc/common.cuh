// Shared internals of the tbgf library: complex arithmetic, status handling,
// the context (device workspace, last error) and host/device staging of
// caller arrays.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tbgf.h"

// ------------------------------------------------------------------ complex
template <typename T>
struct cpx {
    T re, im;
};
typedef cpx<double> c64;
typedef cpx<float> c32;

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) {
    cpx<T> z;
    z.re = r;
    z.im = i;
    return z;
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cdiv(cpx<T> a, cpx<T> b) {
    // Smith's algorithm: avoids overflow of |b|^2 for large |b|
    if (fabs(b.re) >= fabs(b.im)) {
        T r = b.im / b.re, d = b.re + b.im * r;
        return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
    } else {
        T r = b.re / b.im, d = b.re * r + b.im;
        return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
    }
}
template <typename T>
__host__ __device__ __forceinline__ T cabs2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ bool cfinite(c64 a) { return isfinite(a.re) && isfinite(a.im); }
__host__ __device__ __forceinline__ c32 to32(c64 a) { return mk((float)a.re, (float)a.im); }
__host__ __device__ __forceinline__ c64 to64(c32 a) { return mk((double)a.re, (double)a.im); }
__host__ __device__ __forceinline__ c64 to64(c64 a) { return a; }

// ------------------------------------------------------------------ status
struct tb_tune_key {
    int64_t n_brows, nnzb, n_rhs_cap;
    int32_t bdim, has_s, precision, n_z;
    bool operator==(const tb_tune_key &o) const {
        return n_brows == o.n_brows && nnzb == o.nnzb && n_rhs_cap == o.n_rhs_cap && bdim == o.bdim &&
               has_s == o.has_s && precision == o.precision && n_z == o.n_z;
    }
};

struct tb_ctx {
    int device = 0;
    std::string last_error;
    // autotuned (panel width, CTAs per SM) per problem shape
    std::vector<std::pair<tb_tune_key, std::pair<int, int>>> tuned;
    // grow-only device workspace slots owned by the context
    std::vector<void *> ws_ptr;
    std::vector<size_t> ws_size;
};

namespace tbgf {

int set_error(tb_ctx *ctx, int code, const char *fmt, ...);

#define TB_CUDA_TRY(ctx, call)                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return ::tbgf::set_error((ctx), TB_ERR_CUDA, "%s failed: %s (%s:%d)", #call,          \
                                     cudaGetErrorString(e_), __FILE__, __LINE__);                \
    } while (0)

#define TB_CHECK(ctx, cond, code, ...)                                                           \
    do {                                                                                         \
        if (!(cond)) return ::tbgf::set_error((ctx), (code), __VA_ARGS__);                       \
    } while (0)

// Device workspace slot `slot` of at least `bytes` (grow-only, owned by ctx).
int ws_get(tb_ctx *ctx, int slot, size_t bytes, void **out);

enum WsSlot {
    WS_SPMM_STAGE = 0,  // staging for tb_bsr_spmm
    WS_SOLVE_VEC = 1,   // panel vectors of the solver
    WS_SOLVE_SMALL = 2, // per-column / per-shift state, partials, control
    WS_SOLVE_PROJ = 3,  // projected solutions
    WS_STAGE_IN = 4,    // staged host inputs
    WS_STAGE_OUT = 5,   // staged host outputs
    WS_MATRIX32 = 6,    // FP32 copies of matrix values (mixed precision)
    WS_REDUCE = 7,      // gf_reduce staging
    WS_COUNT = 8
};

bool is_device_ptr(const void *p);

// Stages a list of caller arrays into one device buffer when they are in
// host memory.  Inputs are copied at add(); outputs are copied back by finish().
class Stager {
  public:
    Stager(tb_ctx *ctx, int slot, cudaStream_t s) : ctx_(ctx), slot_(slot), stream_(s) {}
    // Registers an array; returns its device address (the caller's own pointer
    // when it already is device memory).  Must be called for all arrays before
    // commit(); addresses are final only after commit().
    void add(const void *p, size_t bytes, bool is_input, bool is_output, void **dev_out);
    int commit();
    int finish(); // copies outputs back; synchronises if any output is host memory
    bool any_host() const { return any_host_; }

  private:
    struct Item {
        const void *host;
        size_t bytes, offset;
        bool in, out;
        void **dev_out;
    };
    tb_ctx *ctx_;
    int slot_;
    cudaStream_t stream_;
    std::vector<Item> items_;
    size_t total_ = 0;
    bool any_host_ = false;
    char *base_ = nullptr;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Checks a device BSR structure (row_ptr monotone from 0 to nnzb, col_idx in
// range and ascending within each block row) and the 16-byte alignment of its
// values; returns TB_OK or TB_ERR_STRUCTURE / TB_ERR_ARG.  Synchronises `s`.
// Structure check of validate_bsr as a kernel: ORs 1 into *bad for a bad
// row pointer, 2 for a column index out of range or out of order.
__global__ void k_validate_bsr(const int64_t *rp, const int32_t *ci, int64_t n_brows, int64_t nnzb, int *bad);

int validate_bsr(tb_ctx *ctx, const int64_t *row_ptr, const int32_t *col_idx, const void *val, int64_t n_brows,
                 int64_t nnzb, cudaStream_t s, const char *name);

} // namespace tbgf

// ------------------------------------------------- device helpers (reductions)
#define TB_FULL_MASK 0xffffffffu

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(TB_FULL_MASK, v, o);
    return v;
}

// True in every thread of the CTA that arrives last at `counter` (which it
// resets to zero for the next launch).  Uses one int of shared memory.
__device__ __forceinline__ bool last_cta_arrival(unsigned int *counter) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}
