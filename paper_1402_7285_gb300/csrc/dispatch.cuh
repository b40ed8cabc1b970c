// Compile-time variants: value type (FP64 / FP32), block edge B and panel width W.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tbgf {

// Block edges with compiled kernels: 1 (scalar CSR), 4 (s+p) and 9 (s+p+d).
inline bool supported_bdim(int b) { return b == 1 || b == 4 || b == 9; }

// Panel widths with compiled kernels (complex columns).
inline int panel_width_for(int ncols) {
    if (ncols <= 8) return 8;
    if (ncols <= 16) return 16;
    if (ncols <= 32) return 32;
    return 64;
}

template <typename T, int B, class F>
bool dispatch_w(F &f, int W) {
    switch (W) {
    case 8: f.template run<T, B, 8>(); return true;
    case 16: f.template run<T, B, 16>(); return true;
    case 32: f.template run<T, B, 32>(); return true;
    case 64: f.template run<T, B, 64>(); return true;
    }
    return false;
}

template <typename T, class F>
bool dispatch_bw(F &f, int b, int W) {
    switch (b) {
    case 1: return dispatch_w<T, 1>(f, W);
    case 4: return dispatch_w<T, 4>(f, W);
    case 9: return dispatch_w<T, 9>(f, W);
    }
    return false;
}

template <class F>
bool dispatch_tbw(F &f, bool f32, int b, int W) {
    return f32 ? dispatch_bw<float>(f, b, W) : dispatch_bw<double>(f, b, W);
}

void launch_to_float(const double *src, float *dst, int64_t n, cudaStream_t s);
// FP64 matrix values -> the precision's value type (FP32 or df) in dst
void convert_values(int precision, const double *src, void *dst, int64_t n, cudaStream_t s);

} // namespace tbgf
