// Iteration-count predictor: MLP 32 -> 64 -> 64 -> 1 (tanh), FP16 weights in
// the forward pass, FP32 accumulation, FP32 master weights updated by Adam
// (Kingma & Ba, 2015), mean squared error loss.  The paper has no learned
// component: this is the project's scheduler model (predicts each column's
// iterations to tolerance so columns can be ordered / binned).
//
// Kernels: per-sample forward (+ backward deltas), per-parameter gradient
// reduction over the minibatch (a fixed summation order: deterministic), Adam.
// Parameter layout (floats): W1[64][32] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int DI = 32, DH = 64;
constexpr int O_W1 = 0, O_B1 = O_W1 + DH * DI, O_W2 = O_B1 + DH, O_B2 = O_W2 + DH * DH, O_W3 = O_B2 + DH,
              O_B3 = O_W3 + DH, NPARAM = O_B3 + 1;
constexpr int FNT = 128;

// Forward (and, with T != nullptr, backward deltas) for samples [s0, s0 + n).
__global__ void __launch_bounds__(FNT) k_mlp_fwd(const __half *__restrict__ w16, const float *__restrict__ X,
                                                 const float *__restrict__ tgt, int64_t s0, int64_t n,
                                                 float inv_batch, float *__restrict__ pred,
                                                 float *__restrict__ H1, float *__restrict__ H2,
                                                 float *__restrict__ DZ1, float *__restrict__ DZ2,
                                                 float *__restrict__ DY, float *__restrict__ sqerr) {
    __shared__ float w[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += FNT) w[i] = __half2float(w16[i]);
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)FNT + threadIdx.x;
    float err2 = 0.f;
    if (t < n) {
        const int64_t s = s0 + t;
        float x[DI], h1[DH], h2[DH];
#pragma unroll
        for (int k = 0; k < DI; ++k) x[k] = X[s * DI + k];
#pragma unroll 4
        for (int i = 0; i < DH; ++i) {
            float acc = w[O_B1 + i];
#pragma unroll
            for (int k = 0; k < DI; ++k) acc = fmaf(w[O_W1 + i * DI + k], x[k], acc);
            h1[i] = tanhf(acc);
        }
        float y = w[O_B3];
#pragma unroll 4
        for (int i = 0; i < DH; ++i) {
            float acc = w[O_B2 + i];
#pragma unroll
            for (int k = 0; k < DH; ++k) acc = fmaf(w[O_W2 + i * DH + k], h1[k], acc);
            h2[i] = tanhf(acc);
            y = fmaf(w[O_W3 + i], h2[i], y);
        }
        if (pred) pred[s] = y;
        if (tgt) {
            const float e = y - tgt[s];
            err2 = e * e;
            if (DZ1) {
                const float dy = 2.f * e * inv_batch;
                DY[t] = dy;
                float dz2[DH];
#pragma unroll
                for (int i = 0; i < DH; ++i) {
                    dz2[i] = dy * w[O_W3 + i] * (1.f - h2[i] * h2[i]);
                    DZ2[t * DH + i] = dz2[i];
                    H2[t * DH + i] = h2[i];
                }
#pragma unroll 4
                for (int k = 0; k < DH; ++k) {
                    float acc = 0.f;
#pragma unroll
                    for (int i = 0; i < DH; ++i) acc = fmaf(w[O_W2 + i * DH + k], dz2[i], acc);
                    DZ1[t * DH + k] = acc * (1.f - h1[k] * h1[k]);
                    H1[t * DH + k] = h1[k];
                }
            }
        }
    }
    if (sqerr) {
        // per-CTA partial of the squared error (FP64 partials, fixed order)
        __shared__ float red[FNT];
        red[threadIdx.x] = err2;
        __syncthreads();
        for (int o = FNT / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) sqerr[blockIdx.x] = red[0];
    }
}

// grad[p] = sum over the n samples of the batch, one thread per parameter.
__global__ void k_mlp_wgrad(const float *__restrict__ X, int64_t s0, int64_t n, const float *__restrict__ H1,
                            const float *__restrict__ H2, const float *__restrict__ DZ1,
                            const float *__restrict__ DZ2, const float *__restrict__ DY, float *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float acc = 0.f;
    if (p < O_B1) {
        const int i = p / DI, k = p % DI;
        for (int64_t t = 0; t < n; ++t) acc = fmaf(DZ1[t * DH + i], X[(s0 + t) * DI + k], acc);
    } else if (p < O_W2) {
        const int i = p - O_B1;
        for (int64_t t = 0; t < n; ++t) acc += DZ1[t * DH + i];
    } else if (p < O_B2) {
        const int q = p - O_W2, i = q / DH, k = q % DH;
        for (int64_t t = 0; t < n; ++t) acc = fmaf(DZ2[t * DH + i], H1[t * DH + k], acc);
    } else if (p < O_W3) {
        const int i = p - O_B2;
        for (int64_t t = 0; t < n; ++t) acc += DZ2[t * DH + i];
    } else if (p < O_B3) {
        const int k = p - O_W3;
        for (int64_t t = 0; t < n; ++t) acc = fmaf(DY[t], H2[t * DH + k], acc);
    } else {
        for (int64_t t = 0; t < n; ++t) acc += DY[t];
    }
    grad[p] = acc;
}

__global__ void k_adam(float *__restrict__ w, __half *__restrict__ w16, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.f - powf(b1, (float)t));
    const float vh = vp / (1.f - powf(b2, (float)t));
    const float wp = w[p] - lr * mh / (sqrtf(vh) + eps);
    w[p] = wp;
    w16[p] = __float2half_rn(wp);
}

__global__ void k_to_half(const float *__restrict__ w, __half *__restrict__ w16) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) w16[p] = __float2half_rn(w[p]);
}

struct MlpWs {
    float *w, *g, *m, *v, *H1, *H2, *DZ1, *DZ2, *DY, *sq;
    __half *w16;
};

int mlp_workspace(tb_ctx *ctx, int64_t batch, int64_t nblk_max, MlpWs &o) {
    using namespace tbgf;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t x = off;
        off = align_up(off + bytes, 256);
        return x;
    };
    const size_t ow = take(4 * NPARAM), og = take(4 * NPARAM), om = take(4 * NPARAM), ov = take(4 * NPARAM);
    const size_t o16 = take(2 * NPARAM);
    const size_t oh1 = take(4 * batch * DH), oh2 = take(4 * batch * DH), odz1 = take(4 * batch * DH),
                 odz2 = take(4 * batch * DH), ody = take(4 * batch), osq = take(4 * nblk_max);
    void *base = nullptr;
    int rc = ws_get(ctx, WS_SPMM_STAGE, off, &base);
    if (rc) return rc;
    char *b = (char *)base;
    o.w = (float *)(b + ow), o.g = (float *)(b + og), o.m = (float *)(b + om), o.v = (float *)(b + ov);
    o.w16 = (__half *)(b + o16);
    o.H1 = (float *)(b + oh1), o.H2 = (float *)(b + oh2), o.DZ1 = (float *)(b + odz1), o.DZ2 = (float *)(b + odz2);
    o.DY = (float *)(b + ody), o.sq = (float *)(b + osq);
    return TB_OK;
}

} // namespace

extern "C" {

int mlp_param_count(void) { return NPARAM; }

int mlp_grad(tb_ctx *ctx, const float *params, const float *X, const float *y, int64_t n, float *grad,
             double *loss, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, params && X && y && grad && n >= 1 && n <= (1 << 24), TB_ERR_ARG, "mlp_grad: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Stager st(ctx, WS_STAGE_IN, s);
    void *dp, *dX, *dy, *dg;
    st.add(params, 4 * NPARAM, true, false, &dp);
    st.add(X, 4 * n * DI, true, false, &dX);
    st.add(y, 4 * n, true, false, &dy);
    st.add(grad, 4 * NPARAM, false, true, &dg);
    int rc = st.commit();
    if (rc) return rc;
    const int64_t nblk = (n + FNT - 1) / FNT;
    MlpWs w;
    rc = mlp_workspace(ctx, n, nblk, w);
    if (rc) return rc;
    k_to_half<<<(NPARAM + 255) / 256, 256, 0, s>>>((const float *)dp, w.w16);
    k_mlp_fwd<<<(int)nblk, FNT, 0, s>>>(w.w16, (const float *)dX, (const float *)dy, 0, n, 1.f / (float)n, nullptr,
                                        w.H1, w.H2, w.DZ1, w.DZ2, w.DY, w.sq);
    k_mlp_wgrad<<<(NPARAM + 127) / 128, 128, 0, s>>>((const float *)dX, 0, n, w.H1, w.H2, w.DZ1, w.DZ2, w.DY,
                                                      (float *)dg);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    if (loss) {
        std::vector<float> sq(nblk);
        TB_CUDA_TRY(ctx, cudaMemcpyAsync(sq.data(), w.sq, 4 * nblk, cudaMemcpyDeviceToHost, s));
        TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        double acc = 0;
        for (float v : sq) acc += v;
        *loss = acc / (double)n;
    }
    return st.finish();
}

int mlp_train(tb_ctx *ctx, const float *X, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
              float *params, double *loss_hist, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, X && y && params && n >= 1 && epochs >= 0 && batch >= 1 && batch <= 65536 && lr > 0.f,
             TB_ERR_ARG, "mlp_train: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Stager st(ctx, WS_STAGE_IN, s);
    void *dX, *dy, *dp;
    st.add(X, 4 * n * DI, true, false, &dX);
    st.add(y, 4 * n, true, false, &dy);
    st.add(params, 4 * NPARAM, true, true, &dp);
    int rc = st.commit();
    if (rc) return rc;
    const int64_t bmax = std::min<int64_t>(batch, n);
    const int64_t nblk = (n + FNT - 1) / FNT;
    MlpWs w;
    rc = mlp_workspace(ctx, bmax, nblk, w);
    if (rc) return rc;
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(w.w, dp, 4 * NPARAM, cudaMemcpyDeviceToDevice, s));
    TB_CUDA_TRY(ctx, cudaMemsetAsync(w.m, 0, 4 * NPARAM, s));
    TB_CUDA_TRY(ctx, cudaMemsetAsync(w.v, 0, 4 * NPARAM, s));
    k_to_half<<<(NPARAM + 255) / 256, 256, 0, s>>>(w.w, w.w16);
    int t = 0;
    std::vector<float> sq(nblk);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t s0 = 0; s0 < n; s0 += bmax) {
            const int64_t nb = std::min<int64_t>(bmax, n - s0);
            k_mlp_fwd<<<(int)((nb + FNT - 1) / FNT), FNT, 0, s>>>(w.w16, (const float *)dX, (const float *)dy, s0, nb,
                                                                 1.f / (float)nb, nullptr, w.H1, w.H2, w.DZ1, w.DZ2,
                                                                 w.DY, nullptr);
            k_mlp_wgrad<<<(NPARAM + 127) / 128, 128, 0, s>>>((const float *)dX, s0, nb, w.H1, w.H2, w.DZ1, w.DZ2,
                                                              w.DY, w.g);
            ++t;
            k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(w.w, w.w16, w.g, w.m, w.v, t, lr, 0.9f, 0.999f, 1e-8f);
        }
        if (loss_hist) {
            k_mlp_fwd<<<(int)nblk, FNT, 0, s>>>(w.w16, (const float *)dX, (const float *)dy, 0, n, 0.f, nullptr,
                                                nullptr, nullptr, nullptr, nullptr, nullptr, w.sq);
            TB_CUDA_TRY(ctx, cudaMemcpyAsync(sq.data(), w.sq, 4 * nblk, cudaMemcpyDeviceToHost, s));
            TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            double acc = 0;
            for (float v : sq) acc += v;
            loss_hist[ep] = acc / (double)n;
        }
    }
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(dp, w.w, 4 * NPARAM, cudaMemcpyDeviceToDevice, s));
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}

int mlp_predict(tb_ctx *ctx, const float *params, const float *X, int64_t n, float *pred, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, params && X && pred && n >= 1, TB_ERR_ARG, "mlp_predict: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Stager st(ctx, WS_STAGE_IN, s);
    void *dp, *dX, *dpred;
    st.add(params, 4 * NPARAM, true, false, &dp);
    st.add(X, 4 * n * DI, true, false, &dX);
    st.add(pred, 4 * n, false, true, &dpred);
    int rc = st.commit();
    if (rc) return rc;
    MlpWs w;
    rc = mlp_workspace(ctx, 1, 1, w);
    if (rc) return rc;
    k_to_half<<<(NPARAM + 255) / 256, 256, 0, s>>>((const float *)dp, w.w16);
    k_mlp_fwd<<<(int)((n + FNT - 1) / FNT), FNT, 0, s>>>(w.w16, (const float *)dX, nullptr, 0, n, 0.f,
                                                        (float *)dpred, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                        nullptr);
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}

} // extern "C"
