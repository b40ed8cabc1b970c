// Kernels of the panel shifted-COCG solver (generalized shifted COCG, Sec. 3, Eq. 2).
//
// A panel holds W right-hand sides e_j ("slots"), each its own seed COCG in the
// S-bilinear form <u, v> = u^T S v with the same seed shift z_s; the shifted
// systems follow through the collinear residuals r^m = r / pi^m.  Per outer
// iteration n (restated from the shifted-Krylov mathematics; rt = S r is the
// residual of the original equation):
//   A : p_n = r_n + beta_{n-1} p_{n-1};  Sp_n = rt_n + beta_{n-1} Sp_{n-1};
//       Hp_n = H r_n + beta_{n-1} Hp_{n-1} (FP32 panels: H p_n);
//       u = z_s Sp_n - Hp_n;  mu_n = p_n^T u;         (one BSR product with H)
//       per (slot, shift): pi rotation, residual test, p^m_n on the kept rows;
//       last CTA: alpha_n = rho_n / mu_n, column done/breakdown, panel done.
//   B : (S = I) rt_{n+1} = rt_n - alpha_n u; rho_{n+1} = rt^T rt; ||rt||^2;
//       per (slot, shift): pi_{n+1}, alpha^m_n, x^m += alpha^m_n p^m_n;
//       last CTA: beta_n, iteration count, loop condition.
//   B': (S != I) rt_{n+1} = rt_n - alpha_n u; y_0 = r_n - alpha_n u;
//       t_0 = rt_{n+1} - S y_0 (one BSR product with S); shifted updates as B;
//       then the inner CG on S: IC_A (d = t + b d, a = S d, d^H a) and
//       IC_B (y += a d, t -= a a, t^H t), repeated in a device-side loop;
//   C : rho_{n+1} = r_{n+1}^T rt_{n+1}; last CTA as in B.
// All recurrence scalars are FP64.  The loop runs as CUDA-graph conditional
// WHILE nodes whose conditions the last CTA of B / C / IC_B sets; every loop
// has a hard iteration cap, so the device loop always ends.
#pragma once

#include "common.cuh"
#include "spmm.cuh"

namespace tbgf {

struct ColState {
    c64 rho;        // rho_n  = r_n^T rt_n
    c64 alpha;      // alpha_n (0 when the column is done)
    c64 alpha_prev; // alpha_{n-1}
    c64 beta_prev;  // beta_{n-1}
    c64 rho_next;   // rho_{n+1} (between B/C row work and finalize)
    double rn2;     // ||rt_n||^2
    double in_rr;   // inner CG: t^H t
    double in_alpha, in_beta, in_tol2;
    int32_t done, status, iters, n_active, in_done, breakdown;
    int64_t row;    // right-hand side row j (-1: empty slot)
    int64_t dst;    // column index of the solve (-1: empty slot, or results already written)
    int64_t ent0;   // first kept-row entry of the column (index into G's rows)
    int32_t n_ent;  // kept rows of the column
    int32_t fresh;  // 1 from the moment a slot takes a new column until its first iteration ends
    c64 zs;         // this column's seed shift (changes on a restart)
    double chk_w;   // worst active shift residual at the last stagnation check
    int32_t chk_n;  // iteration of that check (-1: none yet)
    int32_t restarts, restart; // restarts so far; 1 while a restart is in flight
    int32_t s_bad;  // the inner CG met a direction with d^H S d <= 0 (S not positive definite)
    // inner solve by refinement (df panels): the true residual t = rt - S y in df,
    // FP32 CG sweeps on S c = t, y += c after each sweep
    int32_t in_sweep;   // 1 while this column's inner solve is still refining
    int32_t in_conv;    // 1 once ||t|| <= inner_tol ||rt|| (or the refinement cap is reached)
    int32_t in_refines; // refinements made in this outer iteration
    int32_t pad_;
    double in_t2;       // ||t||^2 of the true residual at the last refinement
    double in_sig;      // scale of the current FP32 sweep: it solves S c' = t / in_sig
};

// A residual norm usable as a scale (1 when it is zero or not finite).
__host__ __device__ __forceinline__ double safe_scale(double norm2) {
    return (norm2 > 1e-300 && norm2 < 1e300) ? sqrt(norm2) : 1.0;
}

struct ShiftState {
    c64 pi, pi_prev, pi_next; // pi_{n-1}, pi_{n-2}, pi_n at the start of A(n)
    c64 alpha_s;
    double resid;
    int32_t active, conv_it;
    // QMR smoothing (gsQMR): sum over the iterates so far of 1 / omega_k^2, omega_k
    // the quasi-norm sqrt|rho_k| / |pi_k| of the shift's COCG residual, and its
    // first term (the quasi-residual of the zero start)
    double qinv, qinv0;
};

struct Ctrl {
    unsigned int arrive;  // last-CTA arrival counter (reset by the last CTA)
    int32_t n;            // outer iteration of the panel (buffer parity)
    int32_t k;            // inner iteration (buffer parity)
    int32_t panel_done;
    int32_t inner_done;
    int32_t in_ctr;       // inner loop executions in this outer iteration (hard cap)
    int32_t pad0;
    int64_t iter_ctr;     // outer loop executions (hard cap)
    int64_t next_col;     // next column of the queue to load into a slot that retires
    int64_t inner_total;  // inner iterations summed over the panel
    int64_t refine_total; // refinement passes (df panels) summed over the panel
    int32_t refine_now;   // set by the last FP32 sweep step: the next refinement kernel does its work
    int32_t pad32;
    int64_t light_total;  // of those, passes that took S c in FP32
    int64_t pad[1];
};

// Vectors of the inner CG on S that only steer it: its search direction d and
// its starting guess y_0.  With df panels they are FP32 (a perturbation of a
// direction or of a starting guess changes which iterate the inner CG visits,
// not what it converges to: the products S d, the residual t and the solution
// y stay df, and y and t are updated with the same d, so t = rt - S y holds
// to df rounding whatever d is).  FP64 and FP32 panels keep their own type.
template <typename T>
struct DirOf {
    typedef T type;
};
template <>
struct DirOf<df> {
    typedef float type;
};

template <typename T>
struct Panel {
    // matrices (values in T)
    const int64_t *h_rp;
    const int32_t *h_ci;
    const T *h_val;
    const int64_t *s_rp;
    const int32_t *s_ci;
    const T *s_val;
    int32_t s_unit;   // every diagonal block of S is the identity
    int64_t n_brows;
    // panel vectors [n_rows][W] complex T
    T *R[2], *RT, *P[2], *SP, *U, *Tv, *Av;
    T *HP;                         // H p_n by recurrence (FP64 and df panels; null for FP32)
    typename DirOf<T>::type *D[2]; // inner CG directions (FP32 for df panels)
    // inner solve by refinement (df panels with S): FP32 sweep residual, sweep
    // correction and product S d, and an FP32 copy of S's values
    float *T32, *C32, *A32;
    const float *s_val32;
    int32_t ir;          // 1: the inner solve on S runs as FP32 sweeps with df refinement
    int32_t refine_max;  // refinements per outer iteration at most
    double sweep_red;    // an FP32 sweep stops when its residual fell by this factor
    // state
    ColState *col;   // [W]
    ShiftState *sh;  // [W][nz]
    int32_t nz;
    int32_t seed;
    c64 zs;
    const c64 *z;    // [nz]
    // kept rows (projection entries): a region of max_col_ent entries per slot
    c64 *xs, *ps;    // [W][max_col_ent][nz]
    c64 *xq;         // gsQMR: the QMR-smoothed iterates, same layout (null for gsCOCG)
    int32_t qmr;     // 1: gsQMR (results and stopping test from the smoothed iterates)
    // many kept rows (full-vector shifted solutions): the pair steps leave their
    // per-pair coefficients here and k_rows_A / k_rows_B apply them over every
    // (column, kept row, shift), shifts fastest
    int32_t rowpar;
    c64 *coefA;      // [W][nz][2]: 1/pi_n, beta^m_{n-1} (p^m update)
    c64 *coefB;      // [W][nz]: alpha^m_n (x^m update)
    double *etaA;    // [W][nz]: QMR smoothing weight
    int32_t *flagA;  // [W][nz]: bit 0 p^m update, bit 1 smoothing update
    int32_t *flagB;  // [W][nz]: x^m update
    // the column queue (device): columns are loaded into slots in this order
    const int64_t *col_row;     // [n_cols]   right-hand side row j of each column
    const int64_t *col_ptr;     // [n_cols+1] kept-row offsets (rows of G) of each column
    const int64_t *ent_row;     // [col_ptr[n_cols]] kept rows
    int64_t n_cols;
    // reductions
    void *part;      // [W*4][ncta] partials (double or float2)
    Ctrl *ctl;
    cudaGraphConditionalHandle h_outer, h_inner;
    double tol;
    double inner_tol;
    double stall2;    // seed residual^2 below which a stagnating column restarts (0: never)
    int32_t max_iter;
    int32_t inner_max;
    int64_t outer_cap;
    int32_t in_graph; // 1: kernels run inside the solve graph and set its loop conditions
    int32_t max_col_ent; // largest number of kept rows of one column
    // outputs (device)
    c64 *G;
    int32_t *iters;
    double *resid;
    int32_t *status;
    int64_t *stats;  // [4] = (outer iterations, inner iterations, refinements, FP32 refinements)
};

// ---------------------------------------------------------------- accumulators
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s;
    typedef double P;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void add(const Acc &o) { s += o.s; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ P pack() const { return s; }
    __device__ __forceinline__ static Acc unpack(P p) {
        Acc a;
        a.s = p;
        return a;
    }
};
// FP32 two-float (hi + lo) accumulation: TwoSum on every addition, so long
// sums of FP32 terms keep about 48 bits without FP64 instructions.
template <>
struct Acc<float> {
    float hi, lo;
    typedef float2 P;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void add(const Acc &o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ P pack() const { return make_float2(hi, lo); }
    __device__ __forceinline__ static Acc unpack(P p) {
        Acc a;
        a.hi = p.x;
        a.lo = p.y;
        return a;
    }
};

// df values accumulate like FP32 two-float sums (hi by TwoSum, lo added).
template <>
struct Acc<df> {
    float hi, lo;
    typedef float2 P;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void add(df x) {
        add(x.hi);
        lo += x.lo;
    }
    __device__ __forceinline__ void add(const Acc &o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ P pack() const { return make_float2(hi, lo); }
    __device__ __forceinline__ static Acc unpack(P p) {
        Acc a;
        a.hi = p.x;
        a.lo = p.y;
        return a;
    }
};

// Sums per-thread accumulators acc[CPT][K] over the CTA per column and writes
// the CTA partials to part[(c*K + k) * gridDim.x + blockIdx.x].
template <typename T, int W, int NT, int K>
__device__ __forceinline__ void cta_partials(Acc<T> (&acc)[PanelVec<T>::CPT][K], void *part) {
    using TM = Teams<T, W, NT>;
    constexpr int CPT = TM::CPT;
    typedef typename Acc<T>::P P;
    __shared__ P sh[TM::PER_CTA][W * K];
    const int team = threadIdx.x / TM::TPR, lane = threadIdx.x % TM::TPR;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[team][(lane * CPT + cc) * K + k] = acc[cc][k].pack();
    __syncthreads();
    for (int q = threadIdx.x; q < W * K; q += NT) {
        Acc<T> s;
        s.zero();
        for (int t = 0; t < TM::PER_CTA; ++t) s.add(Acc<T>::unpack(sh[t][q]));
        reinterpret_cast<P *>(part)[(int64_t)q * gridDim.x + blockIdx.x] = s.pack();
    }
    __syncthreads();
}

// Warp-wide sum of an accumulator (two-float for FP32: no FP64 instructions).
__device__ __forceinline__ void warp_reduce(Acc<double> &s) { s.s = warp_sum(s.s); }
template <typename A>
__device__ __forceinline__ void warp_reduce_pair(A &s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        A t;
        t.hi = __shfl_xor_sync(TB_FULL_MASK, s.hi, o);
        t.lo = __shfl_xor_sync(TB_FULL_MASK, s.lo, o);
        s.add(t);
    }
}
__device__ __forceinline__ void warp_reduce(Acc<df> &s) { warp_reduce_pair(s); }
__device__ __forceinline__ void warp_reduce(Acc<float> &s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc<float> t;
        t.hi = __shfl_xor_sync(TB_FULL_MASK, s.hi, o);
        t.lo = __shfl_xor_sync(TB_FULL_MASK, s.lo, o);
        s.add(t);
    }
}

// Lane-group sum over R consecutive lanes (R a power of two <= 32), in a fixed order.
__device__ __forceinline__ void group_reduce(Acc<double> &s, int R) {
    for (int o = R / 2; o > 0; o >>= 1) s.s += __shfl_xor_sync(TB_FULL_MASK, s.s, o);
}
template <typename A>
__device__ __forceinline__ void group_reduce(A &s, int R) {
    for (int o = R / 2; o > 0; o >>= 1) {
        A t;
        t.hi = __shfl_xor_sync(TB_FULL_MASK, s.hi, o);
        t.lo = __shfl_xor_sync(TB_FULL_MASK, s.lo, o);
        s.add(t);
    }
}

// In the last CTA: out[q] = sum over CTAs of part[q][*] for q < W*K.  The
// last CTA runs alone, so what counts is how many L2 round trips it waits for:
// RG = NT / (W*K) threads (rounded down to a power of two, at most 32) share a
// row, each keeps RED_U independent loads in flight, and the RG sums of a row
// are combined by shuffles.  The order of the additions depends only on the
// grid and the template arguments, so the sums are reproducible.
template <typename T, int W, int NT, int K>
__device__ __forceinline__ void reduce_partials(const void *part, double *out) {
    typedef typename Acc<T>::P P;
    constexpr int ROWS = W * K;
    constexpr int FIT = NT / ROWS >= 32 ? 32 : (NT / ROWS >= 1 ? NT / ROWS : 1);
    constexpr int RG = FIT >= 16 ? (FIT >= 32 ? 32 : 16) : (FIT >= 8 ? 8 : (FIT >= 4 ? 4 : (FIT >= 2 ? 2 : 1)));
    constexpr int PASS = NT / RG; // rows per pass
    constexpr int RED_U = 16;
    const P *pp = reinterpret_cast<const P *>(part);
    const int G = (int)gridDim.x;
    Acc<T> z;
    z.zero();
    const P zp = z.pack();
    const int sub = threadIdx.x % RG;
    for (int q0 = 0; q0 < ROWS; q0 += PASS) {
        const int q = q0 + (int)threadIdx.x / RG;
        Acc<T> s;
        s.zero();
        if (q < ROWS) {
            const P *row = pp + (int64_t)q * G;
            for (int b0 = sub; b0 < G; b0 += RG * RED_U) {
                P v[RED_U];
#pragma unroll
                for (int u = 0; u < RED_U; ++u) {
                    const int b = b0 + u * RG;
                    v[u] = b < G ? __ldcg(row + b) : zp;
                }
#pragma unroll
                for (int u = 0; u < RED_U; ++u) s.add(Acc<T>::unpack(v[u]));
            }
        }
        group_reduce(s, RG);
        if (sub == 0 && q < ROWS) out[q] = s.value();
    }
    __syncthreads();
}

// Work item index spread round-robin over the CTAs (so small per-pair loops do
// not land on the first few SMs).
__device__ __forceinline__ int64_t spread_index() { return (int64_t)threadIdx.x * gridDim.x + blockIdx.x; }

__device__ __forceinline__ c64 cadd(c64 a, c64 b) { return a + b; }

// ------------------------------------------------------------ loader functors
// x = a(row) + s .* b(row)   (per-column complex scalars s; b may be absent)
template <typename T, int W>
struct LdAxpy {
    const T *a;
    const T *b;
    cpx<T> s[PanelVec<T>::CPT];
    int lane;
    __device__ __forceinline__ void operator()(int64_t row, cpx<T> (&x)[PanelVec<T>::CPT]) const {
        ld_row<T, W>(a, row, lane, x);
        if (b) {
            cpx<T> y[PanelVec<T>::CPT];
            ld_row<T, W>(b, row, lane, y);
#pragma unroll
            for (int c = 0; c < PanelVec<T>::CPT; ++c) x[c] = x[c] + s[c] * y[c];
        }
    }
};


template <typename T>
__device__ __forceinline__ cpx<T> cvt(c64 v) {
    return mk((T)v.re, (T)v.im);
}

// Load / store CPT complex values of a direction panel row (layout of the
// panel type T, element type DirOf<T>: a df panel's directions are one
// float2 per lane).
template <typename T, int W>
__device__ __forceinline__ void ld_dir(const typename DirOf<T>::type *__restrict__ base, int64_t row, int lane,
                                       cpx<typename DirOf<T>::type> (&x)[PanelVec<T>::CPT]) {
    if constexpr (std::is_same<T, df>::value) {
        const float2 v = *reinterpret_cast<const float2 *>(base + (row * W + lane) * 2);
        x[0] = mk(v.x, v.y);
    } else {
        ld_row<T, W>(base, row, lane, x);
    }
}
template <typename T, int W>
__device__ __forceinline__ void st_dir(typename DirOf<T>::type *__restrict__ base, int64_t row, int lane,
                                       const cpx<typename DirOf<T>::type> (&x)[PanelVec<T>::CPT]) {
    if constexpr (std::is_same<T, df>::value) {
        *reinterpret_cast<float2 *>(base + (row * W + lane) * 2) = make_float2(x[0].re, x[0].im);
    } else {
        st_row<T, W>(base, row, lane, x);
    }
}

// a * b and c + a * b with b of the direction type
__device__ __forceinline__ df mul_x(df a, float b) { return mul_f(a, b); }
__device__ __forceinline__ float mul_x(float a, float b) { return a * b; }
__device__ __forceinline__ double mul_x(double a, double b) { return a * b; }
__device__ __forceinline__ df fma_x(df a, float b, df c) { return fma_f(a, b, c); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_x(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ df fma_x(df a, df b, df c) { return fma(a, b, c); }

// Inner CG direction d_k = t_k + beta d_{k-1} (real beta per column; d_{k-1}
// absent at k = 0), formed in the direction type.
template <typename T, int W>
struct LdDir {
    typedef typename DirOf<T>::type X;
    const T *t;
    const X *d;
    X s[PanelVec<T>::CPT];
    int lane;
    __device__ __forceinline__ void operator()(int64_t row, cpx<X> (&x)[PanelVec<T>::CPT]) const {
        constexpr int CPT = PanelVec<T>::CPT;
        if constexpr (std::is_same<T, df>::value) {
            cpx<df> tv[1];
            ld_row<df, W>(t, row, lane, tv);
            x[0] = mk(tv[0].re.hi, tv[0].im.hi);
        } else {
            ld_row<T, W>(t, row, lane, x);
        }
        if (d) {
            cpx<X> y[CPT];
            ld_dir<T, W>(d, row, lane, y);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                x[c].re = fma_x(s[c], y[c].re, x[c].re);
                x[c].im = fma_x(s[c], y[c].im, x[c].im);
            }
        }
    }
};

// An FP32 complex panel read in the team layout of a df panel (one complex per
// lane, float2): the correction of an FP32 sweep as the operand of a df product.
template <int W>
struct LdF32 {
    const float *c;
    int lane;
    __device__ __forceinline__ void operator()(int64_t row, cpx<float> (&x)[1]) const {
        const float2 v = *reinterpret_cast<const float2 *>(c + (row * W + lane) * 2);
        x[0] = mk(v.x, v.y);
    }
};

// Starting guess of the inner CG, y_0 = r_n - alpha_n u (complex alpha per
// column), formed in the direction type; e_j for a column that a slot has just
// taken from the queue (its r_n belongs to the slot's previous column).
template <typename T, int W>
struct LdGuess {
    typedef typename DirOf<T>::type X;
    const T *r;
    const T *u;
    cpx<X> s[PanelVec<T>::CPT]; // -alpha_n
    int64_t fresh_row[PanelVec<T>::CPT]; // row j of a fresh column, -1 otherwise
    int lane;
    __device__ __forceinline__ void operator()(int64_t row, cpx<X> (&x)[PanelVec<T>::CPT]) const {
        constexpr int CPT = PanelVec<T>::CPT;
        guess(row, x);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (fresh_row[c] >= 0) x[c] = mk((X)(row == fresh_row[c] ? 1 : 0), (X)0);
    }
    __device__ __forceinline__ void guess(int64_t row, cpx<X> (&x)[PanelVec<T>::CPT]) const {
        constexpr int CPT = PanelVec<T>::CPT;
        if constexpr (std::is_same<T, df>::value) {
            cpx<df> rv[1], uv[1];
            ld_row<df, W>(r, row, lane, rv);
            ld_row<df, W>(u, row, lane, uv);
            const float ur = uv[0].re.hi, ui = uv[0].im.hi;
            x[0].re = fmaf(s[0].re, ur, fmaf(-s[0].im, ui, rv[0].re.hi));
            x[0].im = fmaf(s[0].re, ui, fmaf(s[0].im, ur, rv[0].im.hi));
        } else {
            cpx<T> uv[CPT];
            ld_row<T, W>(r, row, lane, x);
            ld_row<T, W>(u, row, lane, uv);
#pragma unroll
            for (int c = 0; c < CPT; ++c) x[c] = x[c] + s[c] * uv[c];
        }
    }
};

} // namespace tbgf
