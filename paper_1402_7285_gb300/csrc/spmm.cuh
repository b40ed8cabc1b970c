// Block-sparse (BSR) product of a real matrix with a complex panel: the one
// sparse product per COCG iteration that every shift shares (Sec. 3, Eq. 2).
//
// Panel layout: [n_rows][W] complex, row-major, (re, im) interleaved; a panel
// row of W complex values is contiguous.  A "team" of W / CPT threads owns one
// block row at a time: lane l holds complex columns l*CPT .. l*CPT+CPT-1, so
// a team reads each neighbour panel row as one coalesced run of vector loads
// (float4 = 2 complex FP32, double2 = 1 complex FP64).  The b x b block values
// are read once per team (broadcast within the team).  Accumulation is in the
// panel's type T.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"

template <typename T>
struct PanelVec;
template <>
struct PanelVec<float> {
    typedef float4 V;
    static constexpr int CPT = 2;
};
template <>
struct PanelVec<double> {
    typedef double2 V;
    static constexpr int CPT = 1;
};
// one complex df (re.hi, re.lo, im.hi, im.lo) per 16-byte vector
template <>
struct PanelVec<df> {
    typedef float4 V;
    static constexpr int CPT = 1;
};

// load / store CPT complex values of one panel row for lane `lane`
template <typename T, int W>
__device__ __forceinline__ void ld_row(const T *__restrict__ base, int64_t row, int lane,
                                       cpx<T> (&x)[PanelVec<T>::CPT]) {
    typedef typename PanelVec<T>::V V;
    const V v = *reinterpret_cast<const V *>(base + (row * W + (int64_t)lane * PanelVec<T>::CPT) * 2);
    if constexpr (std::is_same<T, df>::value) {
        x[0] = mk(df(v.x, v.y), df(v.z, v.w));
    } else if constexpr (PanelVec<T>::CPT == 2) {
        x[0] = mk(v.x, v.y);
        x[1] = mk(v.z, v.w);
    } else {
        x[0] = mk(v.x, v.y);
    }
}

template <typename T, int W>
__device__ __forceinline__ void st_row(T *__restrict__ base, int64_t row, int lane,
                                       const cpx<T> (&x)[PanelVec<T>::CPT]) {
    typedef typename PanelVec<T>::V V;
    V v;
    if constexpr (std::is_same<T, df>::value) {
        v.x = x[0].re.hi, v.y = x[0].re.lo, v.z = x[0].im.hi, v.w = x[0].im.lo;
    } else if constexpr (PanelVec<T>::CPT == 2) {
        v.x = x[0].re, v.y = x[0].im, v.z = x[1].re, v.w = x[1].im;
    } else {
        v.x = x[0].re, v.y = x[0].im;
    }
    *reinterpret_cast<V *>(base + (row * W + (int64_t)lane * PanelVec<T>::CPT) * 2) = v;
}

// Read the B x B block at `blk` into registers (vector loads when aligned).
template <typename T, int B>
__device__ __forceinline__ void ld_block(const T *__restrict__ blk, T (&a)[B * B]) {
    if constexpr (std::is_same<T, df>::value && (B * B * sizeof(T)) % 16 == 0) {
#pragma unroll
        for (int q = 0; q < B * B / 2; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(blk) + q);
            a[2 * q] = df(v.x, v.y), a[2 * q + 1] = df(v.z, v.w);
        }
    } else if constexpr ((B * B * sizeof(T)) % 16 == 0) {
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < B * B / PER; ++q) {
            if constexpr (sizeof(T) == 4) {
                float4 v = __ldg(reinterpret_cast<const float4 *>(blk) + q);
                a[4 * q] = v.x, a[4 * q + 1] = v.y, a[4 * q + 2] = v.z, a[4 * q + 3] = v.w;
            } else {
                double2 v = __ldg(reinterpret_cast<const double2 *>(blk) + q);
                a[2 * q] = v.x, a[2 * q + 1] = v.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < B * B; ++q) a[q] = ldg_val(blk + q);
    }
}

// acc[i][c] = sum over the blocks of block row br of A_blk(i, j) * v(col*B + j)[c],
// where v(row) is produced by the loader functor `ld(row, x)`.  The operand
// type X is T, or float for df matrices times an FP32 panel (the products and
// sums stay df).  unit_row = br declares the diagonal block of this row to be
// the identity (an overlap matrix of orthonormal on-site orbitals): its
// products are replaced by additions of the operand, which gives the same bits
// (products with 1 and 0 are exact, and adding an exact zero changes nothing).
template <typename T, int B, typename X = T, int UNR = 2, class Loader>
__device__ __forceinline__ void bsr_row_product(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                const T *__restrict__ val, int64_t br, Loader &ld,
                                                cpx<T> (&acc)[B][PanelVec<T>::CPT], int64_t unit_row = -1) {
    constexpr int CPT = PanelVec<T>::CPT;
    static_assert(std::is_same<X, T>::value || (std::is_same<T, df>::value && std::is_same<X, float>::value),
                  "operand type");
    const int64_t k0 = __ldg(rp + br), k1 = __ldg(rp + br + 1);
    if constexpr (std::is_same<T, df>::value) {
        DfSum sr[B], si[B];
#pragma unroll
        for (int i = 0; i < B; ++i) sr[i].zero(), si[i].zero();
        int64_t col_n = k0 < k1 ? (int64_t)__ldg(ci + k0) : 0;
#pragma unroll(B <= 4 ? 2 : 1)
        for (int64_t k = k0; k < k1; ++k) {
            // the next block's column is loaded a block ahead, so the operand
            // loads never wait for an index load
            const int64_t col = col_n;
            if (k + 1 < k1) col_n = __ldg(ci + k + 1);
            cpx<X> x[B][CPT];
#pragma unroll
            for (int j = 0; j < B; ++j) ld(col * B + j, x[j]);
            if (col == unit_row) {
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    sr[i].add_val(x[i][0].re);
                    si[i].add_val(x[i][0].im);
                }
            } else {
                T a[B * B];
                ld_block<T, B>(val + k * (int64_t)(B * B), a);
#pragma unroll
                for (int i = 0; i < B; ++i)
#pragma unroll
                    for (int j = 0; j < B; ++j) {
                        sr[i].add_prod(a[i * B + j], x[j][0].re);
                        si[i].add_prod(a[i * B + j], x[j][0].im);
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < B; ++i) acc[i][0] = mk(sr[i].value(), si[i].value());
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[i][c] = mk<T>(0, 0);
        // two blocks per trip keep twice the neighbour loads in flight (small
        // blocks; UNR sets it, 1 where registers are short)
        int64_t col_n = k0 < k1 ? (int64_t)__ldg(ci + k0) : 0;
#pragma unroll(B <= 4 ? UNR : 1)
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t col = col_n;
            if (k + 1 < k1) col_n = __ldg(ci + k + 1);
            cpx<T> x[B][CPT];
#pragma unroll
            for (int j = 0; j < B; ++j) ld(col * B + j, x[j]);
            if (col == unit_row) {
#pragma unroll
                for (int i = 0; i < B; ++i)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        acc[i][c].re = acc[i][c].re + x[i][c].re;
                        acc[i][c].im = acc[i][c].im + x[i][c].im;
                    }
            } else {
                T a[B * B];
                ld_block<T, B>(val + k * (int64_t)(B * B), a);
#pragma unroll
                for (int i = 0; i < B; ++i)
#pragma unroll
                    for (int j = 0; j < B; ++j)
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            acc[i][c].re = fma(a[i * B + j], x[j][c].re, acc[i][c].re);
                            acc[i][c].im = fma(a[i * B + j], x[j][c].im, acc[i][c].im);
                        }
            }
        }
    }
}

// Team geometry for a CTA of NT threads and panel width W.
template <typename T, int W, int NT>
struct Teams {
    static constexpr int CPT = PanelVec<T>::CPT;
    static constexpr int TPR = W / CPT;      // threads per block row
    static constexpr int PER_CTA = NT / TPR; // block rows in flight per CTA
    static_assert(W % CPT == 0, "panel width must be a multiple of the vector width");
    static_assert(NT % TPR == 0, "CTA size must be a multiple of the team size");
};

// Block-row order of the product kernels: groups of PER_CTA consecutive block
// rows (one per team) are dealt to the CTAs in turn, group g to CTA g mod
// grid.  The rows in flight at any moment then form one window that sweeps
// through the matrix, so the neighbour rows its products read (for a lattice
// numbered plane by plane, within a plane or two of the window) are still in
// L2 when the next rows ask for them; contiguous per-CTA ranges would spread
// the front over the whole vector and overflow L2.
