// tb_descriptors: 32 local-environment numbers per right-hand side, the input
// of the iteration-count predictor (the paper has no learned component; the
// definition is the project's own and is listed in include/tbgf.h).
//
// One CTA per column: the hop-shell subspace's block structure and two FP64
// vectors live in shared memory; hop distances come from a level-synchronous
// breadth-first search inside the subspace; the spectral moments
// m_k = e_j^T (H_OO - H_jj)^k e_j (k = 2..9) from v_{k+1} = (H_OO - H_jj) v_k
// with m_{2k} = v_k.v_k and m_{2k+1} = v_k.v_{k+1}.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int DNT = 256;
constexpr int NDESC = 32;

__device__ __forceinline__ int find_atom(const int32_t *atoms, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int64_t v = atoms[mid];
        if (v == g) return mid;
        if (v < g) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// CTA sum of one double (FP64: descriptors are a one-off per column)
__device__ __forceinline__ double cta_sum_d(double v, double *scratch) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < DNT / 32; ++w) s += scratch[w];
        scratch[DNT / 32] = s;
    }
    __syncthreads();
    s = scratch[DNT / 32];
    __syncthreads();
    return s;
}

template <int B>
__global__ void __launch_bounds__(DNT) k_desc(const int64_t *__restrict__ h_rp, const int32_t *__restrict__ h_ci,
                                              const double *__restrict__ h_val, const double *__restrict__ s_val,
                                              const int64_t *__restrict__ rhs, const int32_t *__restrict__ radii,
                                              const int64_t *__restrict__ sub_ptr,
                                              const int32_t *__restrict__ sub_atoms, int64_t n, int maxa, int dmax,
                                              float *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int maxr = maxa * B;
    double *v0 = reinterpret_cast<double *>(smem);
    double *v1 = v0 + maxr;
    int32_t *atoms = reinterpret_cast<int32_t *>(v1 + maxr);
    int32_t *nbk = atoms + maxa;
    int16_t *nbl = reinterpret_cast<int16_t *>(nbk + maxa * dmax);
    int16_t *cnt = nbl + maxa * dmax;
    int16_t *dist = cnt + maxa;
    __shared__ double scratch[DNT / 32 + 1];
    __shared__ int s_changed;
    const int tid = threadIdx.x;
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        const int64_t a0 = sub_ptr[c];
        const int nat = (int)(sub_ptr[c + 1] - a0);
        const int64_t j = rhs[c];
        const int R = radii[c];
        for (int l = tid; l < nat; l += DNT) atoms[l] = sub_atoms[a0 + l];
        __syncthreads();
        for (int l = tid; l < nat; l += DNT) {
            const int64_t g = atoms[l];
            int k2 = 0;
            for (int64_t k = h_rp[g]; k < h_rp[g + 1] && k2 < dmax; ++k) {
                const int lc = find_atom(atoms, nat, h_ci[k]);
                if (lc >= 0) {
                    nbl[l * dmax + k2] = (int16_t)lc;
                    nbk[l * dmax + k2] = (int32_t)k;
                    ++k2;
                }
            }
            cnt[l] = (int16_t)k2;
            dist[l] = -1;
        }
        __syncthreads();
        const int la = find_atom(atoms, nat, j / B);
        const int jl = la * B + (int)(j % B);
        if (tid == 0) dist[la] = 0;
        __syncthreads();
        for (int d = 0; d < R; ++d) {
            for (int l = tid; l < nat; l += DNT) {
                if (dist[l] != d) continue;
                for (int s = 0; s < cnt[l]; ++s) {
                    const int lc = nbl[l * dmax + s];
                    if (dist[lc] < 0) dist[lc] = (int16_t)(d + 1); // every writer stores the same value
                }
            }
            __syncthreads();
        }
        const int nrows = nat * B;
        // --- shell counts, surface fraction
        double shell[6] = {0, 0, 0, 0, 0, 0};
        int dmx_local = 0;
        for (int l = tid; l < nat; l += DNT) {
            const int dd = dist[l];
            if (dd >= 1 && dd <= 5) shell[dd] += 1.0;
            dmx_local = max(dmx_local, (int)dd);
        }
        double shells[6];
        for (int s = 1; s <= 5; ++s) shells[s] = cta_sum_d(shell[s], scratch);
        // max hop distance in the subspace = number of levels actually reached
        double dm = cta_sum_d(0.0, scratch); // sync point
        (void)dm;
        if (tid == 0) s_changed = 0;
        __syncthreads();
        atomicMax(&s_changed, dmx_local);
        __syncthreads();
        const int dmax_reached = s_changed;
        double surf = 0.0;
        for (int l = tid; l < nat; l += DNT) surf += (dist[l] == dmax_reached) ? 1.0 : 0.0;
        surf = cta_sum_d(surf, scratch);
        // --- diagonal statistics and row-j sums
        double dsum = 0, dsq = 0, dmin = 1e300, dmaxv = -1e300, hrow = 0, srow = 0, hjj = 0;
        for (int l = tid; l < nrows; l += DNT) {
            const int lat = l / B, i = l % B;
            for (int s = 0; s < cnt[lat]; ++s) {
                const int lc = nbl[lat * dmax + s];
                const int64_t kb = nbk[lat * dmax + s];
                if (lc == lat) {
                    const double h = h_val[kb * B * B + i * B + i];
                    dsum += h;
                    dsq += h * h;
                    dmin = fmin(dmin, h);
                    dmaxv = fmax(dmaxv, h);
                }
                if (l == jl) {
                    for (int q = 0; q < B; ++q) {
                        const int col = lc * B + q;
                        if (col == jl) {
                            hjj = h_val[kb * B * B + i * B + q];
                            continue;
                        }
                        const double h = h_val[kb * B * B + i * B + q];
                        hrow += h * h;
                        if (s_val) {
                            const double sv = s_val[kb * B * B + i * B + q];
                            srow += sv * sv;
                        }
                    }
                }
            }
        }
        const double dmean = cta_sum_d(dsum, scratch) / nrows;
        const double dvar = cta_sum_d(dsq, scratch) / nrows - dmean * dmean;
        hjj = cta_sum_d(hjj, scratch);
        hrow = cta_sum_d(hrow, scratch);
        srow = cta_sum_d(srow, scratch);
        // min / max through warp reductions of the negated / plain values
        double mn = dmin, mx = dmaxv;
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_xor_sync(TB_FULL_MASK, mn, o));
            mx = fmax(mx, __shfl_xor_sync(TB_FULL_MASK, mx, o));
        }
        __shared__ double s_mn[DNT / 32], s_mx[DNT / 32];
        if ((tid & 31) == 0) s_mn[tid >> 5] = mn, s_mx[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < DNT / 32; ++w) s_mn[0] = fmin(s_mn[0], s_mn[w]), s_mx[0] = fmax(s_mx[0], s_mx[w]);
        }
        __syncthreads();
        const double gmin = s_mn[0], gmax = s_mx[0];
        // --- mean Frobenius norm of the in-subspace neighbour blocks of atom a
        double fsum = 0.0, fcnt = 0.0;
        for (int s = tid; s < cnt[la]; s += DNT) {
            const int lc = nbl[la * dmax + s];
            if (lc == la) continue;
            const int64_t kb = nbk[la * dmax + s];
            double f = 0.0;
            for (int q = 0; q < B * B; ++q) f += h_val[kb * B * B + q] * h_val[kb * B * B + q];
            fsum += sqrt(f);
            fcnt += 1.0;
        }
        fsum = cta_sum_d(fsum, scratch);
        fcnt = cta_sum_d(fcnt, scratch);
        // --- spectral moments
        for (int l = tid; l < nrows; l += DNT) v0[l] = (l == jl) ? 1.0 : 0.0;
        __syncthreads();
        double mom[10];
        double *cur = v0, *nxt = v1;
        for (int k = 0; k < 5; ++k) {
            double d1 = 0.0, d2 = 0.0;
            for (int l = tid; l < nrows; l += DNT) {
                const int lat = l / B, i = l % B;
                double y = -hjj * cur[l];
                for (int s = 0; s < cnt[lat]; ++s) {
                    const int lc = nbl[lat * dmax + s];
                    const int64_t kb = nbk[lat * dmax + s];
                    for (int q = 0; q < B; ++q) y = fma(h_val[kb * B * B + i * B + q], cur[lc * B + q], y);
                }
                nxt[l] = y;
                d1 += cur[l] * cur[l];
                d2 += cur[l] * y;
            }
            // v_k . v_k = m_{2k},  v_k . v_{k+1} = m_{2k+1}
            mom[2 * k] = cta_sum_d(d1, scratch);
            mom[2 * k + 1] = cta_sum_d(d2, scratch);
            double *t = cur;
            cur = nxt;
            nxt = t;
        }
        if (tid == 0) {
            float *o = out + c * NDESC;
            for (int q = 0; q < NDESC; ++q) o[q] = 0.f;
            o[0] = (float)(R / 5.0);
            o[1] = (float)(log((double)nat) / log(1000.0));
            for (int s = 1; s <= 5; ++s) o[1 + s] = (float)(shells[s] / 100.0);
            o[7] = (float)((double)(h_rp[j / B + 1] - h_rp[j / B] - 1) / 12.0);
            o[8] = (float)hjj;
            for (int k = 2; k <= 9; ++k) {
                const double m = mom[k];
                o[9 + k - 2] = (float)((m < 0 ? -1.0 : 1.0) * pow(fabs(m), 1.0 / k));
            }
            o[17] = (float)srow;
            o[18] = (float)dmean;
            o[19] = (float)sqrt(fmax(dvar, 0.0));
            o[20] = (float)gmin;
            o[21] = (float)gmax;
            o[22] = (float)hrow;
            o[23] = (float)(fcnt > 0 ? fsum / fcnt : 0.0);
            o[24] = (float)(nrows / 1000.0);
            o[25] = (float)(surf / nat);
        }
        __syncthreads();
    }
}

} // namespace

extern "C" int tb_descriptors(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const int64_t *rhs_rows,
                              const int32_t *radii, int64_t n_rhs, const int64_t *sub_ptr, const int32_t *sub_atoms,
                              float *out, void *stream) {
    using namespace tbgf;
    if (!ctx) return TB_ERR_ARG;
    TB_CHECK(ctx, H && H->row_ptr && H->col_idx && H->val && n_rhs >= 0, TB_ERR_ARG, "tb_descriptors: bad arguments");
    TB_CHECK(ctx, H->bdim == 1 || H->bdim == 4 || H->bdim == 9, TB_ERR_UNSUPPORTED, "bdim %d", H->bdim);
    TB_CHECK(ctx, !S || (S->nnzb == H->nnzb && S->bdim == H->bdim), TB_ERR_ARG, "S must have H's block pattern");
    if (n_rhs == 0) return TB_OK;
    TB_CHECK(ctx, rhs_rows && radii && sub_ptr && sub_atoms && out, TB_ERR_ARG, "tb_descriptors: arrays missing");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = H->bdim;
    std::vector<int64_t> h_sptr(n_rhs + 1), h_rp(H->n_brows + 1), h_rhs(n_rhs);
    std::vector<int32_t> h_rad(n_rhs);
    auto fetch = [&](void *dst, const void *src, size_t bytes) -> int {
        if (is_device_ptr(src)) {
            TB_CUDA_TRY(ctx, cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(dst, src, bytes);
        }
        return TB_OK;
    };
    int rc = fetch(h_sptr.data(), sub_ptr, 8 * (n_rhs + 1));
    if (!rc) rc = fetch(h_rp.data(), H->row_ptr, 8 * (H->n_brows + 1));
    if (!rc) rc = fetch(h_rhs.data(), rhs_rows, 8 * n_rhs);
    if (!rc) rc = fetch(h_rad.data(), radii, 4 * n_rhs);
    if (rc) return rc;
    int maxa = 1, dmax = 1;
    for (int64_t a = 0; a < H->n_brows; ++a) dmax = std::max<int64_t>(dmax, h_rp[a + 1] - h_rp[a]);
    for (int64_t c = 0; c < n_rhs; ++c) {
        const int64_t na = h_sptr[c + 1] - h_sptr[c];
        TB_CHECK(ctx, na >= 1 && na <= 32767 && h_rad[c] >= 0 && h_rad[c] <= 64 && h_rhs[c] >= 0 &&
                          h_rhs[c] < H->n_brows * b,
                 TB_ERR_ARG, "tb_descriptors: column %lld out of range", (long long)c);
        maxa = std::max<int64_t>(maxa, na);
    }
    const int64_t n_sub = h_sptr[n_rhs];
    Stager st(ctx, WS_STAGE_IN, s);
    void *drp, *dci, *dval, *dsval = nullptr, *drhs, *drad, *dsptr, *datoms, *dout;
    const int64_t bb = (int64_t)b * b;
    st.add(H->row_ptr, 8 * (H->n_brows + 1), true, false, &drp);
    st.add(H->col_idx, 4 * H->nnzb, true, false, &dci);
    st.add(H->val, 8 * H->nnzb * bb, true, false, &dval);
    if (S) st.add(S->val, 8 * S->nnzb * bb, true, false, &dsval);
    st.add(rhs_rows, 8 * n_rhs, true, false, &drhs);
    st.add(radii, 4 * n_rhs, true, false, &drad);
    st.add(sub_ptr, 8 * (n_rhs + 1), true, false, &dsptr);
    st.add(sub_atoms, 4 * n_sub, true, false, &datoms);
    st.add(out, 4 * 32 * n_rhs, false, true, &dout);
    rc = st.commit();
    if (rc) return rc;
    rc = validate_bsr(ctx, (const int64_t *)drp, (const int32_t *)dci, dval, H->n_brows, H->nnzb, s, "H");
    if (rc) return rc;
    const size_t sm = (size_t)2 * maxa * b * 8 + (size_t)maxa * 4 + (size_t)maxa * dmax * 6 + (size_t)maxa * 4 + 64;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    TB_CHECK(ctx, sm <= (size_t)optin, TB_ERR_SIZE, "descriptor subspace needs %zu bytes of shared memory", sm);
    const void *fn = b == 1 ? (const void *)k_desc<1> : b == 4 ? (const void *)k_desc<4> : (const void *)k_desc<9>;
    TB_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int grid = (int)std::min<int64_t>(n_rhs, 152 * 4);
#define TB_DESC_ARGS                                                                                          \
    (const int64_t *)drp, (const int32_t *)dci, (const double *)dval, (const double *)dsval, (const int64_t *)drhs, \
        (const int32_t *)drad, (const int64_t *)dsptr, (const int32_t *)datoms, n_rhs, maxa, dmax, (float *)dout
    if (b == 1)
        k_desc<1><<<grid, DNT, sm, s>>>(TB_DESC_ARGS);
    else if (b == 4)
        k_desc<4><<<grid, DNT, sm, s>>>(TB_DESC_ARGS);
    else
        k_desc<9><<<grid, DNT, sm, s>>>(TB_DESC_ARGS);
#undef TB_DESC_ARGS
    TB_CUDA_TRY(ctx, cudaGetLastError());
    return st.finish();
}
