// tb_build_bsr / tb_build_csr: synthetic tight-binding H and S (host, OpenMP).
//
// The matrices have the structure Sec. 8 gives for the LCAO Hamiltonian and
// overlap of Eq. 1 and Eq. 2: real symmetric, S with unit diagonal, off-diagonal
// magnitudes below one and positive definite, M proportional to the atom count.
// Lattices:
//   SC periodic: atom a = x + L (y + L z), six wrapped nearest neighbours.
//   FCC cluster: integer sites (half lattice constant units) with x + y + z
//     even; the n_sites closest to the origin by (r^2, x, y, z); optional
//     vacancies and slab cut; kept atoms numbered in (z, y, x) raster order;
//     neighbours at the twelve (+-1, +-1, 0)-type offsets.
// Random values: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed,
// counter (index lo, index hi, stream, 0); uniform u = 53 high bits of
// (w0 << 32 | w1); normal = sqrt(-2 ln(1 - u_a)) cos(2 pi u_b).  Streams:
// 1 onsite, 2 hopping, 3 overlap, 4 vacancy, 5 slab, 6 substitution.  A pair
// (a, a + d) with d a "positive" direction draws entry (k, l) at index
// (a * n_pos + d) * b^2 + k * b + l; the other atom stores the transpose.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/tbgf.h"

namespace {

struct Philox {
    static inline void mulhilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
        uint64_t p = (uint64_t)a * (uint64_t)b;
        hi = (uint32_t)(p >> 32);
        lo = (uint32_t)p;
    }
    // 10 rounds; ctr[4] in/out, key[2]
    static inline void run(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
        const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
        for (int r = 0; r < 10; ++r) {
            if (r) {
                k0 += W0;
                k1 += W1;
            }
            uint32_t hi0, lo0, hi1, lo1;
            mulhilo(M0, ctr[0], hi0, lo0);
            mulhilo(M1, ctr[2], hi1, lo1);
            uint32_t n0 = hi1 ^ ctr[1] ^ k0, n2 = hi0 ^ ctr[3] ^ k1;
            ctr[0] = n0;
            ctr[1] = lo1;
            ctr[2] = n2;
            ctr[3] = lo0;
        }
    }
};

struct Rng {
    uint64_t seed;
    inline void words(uint32_t stream, uint64_t idx, uint32_t w[4]) const {
        w[0] = (uint32_t)idx;
        w[1] = (uint32_t)(idx >> 32);
        w[2] = stream;
        w[3] = 0;
        Philox::run(w, (uint32_t)seed, (uint32_t)(seed >> 32));
    }
    static inline double u53(uint32_t a, uint32_t b) {
        uint64_t v = (((uint64_t)a << 32) | b) >> 11;
        return (double)v * (1.0 / 9007199254740992.0);
    }
    inline double uniform(uint32_t stream, uint64_t idx) const {
        uint32_t w[4];
        words(stream, idx, w);
        return u53(w[0], w[1]);
    }
    inline double normal(uint32_t stream, uint64_t idx) const {
        uint32_t w[4];
        words(stream, idx, w);
        double ua = u53(w[0], w[1]), ub = u53(w[2], w[3]);
        return std::sqrt(-2.0 * std::log(1.0 - ua)) * std::cos(2.0 * M_PI * ub);
    }
};

enum { ST_ONSITE = 1, ST_HOP = 2, ST_OVERLAP = 3, ST_VACANCY = 4, ST_SLAB = 5, ST_SUBST = 6 };

struct Site {
    int64_t x, y, z;
};

// One stored off-diagonal block: neighbour atom and its pair key.
struct Nb {
    int64_t col;
    int64_t owner;
    int32_t dir;   // -1 for the diagonal block
    int32_t trans; // 1: the stored block is the transpose of the pair's draw
};

struct Structure {
    int64_t n = 0;
    int n_pos = 0;
    std::vector<int64_t> row_ptr;
    std::vector<Nb> nb;
};

const int SC_DIRS[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
const int FCC_DIRS[6][3] = {{1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};

int build_sc(int64_t L, Structure &st) {
    if (L < 3) return TB_ERR_ARG;
    const int64_t n = L * L * L;
    st.n = n;
    st.n_pos = 3;
    st.row_ptr.assign(n + 1, 0);
    st.nb.resize(n * 7);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        int64_t x = a % L, y = (a / L) % L, z = a / (L * L);
        Nb e[7];
        e[0] = Nb{a, a, -1, 0};
        int k = 1;
        for (int d = 0; d < 3; ++d) {
            for (int s = 1; s >= -1; s -= 2) {
                int64_t cx = (x + s * SC_DIRS[d][0] + L) % L, cy = (y + s * SC_DIRS[d][1] + L) % L,
                        cz = (z + s * SC_DIRS[d][2] + L) % L;
                int64_t c = cx + L * (cy + L * cz);
                e[k++] = (s == 1) ? Nb{c, a, d, 0} : Nb{c, c, d, 1};
            }
        }
        std::sort(e, e + 7, [](const Nb &p, const Nb &q) { return p.col < q.col; });
        for (int i = 0; i < 7; ++i) st.nb[a * 7 + i] = e[i];
        st.row_ptr[a + 1] = (a + 1) * 7;
    }
    return TB_OK;
}

int fcc_sites(const tb_system_spec &sp, const Rng &rng, std::vector<Site> &out) {
    const int64_t n = sp.n_sites;
    if (n <= 0) return TB_ERR_ARG;
    int64_t R = (int64_t)std::ceil(std::cbrt(3.0 * (double)n / (2.0 * M_PI))) + 3;
    std::vector<Site> cand;
    for (;;) {
        std::vector<Site> pts;
        for (int64_t x = -R; x <= R; ++x)
            for (int64_t y = -R; y <= R; ++y)
                for (int64_t z = -R; z <= R; ++z)
                    if (((x + y + z) % 2 + 2) % 2 == 0) pts.push_back(Site{x, y, z});
        auto key_less = [](const Site &p, const Site &q) {
            int64_t rp = p.x * p.x + p.y * p.y + p.z * p.z, rq = q.x * q.x + q.y * q.y + q.z * q.z;
            if (rp != rq) return rp < rq;
            if (p.x != q.x) return p.x < q.x;
            if (p.y != q.y) return p.y < q.y;
            return p.z < q.z;
        };
        if ((int64_t)pts.size() >= n) {
            std::nth_element(pts.begin(), pts.begin() + (n - 1), pts.end(), key_less);
            const Site &last = pts[n - 1];
            if (last.x * last.x + last.y * last.y + last.z * last.z < R * R) {
                pts.resize(n);
                cand.swap(pts);
                break;
            }
        }
        R += 4;
    }
    // raster order (z, y, x)
    std::sort(cand.begin(), cand.end(), [](const Site &p, const Site &q) {
        if (p.z != q.z) return p.z < q.z;
        if (p.y != q.y) return p.y < q.y;
        return p.x < q.x;
    });
    int64_t zmin = cand.front().z, zmax = cand.back().z;
    double zcut = 0.0;
    if (sp.slab) zcut = (double)zmin + (double)(zmax - zmin) * (2.0 / 3.0 + rng.uniform(ST_SLAB, 0) / 3.0);
    out.clear();
    out.reserve(cand.size());
    for (int64_t s = 0; s < (int64_t)cand.size(); ++s) {
        if (sp.vacancy_frac > 0.0 && rng.uniform(ST_VACANCY, (uint64_t)s) < sp.vacancy_frac) continue;
        if (sp.slab && (double)cand[s].z > zcut) continue;
        out.push_back(cand[s]);
    }
    return TB_OK;
}

int build_fcc(const std::vector<Site> &sites, Structure &st) {
    const int64_t n = (int64_t)sites.size();
    st.n = n;
    st.n_pos = 6;
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (n) {
        lo[0] = hi[0] = sites[0].x;
        lo[1] = hi[1] = sites[0].y;
        lo[2] = hi[2] = sites[0].z;
    }
    for (const Site &s : sites) {
        lo[0] = std::min(lo[0], s.x), hi[0] = std::max(hi[0], s.x);
        lo[1] = std::min(lo[1], s.y), hi[1] = std::max(hi[1], s.y);
        lo[2] = std::min(lo[2], s.z), hi[2] = std::max(hi[2], s.z);
    }
    // dense grid lookup with a one-site margin
    const int64_t ex = hi[0] - lo[0] + 3, ey = hi[1] - lo[1] + 3, ez = hi[2] - lo[2] + 3;
    std::vector<int64_t> grid((size_t)(ex * ey * ez), -1);
    auto gidx = [&](int64_t x, int64_t y, int64_t z) {
        return ((z - lo[2] + 1) * ey + (y - lo[1] + 1)) * ex + (x - lo[0] + 1);
    };
    for (int64_t a = 0; a < n; ++a) grid[gidx(sites[a].x, sites[a].y, sites[a].z)] = a;
    std::vector<int32_t> cnt(n);
    std::vector<Nb> tmp((size_t)n * 13);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        Nb e[13];
        int k = 0;
        e[k++] = Nb{a, a, -1, 0};
        for (int d = 0; d < 6; ++d) {
            for (int s = 1; s >= -1; s -= 2) {
                int64_t cx = sites[a].x + s * FCC_DIRS[d][0], cy = sites[a].y + s * FCC_DIRS[d][1],
                        cz = sites[a].z + s * FCC_DIRS[d][2];
                int64_t c = grid[gidx(cx, cy, cz)];
                if (c < 0) continue;
                e[k++] = (s == 1) ? Nb{c, a, d, 0} : Nb{c, c, d, 1};
            }
        }
        std::sort(e, e + k, [](const Nb &p, const Nb &q) { return p.col < q.col; });
        for (int i = 0; i < k; ++i) tmp[a * 13 + i] = e[i];
        cnt[a] = k;
    }
    st.row_ptr.assign(n + 1, 0);
    for (int64_t a = 0; a < n; ++a) st.row_ptr[a + 1] = st.row_ptr[a] + cnt[a];
    st.nb.resize(st.row_ptr[n]);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a)
        for (int i = 0; i < cnt[a]; ++i) st.nb[st.row_ptr[a] + i] = tmp[a * 13 + i];
    return TB_OK;
}

// Fill H (overlap == false) or S values for every stored block.
void fill_values(const tb_system_spec &sp, const Structure &st, const Rng &rng, bool overlap, double s_param,
                 double *val) {
    const int b = sp.bdim;
    const int64_t bb = (int64_t)b * b;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < st.n; ++a) {
        for (int64_t k = st.row_ptr[a]; k < st.row_ptr[a + 1]; ++k) {
            const Nb &e = st.nb[k];
            double *blk = val + k * bb;
            if (e.dir < 0) { // onsite block
                std::memset(blk, 0, sizeof(double) * bb);
                if (overlap) {
                    for (int i = 0; i < b; ++i) blk[i * b + i] = 1.0;
                    continue;
                }
                if (sp.onsite_mode == TB_ONSITE_UNIFORM) {
                    double u = rng.uniform(ST_ONSITE, (uint64_t)a);
                    double e0 = sp.onsite_lo + (sp.onsite_hi - sp.onsite_lo) * u;
                    for (int i = 0; i < b; ++i) blk[i * b + i] = e0;
                } else {
                    double N[256];
                    for (int64_t q = 0; q < bb; ++q)
                        N[q] = sp.onsite_sigma * rng.normal(ST_ONSITE, (uint64_t)a * bb + q);
                    for (int i = 0; i < b; ++i)
                        for (int j = 0; j < b; ++j) blk[i * b + j] = 0.5 * (N[i * b + j] + N[j * b + i]);
                    for (int i = 0; i < b; ++i) blk[i * b + i] += sp.onsite_diag[i];
                }
                if (sp.subst_frac > 0.0 && rng.uniform(ST_SUBST, (uint64_t)a) < sp.subst_frac)
                    for (int i = 0; i < b; ++i) blk[i * b + i] += sp.subst_shift;
                continue;
            }
            const bool is_const = overlap ? (sp.s_mode == TB_S_CONST) : (sp.hop_mode == TB_HOP_CONST);
            if (is_const) {
                const double c = overlap ? s_param : sp.hop_t;
                std::memset(blk, 0, sizeof(double) * bb);
                for (int i = 0; i < b; ++i) blk[i * b + i] = c;
                continue;
            }
            const double sigma = overlap ? s_param : sp.hop_sigma;
            const uint32_t stream = overlap ? ST_OVERLAP : ST_HOP;
            const uint64_t base = ((uint64_t)e.owner * (uint64_t)st.n_pos + (uint64_t)e.dir) * (uint64_t)bb;
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j) {
                    // stored block (i, j) is draw (i, j) of the pair, or draw (j, i) when transposed
                    const int q = e.trans ? (j * b + i) : (i * b + j);
                    blk[i * b + j] = sigma * rng.normal(stream, base + q);
                }
        }
    }
}

double gershgorin_offdiag_max(const Structure &st, int b, const double *val) {
    double worst = 0.0;
    const int64_t bb = (int64_t)b * b;
#pragma omp parallel for reduction(max : worst) schedule(static)
    for (int64_t a = 0; a < st.n; ++a) {
        for (int i = 0; i < b; ++i) {
            double s = 0.0;
            for (int64_t k = st.row_ptr[a]; k < st.row_ptr[a + 1]; ++k) {
                const double *blk = val + k * bb + (int64_t)i * b;
                for (int j = 0; j < b; ++j) {
                    bool diag = (st.nb[k].col == a) && (j == i);
                    s += diag ? std::fabs(blk[j] - 1.0) : std::fabs(blk[j]);
                }
            }
            worst = std::max(worst, s);
        }
    }
    return worst;
}

int validate(const tb_system_spec *sp) {
    if (!sp) return TB_ERR_ARG;
    if (sp->bdim < 1 || sp->bdim > 16) return TB_ERR_ARG;
    if (sp->lattice == TB_LATTICE_SC_PERIODIC) {
        if (sp->L < 3) return TB_ERR_ARG;
        if (sp->vacancy_frac != 0.0 || sp->slab) return TB_ERR_ARG;
    } else if (sp->lattice == TB_LATTICE_FCC_CLUSTER) {
        if (sp->n_sites < 1) return TB_ERR_ARG;
    } else {
        return TB_ERR_ARG;
    }
    if (sp->onsite_mode != TB_ONSITE_UNIFORM && sp->onsite_mode != TB_ONSITE_DIAG_NORMAL) return TB_ERR_ARG;
    if (sp->hop_mode != TB_HOP_CONST && sp->hop_mode != TB_HOP_NORMAL) return TB_ERR_ARG;
    if (sp->s_mode != TB_S_IDENTITY && sp->s_mode != TB_S_NORMAL && sp->s_mode != TB_S_CONST) return TB_ERR_ARG;
    if (sp->vacancy_frac < 0.0 || sp->vacancy_frac >= 1.0) return TB_ERR_ARG;
    return TB_OK;
}

int build(const tb_system_spec *sp, uint64_t seed, tb_bsr *H, tb_bsr *S, uint64_t *overlap_seed) {
    int rc = validate(sp);
    if (rc != TB_OK) return rc;
    if (!H) return TB_ERR_ARG;
    const bool want_s = sp->s_mode != TB_S_IDENTITY;
    if (want_s && !S) return TB_ERR_ARG;
    Rng rng{seed};
    Structure st;
    if (sp->lattice == TB_LATTICE_SC_PERIODIC) {
        if ((int64_t)sp->L * sp->L * sp->L > (int64_t)INT32_MAX) return TB_ERR_SIZE;
        rc = build_sc(sp->L, st);
    } else {
        std::vector<Site> sites;
        rc = fcc_sites(*sp, rng, sites);
        if (rc == TB_OK) {
            if ((int64_t)sites.size() > (int64_t)INT32_MAX) return TB_ERR_SIZE;
            rc = build_fcc(sites, st);
        }
    }
    if (rc != TB_OK) return rc;
    const int64_t nnzb = st.row_ptr[st.n];
    const int b = sp->bdim;
    auto fill_header = [&](tb_bsr *M) {
        M->n_brows = st.n;
        M->bdim = b;
        M->nnzb = nnzb;
    };
    const bool sizes_only = (H->row_ptr == nullptr);
    fill_header(H);
    if (want_s) fill_header(S);
    if (sizes_only) return TB_OK;
    if (!H->col_idx || !H->val) return TB_ERR_ARG;
    if (want_s && (!S->row_ptr || !S->col_idx || !S->val)) return TB_ERR_ARG;
    auto fill_structure = [&](tb_bsr *M) {
        std::memcpy(M->row_ptr, st.row_ptr.data(), sizeof(int64_t) * (st.n + 1));
        for (int64_t k = 0; k < nnzb; ++k) M->col_idx[k] = (int32_t)st.nb[k].col;
    };
    fill_structure(H);
    fill_values(*sp, st, rng, false, 0.0, H->val);
    uint64_t s_seed = seed;
    if (want_s) {
        fill_structure(S);
        if (sp->s_mode == TB_S_CONST) {
            fill_values(*sp, st, rng, true, sp->s_param, S->val);
        } else {
            bool ok = false;
            for (int attempt = 0; attempt < 64 && !ok; ++attempt) {
                s_seed = seed + (uint64_t)attempt;
                Rng rs{s_seed};
                fill_values(*sp, st, rs, true, sp->s_param, S->val);
                ok = gershgorin_offdiag_max(st, b, S->val) < 1.0;
            }
            if (!ok) return TB_ERR_ARG;
        }
    }
    if (overlap_seed) *overlap_seed = s_seed;
    return TB_OK;
}

} // namespace

extern "C" {

int tb_build_bsr(const tb_system_spec *spec, uint64_t seed, tb_bsr *H, tb_bsr *S, uint64_t *overlap_seed) {
    return build(spec, seed, H, S, overlap_seed);
}

int tb_build_csr(const tb_system_spec *spec, uint64_t seed, tb_bsr *H, tb_bsr *S, uint64_t *overlap_seed) {
    if (!spec || spec->bdim != 1) return TB_ERR_ARG;
    return build(spec, seed, H, S, overlap_seed);
}

} // extern "C"
