// tb_local_subspaces: hop-shell local subspaces of right-hand-side atoms (host, OpenMP).
//
// Sec. 2 rests order-N on locality: the Green's-function column of an atom is
// computed on the atoms near it.  The subspace of radius R around the atom of
// row j holds every atom within R hops of it in the nearest-neighbour graph
// (the block pattern of H without its diagonal); its rows are all orbitals of
// those atoms.  Output per column: the atoms, ascending.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/tbgf.h"

namespace {

// Breadth-first search to depth `radius`; `mark` is a per-thread scratch array
// (all -1 on entry and on exit).
void bfs(const int64_t *rp, const int32_t *ci, int64_t start, int radius, std::vector<int32_t> &mark,
         std::vector<int64_t> &out) {
    out.clear();
    out.push_back(start);
    mark[start] = 0;
    size_t head = 0;
    while (head < out.size()) {
        const int64_t a = out[head++];
        const int d = mark[a];
        if (d >= radius) continue;
        for (int64_t k = rp[a]; k < rp[a + 1]; ++k) {
            const int64_t c = ci[k];
            if (c == a || mark[c] >= 0) continue;
            mark[c] = d + 1;
            out.push_back(c);
        }
    }
    for (int64_t a : out) mark[a] = -1;
    std::sort(out.begin(), out.end());
}

} // namespace

extern "C" int tb_local_subspaces(const tb_bsr *A, const int64_t *rhs_rows, const int32_t *radii, int64_t n_rhs,
                                  int64_t *sub_ptr, int32_t *sub_atoms) {
    if (!A || !A->row_ptr || !A->col_idx || A->n_brows <= 0 || A->bdim < 1 || n_rhs < 0 || !sub_ptr) return TB_ERR_ARG;
    if (n_rhs > 0 && (!rhs_rows || !radii)) return TB_ERR_ARG;
    const int64_t n = A->n_brows, b = A->bdim;
    for (int64_t c = 0; c < n_rhs; ++c)
        if (rhs_rows[c] < 0 || rhs_rows[c] >= n * b || radii[c] < 0 || radii[c] > 64) return TB_ERR_ARG;
    for (int64_t a = 0; a < n; ++a)
        if (A->row_ptr[a + 1] < A->row_ptr[a]) return TB_ERR_STRUCTURE;
    for (int64_t k = 0; k < A->row_ptr[n]; ++k)
        if (A->col_idx[k] < 0 || A->col_idx[k] >= n) return TB_ERR_STRUCTURE;
    std::vector<int64_t> counts(n_rhs);
    int err = 0;
#pragma omp parallel
    {
        std::vector<int32_t> mark(n, -1);
        std::vector<int64_t> atoms;
#pragma omp for schedule(dynamic, 64)
        for (int64_t c = 0; c < n_rhs; ++c) {
            bfs(A->row_ptr, A->col_idx, rhs_rows[c] / b, radii[c], mark, atoms);
            counts[c] = (int64_t)atoms.size();
            if (sub_atoms) {
                // sub_ptr was filled by the sizing call; check it still matches
                if (sub_ptr[c + 1] - sub_ptr[c] != counts[c]) {
#pragma omp atomic write
                    err = 1;
                } else {
                    for (size_t i = 0; i < atoms.size(); ++i) sub_atoms[sub_ptr[c] + i] = (int32_t)atoms[i];
                }
            }
        }
    }
    if (!sub_atoms) {
        sub_ptr[0] = 0;
        for (int64_t c = 0; c < n_rhs; ++c) sub_ptr[c + 1] = sub_ptr[c] + counts[c];
    }
    return err ? TB_ERR_ARG : TB_OK;
}
