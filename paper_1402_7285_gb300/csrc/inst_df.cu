// Instantiations of the panel and local solvers for df panel vectors.
#include "cocg_impl.cuh"
#include "local_impl.cuh"

namespace tbgf {

bool launch_panel_df(SolveLaunch &L, int b, int W) { return dispatch_bw<df>(L, b, W); }

bool launch_local_df(LocalLaunch &L, int b) { return dispatch_bw<df>(L, b, 8); }

} // namespace tbgf
