// Instantiations of the panel and local solvers for double panel vectors.
#include "cocg_impl.cuh"
#include "local_impl.cuh"

namespace tbgf {

bool launch_panel_f64(SolveLaunch &L, int b, int W) { return dispatch_bw<double>(L, b, W); }

bool launch_local_f64(LocalLaunch &L, int b) { return dispatch_bw<double>(L, b, 8); }

} // namespace tbgf
