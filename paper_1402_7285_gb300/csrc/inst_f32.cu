// Instantiations of the panel and local solvers for float panel vectors.
#include "cocg_impl.cuh"
#include "local_impl.cuh"

namespace tbgf {

bool launch_panel_f32(SolveLaunch &L, int b, int W) { return dispatch_bw<float>(L, b, W); }

bool launch_local_f32(LocalLaunch &L, int b) { return dispatch_bw<float>(L, b, 8); }

} // namespace tbgf
