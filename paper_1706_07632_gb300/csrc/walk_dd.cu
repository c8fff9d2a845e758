// FP64 panel walks (every product in FP64).
#include <algorithm>

#include "walk_impl.cuh"

namespace fhmg {
int walk_launch_dd(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used) {
  if (jobs[0].mode == MODE_SMOOTH) return panel_dispatch<double, double, MODE_SMOOTH>(st, jobs, njobs, err, tile_used);
  return panel_dispatch<double, double, MODE_MATVEC>(st, jobs, njobs, err, tile_used);
}
}  // namespace fhmg
