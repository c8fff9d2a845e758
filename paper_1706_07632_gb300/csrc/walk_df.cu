// Mixed panel walks: FP64 grid functions, stencil and diagonal; FP32 H-matrix products.
#include <algorithm>

#include "walk_impl.cuh"

namespace fhmg {
int walk_launch_df(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used) {
  if (jobs[0].mode == MODE_SMOOTH) return panel_dispatch<double, float, MODE_SMOOTH>(st, jobs, njobs, err, tile_used);
  return panel_dispatch<double, float, MODE_MATVEC>(st, jobs, njobs, err, tile_used);
}
}  // namespace fhmg
