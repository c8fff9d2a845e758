// FP32 panel walks: FP32 grid functions and products (inner cycles on well-conditioned grids).
#include <algorithm>

#include "walk_impl.cuh"

namespace fhmg {
int walk_launch_ff(cudaStream_t st, const WalkArgsT<float>* jobs, int njobs, std::string* err, int* tile_used) {
  if (jobs[0].mode == MODE_SMOOTH) return panel_dispatch<float, float, MODE_SMOOTH>(st, jobs, njobs, err, tile_used);
  return panel_dispatch<float, float, MODE_MATVEC>(st, jobs, njobs, err, tile_used);
}
}  // namespace fhmg
