// Mixed panel walks: FP64 grid functions, stencil and diagonal; FP32 H-matrix products.
#include <algorithm>

#include "walk_impl.cuh"

namespace fhmg {
int walk_launch_df(cudaStream_t st, const WalkArgs& a, std::string* err, int* tile_used) {
  if (a.mode == MODE_SMOOTH) return panel_dispatch<float, MODE_SMOOTH>(st, a, err, tile_used);
  return panel_dispatch<float, MODE_MATVEC>(st, a, err, tile_used);
}
}  // namespace fhmg
