// FP64 panel walks (every product in FP64).
#include <algorithm>

#include "walk_impl.cuh"

namespace fhmg {
int walk_launch_dd(cudaStream_t st, const WalkArgs& a, std::string* err, int* tile_used) {
  if (a.mode == MODE_SMOOTH) return panel_dispatch<double, MODE_SMOOTH>(st, a, err, tile_used);
  return panel_dispatch<double, MODE_MATVEC>(st, a, err, tile_used);
}
}  // namespace fhmg
