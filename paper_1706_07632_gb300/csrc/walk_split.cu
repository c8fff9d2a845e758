// Launcher of the tensor-core defect by digit splitting (split.cuh).
#include <cstdio>
#include <string>

#include "split.cuh"
#include "walk.h"

namespace fhmg {

namespace {
KernelCache g_split_cache;
}

int split_defect_launch(cudaStream_t st, const SplitArgs& a0, std::string* err) {
  if (a0.M % kSplitRows != 0 || a0.M > kSplitMaxM || a0.ld < 1 || !a0.U || !a0.F || !a0.OUT || !a0.fe || !a0.At ||
      !a0.pairs || !a0.rexp) {
    if (err) *err = "split defect: unsupported arguments";
    return 2;
  }
  SplitArgs a = a0;
  a.ntiles = (a.ld + kSpCols - 1) / kSpCols;
  if (a.spin <= 0) a.spin = kSpinLimit;
  const int sms = device_sms();
  // the exponents of u per grid point and B = F - A_h u into OUT (one pass, grid-stride)
  split_prep_kernel<<<grid_for(a.ld, 8), 256, 0, st>>>(a.U, a.F, a.OUT, a.fe, a.ld, a.M, a.dim, a.N, a.inv_h2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (err) *err = std::string("split_prep_kernel: ") + cudaGetErrorString(e);
    return 1;
  }
  a.ns = 4;
  const size_t smem = split_smem(a.ns).total + 1024;  // + the alignment of the swizzled tiles
  int occ = 1;
  e = prepare_launch(split_defect_kernel, kSpBlock, smem, g_split_cache, &occ);
  if (e != cudaSuccess) {
    if (err) *err = std::string("split_defect_kernel attributes: ") + cudaGetErrorString(e);
    return 1;
  }
  const long long grid = std::min<long long>(a.ntiles, (long long)sms * occ);
  split_defect_kernel<<<(unsigned)grid, kSpBlock, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (err) *err = std::string("split_defect_kernel: ") + cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

}  // namespace fhmg
