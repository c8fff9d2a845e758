// Launchers of the tensor-core panel walk (FP32 products, leaf 64, column tile 16 or 32).
#include <algorithm>
#include <string>

#include "mma.cuh"
#include "walk.h"

namespace fhmg {
namespace {

constexpr int kMmaBlock = 256 + 32;  // consumer warps + producer warp
constexpr size_t kMmaSmemMax = 227 * 1024;

template <typename T, int TC, int MODE>
int mma_launch_t(cudaStream_t st, WalkBatch<T, float>& B, std::string* err) {
  auto kern = hmma_kernel<T, TC, MODE>;
  // the deepest chunk ring that fits beside the x tiles and the z pool
  const size_t other = mma_smem(TC, B.pool, B.W, B.slot_bytes, 0).total + 64;
  int ns = other < kMmaSmemMax ? (int)((kMmaSmemMax - other) / (size_t)B.slot_bytes) : 0;
  ns = std::min(ns, 8);
  if (ns < 2) {
    *err = "tensor-core walk: no room for two chunk slots in shared memory";
    return 2;
  }
  B.ns = ns;
  const size_t smem = mma_smem(TC, B.pool, B.W, B.slot_bytes, ns).total;
  static KernelCache cache;
  int occ = 1;
  {
    cudaError_t e = prepare_launch(kern, kMmaBlock, smem, cache, &occ);
    if (e != cudaSuccess) {
      *err = std::string("tensor-core walk set-up: ") + cudaGetErrorString(e);
      return 1;
    }
  }
  if (B.ntiles <= 0) return 0;
  const long long grid = std::min<long long>(B.ntiles, (long long)device_sms() * occ);
  kern<<<(unsigned)grid, kMmaBlock, smem, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("tensor-core walk launch: ") + cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

template <typename T>
int mma_dispatch(cudaStream_t st, WalkBatch<T, float>& B, int TC, int mode, std::string* err) {
  if (TC == 16) return mode == MODE_SMOOTH ? mma_launch_t<T, 16, MODE_SMOOTH>(st, B, err)
                                           : mma_launch_t<T, 16, MODE_MATVEC>(st, B, err);
  if (TC == 32) return mode == MODE_SMOOTH ? mma_launch_t<T, 32, MODE_SMOOTH>(st, B, err)
                                           : mma_launch_t<T, 32, MODE_MATVEC>(st, B, err);
  *err = "tensor-core walk: column tile must be 16 or 32";
  return 2;
}

}  // namespace

int mma_launch_df(cudaStream_t st, WalkBatch<double, float>& B, int TC, int mode, std::string* err) {
  return mma_dispatch<double>(st, B, TC, mode, err);
}
int mma_launch_ff(cudaStream_t st, WalkBatch<float, float>& B, int TC, int mode, std::string* err) {
  return mma_dispatch<float>(st, B, TC, mode, err);
}

}  // namespace fhmg
