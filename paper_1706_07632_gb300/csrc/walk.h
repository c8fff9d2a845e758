// Host-side launchers of the panel walk kernel, one translation unit per precision pair
// (compiled in parallel).  Returns 0 on success, 1 on a CUDA error, 2 if no kernel matches.
#pragma once
#include <string>

#include "panel.cuh"

namespace fhmg {

// One walk job (one instance).
template <typename T>
struct WalkArgsT {
  PanelDev P;                  // ns is chosen by the launcher
  int mode;                    // MODE_SMOOTH / MODE_MATVEC (the same for every job of a launch)
  Geo geo;
  long long ncols;
  T* X;
  const T* B;
  T* OUT;
  const void* Dinv;            // TM*, level inverses (smoother)
  long long dinv_cstride;      // 0, or per-column inverse sets (forces a column tile of 1)
  const T* ddiag;              // FP32 products: diagonal of the DIAG blocks (see WalkJob)
  unsigned long long* norm;
  int* err;                    // device error word (bounded-wait timeout); the first job's is used
  int tile;                    // 0: automatic, else the column tile TC (the first job's is used)
};
using WalkArgs = WalkArgsT<double>;

// Launches njobs (1..kMaxJobs) jobs with the same leaf size and mode as one persistent kernel.
// dd: FP64 storage, FP64 products; df: FP64 storage, FP32 products; ff: FP32 storage and products.
int walk_launch_dd(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used);
int walk_launch_df(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used);
int walk_launch_ff(cudaStream_t st, const WalkArgsT<float>* jobs, int njobs, std::string* err, int* tile_used);

}  // namespace fhmg
