// Host-side launchers of the panel walk kernel, one translation unit per precision pair
// (compiled in parallel).  Returns 0 on success, 1 on a CUDA error, 2 if no kernel matches.
#pragma once
#include <string>

#include "panel.cuh"

namespace fhmg {

struct WalkArgs {
  PanelDev P;                  // ns is chosen by the launcher
  int mode;                    // MODE_SMOOTH / MODE_MATVEC
  Geo geo;
  long long ncols;
  double* X;
  const double* B;
  double* OUT;
  const void* Dinv;            // TM*, level inverses (smoother)
  const double* ddiag;         // mixed path only
  unsigned long long* norm;
  int* err;                    // device error word (bounded-wait timeout)
  int tile;                    // 0: automatic, else the column tile TC
};

int walk_launch_dd(cudaStream_t st, const WalkArgs& a, std::string* err, int* tile_used);
int walk_launch_df(cudaStream_t st, const WalkArgs& a, std::string* err, int* tile_used);

}  // namespace fhmg
