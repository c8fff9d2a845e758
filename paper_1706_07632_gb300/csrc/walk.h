// Host-side launchers of the panel walk kernel, one translation unit per precision pair
// (compiled in parallel).  Returns 0 on success, 1 on a CUDA error, 2 if no kernel matches.
#pragma once
#include <string>

#include "devinfo.h"

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
  PanelDev PM;                 // FP32 products only: the stream in the tensor-core layout (pkg NULL: none)
  const void* DinvM;           // and the level inverses in that layout
  PanelDev PU;                 // FP32-storage walks of BF16 problems: the tcgen05 stream (pkg NULL: none)
  const void* DinvU;           // and the level inverses in that layout
  long long spin;              // consumer-side poll limit of the bounded waits (0: kSpinLimit; first job's)
  long long withhold;          // test hook, 0: off; else the producers withhold chunk withhold - 1 (first job's)
};
using WalkArgs = WalkArgsT<double>;

// Launches njobs (1..kMaxJobs) jobs with the same leaf size and mode as one persistent kernel.
// dd: FP64 storage, FP64 products; df: FP64 storage, FP32 products; ff: FP32 storage and products.
int walk_launch_dd(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used);
int walk_launch_df(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used);
int walk_launch_ff(cudaStream_t st, const WalkArgsT<float>* jobs, int njobs, std::string* err, int* tile_used);

// FP64-accurate walks in double-float arithmetic, walk_dfd.cu: products (MODE_MATVEC) or line solves
// on compact columns (MODE_SMOOTH, geo.dim 0; Dinv: inverses as float pairs, 2 L^2 floats per leaf,
// dinv_cstride floats per column); the jobs' P is the build_panel_df stream; tile 1, 4, 8 or 16
// (0: automatic; 1 whenever columns have their own inverses).
// tcgen05 walks (BF16 products, FP32 storage, leaf 64, 128-column tiles), walk_umma.cu: the jobs' PU
// stream and DinvU inverses.  Returns 2 (no kernel) if a job lacks them or needs far near-field blocks.
int walk_launch_umma(cudaStream_t st, const WalkArgsT<float>* jobs, int njobs, std::string* err);
constexpr int kUmmaL = 64;  // leaf size of the tcgen05 walk

// FP64-accurate finest-grid defect r = F - A_h u - (R~ (x) I) u on the tcgen05 tensor cores by
// digit splitting of R~ and u (split.cuh, walk_split.cu): time matrices with M a multiple of
// kSplitRows and at most kSplitMaxM levels.  Launches the exponent pass and the defect kernel;
// returns 2 for unsupported arguments.
constexpr int kSplitRows = 128;
constexpr int kSplitMaxM = 512;
struct SplitArgs {
  const double* U;            // u, [M][ld]
  const double* F;            // F = f + d g, [M][ld]
  double* OUT;                // r, [M][ld]
  unsigned long long* norm;   // max |r| as FP64 bits (atomicMax), or NULL
  int* fe;                    // scratch, ld ints: per grid point the largest biased FP64 exponent of u
  const unsigned char* At;    // R~ digit tiles (build_split)
  const int4* pairs;          // per (I, J), I-major: {digit mask, first tile, 0, 0}
  const int* rexp;            // E_m per time row
  int* err;                   // device error word (bounded-wait timeout)
  long long ld;               // points per time level (N^dim)
  long long ntiles;           // set by the launcher
  int dim, N, M;
  double inv_h2;              // 1 / h^2
  int ns;                     // ring slots, set by the launcher
  long long spin;             // consumer / MMA poll limit (0: kSpinLimit)
  long long withhold;         // test hook (0 off): the producer withholds digit tile withhold - 1
};
int split_defect_launch(cudaStream_t st, const SplitArgs& a, std::string* err);

int walk_launch_dfprod(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used);

// Tensor-core walks (FP32 products, leaf 64, TC 16 or 32), walk_mma.cu.  B.ns is chosen here.
int mma_launch_df(cudaStream_t st, WalkBatch<double, float>& B, int TC, int mode, std::string* err);
int mma_launch_ff(cudaStream_t st, WalkBatch<float, float>& B, int TC, int mode, std::string* err);
template <typename T>
inline int mma_launch(cudaStream_t st, WalkBatch<T, float>& B, int TC, int mode, std::string* err);
template <>
inline int mma_launch<double>(cudaStream_t st, WalkBatch<double, float>& B, int TC, int mode, std::string* err) {
  return mma_launch_df(st, B, TC, mode, err);
}
template <>
inline int mma_launch<float>(cudaStream_t st, WalkBatch<float, float>& B, int TC, int mode, std::string* err) {
  return mma_launch_ff(st, B, TC, mode, err);
}

}  // namespace fhmg
