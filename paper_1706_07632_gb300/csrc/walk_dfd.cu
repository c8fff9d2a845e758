// Launcher of the double-float walks (hdf_kernel, df.cuh): FP64 arrays, FP64-accurate H-matrix
// products (defects) and line solves on compact columns (the exactly solved level's modes) in
// FP32-pair arithmetic.
#include <algorithm>
#include <string>

#include "df.cuh"
#include "walk.h"

namespace fhmg {
namespace {

constexpr int kDfBlock = 256 + 32;
constexpr size_t kDfSmemMax = 227 * 1024;

template <int L, int TC, int MODE>
int df_launch_t(cudaStream_t st, WalkBatch<double, float>& B, std::string* err) {
  auto kern = hdf_kernel<L, TC, MODE>;
  // with more tiles than SMs and a tile that leaves room for two CTAs' registers (TC <= 8), size
  // the ring for two CTAs per SM (16 consumer warps hide the latency of the double-float chains
  // better than a deeper ring: 3.9 vs 5.3 ms for 4095 columns x M = 4096); else the deepest ring
  const size_t other = df_smem(L, TC, B.pool, B.W, B.slot_bytes, 0).total + 64;
  const size_t budget = (TC <= 8 && B.ntiles > device_sms()) ? kDfSmemMax / 2 - 1024 : kDfSmemMax;
  int ns = other < budget ? (int)((budget - other) / (size_t)B.slot_bytes) : 0;
  ns = std::min(ns, 8);
  if (ns < 2 && budget < kDfSmemMax)
    ns = std::min(8, other < kDfSmemMax ? (int)((kDfSmemMax - other) / (size_t)B.slot_bytes) : 0);
  if (ns < 2) {
    *err = "double-float walk: no room for two chunk slots in shared memory";
    return 2;
  }
  B.ns = ns;
  const size_t smem = df_smem(L, TC, B.pool, B.W, B.slot_bytes, ns).total;
  static KernelCache cache;
  int occ = 1;
  {
    cudaError_t e = prepare_launch(kern, kDfBlock, smem, cache, &occ);
    if (e != cudaSuccess) {
      *err = std::string("double-float walk set-up: ") + cudaGetErrorString(e);
      return 1;
    }
  }
  if (B.ntiles <= 0) return 0;
  const long long grid = std::min<long long>(B.ntiles, (long long)device_sms() * occ);
  kern<<<(unsigned)grid, kDfBlock, smem, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("double-float walk launch: ") + cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

}  // namespace

int walk_launch_dfprod(cudaStream_t st, const WalkArgsT<double>* jobs, int njobs, std::string* err, int* tile_used) {
  if (njobs < 1 || njobs > kMaxJobs) {
    *err = "double-float walk needs 1.." + std::to_string(kMaxJobs) + " jobs";
    return 2;
  }
  const int L = jobs[0].P.L;
  const int mode = jobs[0].mode;
  WalkBatch<double, float> B;
  B.njobs = njobs;
  B.pool = 0;
  B.W = 1;
  B.slot_bytes = 16;
  B.err = jobs[0].err;
  B.spin = jobs[0].spin > 0 ? jobs[0].spin : kSpinLimit;
  B.withhold = jobs[0].withhold;
  long long cols = 0;
  for (int j = 0; j < njobs; ++j) {
    if (jobs[j].P.L != L || jobs[j].mode != mode || (mode == MODE_SMOOTH && jobs[j].geo.dim != 0)) {
      *err = "double-float walk: jobs of one leaf size and mode; solves on compact columns only";
      return 2;
    }
    B.pool = std::max(B.pool, jobs[j].P.pool);
    B.W = std::max(B.W, jobs[j].P.W);
    B.slot_bytes = std::max(B.slot_bytes, jobs[j].P.slot_bytes);
    cols += jobs[j].ncols;
  }
  // column tile: 8 once the columns give every SM a tile of 8 (two CTAs per SM), else 4
  int TC = jobs[0].tile;
  if (TC != 1 && TC != 4 && TC != 8 && TC != 16) TC = cols >= 8LL * device_sms() ? 8 : cols >= 4LL * device_sms() ? 4 : 1;
  bool per_column = false;
  for (int j = 0; j < njobs; ++j) per_column |= jobs[j].dinv_cstride != 0;
  if (per_column) TC = 1;  // each column streams its own inverses
  if (tile_used) *tile_used = TC;
  long long tiles = 0;
  for (int j = 0; j < njobs; ++j) {
    WalkJob<double, float>& J = B.job[j];
    J.P = jobs[j].P;
    J.geo = jobs[j].geo;
    J.ncols = jobs[j].ncols;
    J.tile0 = tiles;
    J.X = jobs[j].X;
    J.B = jobs[j].B;
    J.OUT = jobs[j].OUT;
    J.Dinv = (const float*)jobs[j].Dinv;
    J.dinv_cstride = jobs[j].dinv_cstride;
    J.ddiag = nullptr;
    J.norm = jobs[j].norm;
    tiles += (jobs[j].ncols + TC - 1) / TC;
  }
  B.ntiles = tiles;
  B.ns = 2;
#define FHMG_DF(LL, TT)                                                                              \
  if (L == LL && TC == TT)                                                                             \
    return mode == MODE_SMOOTH ? df_launch_t<LL, TT, MODE_SMOOTH>(st, B, err)                          \
                               : df_launch_t<LL, TT, MODE_MATVEC>(st, B, err);
  FHMG_DF(64, 1) FHMG_DF(64, 4) FHMG_DF(64, 8) FHMG_DF(64, 16)
  FHMG_DF(32, 1) FHMG_DF(32, 4) FHMG_DF(32, 8) FHMG_DF(32, 16)
#undef FHMG_DF
  *err = "no double-float walk for leaf " + std::to_string(L);
  return 2;
}

}  // namespace fhmg
