// Template dispatch of hpanel_kernel over (leaf, column tile); included by the per-precision
// translation units.
#pragma once
#include <algorithm>
#include <string>

#include "walk.h"

namespace fhmg {

constexpr int kPanelThreads = 256;                  // consumer threads of the walk
constexpr int kPanelBlock = kPanelThreads + 32;     // + the producer warp
constexpr size_t kPanelSmemCap = 200 * 1024;

inline int panel_slots(int slot_bytes) {
  int ns = (int)((96 * 1024) / (size_t)slot_bytes);
  return ns < 2 ? 2 : (ns > 16 ? 16 : ns);
}

template <typename T, typename TM>
size_t panel_bytes(int L, int TC, int pool, int W, int slot_bytes, int ns) {
  return panel_smem(L, TC, pool, W, slot_bytes, ns, sizeof(TM)).total;
}

template <typename T, typename TM, int L, int TC, int MODE>
int panel_launch_t(cudaStream_t st, const WalkBatch<T, TM>& B, std::string* err) {
  auto kern = hpanel_kernel<T, TM, L, TC, MODE, kPanelThreads>;
  const size_t smem = panel_bytes<T, TM>(L, TC, B.pool, B.W, B.slot_bytes, B.ns);
  static KernelCache cache;
  int occ = 1;
  {
    cudaError_t e = prepare_launch(kern, kPanelBlock, smem, cache, &occ);
    if (e != cudaSuccess) {
      *err = std::string("panel launch set-up: ") + cudaGetErrorString(e);
      return 1;
    }
  }
  if (B.ntiles <= 0) return 0;
  const long long grid = std::min<long long>(B.ntiles, (long long)device_sms() * occ);
  kern<<<(unsigned)grid, kPanelBlock, smem, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("panel launch: ") + cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

// Column tile: the largest TC whose tiles still cover every SM (persistent CTAs reuse each
// staged chunk for all TC columns), TC = 1 when there are fewer columns than SMs; shrunk until
// the shared-memory layout fits.
template <typename T, typename TM>
int panel_pick(int L, int pool, int W, int slot_bytes, int ns, long long ncols, int sms) {
  const int tcmax = (L == 64 && sizeof(TM) == 8) ? 16 : 32;  // FP64 leaf-64 tiles of 32 spill
  int tc = 1;
  while (tc < tcmax && (ncols + 2 * tc - 1) / (2 * tc) >= sms) tc *= 2;
  while (tc > 1 && panel_bytes<T, TM>(L, tc, pool, W, slot_bytes, ns) > kPanelSmemCap) tc /= 2;
  return tc;
}

template <typename T, typename TM, int MODE>
int panel_dispatch(cudaStream_t st, const WalkArgsT<T>* jobs, int njobs, std::string* err, int* tile_used) {
  if (njobs < 1 || njobs > kMaxJobs) {
    *err = "walk launch needs 1.." + std::to_string(kMaxJobs) + " jobs";
    return 2;
  }
  const int L = jobs[0].P.L;
  const int sms = device_sms();
  int pool = 0, W = 1, slot = 16;
  long long cols = 0;
  for (int j = 0; j < njobs; ++j) {
    if (jobs[j].P.L != L) {
      *err = "jobs of one walk launch must share the leaf size";
      return 2;
    }
    if (sizeof(TM) < 8 && jobs[j].ddiag == nullptr) {
      *err = "FP32 products need the diagonal of the streamed DIAG blocks (ddiag)";
      return 2;
    }
    pool = std::max(pool, jobs[j].P.pool);
    W = std::max(W, jobs[j].P.W);
    slot = std::max(slot, jobs[j].P.slot_bytes);
    cols = std::max(cols, jobs[j].ncols);
  }
  int ns = panel_slots(slot);
  long long total_cols = 0;
  for (int j = 0; j < njobs; ++j) total_cols += jobs[j].ncols;
  if constexpr (sizeof(TM) == 4) {
    // FP32 products on the tensor cores: leaf 64, tile 16 or 32 (tile 16 once the columns fill
    // 128 SMs with 16 each -- below that the SIMT walk with narrower tiles on every SM is faster,
    // e.g. 0.36 vs 0.52 ms at 1024 columns x M = 4096 -- and 32 once they fill every SM with 32)
    bool mma_ok = L == 64;
    for (int j = 0; j < njobs; ++j)
      mma_ok = mma_ok && jobs[j].PM.pkg != nullptr && !jobs[j].PM.far && jobs[j].dinv_cstride == 0;
    if (mma_ok) {
      int tcm = jobs[0].tile;
      if (tcm == 0) tcm = total_cols >= 32LL * sms ? 32 : total_cols >= 2048 ? 16 : 0;
      if (tcm == 16 || tcm == 32) {
        if (tile_used) *tile_used = tcm;
        WalkBatch<T, float> Bm;
        Bm.njobs = njobs;
        Bm.pool = 0;
        Bm.W = 1;
        Bm.slot_bytes = 16;
        Bm.err = jobs[0].err;
        Bm.spin = jobs[0].spin > 0 ? jobs[0].spin : kSpinLimit;
        Bm.withhold = jobs[0].withhold;
        long long tiles = 0;
        for (int j = 0; j < njobs; ++j) {
          Bm.pool = std::max(Bm.pool, jobs[j].PM.pool);
          Bm.W = std::max(Bm.W, jobs[j].PM.W);
          Bm.slot_bytes = std::max(Bm.slot_bytes, jobs[j].PM.slot_bytes);
          WalkJob<T, float>& J = Bm.job[j];
          J.P = jobs[j].PM;
          J.geo = jobs[j].geo;
          J.ncols = jobs[j].ncols;
          J.tile0 = tiles;
          J.X = jobs[j].X;
          J.B = jobs[j].B;
          J.OUT = jobs[j].OUT;
          J.Dinv = (const float*)jobs[j].DinvM;
          J.dinv_cstride = 0;
          J.ddiag = jobs[j].ddiag;
          J.norm = jobs[j].norm;
          tiles += (jobs[j].ncols + tcm - 1) / tcm;
        }
        Bm.ntiles = tiles;
        Bm.ns = 2;
        return mma_launch<T>(st, Bm, tcm, MODE, err);
      }
    }
  }
  bool per_column_inverse = false;
  for (int j = 0; j < njobs; ++j) per_column_inverse |= jobs[j].dinv_cstride != 0;
  const int TC = per_column_inverse ? 1
                 : jobs[0].tile     ? jobs[0].tile
                                    : panel_pick<T, TM>(L, pool, W, slot, ns, total_cols, sms);
  if (tile_used) *tile_used = TC;
  // Pipeline depth: when every tile gets its own SM (one CTA per SM), a CTA has little work per
  // chunk and the copies' latency dominates -- deepen the ring up to ~200 KB of shared memory;
  // otherwise keep ~96 KB of slots so that two CTAs fit per SM.
  long long tiles_all = 0;
  for (int j = 0; j < njobs; ++j) tiles_all += (jobs[j].ncols + TC - 1) / TC;
  if (tiles_all <= sms) {
    const size_t other = panel_bytes<T, TM>(L, TC, pool, W, slot, 0);
    while (ns < 16 && other + (size_t)(ns + 1) * slot + 64 <= kPanelSmemCap) ++ns;
  }
  if (panel_bytes<T, TM>(L, TC, pool, W, slot, ns) > 227 * 1024) {
    *err = "panel shared memory exceeds 227 KB";
    return 2;
  }
  WalkBatch<T, TM> B;
  B.njobs = njobs;
  B.ns = ns;
  B.pool = pool;
  B.W = W;
  B.slot_bytes = slot;
  B.err = jobs[0].err;
  B.spin = jobs[0].spin > 0 ? jobs[0].spin : kSpinLimit;
  B.withhold = jobs[0].withhold;
  long long tiles = 0;
  for (int j = 0; j < njobs; ++j) {
    WalkJob<T, TM>& J = B.job[j];
    J.P = jobs[j].P;
    J.geo = jobs[j].geo;
    J.ncols = jobs[j].ncols;
    J.tile0 = tiles;
    J.X = jobs[j].X;
    J.B = jobs[j].B;
    J.OUT = jobs[j].OUT;
    J.Dinv = (const TM*)jobs[j].Dinv;
    J.dinv_cstride = jobs[j].dinv_cstride;
    J.ddiag = jobs[j].ddiag;
    J.norm = jobs[j].norm;
    tiles += (jobs[j].ncols + TC - 1) / TC;
  }
  B.ntiles = tiles;
#define FHMG_CASE(LL, TT) \
  if (L == LL && TC == TT) return panel_launch_t<T, TM, LL, TT, MODE>(st, B, err);
  FHMG_CASE(16, 1) FHMG_CASE(16, 2) FHMG_CASE(16, 4) FHMG_CASE(16, 8) FHMG_CASE(16, 16) FHMG_CASE(16, 32)
  FHMG_CASE(32, 1) FHMG_CASE(32, 2) FHMG_CASE(32, 4) FHMG_CASE(32, 8) FHMG_CASE(32, 16) FHMG_CASE(32, 32)
  FHMG_CASE(64, 1) FHMG_CASE(64, 2) FHMG_CASE(64, 4) FHMG_CASE(64, 8) FHMG_CASE(64, 16) FHMG_CASE(64, 32)
#undef FHMG_CASE
  *err = "no panel kernel for leaf " + std::to_string(L) + ", tile " + std::to_string(TC);
  return 2;
}

}  // namespace fhmg
