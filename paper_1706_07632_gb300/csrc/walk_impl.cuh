// Template dispatch of hpanel_kernel over (leaf, column tile); included by the per-precision
// translation units.
#pragma once
#include <string>

#include "walk.h"

namespace fhmg {

constexpr int kPanelSMs = 152;
constexpr int kPanelThreads = 256;
constexpr size_t kPanelSmemCap = 200 * 1024;

inline int panel_slots(int slot_bytes) {
  int ns = (int)((96 * 1024) / (size_t)slot_bytes);
  return ns < 2 ? 2 : (ns > 16 ? 16 : ns);
}

template <typename TM>
size_t panel_bytes(const PanelDev& P, int L, int TC) {
  return panel_smem(L, TC, P.pool, P.W, P.slot_bytes, P.ns, sizeof(double), sizeof(TM)).total;
}

template <typename TM, int L, int TC, int MODE>
int panel_launch_t(cudaStream_t st, const WalkArgs& a, PanelDev P, std::string* err) {
  auto kern = hpanel_kernel<double, TM, L, TC, MODE, kPanelThreads>;
  const size_t smem = panel_bytes<TM>(P, L, TC);
  static size_t configured = 48 * 1024;
  static size_t occ_smem = 0;
  static int occ = 1;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
      return 1;
    }
    configured = smem;
  }
  if (occ_smem != smem) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kPanelThreads, smem) != cudaSuccess || o < 1) o = 1;
    occ = o;
    occ_smem = smem;
  }
  const long long ntiles = (a.ncols + TC - 1) / TC;
  if (ntiles <= 0) return 0;
  long long grid = std::min<long long>(ntiles, (long long)kPanelSMs * occ);
  kern<<<(unsigned)grid, kPanelThreads, smem, st>>>(P, a.geo, a.ncols, a.X, a.B, a.OUT, (const TM*)a.Dinv, a.ddiag,
                                                    a.norm, a.err);
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
template <typename TM>
int panel_pick(const PanelDev& P, int L, long long ncols) {
  const int tcmax = (L == 64 && sizeof(TM) == 8) ? 16 : 32;  // FP64 leaf-64 tiles of 32 spill
  int tc = 1;
  while (tc < tcmax && (ncols + 2 * tc - 1) / (2 * tc) >= kPanelSMs) tc *= 2;
  while (tc > 1 && panel_bytes<TM>(P, L, tc) > kPanelSmemCap) tc /= 2;
  return tc;
}

template <typename TM, int MODE>
int panel_dispatch(cudaStream_t st, const WalkArgs& a, std::string* err, int* tile_used) {
  PanelDev P = a.P;
  P.ns = panel_slots(P.slot_bytes);
  const int L = P.L;
  const int TC = a.tile ? a.tile : panel_pick<TM>(P, L, a.ncols);
  if (tile_used) *tile_used = TC;
  if (panel_bytes<TM>(P, L, TC) > 227 * 1024) {
    *err = "panel shared memory exceeds 227 KB";
    return 2;
  }
#define FHMG_CASE(LL, TT) \
  if (L == LL && TC == TT) return panel_launch_t<TM, LL, TT, MODE>(st, a, P, err);
  FHMG_CASE(16, 1) FHMG_CASE(16, 2) FHMG_CASE(16, 4) FHMG_CASE(16, 8) FHMG_CASE(16, 16) FHMG_CASE(16, 32)
  FHMG_CASE(32, 1) FHMG_CASE(32, 2) FHMG_CASE(32, 4) FHMG_CASE(32, 8) FHMG_CASE(32, 16) FHMG_CASE(32, 32)
  FHMG_CASE(64, 1) FHMG_CASE(64, 2) FHMG_CASE(64, 4) FHMG_CASE(64, 8) FHMG_CASE(64, 16) FHMG_CASE(64, 32)
#undef FHMG_CASE
  *err = "no panel kernel for leaf " + std::to_string(L) + ", tile " + std::to_string(TC);
  return 2;
}

}  // namespace fhmg
