// Launcher of the tcgen05 walk (humma_kernel, umma.cuh): FP32 grid functions, BF16 H-matrix products
// with FP32 accumulation in tensor memory, 128 spatial columns per tile.
#include <algorithm>
#include <string>

#include "umma.cuh"
#include "walk.h"

namespace fhmg {
namespace {

constexpr size_t kUmmaSmemMax = 227 * 1024;
constexpr size_t kUmmaTwoPerSM = 112 * 1024;  // two CTAs share an SM's 228 KB (1 KB reserved each)

template <int MODE>
int umma_launch_t(cudaStream_t st, WalkBatch<float, uint16_t>& B, std::string* err) {
  auto kern = humma_kernel<MODE>;
  // two CTAs per SM (their chunk rings and tensor-memory round trips interleave) when at least three
  // slots fit beside the operand tiles, else one CTA with the deepest ring that fits
  const size_t other = umma_smem(B.pool, B.W, B.slot_bytes, 0).total + 128;
  int ns = other < kUmmaTwoPerSM ? (int)((kUmmaTwoPerSM - other) / (size_t)B.slot_bytes) : 0;
  const bool two = ns >= 3;
  if (!two) ns = other < kUmmaSmemMax ? (int)((kUmmaSmemMax - other) / (size_t)B.slot_bytes) : 0;
  ns = std::min(ns, 12);
  if (ns < 2) {
    *err = "tcgen05 walk: no room for two chunk slots in shared memory";
    return 2;
  }
  B.ns = ns;
  const size_t smem = umma_smem(B.pool, B.W, B.slot_bytes, ns).total;
  static KernelCache cache;
  int occ = 1;
  {
    cudaError_t e = prepare_launch(kern, kUmmaBlock, smem, cache, &occ);
    if (e != cudaSuccess) {
      *err = std::string("tcgen05 walk set-up: ") + cudaGetErrorString(e);
      return 1;
    }
  }
  if (B.ntiles <= 0) return 0;
  // two CTAs per SM when the shared memory was planned for two (each allocates half of the SM's
  // tensor memory; the registers of __launch_bounds__(.., 2) allow it), else one.  Persistent CTAs
  // never wait on one another, so a CTA that finds no room simply starts when another one ends.
  const long long per_sm = two ? 2 : 1;
  (void)occ;
  const long long grid = std::min<long long>(B.ntiles, (long long)device_sms() * per_sm);
  kern<<<(unsigned)grid, kUmmaBlock, smem, st>>>(B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("tcgen05 walk launch: ") + cudaGetErrorString(e);
    return 1;
  }
  return 0;
}

}  // namespace

int walk_launch_umma(cudaStream_t st, const WalkArgsT<float>* jobs, int njobs, std::string* err) {
  if (njobs < 1 || njobs > kMaxJobs) {
    *err = "tcgen05 walk needs 1.." + std::to_string(kMaxJobs) + " jobs";
    return 2;
  }
  const int mode = jobs[0].mode;
  WalkBatch<float, uint16_t> B;
  B.njobs = njobs;
  B.pool = 1;
  B.W = 1;
  B.slot_bytes = 16;
  B.err = jobs[0].err;
  B.spin = jobs[0].spin > 0 ? jobs[0].spin : kSpinLimit;
  B.withhold = jobs[0].withhold;
  long long tiles = 0;
  for (int j = 0; j < njobs; ++j) {
    const WalkArgsT<float>& a = jobs[j];
    if (a.mode != mode || a.PU.pkg == nullptr || a.PU.L != kUmmaL || a.PU.far || a.dinv_cstride != 0 ||
        a.ddiag == nullptr || (mode == MODE_SMOOTH && a.DinvU == nullptr)) {
      *err = "tcgen05 walk: needs leaf 64, its stream and inverses, no far near-field blocks, shared inverses";
      return 2;
    }
    B.pool = std::max(B.pool, a.PU.pool);
    B.W = std::max(B.W, a.PU.W);
    B.slot_bytes = std::max(B.slot_bytes, a.PU.slot_bytes);
    WalkJob<float, uint16_t>& J = B.job[j];
    J.P = a.PU;
    J.geo = a.geo;
    J.ncols = a.ncols;
    J.tile0 = tiles;
    J.X = a.X;
    J.B = a.B;
    J.OUT = a.OUT;
    J.Dinv = (const uint16_t*)a.DinvU;
    J.dinv_cstride = 0;
    J.ddiag = a.ddiag;
    J.norm = a.norm;
    tiles += (a.ncols + kUmmaCols - 1) / kUmmaCols;
  }
  B.ntiles = tiles;
  B.ns = 2;
  return mode == MODE_SMOOTH ? umma_launch_t<MODE_SMOOTH>(st, B, err) : umma_launch_t<MODE_MATVEC>(st, B, err);
}

}  // namespace fhmg
