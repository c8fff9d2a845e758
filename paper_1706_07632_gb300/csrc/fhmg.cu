// C-ABI and V-cycle driver (Algorithm 2) over the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fhmg.h"
#include "hbuild.h"
#include "kernels.cuh"

using fhmg::Geo;
using fhmg::HDev;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(x)                                                                         \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) return fail(FHMG_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)
#define TRY(...)                    \
  do {                              \
    int s_ = (__VA_ARGS__);         \
    if (s_ != FHMG_OK) return s_;   \
  } while (0)

constexpr int kSMs = 152;

}  // namespace

struct fhmg_hmatrix_s {
  fhmg::HostH host;
  fhmg::FlatH flat;
};

namespace {

template <typename T>
struct DevH {
  std::vector<void*> allocs;
  HDev<T> d{};
  size_t bytes = 0;
};

struct LevelData {
  int N = 0;
  long long npts = 0;
  double h = 0, inv_h2 = 0, shift = 0;
  double* E = nullptr;   // unknown of the coarse-grid correction (coarse levels)
  double* RC = nullptr;  // restricted defect (coarse levels)
  double* Dinv64 = nullptr;
  float* Dinv32 = nullptr;
  int tc_smooth[2] = {0, 0};
  int tc_matvec = 0;
};

}  // namespace

struct fhmg_problem_s {
  fhmg_hmatrix H = nullptr;
  int dim = 1, N = 0, nlev = 0, prec = 0;
  double Lx = 1.0;
  cudaStream_t st = nullptr;
  int M = 0, L = 0, nb = 0;
  DevH<double> h64;
  DevH<float> h32;
  std::vector<LevelData> lev;
  double* Xs = nullptr;  // scratch, >= max(colour-0 count, coarse count) * M
  double* Rs = nullptr;  // scratch, fine points * M
  double* Ff = nullptr;  // f + d g when g is given
  double* dmm = nullptr; // d_{m,m}
  unsigned long long* dnorm = nullptr;
  double* hu = nullptr;  // device copies for fhmg_solve_host
  double* hf = nullptr;
  double* hg = nullptr;
  std::vector<void*> allocs;
  long long launches = 0;                 // kernel launches issued (all kernels)
  bool profile = false;                   // record events around finest-level smoother walks
  std::vector<cudaEvent_t> ev;            // start/stop pairs
  size_t ev_used = 0;
};

namespace {

template <typename T>
int dalloc(std::vector<void*>& list, T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) return fail(FHMG_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  list.push_back(*p);
  return FHMG_OK;
}

template <typename T, typename S>
int upload(std::vector<void*>& list, const std::vector<S>& src, const T** out, size_t* bytes) {
  T* p;
  TRY(dalloc(list, &p, src.size()));
  std::vector<T> tmp(src.begin(), src.end());
  if (!tmp.empty()) CK(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = p;
  if (bytes) *bytes += tmp.size() * sizeof(T);
  return FHMG_OK;
}

// row-major -> column-major for a stack of rows x cols blocks
void transpose_into(const double* in, double* out, int rows, int cols) {
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) out[(size_t)c * rows + r] = in[(size_t)r * cols + c];
}

template <typename T>
int upload_h(const fhmg::FlatH& f, DevH<T>& D) {
  const int L = f.L, nb = f.nb;
  std::vector<double> dense(f.dense_data.size()), ud(f.udata.size()), vd(f.vdata.size());
  size_t nd = f.dense_data.size() / ((size_t)L * L);
  for (size_t b = 0; b < nd; ++b)
    transpose_into(&f.dense_data[b * L * L], &dense[b * L * L], L, L);
  for (int i = 0; i < nb; ++i) {
    int K = f.uptr[i + 1] - f.uptr[i];
    if (K) transpose_into(&f.udata[f.uoff[i]], &ud[f.uoff[i]], L, K);
    int Kv = f.vptr[i + 1] - f.vptr[i];
    if (Kv) transpose_into(&f.vdata[f.voff[i]], &vd[f.voff[i]], Kv, L);
  }
  HDev<T>& d = D.d;
  TRY(upload(D.allocs, dense, &d.dense, &D.bytes));
  TRY(upload(D.allocs, f.dptr, &d.dptr, &D.bytes));
  TRY(upload(D.allocs, f.dlist_blk, &d.dblk, &D.bytes));
  TRY(upload(D.allocs, f.dlist_col, &d.dcol, &D.bytes));
  TRY(upload(D.allocs, f.diag_blk, &d.diag, &D.bytes));
  TRY(upload(D.allocs, f.uptr, &d.uptr, &D.bytes));
  TRY(upload(D.allocs, f.uz, &d.uz, &D.bytes));
  TRY(upload(D.allocs, f.uoff, &d.uoff, &D.bytes));
  TRY(upload(D.allocs, ud, &d.udata, &D.bytes));
  TRY(upload(D.allocs, f.vptr, &d.vptr, &D.bytes));
  TRY(upload(D.allocs, f.vz, &d.vz, &D.bytes));
  TRY(upload(D.allocs, f.vinit, &d.vinit, &D.bytes));
  TRY(upload(D.allocs, f.voff, &d.voff, &D.bytes));
  TRY(upload(D.allocs, vd, &d.vdata, &D.bytes));
  d.M = f.M;
  d.L = L;
  d.nb = nb;
  d.pool = f.pool_rows;
  return FHMG_OK;
}

template <typename T>
size_t walk_smem(int L, int TC, int pool) {
  return (size_t)(L * TC + pool * TC) * sizeof(T);
}

template <typename T, int L, int TC, int MODE>
int launch_walk_t(cudaStream_t st, const HDev<T>& H, const Geo& geo, long long ncols, T* X, const T* B,
                  T* OUT, const T* Dinv, unsigned long long* norm) {
  auto kern = fhmg::hwalk_kernel<T, L, TC, MODE>;
  const size_t smem = walk_smem<T>(L, TC, H.pool);
  static size_t configured = 48 * 1024;
  if (smem > configured) {
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  const long long grid = (ncols + TC - 1) / TC;
  if (grid <= 0) return FHMG_OK;
  if (grid > 0x7fffffffLL) return fail(FHMG_EINVAL, "too many columns");
  kern<<<(unsigned)grid, fhmg::Tile<L, TC>::NT, smem, st>>>(H, geo, ncols, X, B, OUT, Dinv, norm);
  CK(cudaGetLastError());
  return FHMG_OK;
}

template <typename T, int MODE>
int launch_walk(fhmg_problem p, const HDev<T>& H, int TC, const Geo& geo, long long ncols, T* X, const T* B,
                T* OUT, const T* Dinv, unsigned long long* norm) {
  cudaStream_t st = p->st;
  if (ncols > 0) ++p->launches;
#define FHMG_CASE(LL, TT)                                                                  \
  if (H.L == LL && TC == TT) return launch_walk_t<T, LL, TT, MODE>(st, H, geo, ncols, X, B, OUT, Dinv, norm);
  FHMG_CASE(16, 1) FHMG_CASE(16, 2) FHMG_CASE(16, 4) FHMG_CASE(16, 8) FHMG_CASE(16, 16)
  FHMG_CASE(32, 1) FHMG_CASE(32, 2) FHMG_CASE(32, 4) FHMG_CASE(32, 8) FHMG_CASE(32, 16)
  FHMG_CASE(64, 1) FHMG_CASE(64, 2) FHMG_CASE(64, 4) FHMG_CASE(64, 8) FHMG_CASE(64, 16)
#undef FHMG_CASE
  return fail(FHMG_EINVAL, "no kernel for leaf %d and column tile %d", H.L, TC);
}

// Column tile: the smallest of 1..16 whose grid fits in about one wave of 7 resident 256-thread
// CTAs per SM (more CTAs than that only adds waves; fewer columns per CTA keeps each CTA's
// sequential leaf chain short), shrunk if the z-pool does not fit in shared memory.
template <typename T>
int pick_tc(const HDev<T>& H, long long ncols) {
  int tc = 1;
  while (tc < 16 && (ncols + tc - 1) / tc > 7LL * kSMs) tc *= 2;
  while (tc > 1 && walk_smem<T>(H.L, tc, H.pool) > 200 * 1024) tc /= 2;
  return tc;
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max(1LL, std::min(b, 152LL * 32));
}

int check_dims(fhmg_problem p) {
  if (!p) return fail(FHMG_EINVAL, "null problem");
  return FHMG_OK;
}

int record_event(fhmg_problem p) {
  if (p->ev_used == p->ev.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    p->ev.push_back(e);
  }
  CK(cudaEventRecord(p->ev[p->ev_used++], p->st));
  return FHMG_OK;
}

// ---------------------------------------------------------------- driver steps (FP64)

int sweep(fhmg_problem p, int l, double* u, const double* F) {
  LevelData& lv = p->lev[l];
  for (int colour = 0; colour < 2; ++colour) {
    const long long nc = fhmg::colour_count(p->dim, lv.N, colour);
    if (nc == 0) continue;
    Geo g{p->dim, lv.N, colour, lv.npts, lv.inv_h2};
    int tc = lv.tc_smooth[colour] ? lv.tc_smooth[colour] : pick_tc(p->h64.d, nc);
    const bool rec = p->profile && l == p->nlev - 1;
    if (rec) TRY(record_event(p));
    TRY(launch_walk<double, fhmg::MODE_SMOOTH>(p, p->h64.d, tc, g, nc, u, F, nullptr, lv.Dinv64, nullptr));
    if (rec) TRY(record_event(p));
  }
  return FHMG_OK;
}

// rc = FW(F - A_h u) - R~ FW(u) on level l-1
int restrict_defect(fhmg_problem p, int l, const double* u, const double* F, double* rc) {
  LevelData& lv = p->lev[l];
  LevelData& lc = p->lev[l - 1];
  const long long n = lc.npts * p->M;
  fhmg::restrict_pre_kernel<double><<<blocks_for(n), 256, 0, p->st>>>(p->dim, lv.N, lv.inv_h2, p->M, u, F, p->Xs, rc);
  ++p->launches;
  CK(cudaGetLastError());
  Geo g{0, 0, 0, lc.npts, 0.0};
  int tc = lc.tc_matvec ? lc.tc_matvec : pick_tc(p->h64.d, lc.npts);
  return launch_walk<double, fhmg::MODE_MATVEC>(p, p->h64.d, tc, g, lc.npts, p->Xs, rc, rc, nullptr, nullptr);
}

int prolong_add(fhmg_problem p, int l, const double* e, double* u) {
  const long long n = p->lev[l].npts * p->M;
  fhmg::prolong_add_kernel<double><<<blocks_for(n), 256, 0, p->st>>>(p->dim, p->lev[l].N, p->M, e, u);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int vcycle_rec(fhmg_problem p, int l, double* u, const double* F, int nu1, int nu2) {
  if (l == 0) return sweep(p, 0, u, F);  // one interior point: the colour-0 solve is exact
  for (int s = 0; s < nu1; ++s) TRY(sweep(p, l, u, F));
  LevelData& lc = p->lev[l - 1];
  TRY(restrict_defect(p, l, u, F, lc.RC));
  CK(cudaMemsetAsync(lc.E, 0, sizeof(double) * lc.npts * p->M, p->st));
  TRY(vcycle_rec(p, l - 1, lc.E, lc.RC, nu1, nu2));
  TRY(prolong_add(p, l, lc.E, u));
  for (int s = 0; s < nu2; ++s) TRY(sweep(p, l, u, F));
  return FHMG_OK;
}

// max |F - A_{h,tau} u| on the finest grid; colour0_only after a completed red-black sweep
// (the defect then vanishes on colour 1 up to rounding).
int fine_norm(fhmg_problem p, const double* u, const double* F, bool colour0_only, double* out) {
  LevelData& lv = p->lev[p->nlev - 1];
  CK(cudaMemsetAsync(p->dnorm, 0, sizeof(unsigned long long), p->st));
  if (colour0_only && lv.npts > 1) {
    const long long nc = fhmg::colour_count(p->dim, lv.N, 0);
    fhmg::gather_defect_kernel<double><<<blocks_for(nc * p->M), 256, 0, p->st>>>(p->dim, lv.N, 0, lv.inv_h2, p->M, u, F,
                                                                                  p->Xs, p->Rs);
    ++p->launches;
    CK(cudaGetLastError());
    Geo g{0, 0, 0, nc, 0.0};
    TRY(launch_walk<double, fhmg::MODE_MATVEC>(p, p->h64.d, pick_tc(p->h64.d, nc), g, nc, p->Xs, p->Rs, nullptr,
                                               nullptr, p->dnorm));
  } else {
    fhmg::gather_defect_kernel<double><<<blocks_for(lv.npts * p->M), 256, 0, p->st>>>(p->dim, lv.N, -1, lv.inv_h2, p->M,
                                                                                       u, F, nullptr, p->Rs);
    ++p->launches;
    CK(cudaGetLastError());
    Geo g{0, 0, 0, lv.npts, 0.0};
    TRY(launch_walk<double, fhmg::MODE_MATVEC>(p, p->h64.d, pick_tc(p->h64.d, lv.npts), g, lv.npts,
                                               const_cast<double*>(u), p->Rs, nullptr, nullptr, p->dnorm));
  }
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, p->dnorm, sizeof bits, cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  double v;
  std::memcpy(&v, &bits, sizeof v);
  *out = v;
  return FHMG_OK;
}

// F = f + d g into the problem's buffer (or f itself when g is NULL)
int full_rhs(fhmg_problem p, const double* f, const double* g, const double** F) {
  if (!f) return fail(FHMG_EINVAL, "f is NULL");
  if (!g) {
    *F = f;
    return FHMG_OK;
  }
  const long long npts = p->lev[p->nlev - 1].npts;
  if (!p->Ff) TRY(dalloc(p->allocs, &p->Ff, (size_t)npts * p->M));
  fhmg::add_initial_kernel<double><<<blocks_for(npts * p->M), 256, 0, p->st>>>(npts, p->M, f, p->dmm, g, p->Ff);
  ++p->launches;
  CK(cudaGetLastError());
  *F = p->Ff;
  return FHMG_OK;
}

__global__ void scale_kernel(double* y, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] *= a;
}

}  // namespace

// ================================================================ C-ABI

extern "C" {

const char* fhmg_last_error(void) { return g_err.c_str(); }

int fhmg_build_hmatrix(double alpha, double gamma, double T, int M, int leaf, int rank, double tol,
                       fhmg_hmatrix* out) {
  if (!out) return fail(FHMG_EINVAL, "out is NULL");
  if (!(leaf == 16 || leaf == 32 || leaf == 64) && leaf < M)
    return fail(FHMG_EINVAL, "leaf must be 16, 32 or 64 (got %d)", leaf);
  int L = std::min(leaf, M);
  if (!(L == 16 || L == 32 || L == 64)) return fail(FHMG_EINVAL, "leaf size min(leaf, M) = %d not in {16,32,64}", L);
  fhmg_hmatrix h = new (std::nothrow) fhmg_hmatrix_s;
  if (!h) return fail(FHMG_ENOMEM, "host allocation failed");
  if (fhmg::build_hmatrix(alpha, gamma, T, M, leaf, rank, tol, h->host) != 0) {
    delete h;
    return fail(FHMG_EINVAL,
                "invalid arguments: need 0<alpha<1, gamma>=1, T>0, M = leaf*2^p, 0<=rank<=64, tol>=0");
  }
  fhmg::flatten(h->host, h->flat);
  *out = h;
  return FHMG_OK;
}

int fhmg_hmatrix_info(fhmg_hmatrix h, int* n_dense, int* n_lowrank, int* max_rank, size_t* bytes) {
  if (!h) return fail(FHMG_EINVAL, "null hmatrix");
  if (n_dense) *n_dense = (int)h->host.dense.size();
  if (n_lowrank) *n_lowrank = (int)h->host.rk.size();
  if (max_rank) *max_rank = h->host.max_rank;
  if (bytes)
    *bytes = sizeof(double) * (h->flat.dense_data.size() + h->flat.udata.size() + h->flat.vdata.size());
  return FHMG_OK;
}

int fhmg_hmatrix_mesh(fhmg_hmatrix h, double* t_out, double* dmm_out) {
  if (!h) return fail(FHMG_EINVAL, "null hmatrix");
  if (t_out) std::memcpy(t_out, h->host.t.data(), sizeof(double) * h->host.t.size());
  if (dmm_out) std::memcpy(dmm_out, h->host.dmm.data(), sizeof(double) * h->host.dmm.size());
  return FHMG_OK;
}

int fhmg_hmatrix_dense(fhmg_hmatrix h, double* R) {
  if (!h || !R) return fail(FHMG_EINVAL, "null argument");
  const int M = h->host.M, L = h->host.L;
  std::memset(R, 0, sizeof(double) * M * M);
  for (auto& d : h->host.dense)
    for (int r = 0; r < L; ++r)
      for (int c = 0; c < L; ++c) R[(size_t)(d.bi * L + r) * M + d.bj * L + c] = d.D[(size_t)r * L + c];
  for (auto& b : h->host.rk)
    for (int r = b.r0; r < b.r1; ++r)
      for (int c = b.c0; c < b.c1; ++c) {
        double s = 0.0;
        for (int k = 0; k < b.k; ++k) s += b.U[(size_t)(r - b.r0) * b.k + k] * b.V[(size_t)(c - b.c0) * b.k + k];
        R[(size_t)r * M + c] = s;
      }
  return FHMG_OK;
}

int fhmg_hmatrix_flops(fhmg_hmatrix h, double* flops_per_column) {
  if (!h || !flops_per_column) return fail(FHMG_EINVAL, "null argument");
  *flops_per_column = (double)h->flat.flops_per_col_matvec;
  return FHMG_OK;
}

int fhmg_hmatrix_destroy(fhmg_hmatrix h) {
  delete h;
  return FHMG_OK;
}

int fhmg_problem_destroy(fhmg_problem p) {
  if (!p) return FHMG_OK;
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  for (void* a : p->allocs) cudaFree(a);
  for (void* a : p->h64.allocs) cudaFree(a);
  for (void* a : p->h32.allocs) cudaFree(a);
  delete p;
  return FHMG_OK;
}

int fhmg_problem_create(fhmg_hmatrix h, int dim, int N, double Lx, int prec, void* stream, fhmg_problem* out) {
  if (!h || !out) return fail(FHMG_EINVAL, "null argument");
  if (dim != 1 && dim != 2) return fail(FHMG_EINVAL, "dim must be 1 or 2");
  if (N < 1 || ((N + 1) & N) != 0) return fail(FHMG_EINVAL, "N must be 2^levels - 1 (got %d)", N);
  if (!(Lx > 0)) return fail(FHMG_EINVAL, "Lx must be > 0");
  if (prec != FHMG_FP64 && prec != FHMG_MIXED_FP32) return fail(FHMG_EINVAL, "unknown precision %d", prec);
  fhmg_problem p = new (std::nothrow) fhmg_problem_s;
  if (!p) return fail(FHMG_ENOMEM, "host allocation failed");
  p->H = h;
  p->dim = dim;
  p->N = N;
  p->Lx = Lx;
  p->prec = prec;
  p->st = (cudaStream_t)stream;
  p->M = h->host.M;
  p->L = h->host.L;
  p->nb = h->host.nb;
  int nlev = 0;
  while ((1 << nlev) - 1 < N) ++nlev;
  p->nlev = nlev;
  p->lev.resize(nlev);
  int st = FHMG_OK;
  auto bail = [&](int s) {
    fhmg_problem_destroy(p);
    return s;
  };
  if ((st = upload_h(h->flat, p->h64)) != FHMG_OK) return bail(st);
  if (prec == FHMG_MIXED_FP32 && (st = upload_h(h->flat, p->h32)) != FHMG_OK) return bail(st);
  const int M = p->M;
  for (int l = 0; l < nlev; ++l) {
    LevelData& lv = p->lev[l];
    lv.N = (1 << (l + 1)) - 1;
    lv.npts = dim == 1 ? lv.N : (long long)lv.N * lv.N;
    lv.h = Lx / (lv.N + 1);
    lv.inv_h2 = 1.0 / (lv.h * lv.h);
    lv.shift = (dim == 1 ? 2.0 : 4.0) * lv.inv_h2;
    std::vector<double> inv;
    fhmg::diag_inverses(h->host, h->flat, lv.shift, inv);
    std::vector<double> invT(inv.size());
    for (int i = 0; i < p->nb; ++i) transpose_into(&inv[(size_t)i * p->L * p->L], &invT[(size_t)i * p->L * p->L], p->L, p->L);
    const double* d64;
    if ((st = upload(p->allocs, invT, &d64, nullptr)) != FHMG_OK) return bail(st);
    lv.Dinv64 = const_cast<double*>(d64);
    if (prec == FHMG_MIXED_FP32) {
      const float* d32;
      if ((st = upload(p->allocs, invT, &d32, nullptr)) != FHMG_OK) return bail(st);
      lv.Dinv32 = const_cast<float*>(d32);
    }
    if (l < nlev - 1) {
      if ((st = dalloc(p->allocs, &lv.E, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
      if ((st = dalloc(p->allocs, &lv.RC, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
    }
  }
  const LevelData& fine = p->lev[nlev - 1];
  long long c0 = fhmg::colour_count(dim, N, 0);
  long long coarse = nlev > 1 ? p->lev[nlev - 2].npts : 1;
  if ((st = dalloc(p->allocs, &p->Xs, (size_t)std::max(c0, coarse) * M)) != FHMG_OK) return bail(st);
  if ((st = dalloc(p->allocs, &p->Rs, (size_t)fine.npts * M)) != FHMG_OK) return bail(st);
  const double* dm;
  if ((st = upload(p->allocs, h->host.dmm, &dm, nullptr)) != FHMG_OK) return bail(st);
  p->dmm = const_cast<double*>(dm);
  if ((st = dalloc(p->allocs, &p->dnorm, 1)) != FHMG_OK) return bail(st);
  if (walk_smem<double>(p->L, 1, p->h64.d.pool) > 200 * 1024) return bail(fail(FHMG_EINVAL, "H-matrix z-pool too large"));
  *out = p;
  return FHMG_OK;
}

int fhmg_problem_autotune(fhmg_problem p) { return check_dims(p); }

int fhmg_problem_profile(fhmg_problem p, int enable) {
  TRY(check_dims(p));
  CK(cudaStreamSynchronize(p->st));
  p->profile = enable != 0;
  p->ev_used = 0;
  p->launches = 0;
  return FHMG_OK;
}

int fhmg_problem_counters(fhmg_problem p, long long* launches, long long* smooth_launches, double* smooth_ms) {
  TRY(check_dims(p));
  CK(cudaStreamSynchronize(p->st));
  double ms = 0.0;
  for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
    float x = 0.f;
    CK(cudaEventElapsedTime(&x, p->ev[i], p->ev[i + 1]));
    ms += x;
  }
  if (launches) *launches = p->launches;
  if (smooth_launches) *smooth_launches = (long long)(p->ev_used / 2);
  if (smooth_ms) *smooth_ms = ms;
  return FHMG_OK;
}

int fhmg_line_solve(fhmg_problem p, int level, double* X, const double* B, long long ncols) {
  TRY(check_dims(p));
  if (level < 0 || level >= p->nlev) return fail(FHMG_EINVAL, "level out of range");
  if (!X || !B || ncols < 0) return fail(FHMG_EINVAL, "bad arrays");
  Geo g{0, 0, 0, ncols, 0.0};
  return launch_walk<double, fhmg::MODE_SMOOTH>(p, p->h64.d, pick_tc(p->h64.d, ncols), g, ncols, X, B, nullptr,
                                                p->lev[level].Dinv64, nullptr);
}

int fhmg_hmatvec(fhmg_problem p, double* Y, const double* X, long long ncols) {
  TRY(check_dims(p));
  if (!X || !Y || ncols < 0 || X == Y) return fail(FHMG_EINVAL, "bad arrays");
  CK(cudaMemsetAsync(Y, 0, sizeof(double) * ncols * p->M, p->st));
  Geo g{0, 0, 0, ncols, 0.0};
  TRY(launch_walk<double, fhmg::MODE_MATVEC>(p, p->h64.d, pick_tc(p->h64.d, ncols), g, ncols,
                                             const_cast<double*>(X), Y, Y, nullptr, nullptr));
  scale_kernel<<<blocks_for(ncols * p->M), 256, 0, p->st>>>(Y, ncols * p->M, -1.0);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int fhmg_smooth(fhmg_problem p, double* u, const double* F, int nsweeps) {
  TRY(check_dims(p));
  if (!u || !F || nsweeps < 0) return fail(FHMG_EINVAL, "bad arguments");
  for (int s = 0; s < nsweeps; ++s) TRY(sweep(p, p->nlev - 1, u, F));
  return FHMG_OK;
}

int fhmg_residual(fhmg_problem p, const double* u, const double* f, const double* g, double* r) {
  TRY(check_dims(p));
  if (!u || !r) return fail(FHMG_EINVAL, "bad arrays");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  LevelData& lv = p->lev[p->nlev - 1];
  fhmg::gather_defect_kernel<double><<<blocks_for(lv.npts * p->M), 256, 0, p->st>>>(p->dim, lv.N, -1, lv.inv_h2, p->M, u, F,
                                                                                     nullptr, r);
  ++p->launches;
  CK(cudaGetLastError());
  Geo geo{0, 0, 0, lv.npts, 0.0};
  return launch_walk<double, fhmg::MODE_MATVEC>(p, p->h64.d, pick_tc(p->h64.d, lv.npts), geo, lv.npts,
                                                const_cast<double*>(u), r, r, nullptr, nullptr);
}

int fhmg_restrict_residual(fhmg_problem p, const double* u, const double* F, double* rc) {
  TRY(check_dims(p));
  if (p->nlev < 2) return fail(FHMG_EINVAL, "no coarser grid");
  if (!u || !F || !rc) return fail(FHMG_EINVAL, "bad arrays");
  return restrict_defect(p, p->nlev - 1, u, F, rc);
}

int fhmg_prolong_correct(fhmg_problem p, double* u, const double* e) {
  TRY(check_dims(p));
  if (p->nlev < 2) return fail(FHMG_EINVAL, "no coarser grid");
  if (!u || !e) return fail(FHMG_EINVAL, "bad arrays");
  return prolong_add(p, p->nlev - 1, e, u);
}

int fhmg_vcycle(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2) {
  TRY(check_dims(p));
  if (!u || nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0) return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  return vcycle_rec(p, p->nlev - 1, u, F, nu1, nu2);
}

int fhmg_residual_norm(fhmg_problem p, const double* u, const double* f, const double* g, double* out) {
  TRY(check_dims(p));
  if (!u || !out) return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  double v;
  TRY(fine_norm(p, u, F, false, &v));
  *out = v;
  return FHMG_OK;
}

int fhmg_solve(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2, double rtol,
               int max_cycles, int* cycles_out, double* relres_out) {
  TRY(check_dims(p));
  if (!u || nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0 || !(rtol >= 0) || max_cycles < 0)
    return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  double r0, r;
  TRY(fine_norm(p, u, F, false, &r0));
  if (!std::isfinite(r0)) return fail(FHMG_ENAN, "initial residual is not finite");
  r = r0;
  int k = 0;
  while (r > rtol * r0 && k < max_cycles) {
    TRY(vcycle_rec(p, p->nlev - 1, u, F, nu1, nu2));
    TRY(fine_norm(p, u, F, nu2 > 0, &r));
    ++k;
    if (!std::isfinite(r)) return fail(FHMG_ENAN, "residual became non-finite after %d cycles", k);
  }
  if (cycles_out) *cycles_out = k;
  if (relres_out) *relres_out = r0 > 0 ? r / r0 : 0.0;
  if (r > rtol * r0) return fail(FHMG_ENOTCONV, "relative residual %.3e after %d cycles", r0 > 0 ? r / r0 : 0.0, k);
  return FHMG_OK;
}

int fhmg_solve_host(fhmg_problem p, double* u_host, const double* f_host, const double* g_host, int nu1, int nu2,
                    double rtol, int max_cycles, int* cycles_out, double* relres_out) {
  TRY(check_dims(p));
  if (!u_host || !f_host) return fail(FHMG_EINVAL, "bad arrays");
  const size_t n = (size_t)p->lev[p->nlev - 1].npts * p->M;
  const size_t ng = (size_t)p->lev[p->nlev - 1].npts;
  if (!p->hu) TRY(dalloc(p->allocs, &p->hu, n));
  if (!p->hf) TRY(dalloc(p->allocs, &p->hf, n));
  if (g_host && !p->hg) TRY(dalloc(p->allocs, &p->hg, ng));
  CK(cudaMemcpyAsync(p->hu, u_host, n * sizeof(double), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->hf, f_host, n * sizeof(double), cudaMemcpyHostToDevice, p->st));
  if (g_host) CK(cudaMemcpyAsync(p->hg, g_host, ng * sizeof(double), cudaMemcpyHostToDevice, p->st));
  int st = fhmg_solve(p, p->hu, p->hf, g_host ? p->hg : nullptr, nu1, nu2, rtol, max_cycles, cycles_out, relres_out);
  if (st != FHMG_OK && st != FHMG_ENOTCONV) return st;
  CK(cudaMemcpyAsync(u_host, p->hu, n * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return st;
}

}  // extern "C"
