// C-ABI and V-cycle driver (Algorithm 2) over the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "coarse.cuh"
#include "fhmg.h"
#include "hbuild.h"
#include "kernels.cuh"
#include "walk.h"

using fhmg::Geo;

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

#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return fail(FHMG_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));       \
  } while (0)
#define TRY(...)                    \
  do {                              \
    int s_ = (__VA_ARGS__);         \
    if (s_ != FHMG_OK) return s_;   \
  } while (0)

}  // namespace

struct fhmg_hmatrix_s {
  fhmg::HostH host;
  fhmg::FlatH flat;
};

namespace {

struct DevPanel {
  std::vector<void*> allocs;
  fhmg::PanelDev d{};
  size_t bytes = 0;
};

struct LevelData {
  int N = 0;
  long long npts = 0;
  double h = 0, inv_h2 = 0, shift = 0;
  double* E = nullptr;         // unknown of the coarse-grid correction (coarse levels)
  double* RC = nullptr;        // restricted defect (coarse levels)
  float* E32 = nullptr;        // FP32 copies for the FP32 inner cycles of the mixed path
  float* RC32 = nullptr;
  double* Dinv64 = nullptr;    // (D_ii + s I)^{-1}, FP64, in the chunk layout (to_panel_layout)
  float* Dinv32 = nullptr;     // the same in FP32 without its diagonal (mixed path)
  float* Dinv32m = nullptr;    // ... and as TF32 hi/lo pairs in the tensor-core layout (to_mma_layout)
  uint16_t* Dinv32u = nullptr; // ... and as BF16 in the tcgen05 layout (to_umma_layout; BF16 problems)
  double* dinvdiag = nullptr;  // the inverses' diagonal, FP64 (mixed path) ...
  float* dinvdiag32 = nullptr; // ... and FP32 (FP32 inner cycles)
};

}  // namespace

struct fhmg_problem_s {
  fhmg_hmatrix H = nullptr;
  int dev = 0;  // the CUDA device the problem was created on (made current by every call)
  int dim = 1, N = 0, nlev = 0, prec = 0;
  double Lx = 1.0;
  cudaStream_t st = nullptr;
  int M = 0, L = 0, nb = 0;
  DevPanel panel64;  // chunk stream, FP64 matrices
  DevPanel panel32;  // chunk stream, FP32 matrices (mixed path)
  DevPanel panel32m; // the same in the tensor-core layout (build_panel_mma)
  DevPanel panel64df; // FP64-accurate products in double-float arithmetic (build_panel_df)
  DevPanel panel32u;  // BF16 products on tcgen05 for the FP32-storage walks (build_panel_umma; BF16 problems)
  int defect_df = 1;  // mixed path, outer FP64 defect: 0 DFMA products, 1 double-float walk, 2 digit
                      // splitting on the tensor cores (where split_ok)
  // tensor-core defect by digit splitting (build_split): digit tiles of the dense R~, pair table,
  // row exponents, per-point exponent scratch; mixed problems with M a multiple of 128, M <= 512
  const unsigned char* spAt = nullptr;
  const int* spPairs = nullptr;
  const int* spRexp = nullptr;
  int* spFe = nullptr;
  double sp_mma_flops = 0;  // BF16 tensor-core flops one split defect executes per grid point
  int use_mma = 1;   // FP32 products on the tensor cores where the column tile allows
  double* rdiag = nullptr;  // FP64 diagonal of R~'s diagonal blocks (mixed path) ...
  float* rdiag32 = nullptr; // ... and its FP32 copy (FP32 inner cycles)
  std::vector<LevelData> lev;
  double* Xs = nullptr;  // scratch, >= max(colour-0 count, coarse count) * M
  double* Rs = nullptr;  // scratch, fine points * M (defect)
  double* Ef = nullptr;  // fine-grid correction of the mixed path
  float* Xs32 = nullptr; // FP32 inner cycles of the mixed path: scratch, defect, correction
  float* Rs32 = nullptr;
  float* Ef32 = nullptr;
  int mixed_storage = 0; // 0 automatic per level, 1 FP64 storage + FP32 products, 2 FP32 storage
  int rtol_ref = 0;      // stopping test relative to: 0 the initial defect, 1 max |F|
  std::map<std::pair<int, long long>, int> tune;  // autotuned column tiles: (kind*2+mode, ncols) -> TC
  double* Ff = nullptr;  // f + d g when g is given
  double* dmm = nullptr; // d_{m,m}
  unsigned long long* dnorm = nullptr;
  int* derr = nullptr;   // device error word of the panel kernels (bounded-wait timeout)
  double* hu = nullptr;  // device copies for fhmg_solve_host
  double* hf = nullptr;
  double* hg = nullptr;
  int inner = 0;         // inner V-cycles per defect-correction step (0: 2 with FP32 storage, 4 otherwise)
  int cycle_index = 1;   // coarse-grid cycles per level (1: V-cycle, 2: W-cycle)
  long long inj_spin = 0;  // armed test hook: the next walk withholds a chunk, consumers poll inj_spin times
  std::vector<void*> allocs;
  // exact coarse-level solve (fhmg_problem_set_coarse_direct), FP64
  int ndirect = 1;              // grid size per dimension solved exactly (1: recursion to one point)
  int lcd = -1;                 // its level index (< nlev - 1), -1: none
  double2* dTw = nullptr;       // FFT twiddles exp(-2 pi i j / P), j < P/2, P = 2 (n + 1)
  double* dModeInv = nullptr;   // (D_ii + lam_k I)^{-1}: modes x nb x L x L, DIAG chunk layout
  float* dModeInvDF = nullptr;  // the same as float pairs (mixed problems: double-float mode solves)
  double* dCA = nullptr;        // scratch, M x points of that level
  double* dCB = nullptr;
  std::vector<void*> dallocs;   // the buffers above
  long long launches = 0;       // kernel launches issued (all kernels)
  bool profile = false;         // record events around finest-level smoother walks
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  size_t ev_used = 0;
  std::vector<cudaEvent_t> evd; // start/stop pairs around finest-grid FP64 defect products
  size_t evd_used = 0;
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

// Uploads the chunk stream of the H-matrix (elem_bytes 8: FP64 products, 4: FP32 products,
// 0: FP32 products in the tensor-core layout, -1: FP64-accurate double-float products, -2: BF16
// products in the tcgen05 layout).
int upload_panel(const fhmg::HostH& h, const fhmg::FlatH& f, int elem_bytes, DevPanel& D) {
  fhmg::PanelHost ph;
  if (elem_bytes == -2)
    fhmg::build_panel_umma(h, f, ph);
  else if (elem_bytes == 0)
    fhmg::build_panel_mma(h, f, ph);
  else if (elem_bytes < 0)
    fhmg::build_panel_df(h, f, ph);
  else
    fhmg::build_panel(h, f, elem_bytes, ph);
  const unsigned char* pkg;
  const int* chunks;
  const int* cptr;
  TRY(upload(D.allocs, ph.pkg, &pkg, &D.bytes));
  TRY(upload(D.allocs, ph.chunks, &chunks, &D.bytes));
  TRY(upload(D.allocs, ph.cptr, &cptr, &D.bytes));
  D.d.pkg = pkg;
  D.d.chunks = reinterpret_cast<const int4*>(chunks);
  D.d.cptr = cptr;
  D.d.nb = f.nb;
  D.d.L = f.L;
  D.d.pool = f.pool_rows;
  D.d.W = ph.W;
  D.d.slot_bytes = ph.slot_bytes;
  D.d.ns = 2;
  D.d.far = ph.far ? 1 : 0;
  return FHMG_OK;
}

int blocks_for(long long n) { return fhmg::grid_for(n, 32); }

// R~ as a dense row-major M x M matrix (near-field blocks as stored, low-rank blocks expanded)
void dense_of(const fhmg::HostH& h, std::vector<double>& R) {
  const int M = h.M, L = h.L;
  R.assign((size_t)M * M, 0.0);
  for (auto& d : h.dense)
    for (int r = 0; r < L; ++r)
      for (int c = 0; c < L; ++c) R[(size_t)(d.bi * L + r) * M + d.bj * L + c] = d.D[(size_t)r * L + c];
  for (auto& b : h.rk)
    for (int r = b.r0; r < b.r1; ++r)
      for (int c = b.c0; c < b.c1; ++c) {
        double s = 0.0;
        for (int k = 0; k < b.k; ++k) s += b.U[(size_t)(r - b.r0) * b.k + k] * b.V[(size_t)(c - b.c0) * b.k + k];
        R[(size_t)r * M + c] = s;
      }
}

// Launch shapes of the grid-function kernels (kernels.cuh): points along x, rows along y, time
// levels strided along z.
dim3 coarse_grid(int dim, int Nf, int M) {
  const int Nc = (Nf - 1) / 2;
  return fhmg::plane_grid(Nc, dim == 1 ? 1 : Nc, M, fhmg::device_sms());
}
dim3 fine_grid(int dim, int N, int M) { return fhmg::plane_grid(N, dim == 1 ? 1 : N, M, fhmg::device_sms()); }
dim3 colour_grid(int dim, int N, int M) {
  return fhmg::plane_grid((N + 1) / 2, dim == 1 ? 1 : N, M, fhmg::device_sms());
}

int check_dims(fhmg_problem p) {
  if (!p) return fail(FHMG_EINVAL, "null problem");
  return FHMG_OK;
}

// Makes a device current for the scope of a call and restores the caller's device afterwards.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Entry of every call on a problem: argument check, then the problem's device made current.
#define ENTER(p)                                                                             \
  TRY(check_dims(p));                                                                        \
  DeviceScope dev_scope_((p)->dev);                                                          \
  if (!dev_scope_.ok) return fail(FHMG_ECUDA, "cannot make the problem's device current")

int record_event(fhmg_problem p, std::vector<cudaEvent_t>& ev, size_t& used) {
  if (used == ev.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ev.push_back(e);
  }
  CK(cudaEventRecord(ev[used++], p->st));
  return FHMG_OK;
}

double pair_ms(const std::vector<cudaEvent_t>& ev, size_t used) {
  double ms = 0.0;
  for (size_t i = 0; i + 1 < used; i += 2) {
    float x = 0.f;
    if (cudaEventElapsedTime(&x, ev[i], ev[i + 1]) == cudaSuccess) ms += x;
  }
  return ms;
}

int walk_status(int s, const std::string& err) {
  if (s == 0) return FHMG_OK;
  return fail(s == 1 ? FHMG_ECUDA : FHMG_EINVAL, "%s", err.c_str());
}

// Arithmetic of a walk: K64 FP64 storage and products; KSPLIT FP64 storage, FP32 products;
// K32 FP32 storage and products (inner cycles on well-conditioned grids).
// KDF: FP64-accurate products in double-float arithmetic (FP64 arrays; products only).
enum { K64 = 0, KSPLIT = 1, K32 = 2, KDF = 3 };

// Column tile chosen by the autotuner for (kind, mode, ncols), 0 if none (automatic).
int tuned_tile(fhmg_problem p, int kind, int mode, long long nc) {
  auto it = p->tune.find(std::make_pair(kind * 2 + mode, nc));
  return it == p->tune.end() ? 0 : it->second;
}

// per-type level buffers
template <typename T> T* lev_E(LevelData& lv);
template <> double* lev_E<double>(LevelData& lv) { return lv.E; }
template <> float* lev_E<float>(LevelData& lv) { return lv.E32; }
template <typename T> T* lev_RC(LevelData& lv);
template <> double* lev_RC<double>(LevelData& lv) { return lv.RC; }
template <> float* lev_RC<float>(LevelData& lv) { return lv.RC32; }
template <typename T> T* scratch_X(fhmg_problem p);
template <> double* scratch_X<double>(fhmg_problem p) { return p->Xs; }
template <> float* scratch_X<float>(fhmg_problem p) { return p->Xs32; }

// A smoother half-sweep / line-solve job on level l (shift of that level).
template <typename T>
fhmg::WalkArgsT<T> smooth_job(fhmg_problem p, int l, int kind, const Geo& g, long long nc, T* X, const T* B) {
  LevelData& lv = p->lev[l];
  fhmg::WalkArgsT<T> a{};
  a.P = kind == K64 ? p->panel64.d : p->panel32.d;
  if (kind != K64 && p->use_mma && p->panel32m.d.pkg) {
    a.PM = p->panel32m.d;
    a.DinvM = lv.Dinv32m;
  }
  a.mode = fhmg::MODE_SMOOTH;
  a.geo = g;
  a.ncols = nc;
  a.X = X;
  a.B = B;
  a.OUT = nullptr;
  a.Dinv = kind == K64 ? (const void*)lv.Dinv64 : (const void*)lv.Dinv32;
  // FP32 products leave the diagonal out of the streamed blocks; it is applied in T
  a.ddiag = kind == KSPLIT ? (const T*)lv.dinvdiag : kind == K32 ? (const T*)lv.dinvdiag32 : nullptr;
  a.norm = nullptr;
  a.err = p->derr;
  a.tile = tuned_tile(p, kind, fhmg::MODE_SMOOTH, nc);
  if (kind == K32 && p->panel32u.d.pkg) {
    a.PU = p->panel32u.d;
    a.DinvU = lv.Dinv32u;
  }
  return a;
}

// A product job: OUT = B - R~ X on nc compact columns (OUT may alias B or be NULL).
template <typename T>
fhmg::WalkArgsT<T> matvec_job(fhmg_problem p, int kind, long long nc, const T* X, const T* B, T* OUT,
                              unsigned long long* norm) {
  fhmg::WalkArgsT<T> a{};
  a.P = kind == K64 ? p->panel64.d : kind == KDF ? p->panel64df.d : p->panel32.d;
  if ((kind == KSPLIT || kind == K32) && p->use_mma && p->panel32m.d.pkg) a.PM = p->panel32m.d;
  a.mode = fhmg::MODE_MATVEC;
  a.geo = Geo{0, 0, 0, nc, 0.0};
  a.ncols = nc;
  a.X = const_cast<T*>(X);
  a.B = B;
  a.OUT = OUT;
  a.Dinv = nullptr;
  a.ddiag = kind == KSPLIT ? (const T*)p->rdiag : kind == K32 ? (const T*)p->rdiag32 : nullptr;
  a.norm = norm;
  a.err = p->derr;
  a.tile = tuned_tile(p, kind, fhmg::MODE_MATVEC, nc);
  if (kind == K32 && p->panel32u.d.pkg) a.PU = p->panel32u.d;
  return a;
}

// Launches a list of jobs of one kind and mode on stream st: one persistent kernel per group of
// up to kMaxJobs jobs with the same leaf size (the tile of each group's first job applies).
int launch_jobs(cudaStream_t st, int kind, std::vector<fhmg::WalkArgsT<double>>& jobs, long long* counter) {
  std::vector<fhmg::WalkArgsT<double>> live;
  for (auto& j : jobs)
    if (j.ncols > 0) live.push_back(j);
  std::stable_sort(live.begin(), live.end(), [](const fhmg::WalkArgsT<double>& x, const fhmg::WalkArgsT<double>& y) {
    return x.P.L < y.P.L;
  });
  size_t i = 0;
  while (i < live.size()) {
    size_t e = i;
    while (e < live.size() && live[e].P.L == live[i].P.L && e - i < (size_t)fhmg::kMaxJobs) ++e;
    std::string err;
    int s = kind == KSPLIT ? fhmg::walk_launch_df(st, &live[i], (int)(e - i), &err, nullptr)
            : kind == KDF  ? fhmg::walk_launch_dfprod(st, &live[i], (int)(e - i), &err, nullptr)
                           : fhmg::walk_launch_dd(st, &live[i], (int)(e - i), &err, nullptr);
    TRY(walk_status(s, err));
    if (counter) ++*counter;
    i = e;
  }
  return FHMG_OK;
}

// FP32-storage walks: BF16 problems run wide panels (every SM gets a 128-column tile) on the
// tcgen05 walk, everything else on the FP32-product walks.
int launch_jobs(cudaStream_t st, int, std::vector<fhmg::WalkArgsT<float>>& jobs, long long* counter) {
  for (auto& j : jobs) {
    if (j.ncols <= 0) continue;
    std::string err;
    int s = 2;
    if (j.PU.pkg && j.ncols >= 128LL * fhmg::device_sms()) s = fhmg::walk_launch_umma(st, &j, 1, &err);
    if (s == 2) s = fhmg::walk_launch_ff(st, &j, 1, &err, nullptr);
    TRY(walk_status(s, err));
    if (counter) ++*counter;
  }
  return FHMG_OK;
}

// The armed timeout test hook (fhmg_problem_inject_timeout) applies to the next walk only.
template <typename T>
void apply_injection(fhmg_problem p, fhmg::WalkArgsT<T>& a) {
  if (p->inj_spin <= 0) return;
  a.spin = p->inj_spin;
  a.withhold = 2;  // the second chunk of every CTA's stream is never issued
  p->inj_spin = 0;
}

template <typename T>
int walk_smooth(fhmg_problem p, int l, int kind, const Geo& g, long long nc, T* X, const T* B) {
  std::vector<fhmg::WalkArgsT<T>> j{smooth_job<T>(p, l, kind, g, nc, X, B)};
  apply_injection(p, j[0]);
  return launch_jobs(p->st, kind, j, &p->launches);
}

template <typename T>
int walk_matvec(fhmg_problem p, int kind, long long nc, const T* X, const T* B, T* OUT, unsigned long long* norm) {
  std::vector<fhmg::WalkArgsT<T>> j{matvec_job<T>(p, kind, nc, X, B, OUT, norm)};
  apply_injection(p, j[0]);
  return launch_jobs(p->st, kind, j, &p->launches);
}

// ---------------------------------------------------------------- driver steps

template <typename T>
int sweep(fhmg_problem p, int l, T* u, const T* F, int kind) {
  LevelData& lv = p->lev[l];
  for (int colour = 0; colour < 2; ++colour) {
    const long long nc = fhmg::colour_count(p->dim, lv.N, colour);
    if (nc == 0) continue;
    Geo g{p->dim, lv.N, colour, lv.npts, lv.inv_h2};
    const bool rec = p->profile && l == p->nlev - 1;
    if (rec) TRY(record_event(p, p->ev, p->ev_used));
    TRY(walk_smooth<T>(p, l, kind, g, nc, u, F));
    if (rec) TRY(record_event(p, p->ev, p->ev_used));
  }
  return FHMG_OK;
}

// rc = FW(F - A_h u) - R~ FW(u) on level l-1
template <typename T>
int restrict_defect(fhmg_problem p, int l, const T* u, const T* F, T* rc, int kind) {
  LevelData& lv = p->lev[l];
  LevelData& lc = p->lev[l - 1];
  T* xs = scratch_X<T>(p);
  fhmg::restrict_pre_kernel<T><<<coarse_grid(p->dim, lv.N, p->M), 256, 0, p->st>>>(p->dim, lv.N, lv.inv_h2, p->M, u, F,
                                                                                  xs, rc);
  ++p->launches;
  CK(cudaGetLastError());
  return walk_matvec<T>(p, kind, lc.npts, xs, rc, rc, nullptr);
}

template <typename T>
int prolong_add(fhmg_problem p, int l, const T* e, T* u) {
  fhmg::prolong_add_kernel<T><<<fine_grid(p->dim, p->lev[l].N, p->M), 256, 0, p->st>>>(p->dim, p->lev[l].N, p->M, e, u);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

// E = exact solution of the level-l system for the right-hand side RC (FP64 throughout):
// sine transform in space, one triangular H-matrix walk per spatial mode, inverse transform.
template <typename T>
int direct_level(fhmg_problem p, int l, T* E, const T* RC) {
  const LevelData& lv = p->lev[l];
  const int n = lv.N;
  const long long M = p->M;
  int log2P = 1;
  while ((1 << log2P) < 2 * (n + 1)) ++log2P;
  const int P = 1 << log2P;
  const int thr = std::min(256, std::max(32, P / 2));
  const size_t smem = 3 * (size_t)P * sizeof(double);
  // sine transform along x (M * ny lines) and, in 2D, along y (M * nx lines)
  const unsigned lines_x = (unsigned)(M * (p->dim == 2 ? n : 1)), lines_y = (unsigned)(M * n);
  if (p->dim == 1) {
    fhmg::sine_fft_kernel<T, double><<<lines_x, thr, smem, p->st>>>(RC, p->dCA, p->dTw, M, 1, n, 0, log2P);
  } else {
    fhmg::sine_fft_kernel<T, double><<<lines_x, thr, smem, p->st>>>(RC, p->dCB, p->dTw, M, n, n, 0, log2P);
    fhmg::sine_fft_kernel<double, double><<<lines_y, thr, smem, p->st>>>(p->dCB, p->dCA, p->dTw, M, n, n, 1, log2P);
    ++p->launches;
  }
  ++p->launches;
  CK(cudaGetLastError());
  // mixed problems: the mode solves in FP64-accurate double-float arithmetic (FP32 pipe)
  const bool df = p->dModeInvDF && p->defect_df;
  fhmg::WalkArgsT<double> a{};
  a.P = df ? p->panel64df.d : p->panel64.d;
  a.mode = fhmg::MODE_SMOOTH;
  a.geo = Geo{0, 0, 0, lv.npts, 0.0};  // compact columns, no stencil: X = (R~ + lam I)^{-1} B
  a.ncols = lv.npts;
  a.X = p->dCB;
  a.B = p->dCA;
  a.Dinv = df ? (const void*)p->dModeInvDF : (const void*)p->dModeInv;
  a.dinv_cstride = (long long)p->nb * p->L * p->L * (df ? 2 : 1);
  a.err = p->derr;
  a.tile = 1;
  std::vector<fhmg::WalkArgsT<double>> j{a};
  TRY(launch_jobs(p->st, df ? KDF : K64, j, &p->launches));
  if (p->dim == 1) {
    fhmg::sine_fft_kernel<double, T><<<lines_x, thr, smem, p->st>>>(p->dCB, E, p->dTw, M, 1, n, 0, log2P);
  } else {
    fhmg::sine_fft_kernel<double, double><<<lines_y, thr, smem, p->st>>>(p->dCB, p->dCA, p->dTw, M, n, n, 1, log2P);
    fhmg::sine_fft_kernel<double, T><<<lines_x, thr, smem, p->st>>>(p->dCA, E, p->dTw, M, n, n, 0, log2P);
    ++p->launches;
  }
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

// FP32 nearest to an FP64 value (ties away from zero), by integer operations: the conversion
// instruction runs on the FP64 pipe, 1/64 of the FP32 rate on GB300.  Below the FP32 normal range: 0;
// above it, and Inf / NaN: Inf / NaN.
__device__ __forceinline__ float d2f_int(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 2047) return __uint_as_float(sign | 0x7F800000u | ((b & 0xFFFFFFFFFFFFFULL) ? 0x400000u : 0u));
  int fe = e - 1023 + 127;
  if (e == 0 || fe <= 0) return __uint_as_float(sign);
  unsigned long long q = (((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52)) + (1ULL << 28)) >> 29;
  if (q >> 24) {
    q >>= 1;
    ++fe;
  }
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((uint32_t)fe << 23) | (uint32_t)(q & 0x7FFFFF));
}

__global__ void to_float_kernel(const double* x, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = d2f_int(x[i]);
}
__global__ void to_double_kernel(const float* x, double* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
__global__ void add_float_kernel(double* y, const float* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += (double)x[i];
}

// Storage of a coarse-grid correction on level l inside FP64-storage inner cycles (automatic
// mixed storage only): FP32 where the stencil's conditioning allows it,
// eps32 * cond(A_h) ~ 6e-8 * 4 (N+1)^2 / pi^2 <= 0.05 (N <= 1023 per dimension).
bool level_fp32(fhmg_problem p, int l) {
  if (p->mixed_storage != 0) return false;
  const double n1 = p->lev[l].N + 1.0;
  return 6e-8 * 4.0 * n1 * n1 / (M_PI * M_PI) <= 0.05;
}

template <typename T>
int vcycle_rec(fhmg_problem p, int l, T* u, const T* F, int nu1, int nu2, int kind);

// The coarse-grid correction of level l (restricted defect in RC of level l - 1, result in E of
// level l - 1): exact solve, FP32-storage cycle, or the recursion in T.
template <typename T>
int coarse_correction(fhmg_problem p, int l, int nu1, int nu2, int kind) {
  LevelData& lc = p->lev[l - 1];
  const long long n = lc.npts * p->M;
  if (l - 1 == p->lcd) return direct_level<T>(p, l - 1, lev_E<T>(lc), lev_RC<T>(lc));
  // cycle index: the coarse problem gets cycle_index cycles (W-cycle: 2) unless it is the
  // one-point level, whose solve is exact
  const int reps = l - 1 > 0 ? p->cycle_index : 1;
  if constexpr (std::is_same<T, double>::value) {
    if (kind == KSPLIT && level_fp32(p, l - 1)) {
      to_float_kernel<<<blocks_for(n), 256, 0, p->st>>>(lc.RC, lc.RC32, n);
      ++p->launches;
      CK(cudaGetLastError());
      CK(cudaMemsetAsync(lc.E32, 0, sizeof(float) * n, p->st));
      for (int r = 0; r < reps; ++r) TRY(vcycle_rec<float>(p, l - 1, lc.E32, lc.RC32, nu1, nu2, K32));
      to_double_kernel<<<blocks_for(n), 256, 0, p->st>>>(lc.E32, lc.E, n);
      ++p->launches;
      CK(cudaGetLastError());
      return FHMG_OK;
    }
  }
  CK(cudaMemsetAsync(lev_E<T>(lc), 0, sizeof(T) * n, p->st));
  for (int r = 0; r < reps; ++r) TRY(vcycle_rec<T>(p, l - 1, lev_E<T>(lc), lev_RC<T>(lc), nu1, nu2, kind));
  return FHMG_OK;
}

template <typename T>
int vcycle_rec(fhmg_problem p, int l, T* u, const T* F, int nu1, int nu2, int kind) {
  if (l == 0) return sweep<T>(p, 0, u, F, kind);  // one interior point: the colour-0 solve is exact
  for (int s = 0; s < nu1; ++s) TRY(sweep<T>(p, l, u, F, kind));
  LevelData& lc = p->lev[l - 1];
  TRY(restrict_defect<T>(p, l, u, F, lev_RC<T>(lc), kind));
  TRY(coarse_correction<T>(p, l, nu1, nu2, kind));
  TRY(prolong_add<T>(p, l, lev_E<T>(lc), u));
  for (int s = 0; s < nu2; ++s) TRY(sweep<T>(p, l, u, F, kind));
  return FHMG_OK;
}

// A walk that gave up set the problem's error word: report it once (FHMG_ETIMEOUT) and clear it,
// so that the problem stays usable.
int report_timeout(fhmg_problem p) {
  CK(cudaMemsetAsync(p->derr, 0, sizeof(int), p->st));
  CK(cudaStreamSynchronize(p->st));
  return fail(FHMG_ETIMEOUT, "a walk kernel gave up waiting on a shared-memory stage");
}

int read_norm(fhmg_problem p, double* out) {
  unsigned long long bits = 0;
  int derr = 0;
  CK(cudaMemcpyAsync(&bits, p->dnorm, sizeof bits, cudaMemcpyDeviceToHost, p->st));
  CK(cudaMemcpyAsync(&derr, p->derr, sizeof derr, cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  if (derr) return report_timeout(p);
  double v;
  std::memcpy(&v, &bits, sizeof v);
  *out = v;
  return FHMG_OK;
}

// Products of the FP64 defect on the finest grid: double-float for mixed problems (unless set
// to FP64 by fhmg_problem_set_defect_arith), FP64 otherwise.
int defect_kind(fhmg_problem p) {
  return (p->prec != FHMG_FP64 && p->defect_df && p->panel64df.d.pkg) ? KDF : K64;
}

// The full FP64-accurate defect on the finest grid into dst (all points), its max-norm folded into
// *norm_word (zeroed by the caller): the tensor-core digit splitting where the problem has it
// (defect arithmetic 2), else the stencil gather and the walk of defect_kind.
int full_defect(fhmg_problem p, const double* u, const double* F, double* dst, unsigned long long* norm_word) {
  LevelData& lv = p->lev[p->nlev - 1];
  if (p->prec != FHMG_FP64 && p->defect_df == 2 && p->spAt) {
    fhmg::SplitArgs a{};
    a.U = u;
    a.F = F;
    a.OUT = dst;
    a.norm = norm_word;
    a.fe = p->spFe;
    a.At = p->spAt;
    a.pairs = reinterpret_cast<const int4*>(p->spPairs);
    a.rexp = p->spRexp;
    a.err = p->derr;
    a.ld = lv.npts;
    a.dim = p->dim;
    a.N = lv.N;
    a.M = p->M;
    a.inv_h2 = lv.inv_h2;
    if (p->inj_spin > 0) {
      a.spin = p->inj_spin;
      a.withhold = 2;
      p->inj_spin = 0;
    }
    if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
    std::string err;
    const int s = fhmg::split_defect_launch(p->st, a, &err);
    p->launches += 2;
    if (s == 1) return fail(FHMG_ECUDA, "%s", err.c_str());
    if (s == 0) {
      if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
      return FHMG_OK;
    }
    return fail(FHMG_EINVAL, "%s", err.c_str());
  }
  fhmg::gather_defect_kernel<double><<<fine_grid(p->dim, lv.N, p->M), 256, 0, p->st>>>(p->dim, lv.N, -1, lv.inv_h2,
                                                                                    p->M, u, F, nullptr, dst);
  ++p->launches;
  CK(cudaGetLastError());
  if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
  TRY(walk_matvec<double>(p, defect_kind(p), lv.npts, u, dst, dst, norm_word));
  if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
  return FHMG_OK;
}

// FP64 defect on the finest grid.  colour0_only (after a completed red-black sweep the defect
// vanishes on colour 1 up to rounding): max-norm over colour 0 only, nothing stored.
// Otherwise the full defect is written to R (if R != NULL) and its max-norm returned.
int fine_defect(fhmg_problem p, const double* u, const double* F, bool colour0_only, double* R, double* out) {
  LevelData& lv = p->lev[p->nlev - 1];
  CK(cudaMemsetAsync(p->dnorm, 0, sizeof(unsigned long long), p->st));
  if (colour0_only && lv.npts > 1) {
    const long long nc = fhmg::colour_count(p->dim, lv.N, 0);
    fhmg::gather_defect_kernel<double><<<colour_grid(p->dim, lv.N, p->M), 256, 0, p->st>>>(p->dim, lv.N, 0, lv.inv_h2,
                                                                                        p->M, u, F, p->Xs, p->Rs);
    ++p->launches;
    CK(cudaGetLastError());
    if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
    TRY(walk_matvec<double>(p, K64, nc, p->Xs, p->Rs, nullptr, p->dnorm));
    if (p->profile) TRY(record_event(p, p->evd, p->evd_used));
  } else {
    TRY(full_defect(p, u, F, R ? R : p->Rs, p->dnorm));
  }
  return read_norm(p, out);
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
  fhmg::add_initial_kernel<double><<<fhmg::plane_grid(npts, 1, p->M, fhmg::device_sms()), 256, 0, p->st>>>(
      npts, p->M, f, p->dmm, g, p->Ff);
  ++p->launches;
  CK(cudaGetLastError());
  *F = p->Ff;
  return FHMG_OK;
}

__global__ void axpy_kernel(double* y, const double* x, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

int axpy(fhmg_problem p, double* y, const double* x, long long n, double a) {
  axpy_kernel<<<blocks_for(n), 256, 0, p->st>>>(y, x, n, a);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

// FP64 path: V-cycles on u until the colour-0 defect norm is below rtol * ||r_0||.
int absmax(fhmg_problem p, const double* x, long long n, double* out);

int solve_fp64(fhmg_problem p, double* u, const double* F, int nu1, int nu2, double rtol, int max_cycles, int* kout,
               double* r0out, double* rout) {
  double r0, r;
  TRY(fine_defect(p, u, F, false, nullptr, &r0));
  if (!std::isfinite(r0)) return fail(FHMG_ENAN, "initial residual is not finite");
  r = r0;
  if (p->rtol_ref) TRY(absmax(p, F, p->lev[p->nlev - 1].npts * p->M, &r0));
  int k = 0;
  while (r > rtol * r0 && k < max_cycles) {
    TRY(vcycle_rec<double>(p, p->nlev - 1, u, F, nu1, nu2, K64));
    TRY(fine_defect(p, u, F, nu2 > 0, nullptr, &r));
    ++k;
    if (!std::isfinite(r)) return fail(FHMG_ENAN, "residual became non-finite after %d cycles", k);
  }
  *kout = k;
  *r0out = r0;
  *rout = r;
  return FHMG_OK;
}


// max |x| as FP64 bits: with the sign cleared, the order of the bit patterns is the order of the
// magnitudes and a NaN compares above every number, so no floating-point operation is needed
__global__ void absmax_kernel(const double* x, long long n, unsigned long long* out) {
  const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(x);
  unsigned long long m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = __ldg(xb + i) & 0x7FFFFFFFFFFFFFFFULL;
    m = a > m ? a : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, m, o);
    m = b > m ? b : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// max |x| over n device doubles (FP64, NaN propagates)
int absmax(fhmg_problem p, const double* x, long long n, double* out) {
  CK(cudaMemsetAsync(p->dnorm, 0, sizeof(unsigned long long), p->st));
  absmax_kernel<<<blocks_for(n), 256, 0, p->st>>>(x, n, p->dnorm);
  ++p->launches;
  CK(cudaGetLastError());
  return read_norm(p, out);
}

// Inner storage of the mixed path: FP32 when the grid is well conditioned for it --
// eps32 * cond(A_h) ~ 6e-8 * 4 (N+1)^2 / pi^2 <= 0.05 (the FP32 rounding of a correction then
// perturbs the defect by at most ~5 %), otherwise FP64 storage with FP32 products.
bool inner_fp32(fhmg_problem p) {
  if (p->mixed_storage == 1) return false;
  if (p->mixed_storage == 2) return true;
  const double n1 = p->N + 1.0;
  return 6e-8 * 4.0 * n1 * n1 / (M_PI * M_PI) <= 0.05;
}

// Mixed path (defect correction): r = F - A u in FP64; p->inner V-cycles on A e = r from e = 0
// (FP32 storage and products, or FP64 storage with FP32 products); u += e; repeat until
// ||r|| <= rtol ||r_0|| in FP64.
int solve_mixed(fhmg_problem p, double* u, const double* F, int nu1, int nu2, double rtol, int max_cycles, int* kout,
                double* r0out, double* rout) {
  const long long n = p->lev[p->nlev - 1].npts * p->M;
  const bool f32 = inner_fp32(p);
  double r0, r;
  // a zero initial guess (the common case) has defect F: skip the FP64 product
  double umax;
  TRY(absmax(p, u, n, &umax));
  if (umax == 0.0) {
    TRY(absmax(p, F, n, &r0));
    CK(cudaMemcpyAsync(p->Rs, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->st));
  } else {
    TRY(fine_defect(p, u, F, false, p->Rs, &r0));
  }
  if (!std::isfinite(r0)) return fail(FHMG_ENAN, "initial residual is not finite");
  r = r0;
  if (p->rtol_ref) TRY(absmax(p, F, n, &r0));
  // FP32 storage limits one defect-correction step to ~1e-2 on these grids (two V-cycles reach
  // it); FP64 storage with FP32 products converges like FP64 (four V-cycles ~ 1e-4)
  const int inner = p->inner > 0 ? p->inner : (f32 ? 2 : 4);
  int k = 0;
  double r_prev = -1.0;
  int last = 0;
  while (r > rtol * r0 && k < max_cycles) {
    // cycles of this round: inner, or fewer where the previous round's contraction per cycle says
    // that fewer reach the target with a factor 2 to spare (the last round then runs no cycle the
    // target does not need; each round costs an FP64-accurate defect)
    int cyc = inner;
    if (r_prev > 0.0 && last > 0 && r < r_prev) {
      const double rho = std::pow(r / r_prev, 1.0 / last);
      if (rho > 0.0 && rho < 0.9) {
        const double need = std::log(0.5 * rtol * r0 / r) / std::log(rho);
        if (need < inner) cyc = std::max(1, (int)std::ceil(need));
      }
    }
    const int k_round = k;
    if (f32) {
      to_float_kernel<<<blocks_for(n), 256, 0, p->st>>>(p->Rs, p->Rs32, n);
      ++p->launches;
      CK(cudaGetLastError());
      CK(cudaMemsetAsync(p->Ef32, 0, sizeof(float) * n, p->st));
      for (int j = 0; j < cyc && k < max_cycles; ++j, ++k)
        TRY(vcycle_rec<float>(p, p->nlev - 1, p->Ef32, p->Rs32, nu1, nu2, K32));
      add_float_kernel<<<blocks_for(n), 256, 0, p->st>>>(u, p->Ef32, n);
      ++p->launches;
      CK(cudaGetLastError());
    } else {
      CK(cudaMemsetAsync(p->Ef, 0, sizeof(double) * n, p->st));
      for (int j = 0; j < cyc && k < max_cycles; ++j, ++k)
        TRY(vcycle_rec<double>(p, p->nlev - 1, p->Ef, p->Rs, nu1, nu2, KSPLIT));
      TRY(axpy(p, u, p->Ef, n, 1.0));
    }
    r_prev = r;
    last = k - k_round;
    TRY(fine_defect(p, u, F, false, p->Rs, &r));
    if (!std::isfinite(r)) return fail(FHMG_ENAN, "residual became non-finite after %d cycles", k);
  }
  *kout = k;
  *r0out = r0;
  *rout = r;
  return FHMG_OK;
}

// ---------------------------------------------------------------- batched solves

// One instance at one depth of a lockstep V-cycle.
struct BLev {
  fhmg_problem p;
  int l;
  double* u;
  const double* F;
};

// Smoother sweeps of a set of instances: every colour is ONE launch over all of them.
int batched_sweeps(cudaStream_t st, std::vector<BLev>& set, int nsweeps, int kind, long long* nl) {
  for (int s = 0; s < nsweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      std::vector<fhmg::WalkArgsT<double>> jobs;
      for (auto& b : set) {
        LevelData& lv = b.p->lev[b.l];
        const long long nc = fhmg::colour_count(b.p->dim, lv.N, colour);
        jobs.push_back(smooth_job<double>(b.p, b.l, kind, Geo{b.p->dim, lv.N, colour, lv.npts, lv.inv_h2}, nc, b.u, b.F));
      }
      TRY(launch_jobs(st, kind, jobs, nl));
    }
  return FHMG_OK;
}

// V-cycle of every instance in lockstep by depth below its finest grid (instances with fewer
// levels reach their coarsest grid earlier).  Capturable: no host synchronisation.
int batched_vcycle(cudaStream_t st, std::vector<BLev> cur, int nu1, int nu2, int kind, long long* nl) {
  std::vector<BLev> coarse, rest;
  for (auto& b : cur) (b.l == 0 ? coarse : rest).push_back(b);
  if (!coarse.empty()) TRY(batched_sweeps(st, coarse, 1, kind, nl));  // the one-point exact solve
  if (rest.empty()) return FHMG_OK;
  TRY(batched_sweeps(st, rest, nu1, kind, nl));
  std::vector<fhmg::WalkArgsT<double>> jobs;
  std::vector<BLev> next;
  for (auto& b : rest) {
    LevelData& lv = b.p->lev[b.l];
    LevelData& lc = b.p->lev[b.l - 1];
    const long long n = lc.npts * b.p->M;
    fhmg::restrict_pre_kernel<double><<<coarse_grid(b.p->dim, lv.N, b.p->M), 256, 0, st>>>(b.p->dim, lv.N, lv.inv_h2,
                                                                                         b.p->M, b.u, b.F, b.p->Xs, lc.RC);
    CK(cudaGetLastError());
    ++*nl;
    jobs.push_back(matvec_job<double>(b.p, kind, lc.npts, b.p->Xs, lc.RC, lc.RC, nullptr));
    CK(cudaMemsetAsync(lc.E, 0, sizeof(double) * n, st));
    next.push_back(BLev{b.p, b.l - 1, lc.E, lc.RC});
  }
  TRY(launch_jobs(st, kind, jobs, nl));
  TRY(batched_vcycle(st, next, nu1, nu2, kind, nl));
  for (auto& b : rest) {
    LevelData& lc = b.p->lev[b.l - 1];
    fhmg::prolong_add_kernel<double><<<fine_grid(b.p->dim, b.p->lev[b.l].N, b.p->M), 256, 0, st>>>(
        b.p->dim, b.p->lev[b.l].N, b.p->M, lc.E, b.u);
    CK(cudaGetLastError());
    ++*nl;
  }
  return batched_sweeps(st, rest, nu2, kind, nl);
}

// FP64 defects of a set of instances (all points) into R_k, their max-norms into each dnorm;
// one product launch for all of them.
int batched_defects(cudaStream_t st, std::vector<BLev>& set, std::vector<double*>& R, long long* nl) {
  std::vector<fhmg::WalkArgsT<double>> jobs;
  for (size_t i = 0; i < set.size(); ++i) {
    fhmg_problem p = set[i].p;
    LevelData& lv = p->lev[p->nlev - 1];
    CK(cudaMemsetAsync(p->dnorm, 0, sizeof(unsigned long long), st));
    fhmg::gather_defect_kernel<double><<<fine_grid(p->dim, lv.N, p->M), 256, 0, st>>>(p->dim, lv.N, -1, lv.inv_h2, p->M,
                                                                                   set[i].u, set[i].F, nullptr, R[i]);
    CK(cudaGetLastError());
    ++*nl;
    jobs.push_back(matvec_job<double>(p, K64, lv.npts, set[i].u, R[i], R[i], p->dnorm));
  }
  return launch_jobs(st, K64, jobs, nl);
}

// FP64 colour-0 defect norms (after completed sweeps) of a set of instances.
int batched_colour0_norms(cudaStream_t st, std::vector<BLev>& set, long long* nl) {
  std::vector<fhmg::WalkArgsT<double>> jobs;
  for (auto& b : set) {
    fhmg_problem p = b.p;
    LevelData& lv = p->lev[p->nlev - 1];
    const long long nc = fhmg::colour_count(p->dim, lv.N, 0);
    CK(cudaMemsetAsync(p->dnorm, 0, sizeof(unsigned long long), st));
    fhmg::gather_defect_kernel<double><<<colour_grid(p->dim, lv.N, p->M), 256, 0, st>>>(p->dim, lv.N, 0, lv.inv_h2, p->M,
                                                                                     b.u, b.F, p->Xs, p->Rs);
    CK(cudaGetLastError());
    ++*nl;
    jobs.push_back(matvec_job<double>(p, K64, nc, p->Xs, p->Rs, nullptr, p->dnorm));
  }
  return launch_jobs(st, K64, jobs, nl);
}

int read_norms(cudaStream_t st, std::vector<BLev>& set, std::vector<double>& out) {
  std::vector<unsigned long long> bits(set.size());
  std::vector<int> errs(set.size());
  for (size_t i = 0; i < set.size(); ++i) {
    CK(cudaMemcpyAsync(&bits[i], set[i].p->dnorm, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&errs[i], set[i].p->derr, 4, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  out.resize(set.size());
  for (size_t i = 0; i < set.size(); ++i)
    if (errs[i]) return report_timeout(set[i].p);
  for (size_t i = 0; i < set.size(); ++i) std::memcpy(&out[i], &bits[i], 8);
  return FHMG_OK;
}

// A CUDA graph of one lockstep V-cycle of a fixed set of instances.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

int capture_cycle(cudaStream_t st, std::vector<BLev>& set, int nu1, int nu2, int kind, long long* nl, CycleGraph& g) {
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  // first run outside the capture: configures kernel attributes (shared-memory opt-in)
  TRY(batched_vcycle(st, set, nu1, nu2, kind, nl));
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  long long dummy = 0;
  int s = batched_vcycle(st, set, nu1, nu2, kind, &dummy);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (s != FHMG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(FHMG_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(FHMG_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  return FHMG_OK;
}

__global__ void scale_kernel(double* y, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] *= a;
}

}  // namespace

// Internal hook for entry points that supply their own scratch (noalloc.cu): the FP64 defect of
// u against F at every finest-grid point written to B (device, M * N^dim doubles), its max-norm
// folded into *norm_word (zeroed here) and returned in *out.  Launches kernels and copies 8 bytes
// to the host; allocates nothing.
int fhmg_internal_defect_norm(fhmg_problem p, const double* u, const double* F, double* B,
                              unsigned long long* norm_word, double* out) {
  ENTER(p);
  LevelData& lv = p->lev[p->nlev - 1];
  CK(cudaMemsetAsync(norm_word, 0, sizeof(unsigned long long), p->st));
  TRY(full_defect(p, u, F, B, norm_word));
  unsigned long long bits = 0;
  int derr = 0;
  CK(cudaMemcpyAsync(&bits, norm_word, sizeof bits, cudaMemcpyDeviceToHost, p->st));
  CK(cudaMemcpyAsync(&derr, p->derr, sizeof derr, cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  if (derr) return report_timeout(p);
  std::memcpy(out, &bits, sizeof bits);
  return FHMG_OK;
}

long long fhmg_internal_grid_elems(fhmg_problem p) { return p->lev[p->nlev - 1].npts * (long long)p->M; }

int fhmg_internal_problem_device(fhmg_problem p) { return p->dev; }

int fhmg_internal_problem_geom(fhmg_problem p, int* dim, int* N, int* M, double* Lx, void** stream,
                               const double** t_host) {
  if (!p) return fail(FHMG_EINVAL, "null problem");
  *dim = p->dim;
  *N = p->N;
  *M = p->M;
  *Lx = p->Lx;
  *stream = (void*)p->st;
  *t_host = p->H->host.t.data();
  return FHMG_OK;
}
int fhmg_internal_fail(int code, const char* msg) { return fail(code, "%s", msg); }

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

int fhmg_build_hmatrix_aca(double alpha, double gamma, double T, int M, int leaf, double tol, fhmg_hmatrix* out) {
  if (!out) return fail(FHMG_EINVAL, "out is NULL");
  if (!(tol > 0.0)) return fail(FHMG_EINVAL, "tol must be > 0");
  const int L = std::min(leaf, M);
  if (!(L == 16 || L == 32 || L == 64)) return fail(FHMG_EINVAL, "leaf size min(leaf, M) = %d not in {16,32,64}", L);
  fhmg_hmatrix h = new (std::nothrow) fhmg_hmatrix_s;
  if (!h) return fail(FHMG_ENOMEM, "host allocation failed");
  if (fhmg::build_hmatrix(alpha, gamma, T, M, leaf, 0, tol, h->host, 1) != 0) {
    delete h;
    return fail(FHMG_EINVAL, "invalid arguments: need 0<alpha<1, gamma>=1, T>0, M = leaf*2^p, tol>0");
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
  std::vector<double> D;
  dense_of(h->host, D);
  std::memcpy(R, D.data(), sizeof(double) * D.size());
  return FHMG_OK;
}

int fhmg_hmatrix_flops(fhmg_hmatrix h, double* flops_per_column) {
  if (!h || !flops_per_column) return fail(FHMG_EINVAL, "null argument");
  *flops_per_column = (double)h->flat.flops_per_col_matvec;
  return FHMG_OK;
}

int fhmg_hmatrix_split_digits(fhmg_hmatrix h, unsigned short* tiles, long long* n_tiles, int* pairs, int* rexp) {
  if (!h || !n_tiles) return fail(FHMG_EINVAL, "null argument");
  const int M = h->host.M;
  if (M % fhmg::kSplitRows != 0 || M > fhmg::kSplitMaxM)
    return fail(FHMG_EINVAL, "digit splitting needs M a multiple of %d and M <= %d (M = %d)", fhmg::kSplitRows,
                fhmg::kSplitMaxM, M);
  std::vector<double> D;
  dense_of(h->host, D);
  fhmg::SplitHost sp;
  fhmg::build_split(D, M, sp);
  const long long nt = (long long)(sp.tiles.size() / ((size_t)fhmg::kSplitRows * 64));
  if (tiles) {
    if (*n_tiles < nt) return fail(FHMG_EINVAL, "tiles holds %lld tiles, %lld needed", *n_tiles, nt);
    std::memcpy(tiles, sp.tiles.data(), sizeof(uint16_t) * sp.tiles.size());
  }
  *n_tiles = nt;
  if (pairs) std::memcpy(pairs, sp.pairs.data(), sizeof(int) * sp.pairs.size());
  if (rexp) std::memcpy(rexp, sp.rexp.data(), sizeof(int) * sp.rexp.size());
  return FHMG_OK;
}

int fhmg_sama_two_grid(fhmg_hmatrix h, int dim, int N, double Lx, int nu1, int nu2, double* rho_out) {
  if (!h || !rho_out) return fail(FHMG_EINVAL, "null argument");
  if (dim != 1 && dim != 2) return fail(FHMG_EINVAL, "dim must be 1 or 2");
  if (N < 3 || ((N + 1) & N) != 0) return fail(FHMG_EINVAL, "N must be 2^levels - 1 >= 3 (got %d)", N);
  if (!(Lx > 0) || nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0) return fail(FHMG_EINVAL, "bad arguments");
  const int L = h->host.L;
  std::vector<double> rdiag((size_t)h->host.M);
  for (int i = 0; i < h->host.nb; ++i)
    for (int r = 0; r < L; ++r) rdiag[(size_t)i * L + r] = h->host.dense[h->host.diag[i]].D[(size_t)r * L + r];
  *rho_out = fhmg::sama_two_grid(rdiag, dim, N, Lx / (N + 1), nu1, nu2);
  return FHMG_OK;
}

int fhmg_hmatrix_destroy(fhmg_hmatrix h) {
  delete h;
  return FHMG_OK;
}

int fhmg_problem_destroy(fhmg_problem p) {
  if (!p) return FHMG_OK;
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : p->evd) cudaEventDestroy(e);
  for (void* a : p->allocs) cudaFree(a);
  for (void* a : p->dallocs) cudaFree(a);
  for (void* a : p->panel64.allocs) cudaFree(a);
  for (void* a : p->panel32.allocs) cudaFree(a);
  for (void* a : p->panel32m.allocs) cudaFree(a);
  for (void* a : p->panel64df.allocs) cudaFree(a);
  for (void* a : p->panel32u.allocs) cudaFree(a);
  delete p;
  return FHMG_OK;
}

int fhmg_problem_create(fhmg_hmatrix h, int dim, int N, double Lx, int prec, void* stream, fhmg_problem* out) {
  if (!h || !out) return fail(FHMG_EINVAL, "null argument");
  if (dim != 1 && dim != 2) return fail(FHMG_EINVAL, "dim must be 1 or 2");
  if (N < 1 || ((N + 1) & N) != 0) return fail(FHMG_EINVAL, "N must be 2^levels - 1 (got %d)", N);
  if (!(Lx > 0)) return fail(FHMG_EINVAL, "Lx must be > 0");
  if (prec != FHMG_FP64 && prec != FHMG_MIXED_FP32 && prec != FHMG_MIXED_BF16)
    return fail(FHMG_EINVAL, "unknown precision %d", prec);
  fhmg_problem p = new (std::nothrow) fhmg_problem_s;
  if (!p) return fail(FHMG_ENOMEM, "host allocation failed");
  p->H = h;
  p->dim = dim;
  p->N = N;
  p->Lx = Lx;
  p->prec = prec;
  p->st = (cudaStream_t)stream;
  if (cudaGetDevice(&p->dev) != cudaSuccess) {
    delete p;
    return fail(FHMG_ECUDA, "cudaGetDevice failed");
  }
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
  const bool mixed = prec != FHMG_FP64;
  const bool umma = prec == FHMG_MIXED_BF16 && p->L == fhmg::kUmmaL;
  if ((st = upload_panel(h->host, h->flat, 8, p->panel64)) != FHMG_OK) return bail(st);
  if (mixed) {
    if (umma && (st = upload_panel(h->host, h->flat, -2, p->panel32u)) != FHMG_OK) return bail(st);
    if ((st = upload_panel(h->host, h->flat, 4, p->panel32)) != FHMG_OK) return bail(st);
    if (p->L == 64 && (st = upload_panel(h->host, h->flat, 0, p->panel32m)) != FHMG_OK) return bail(st);
    if ((st = upload_panel(h->host, h->flat, -1, p->panel64df)) != FHMG_OK) return bail(st);
    std::vector<double> rd((size_t)p->nb * p->L);
    for (int i = 0; i < p->nb; ++i)
      for (int r = 0; r < p->L; ++r) rd[(size_t)i * p->L + r] = h->host.dense[h->host.diag[i]].D[(size_t)r * p->L + r];
    const double* d;
    if ((st = upload(p->allocs, rd, &d, nullptr)) != FHMG_OK) return bail(st);
    p->rdiag = const_cast<double*>(d);
    const float* d32;
    if ((st = upload(p->allocs, rd, &d32, nullptr)) != FHMG_OK) return bail(st);
    p->rdiag32 = const_cast<float*>(d32);
    if (p->M % fhmg::kSplitRows == 0 && p->M <= fhmg::kSplitMaxM) {
      std::vector<double> Rd;
      dense_of(h->host, Rd);
      fhmg::SplitHost sh;
      fhmg::build_split(Rd, p->M, sh);
      const unsigned char* at;
      std::vector<unsigned char> bytes(sh.tiles.size() * 2);
      std::memcpy(bytes.data(), sh.tiles.data(), bytes.size());
      if ((st = upload(p->allocs, bytes, &at, nullptr)) != FHMG_OK) return bail(st);
      p->spAt = at;
      if ((st = upload(p->allocs, sh.pairs, &p->spPairs, nullptr)) != FHMG_OK) return bail(st);
      if ((st = upload(p->allocs, sh.rexp, &p->spRexp, nullptr)) != FHMG_OK) return bail(st);
      long long npts = 1;
      for (int d = 0; d < dim; ++d) npts *= N;
      if ((st = dalloc(p->allocs, &p->spFe, (size_t)npts)) != FHMG_OK) return bail(st);
      // per 64-point tile: every stored digit tile a of a pair meets the u digits b < 7 - a in one
      // 128 x 64 x 64 product each
      double fl = 0;
      for (size_t q = 0; q < sh.pairs.size(); q += 4)
        for (int a = 0; a < 7; ++a)
          if ((sh.pairs[q] >> a) & 1) fl += (7 - a) * 2.0 * 128 * 64 * 64;
      p->sp_mma_flops = fl / 64;
      p->defect_df = 2;
    }
  }
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
    const size_t LL = (size_t)p->L * p->L;
    std::vector<double> invP(inv.size());
    for (int i = 0; i < p->nb; ++i) fhmg::to_panel_layout(&inv[i * LL], p->L, 8, false, &invP[i * LL]);
    const double* d64;
    if ((st = upload(p->allocs, invP, &d64, nullptr)) != FHMG_OK) return bail(st);
    lv.Dinv64 = const_cast<double*>(d64);
    if (mixed) {
      for (int i = 0; i < p->nb; ++i) fhmg::to_panel_layout(&inv[i * LL], p->L, 4, true, &invP[i * LL]);
      const float* d32;
      if ((st = upload(p->allocs, invP, &d32, nullptr)) != FHMG_OK) return bail(st);
      lv.Dinv32 = const_cast<float*>(d32);
      std::vector<double> dg((size_t)p->nb * p->L);
      for (int i = 0; i < p->nb; ++i)
        for (int r = 0; r < p->L; ++r) dg[(size_t)i * p->L + r] = inv[(size_t)i * p->L * p->L + (size_t)r * p->L + r];
      const double* dd;
      if ((st = upload(p->allocs, dg, &dd, nullptr)) != FHMG_OK) return bail(st);
      lv.dinvdiag = const_cast<double*>(dd);
      const float* dd32;
      if ((st = upload(p->allocs, dg, &dd32, nullptr)) != FHMG_OK) return bail(st);
      lv.dinvdiag32 = const_cast<float*>(dd32);
      if (umma) {
        std::vector<uint16_t> u(inv.size());
        for (int i = 0; i < p->nb; ++i) fhmg::to_umma_layout(&inv[i * LL], p->L, true, &u[i * LL]);
        uint16_t* du;
        if ((st = dalloc(p->allocs, &du, u.size())) != FHMG_OK) return bail(st);
        if (cudaMemcpy(du, u.data(), u.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
          return bail(fail(FHMG_ECUDA, "cudaMemcpy failed"));
        lv.Dinv32u = du;
      }
      if (p->L == 64) {
        std::vector<float> m(inv.size() * 2);
        for (int i = 0; i < p->nb; ++i) fhmg::to_mma_layout(&inv[i * LL], p->L, true, &m[i * LL * 2]);
        const float* dm;
        if ((st = upload(p->allocs, m, &dm, nullptr)) != FHMG_OK) return bail(st);
        lv.Dinv32m = const_cast<float*>(dm);
      }
    }
    if (l < nlev - 1) {
      if ((st = dalloc(p->allocs, &lv.E, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
      if ((st = dalloc(p->allocs, &lv.RC, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
      if (mixed) {
        if ((st = dalloc(p->allocs, &lv.E32, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
        if ((st = dalloc(p->allocs, &lv.RC32, (size_t)lv.npts * M)) != FHMG_OK) return bail(st);
      }
    }
  }
  const LevelData& fine = p->lev[nlev - 1];
  long long c0 = fhmg::colour_count(dim, N, 0);
  long long coarse = nlev > 1 ? p->lev[nlev - 2].npts : 1;
  if ((st = dalloc(p->allocs, &p->Xs, (size_t)std::max(c0, coarse) * M)) != FHMG_OK) return bail(st);
  if ((st = dalloc(p->allocs, &p->Rs, (size_t)fine.npts * M)) != FHMG_OK) return bail(st);
  if (mixed) {
    if ((st = dalloc(p->allocs, &p->Ef, (size_t)fine.npts * M)) != FHMG_OK) return bail(st);
    if ((st = dalloc(p->allocs, &p->Xs32, (size_t)std::max(c0, coarse) * M)) != FHMG_OK) return bail(st);
    if ((st = dalloc(p->allocs, &p->Rs32, (size_t)fine.npts * M)) != FHMG_OK) return bail(st);
    if ((st = dalloc(p->allocs, &p->Ef32, (size_t)fine.npts * M)) != FHMG_OK) return bail(st);
  }
  const double* dm;
  if ((st = upload(p->allocs, h->host.dmm, &dm, nullptr)) != FHMG_OK) return bail(st);
  p->dmm = const_cast<double*>(dm);
  if ((st = dalloc(p->allocs, &p->dnorm, 1)) != FHMG_OK) return bail(st);
  if ((st = dalloc(p->allocs, &p->derr, 1)) != FHMG_OK) return bail(st);
  if (cudaMemset(p->derr, 0, sizeof(int)) != cudaSuccess) return bail(fail(FHMG_ECUDA, "cudaMemset failed"));
  *out = p;
  return FHMG_OK;
}

// Autotuner: for every walk the solver issues on this problem (smoother colours of every level,
// products on the coarse columns of every restriction, the finest-grid defects), times each
// column tile TC in {1, 2, 4, 8, 16, 32} that fits in shared memory (3 launches each, CUDA
// events, on zeroed workspaces) and records the fastest; later launches use it.
int fhmg_problem_autotune(fhmg_problem p) {
  ENTER(p);
  const int M = p->M;
  const LevelData& fine = p->lev[p->nlev - 1];
  CK(cudaMemsetAsync(p->Rs, 0, sizeof(double) * fine.npts * M, p->st));
  CK(cudaMemsetAsync(p->Xs, 0, sizeof(double) * std::max(fhmg::colour_count(p->dim, p->N, 0),
                                                         p->nlev > 1 ? p->lev[p->nlev - 2].npts : 1) * M, p->st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<int> kinds{K64};
  if (p->prec != FHMG_FP64) kinds.push_back(KSPLIT);
  int st = FHMG_OK;
  auto time_jobs = [&](int kind, fhmg::WalkArgsT<double> job, float* ms) -> int {
    std::vector<fhmg::WalkArgsT<double>> v{job};
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) CK(cudaEventRecord(e0, p->st));
      int s2 = launch_jobs(p->st, kind, v, nullptr);
      if (s2 != FHMG_OK) return s2;
    }
    CK(cudaEventRecord(e1, p->st));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return FHMG_OK;
  };
  for (int kind : kinds) {
    for (int l = 0; l < p->nlev && st == FHMG_OK; ++l) {
      LevelData& lv = p->lev[l];
      for (int mode = 0; mode < 2 && st == FHMG_OK; ++mode) {
        std::vector<long long> cols;
        if (mode == fhmg::MODE_SMOOTH) {
          cols.push_back(fhmg::colour_count(p->dim, lv.N, 0));
          cols.push_back(fhmg::colour_count(p->dim, lv.N, 1));
        } else {
          cols.push_back(lv.npts);  // restriction into this level / full finest defect
          if (l == p->nlev - 1) cols.push_back(fhmg::colour_count(p->dim, lv.N, 0));
        }
        for (size_t ci = 0; ci < cols.size(); ++ci) {
          const long long nc = cols[ci];
          if (nc <= 0 || p->tune.count(std::make_pair(kind * 2 + mode, nc))) continue;
          float best = 1e30f;
          int best_tc = 0;
          for (int tc = 1; tc <= 32; tc *= 2) {
            fhmg::WalkArgsT<double> job =
                mode == fhmg::MODE_SMOOTH
                    ? smooth_job<double>(p, l, kind, Geo{p->dim, lv.N, (int)ci, lv.npts, lv.inv_h2}, nc, p->Rs, p->Rs)
                    : matvec_job<double>(p, kind, nc, p->Rs, p->Rs, nullptr, nullptr);
            job.tile = tc;
            float ms = 0.f;
            int s2 = time_jobs(kind, job, &ms);
            if (s2 == FHMG_EINVAL) continue;  // this tile does not fit
            if (s2 != FHMG_OK) {
              st = s2;
              break;
            }
            if (ms < best) {
              best = ms;
              best_tc = tc;
            }
          }
          if (best_tc) p->tune[std::make_pair(kind * 2 + mode, nc)] = best_tc;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

int fhmg_problem_set_inner(fhmg_problem p, int inner_cycles) {
  ENTER(p);
  if (inner_cycles < 0) return fail(FHMG_EINVAL, "inner_cycles must be >= 0");
  p->inner = inner_cycles;
  return FHMG_OK;
}

int fhmg_problem_set_mixed_storage(fhmg_problem p, int mode) {
  ENTER(p);
  if (mode < 0 || mode > 2) return fail(FHMG_EINVAL, "mixed storage mode must be 0, 1 or 2");
  p->mixed_storage = mode;
  return FHMG_OK;
}

int fhmg_problem_set_coarse_direct(fhmg_problem p, int n) {
  ENTER(p);
  if (n < 0) return fail(FHMG_EINVAL, "coarse direct size must be >= 0");
  int l = -1;
  if (n > 1) {
    for (int q = 0; q < p->nlev - 1; ++q)
      if (p->lev[q].N == n) l = q;
    if (l < 0) return fail(FHMG_EINVAL, "coarse direct size must be a coarse grid size 2^k - 1 below N (got %d)", n);
    if (p->lev[l].npts > 65535) return fail(FHMG_EINVAL, "coarse direct level has more than 65535 points");
  }
  CK(cudaStreamSynchronize(p->st));
  for (void* a : p->dallocs) cudaFree(a);
  p->dallocs.clear();
  p->dModeInv = p->dCA = p->dCB = nullptr;
  p->dModeInvDF = nullptr;
  p->dTw = nullptr;
  p->ndirect = 1;
  p->lcd = -1;
  if (l < 0) return FHMG_OK;
  const LevelData& lv = p->lev[l];
  const int L = p->L, nb = p->nb;
  const double pi = std::acos(-1.0);
  std::vector<double> lam1(n), lam(lv.npts), Dd((size_t)nb * L * L);
  for (int q = 0; q < n; ++q) {
    const double sn = std::sin(pi * (q + 1) / (2.0 * (n + 1)));
    lam1[q] = 4.0 * lv.inv_h2 * sn * sn;
  }
  for (long long m = 0; m < lv.npts; ++m) lam[m] = p->dim == 1 ? lam1[m] : lam1[m / n] + lam1[m % n];
  for (int i = 0; i < nb; ++i)
    std::memcpy(&Dd[(size_t)i * L * L], p->H->host.dense[p->H->host.diag[i]].D.data(), sizeof(double) * L * L);
  const double *dlam, *dDd, *dtw;
  TRY(upload(p->dallocs, lam, &dlam, nullptr));
  TRY(upload(p->dallocs, Dd, &dDd, nullptr));
  const int P = 2 * (n + 1);
  std::vector<double> tw(P);  // (cos, -sin)(2 pi j / P), j < P/2
  for (int j = 0; j < P / 2; ++j) {
    tw[2 * j] = std::cos(2.0 * pi * j / P);
    tw[2 * j + 1] = -std::sin(2.0 * pi * j / P);
  }
  TRY(upload(p->dallocs, tw, &dtw, nullptr));
  p->dTw = reinterpret_cast<double2*>(const_cast<double*>(dtw));
  TRY(dalloc(p->dallocs, &p->dModeInv, (size_t)lv.npts * nb * L * L));
  if (p->prec != FHMG_FP64 && p->panel64df.d.pkg)
    TRY(dalloc(p->dallocs, &p->dModeInvDF, (size_t)lv.npts * nb * 2 * L * L));
  TRY(dalloc(p->dallocs, &p->dCA, (size_t)lv.npts * p->M));
  TRY(dalloc(p->dallocs, &p->dCB, (size_t)lv.npts * p->M));
  const int smem = 2 * L * L * (int)sizeof(double);
  CK(cudaFuncSetAttribute(fhmg::mode_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  fhmg::mode_inverse_kernel<<<dim3(nb, (unsigned)lv.npts), L, smem, p->st>>>(dDd, dlam, L, nb, p->dModeInv, p->dModeInvDF);
  ++p->launches;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->st));
  p->ndirect = n;
  p->lcd = l;
  return FHMG_OK;
}

int fhmg_problem_split_flops(fhmg_problem p, double* per_point) {
  ENTER(p);
  if (!per_point) return fail(FHMG_EINVAL, "null argument");
  if (!p->spAt) return fail(FHMG_EINVAL, "no split defect for this problem");
  *per_point = p->sp_mma_flops;
  return FHMG_OK;
}

int fhmg_problem_set_defect_arith(fhmg_problem p, int mode) {
  ENTER(p);
  if (mode < 0 || mode > 2) return fail(FHMG_EINVAL, "defect arithmetic must be 0 (FP64), 1 (double-float) or 2 (splitting)");
  if (mode == 2 && !p->spAt)
    return fail(FHMG_EINVAL, "defect arithmetic 2 needs a mixed-precision problem with M a multiple of 128, M <= 512");
  p->defect_df = mode;
  return FHMG_OK;
}

int fhmg_problem_set_tensor_cores(fhmg_problem p, int enable) {
  ENTER(p);
  p->use_mma = enable != 0;
  p->tune.clear();  // tuned tiles were timed with the other kernels
  return FHMG_OK;
}

int fhmg_problem_set_rtol_reference(fhmg_problem p, int ref) {
  ENTER(p);
  if (ref != 0 && ref != 1) return fail(FHMG_EINVAL, "reference must be 0 (initial defect) or 1 (max |F|)");
  p->rtol_ref = ref;
  return FHMG_OK;
}

int fhmg_problem_set_cycle_index(fhmg_problem p, int cycle_index) {
  ENTER(p);
  if (cycle_index < 1 || cycle_index > 4) return fail(FHMG_EINVAL, "cycle index must be 1 (V) .. 4 (got %d)", cycle_index);
  p->cycle_index = cycle_index;
  return FHMG_OK;
}

int fhmg_problem_inject_timeout(fhmg_problem p, long long consumer_spin) {
  ENTER(p);
  if (consumer_spin < 1 || consumer_spin > fhmg::kSpinLimit)
    return fail(FHMG_EINVAL, "consumer spin limit must be in 1..2^24");
  p->inj_spin = consumer_spin;
  return FHMG_OK;
}

int fhmg_problem_profile(fhmg_problem p, int enable) {
  ENTER(p);
  CK(cudaStreamSynchronize(p->st));
  p->profile = enable != 0;
  p->ev_used = 0;
  p->evd_used = 0;
  p->launches = 0;
  return FHMG_OK;
}

int fhmg_problem_counters(fhmg_problem p, long long* launches, long long* smooth_launches, double* smooth_ms) {
  ENTER(p);
  CK(cudaStreamSynchronize(p->st));
  if (launches) *launches = p->launches;
  if (smooth_launches) *smooth_launches = (long long)(p->ev_used / 2);
  if (smooth_ms) *smooth_ms = pair_ms(p->ev, p->ev_used);
  return FHMG_OK;
}

int fhmg_problem_defect_timing(fhmg_problem p, long long* defect_launches, double* defect_ms, long long* columns) {
  ENTER(p);
  CK(cudaStreamSynchronize(p->st));
  if (defect_launches) *defect_launches = (long long)(p->evd_used / 2);
  if (defect_ms) *defect_ms = pair_ms(p->evd, p->evd_used);
  if (columns) *columns = p->lev[p->nlev - 1].npts;
  return FHMG_OK;
}

int fhmg_line_solve(fhmg_problem p, int level, double* X, const double* B, long long ncols) {
  ENTER(p);
  if (level < 0 || level >= p->nlev) return fail(FHMG_EINVAL, "level out of range");
  if (!X || !B || ncols < 0) return fail(FHMG_EINVAL, "bad arrays");
  Geo g{0, 0, 0, ncols, 0.0};
  return walk_smooth<double>(p, level, K64, g, ncols, X, B);
}

int fhmg_hmatvec(fhmg_problem p, double* Y, const double* X, long long ncols) {
  ENTER(p);
  if (!X || !Y || ncols < 0 || X == Y) return fail(FHMG_EINVAL, "bad arrays");
  CK(cudaMemsetAsync(Y, 0, sizeof(double) * ncols * p->M, p->st));
  TRY(walk_matvec<double>(p, K64, ncols, X, Y, Y, nullptr));
  scale_kernel<<<blocks_for(ncols * p->M), 256, 0, p->st>>>(Y, ncols * p->M, -1.0);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int fhmg_line_solve_f32(fhmg_problem p, int level, double* X, const double* B, long long ncols, int tile) {
  ENTER(p);
  if (p->prec == FHMG_FP64) return fail(FHMG_EINVAL, "FP32 products need a mixed-precision problem");
  if (level < 0 || level >= p->nlev) return fail(FHMG_EINVAL, "level out of range");
  if (!X || !B || ncols < 0 || tile < 0 || tile > 32 || (tile & (tile - 1)) != 0)
    return fail(FHMG_EINVAL, "bad arguments");
  Geo g{0, 0, 0, ncols, 0.0};
  std::vector<fhmg::WalkArgsT<double>> j{smooth_job<double>(p, level, KSPLIT, g, ncols, X, B)};
  j[0].tile = tile;
  return launch_jobs(p->st, KSPLIT, j, &p->launches);
}

int fhmg_hmatvec_f32(fhmg_problem p, double* Y, const double* X, long long ncols, int tile) {
  ENTER(p);
  if (p->prec == FHMG_FP64) return fail(FHMG_EINVAL, "FP32 products need a mixed-precision problem");
  if (!X || !Y || ncols < 0 || X == Y || tile < 0 || tile > 32 || (tile & (tile - 1)) != 0)
    return fail(FHMG_EINVAL, "bad arguments");
  CK(cudaMemsetAsync(Y, 0, sizeof(double) * ncols * p->M, p->st));
  std::vector<fhmg::WalkArgsT<double>> j{matvec_job<double>(p, KSPLIT, ncols, X, Y, Y, nullptr)};
  j[0].tile = tile;
  TRY(launch_jobs(p->st, KSPLIT, j, &p->launches));
  scale_kernel<<<blocks_for(ncols * p->M), 256, 0, p->st>>>(Y, ncols * p->M, -1.0);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int fhmg_hmatvec_df(fhmg_problem p, double* Y, const double* X, long long ncols, int tile) {
  ENTER(p);
  if (p->prec == FHMG_FP64) return fail(FHMG_EINVAL, "double-float products need a mixed-precision problem");
  if (!X || !Y || ncols < 0 || X == Y || (tile != 0 && tile != 4 && tile != 8 && tile != 16))
    return fail(FHMG_EINVAL, "bad arguments");
  CK(cudaMemsetAsync(Y, 0, sizeof(double) * ncols * p->M, p->st));
  std::vector<fhmg::WalkArgsT<double>> j{matvec_job<double>(p, KDF, ncols, X, Y, Y, nullptr)};
  j[0].tile = tile;
  TRY(launch_jobs(p->st, KDF, j, &p->launches));
  scale_kernel<<<blocks_for(ncols * p->M), 256, 0, p->st>>>(Y, ncols * p->M, -1.0);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int fhmg_line_solve_s(fhmg_problem p, int level, float* X, const float* B, long long ncols) {
  ENTER(p);
  if (p->prec == FHMG_FP64) return fail(FHMG_EINVAL, "FP32-storage walks need a mixed-precision problem");
  if (level < 0 || level >= p->nlev) return fail(FHMG_EINVAL, "level out of range");
  if (!X || !B || ncols < 0) return fail(FHMG_EINVAL, "bad arrays");
  Geo g{0, 0, 0, ncols, 0.0};
  return walk_smooth<float>(p, level, K32, g, ncols, X, B);
}

__global__ void negate_float_kernel(float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = -y[i];
}

int fhmg_hmatvec_s(fhmg_problem p, float* Y, const float* X, long long ncols) {
  ENTER(p);
  if (p->prec == FHMG_FP64) return fail(FHMG_EINVAL, "FP32-storage walks need a mixed-precision problem");
  if (!X || !Y || ncols < 0 || X == Y) return fail(FHMG_EINVAL, "bad arrays");
  CK(cudaMemsetAsync(Y, 0, sizeof(float) * ncols * p->M, p->st));
  TRY(walk_matvec<float>(p, K32, ncols, X, Y, Y, nullptr));
  negate_float_kernel<<<blocks_for(ncols * p->M), 256, 0, p->st>>>(Y, ncols * p->M);
  ++p->launches;
  CK(cudaGetLastError());
  return FHMG_OK;
}

int fhmg_smooth(fhmg_problem p, double* u, const double* F, int nsweeps) {
  ENTER(p);
  if (!u || !F || nsweeps < 0) return fail(FHMG_EINVAL, "bad arguments");
  for (int s = 0; s < nsweeps; ++s) TRY(sweep<double>(p, p->nlev - 1, u, F, K64));
  return FHMG_OK;
}

int fhmg_residual(fhmg_problem p, const double* u, const double* f, const double* g, double* r) {
  ENTER(p);
  if (!u || !r) return fail(FHMG_EINVAL, "bad arrays");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  double nrm;
  return fine_defect(p, u, F, false, r, &nrm);
}

int fhmg_restrict_residual(fhmg_problem p, const double* u, const double* F, double* rc) {
  ENTER(p);
  if (p->nlev < 2) return fail(FHMG_EINVAL, "no coarser grid");
  if (!u || !F || !rc) return fail(FHMG_EINVAL, "bad arrays");
  return restrict_defect<double>(p, p->nlev - 1, u, F, rc, K64);
}

int fhmg_prolong_correct(fhmg_problem p, double* u, const double* e) {
  ENTER(p);
  if (p->nlev < 2) return fail(FHMG_EINVAL, "no coarser grid");
  if (!u || !e) return fail(FHMG_EINVAL, "bad arrays");
  return prolong_add<double>(p, p->nlev - 1, e, u);
}

int fhmg_vcycle(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2) {
  ENTER(p);
  if (!u || nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0) return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  return vcycle_rec<double>(p, p->nlev - 1, u, F, nu1, nu2, K64);
}

int fhmg_residual_norm(fhmg_problem p, const double* u, const double* f, const double* g, double* out) {
  ENTER(p);
  if (!u || !out) return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  double v;
  TRY(fine_defect(p, u, F, false, nullptr, &v));
  *out = v;
  return FHMG_OK;
}

int fhmg_solve(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2, double rtol,
               int max_cycles, int* cycles_out, double* relres_out) {
  ENTER(p);
  if (!u || nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0 || !(rtol >= 0) || max_cycles < 0)
    return fail(FHMG_EINVAL, "bad arguments");
  const double* F;
  TRY(full_rhs(p, f, g, &F));
  int k = 0;
  double r0 = 0, r = 0;
  if (p->prec != FHMG_FP64)
    TRY(solve_mixed(p, u, F, nu1, nu2, rtol, max_cycles, &k, &r0, &r));
  else
    TRY(solve_fp64(p, u, F, nu1, nu2, rtol, max_cycles, &k, &r0, &r));
  if (cycles_out) *cycles_out = k;
  if (relres_out) *relres_out = r0 > 0 ? r / r0 : 0.0;
  if (r > rtol * r0) return fail(FHMG_ENOTCONV, "relative residual %.3e after %d cycles", r0 > 0 ? r / r0 : 0.0, k);
  return FHMG_OK;
}

int fhmg_solve_host(fhmg_problem p, double* u_host, const double* f_host, const double* g_host, int nu1, int nu2,
                    double rtol, int max_cycles, int* cycles_out, double* relres_out) {
  ENTER(p);
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

int fhmg_ws_solve_host(fhmg_wsnet net, fhmg_problem p, double* u_host, const double* f_host, double alpha, int K,
                       int bf16, int nu1, int nu2, double rtol, int max_cycles, int* cycles_out, double* relres_out) {
  ENTER(p);
  if (!net || !u_host || !f_host) return fail(FHMG_EINVAL, "bad arguments");
  const size_t n = (size_t)p->lev[p->nlev - 1].npts * p->M;
  if (!p->hu) TRY(dalloc(p->allocs, &p->hu, n));
  if (!p->hf) TRY(dalloc(p->allocs, &p->hf, n));
  CK(cudaMemcpyAsync(p->hf, f_host, n * sizeof(double), cudaMemcpyHostToDevice, p->st));
  TRY(fhmg_ws_predict(net, p, p->hf, alpha, K, bf16, p->hu));
  int st = fhmg_solve(p, p->hu, p->hf, nullptr, nu1, nu2, rtol, max_cycles, cycles_out, relres_out);
  if (st != FHMG_OK && st != FHMG_ENOTCONV) return st;
  CK(cudaMemcpyAsync(u_host, p->hu, n * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return st;
}

int fhmg_solve_batched(int n, fhmg_problem* probs, double** u, const double** f, int nu1, int nu2, double rtol,
                       int max_cycles, int* cycles_out, double* relres_out) {
  if (n < 1 || n > 4096 || !probs || !u || !f) return fail(FHMG_EINVAL, "bad batch");
  if (nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0 || !(rtol >= 0) || max_cycles < 0) return fail(FHMG_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i) {
    if (!probs[i] || !u[i] || !f[i]) return fail(FHMG_EINVAL, "null problem or array in the batch");
    if (probs[i]->prec != probs[0]->prec) return fail(FHMG_EINVAL, "all problems of a batch must share the precision");
    if (probs[i]->dev != probs[0]->dev) return fail(FHMG_EINVAL, "all problems of a batch must be on one device");
  }
  DeviceScope dev_scope(probs[0]->dev);
  if (!dev_scope.ok) return fail(FHMG_ECUDA, "cannot make the batch's device current");
  const bool mixed = probs[0]->prec != FHMG_FP64;
  const int kind = mixed ? KSPLIT : K64;  // the batched mixed path keeps FP64 storage (valid for every N)
  cudaStream_t st;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  struct Cleanup {
    cudaStream_t s;
    cudaEvent_t e;
    ~Cleanup() {
      cudaEventDestroy(e);
      cudaStreamDestroy(s);
    }
  } cleanup{st, ev};
  for (int i = 0; i < n; ++i) {  // order after the callers' streams
    CK(cudaEventRecord(ev, probs[i]->st));
    CK(cudaStreamWaitEvent(st, ev, 0));
  }
  long long nl = 0;
  std::vector<BLev> set(n);
  std::vector<double*> R(n);
  for (int i = 0; i < n; ++i) {
    set[i] = BLev{probs[i], probs[i]->nlev - 1, u[i], f[i]};
    R[i] = probs[i]->Rs;
  }
  std::vector<double> r0, r;
  TRY(batched_defects(st, set, R, &nl));
  TRY(read_norms(st, set, r0));
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(r0[i])) return fail(FHMG_ENAN, "initial residual of instance %d is not finite", i);
  r = r0;
  std::vector<int> cyc(n, 0);
  auto active_list = [&]() {
    std::vector<int> a;
    for (int i = 0; i < n; ++i)
      if (r[i] > rtol * r0[i] && cyc[i] < max_cycles) a.push_back(i);
    return a;
  };
  std::vector<int> act = active_list();
  CycleGraph graph;
  std::vector<int> graph_set;
  while (!act.empty()) {
    std::vector<BLev> sub;
    for (int i : act)
      sub.push_back(mixed ? BLev{probs[i], probs[i]->nlev - 1, probs[i]->Ef, probs[i]->Rs} : set[i]);
    // inner cycles of this round, capped so that no instance runs past max_cycles (active
    // instances advance in lockstep, so they share one count)
    const int ncyc = std::min(mixed ? (probs[0]->inner > 0 ? probs[0]->inner : 4) : 1, max_cycles - cyc[act[0]]);
    if (mixed)
      for (int i : act)
        CK(cudaMemsetAsync(probs[i]->Ef, 0, sizeof(double) * probs[i]->lev[probs[i]->nlev - 1].npts * probs[i]->M, st));
    for (int c = 0; c < ncyc; ++c) {
      if (graph_set != act) {
        TRY(capture_cycle(st, sub, nu1, nu2, kind, &nl, graph));  // runs this cycle, then captures it
        graph_set = act;
      } else {
        CK(cudaGraphLaunch(graph.exec, st));
        ++nl;
      }
    }
    for (int i : act) cyc[i] += ncyc;
    std::vector<BLev> chk;
    for (int i : act) chk.push_back(set[i]);
    std::vector<double> rn;
    if (mixed) {
      for (int i : act) {
        const long long ne = probs[i]->lev[probs[i]->nlev - 1].npts * probs[i]->M;
        axpy_kernel<<<blocks_for(ne), 256, 0, st>>>(u[i], probs[i]->Ef, ne, 1.0);
        CK(cudaGetLastError());
        ++nl;
      }
      std::vector<double*> Ra;
      for (int i : act) Ra.push_back(probs[i]->Rs);
      TRY(batched_defects(st, chk, Ra, &nl));
    } else if (nu2 > 0) {
      TRY(batched_colour0_norms(st, chk, &nl));
    } else {
      std::vector<double*> Ra;
      for (int i : act) Ra.push_back(probs[i]->Rs);
      TRY(batched_defects(st, chk, Ra, &nl));
    }
    TRY(read_norms(st, chk, rn));
    for (size_t k = 0; k < act.size(); ++k) {
      if (!std::isfinite(rn[k])) return fail(FHMG_ENAN, "residual of instance %d became non-finite", act[k]);
      r[act[k]] = rn[k];
    }
    act = active_list();
  }
  for (int i = 0; i < n; ++i) {  // the callers' streams wait for the batch
    probs[i]->launches += nl / n;
    if (cycles_out) cycles_out[i] = cyc[i];
    if (relres_out) relres_out[i] = r0[i] > 0 ? r[i] / r0[i] : 0.0;
  }
  CK(cudaEventRecord(ev, st));
  for (int i = 0; i < n; ++i) CK(cudaStreamWaitEvent(probs[i]->st, ev, 0));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i)
    if (r[i] > rtol * r0[i]) return fail(FHMG_ENOTCONV, "instance %d: relative residual %.3e after %d cycles", i,
                                         r0[i] > 0 ? r[i] / r0[i] : 0.0, cyc[i]);
  return FHMG_OK;
}

int fhmg_autotune_hmatrix(double alpha, double gamma, double T, int M, int leaf, double err_target, int* best_rank,
                          double* best_tol, double* best_err, double* best_flops) {
  if (!best_rank || !best_tol) return fail(FHMG_EINVAL, "null argument");
  if (!(err_target >= 0.0)) return fail(FHMG_EINVAL, "err_target must be >= 0");
  // the exact reference: every entry of R (dense mode)
  fhmg::HostH ref;
  if (fhmg::build_hmatrix(alpha, gamma, T, M, leaf, 0, 0.0, ref) != 0)
    return fail(FHMG_EINVAL, "invalid arguments: need 0<alpha<1, gamma>=1, T>0, M = leaf*2^p, leaf in {16,32,64}");
  std::vector<double> R;
  dense_of(ref, R);
  std::vector<double> rowmax((size_t)M, 0.0);
  for (int m = 0; m < M; ++m)
    for (int j = 0; j <= m; ++j) rowmax[m] = std::max(rowmax[m], std::fabs(R[(size_t)m * M + j]));
  // candidates: the paper's Taylor form with k terms, then Taylor + recompression to tol, then R itself
  struct Cand {
    int rank;
    double tol;
  };
  static const Cand cands[] = {{4, 0.0},   {6, 0.0},    {8, 0.0},     {10, 0.0},    {12, 0.0},    {16, 0.0}, {20, 0.0},
                               {0, 1e-6}, {0, 1e-8}, {0, 1e-10}, {0, 1e-12}, {0, 1e-14}, {0, 0.0}};
  int br = -1;
  double bt = 0.0, be = 0.0, bf = 0.0;
  std::vector<double> D;
  for (const Cand& c : cands) {
    fhmg::HostH h;
    double err = 0.0;
    fhmg::FlatH f;
    if (c.rank == 0 && c.tol == 0.0) {
      fhmg::flatten(ref, f);  // R itself: exact
    } else {
      if (fhmg::build_hmatrix(alpha, gamma, T, M, leaf, c.rank, c.tol, h) != 0) continue;
      fhmg::flatten(h, f);
      dense_of(h, D);
      for (int m = 0; m < M; ++m) {
        if (rowmax[m] == 0.0) continue;
        double e = 0.0;
        for (int j = 0; j <= m; ++j) e = std::max(e, std::fabs(D[(size_t)m * M + j] - R[(size_t)m * M + j]));
        err = std::max(err, e / rowmax[m]);
      }
    }
    const double fl = (double)f.flops_per_col_matvec;
    if (err <= err_target && (br < 0 || fl < bf || (fl == bf && err < be))) {
      br = c.rank;
      bt = c.tol;
      be = err;
      bf = fl;
    }
  }
  *best_rank = br;
  *best_tol = bt;
  if (best_err) *best_err = be;
  if (best_flops) *best_flops = bf;
  return FHMG_OK;
}

int fhmg_autotune_leaf(double alpha, double gamma, double T, int M, double tol, int dim, int N, double Lx, int prec,
                       void* stream, int* best_leaf, double* best_ms) {
  if (!best_leaf) return fail(FHMG_EINVAL, "best_leaf is NULL");
  double best = 1e300;
  int bl = 0;
  for (int leaf : {16, 32, 64}) {
    if (leaf > M) continue;
    fhmg_hmatrix h = nullptr;
    if (fhmg_build_hmatrix(alpha, gamma, T, M, leaf, 0, tol, &h) != FHMG_OK) continue;
    fhmg_problem p = nullptr;
    int s = fhmg_problem_create(h, dim, N, Lx, prec, stream, &p);
    if (s != FHMG_OK) {
      fhmg_hmatrix_destroy(h);
      return s;
    }
    s = fhmg_problem_autotune(p);
    // time one V-cycle (after a warm-up cycle) on the zeroed workspace: iterate and right-hand
    // side both in Rs (fine-grid size; values do not change the cost)
    const LevelData& fine = p->lev[p->nlev - 1];
    const int kind = p->prec != FHMG_FP64 ? KSPLIT : K64;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    if (s == FHMG_OK && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
      cudaMemsetAsync(p->Rs, 0, sizeof(double) * fine.npts * p->M, p->st);
      s = vcycle_rec<double>(p, p->nlev - 1, p->Rs, p->Rs, 1, 1, kind);
      cudaEventRecord(e0, p->st);
      if (s == FHMG_OK) s = vcycle_rec<double>(p, p->nlev - 1, p->Rs, p->Rs, 1, 1, kind);
      cudaEventRecord(e1, p->st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fhmg_problem_destroy(p);
    fhmg_hmatrix_destroy(h);
    if (s != FHMG_OK) return s;
    if (ms < best) {
      best = ms;
      bl = leaf;
    }
  }
  if (!bl) return fail(FHMG_EINVAL, "no leaf size could be built for M = %d", M);
  *best_leaf = bl;
  if (best_ms) *best_ms = best;
  return FHMG_OK;
}

}  // extern "C"
