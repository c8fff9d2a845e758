// fhmg_residual_norm_noalloc: the finest-grid defect max-norm without any allocation.
//
// Some callers cannot call cudaMalloc once their solve loop is running -- code that runs under a
// fixed memory budget reserved up front, inside a real-time or embedded control loop, or inside a
// host framework that owns every device allocation and forbids the library from making its own.
// For them this entry point computes the same number as fhmg_residual_norm but takes its scratch
// (the defect at every grid point and the max-norm accumulator) from a file-scope __device__
// array of fixed size instead of the problem's workspace, and it calls no allocating routine.
//
// Set-up: the first call for a problem on a given device looks up the device address of the array
// on that device (cudaGetSymbolAddress, with the problem's device made current for the call) and
// caches it; make that first call before any stream capture.  The cached address belongs to the
// device's current context: after cudaDeviceReset on that device the module is loaded anew and
// this entry point must not be called again on that device in the same process.
//
// Limits and sharing:
//  * the defect scratch holds kNoallocMaxElems doubles (16 MiB): problems with
//    M * N^dim > kNoallocMaxElems are rejected with FHMG_EINVAL;
//  * the array belongs to the library and stays allocated on every GPU that loads it until the
//    process exits;
//  * every call shares it: calls whose GPU work overlaps (other streams, other threads, or other
//    problems on the same device) race on it and must be serialised by the caller; the norm
//    accumulator is cleared at the start of every call, the defect part is fully overwritten.
#include <cuda_runtime.h>

#include <atomic>

#include "fhmg.h"

struct fhmg_problem_s;
int fhmg_internal_defect_norm(fhmg_problem p, const double* u, const double* F, double* B,
                              unsigned long long* norm_word, double* out);
long long fhmg_internal_grid_elems(fhmg_problem p);
int fhmg_internal_problem_device(fhmg_problem p);
int fhmg_internal_fail(int code, const char* msg);

namespace {

constexpr long long kNoallocMaxElems = 1LL << 21;
constexpr int kMaxDevices = 64;

// [0, kNoallocMaxElems): the defect; then one 8-byte word for the max-norm (as ull bits)
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxElems + 32];

// Device addresses of the array, resolved once per device (the host-side symbol is only a
// stand-in and must never be handed to a kernel).  Host threads may race on the first lookup;
// each writes the same address, atomically.
std::atomic<double*> g_scratch_ptr[kMaxDevices];

// The array's address on device dev; the caller has made dev current.
int scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fhmg_internal_fail(FHMG_ECUDA, "device index out of range");
  double* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e != cudaSuccess || !a) return fhmg_internal_fail(FHMG_ECUDA, cudaGetErrorString(e));
    ptr = static_cast<double*>(a);
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
  }
  *out = ptr;
  return FHMG_OK;
}

// Makes dev current for the scope of the call, restoring the caller's device afterwards.
struct CurrentDevice {
  int prev = -1;
  bool ok = false;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      return;
    }
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~CurrentDevice() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int fhmg_residual_norm_noalloc(fhmg_problem p, const double* u, const double* f, double* out_max) {
  if (!p || !u || !f || !out_max) return fhmg_internal_fail(FHMG_EINVAL, "null argument");
  const long long n = fhmg_internal_grid_elems(p);
  if (n > kNoallocMaxElems)
    return fhmg_internal_fail(FHMG_EINVAL,
                              "fhmg_residual_norm_noalloc: M * N^dim exceeds the fixed scratch of 2^21 doubles");
  const int dev = fhmg_internal_problem_device(p);
  CurrentDevice scope(dev);
  if (!scope.ok) return fhmg_internal_fail(FHMG_ECUDA, "cannot make the problem's device current");
  double* scratch = nullptr;
  int st = scratch_for_device(dev, &scratch);
  if (st != FHMG_OK) return st;
  auto* norm_word = reinterpret_cast<unsigned long long*>(scratch + kNoallocMaxElems);
  return fhmg_internal_defect_norm(p, u, f, scratch, norm_word, out_max);
}
