// Learned warm start: a small spectral network, trained and run by the kernels of this file.
//
// For a source that is constant in time and a finite sine series, f = sum_pq c_pq s_pq(x, y),
// each spatial eigenmode s_pq of A_h (eigenvalue lam_pq) is carried independently through the
// time discretisation: u = sum_pq c_pq w_pq(t) s_pq with (R + lam_pq I) w_pq = 1.  The network
// predicts y = lam * w(t) in [0, 1) from features of (lam, alpha, t); the warm start projects f
// onto the K x K leading modes, evaluates the network for every (mode, time level) and
// synthesises u0 = sum_pq c_pq w_pq(t_m) s_pq.  Multigrid then solves from u0 and measures
// its error (and is the fallback: u0 = 0).
//
// Network: F = 6 input features -> H -> H -> H -> 1, SiLU activations, FP32 training (Adam), FP32
// or BF16 inference.  Layer l maps width n_l to n_{l+1} with weights W_l (n_{l+1} x n_l,
// row-major) and bias b_l; all parameters live in one FP32 array in layer order (W_0, b_0, W_1,
// b_1, ...).  Kernels: tiled FP32 GEMM (64 x 64 tiles, 4 x 4 per thread, both transposes),
// BF16 tensor-core GEMMs for inference (hidden layers with bias and SiLU fused), bias + SiLU forward /
// backward, MSE loss, column sums, Adam, feature build, spectral
// projection and synthesis.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "devinfo.h"
#include "fhmg.h"

// Kernel launches issued by this file (network training / inference, warm-start projection and
// synthesis), reported by fhmg_wsnet_launches.
static std::atomic<long long> g_nn_launches{0};

int fhmg_internal_fail(int code, const char* msg);

namespace {

constexpr int kFeat = 6;

#define NCK(x)                                                                     \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) return fhmg_internal_fail(FHMG_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

// C (M x N, ldc) = alpha * op(A) op(B) + beta * C;  op(A) is M x K, op(B) is K x N.
// ta: A stored K x M (lda) and transposed; tb: B stored N x K (ldb) and transposed.
// Batched over blockIdx.z with element strides sA, sB, sC.
__global__ void __launch_bounds__(256) gemm_f32(int M, int N, int K, float alpha, const float* A, int lda,
                                                long long sA, int ta, const float* B, int ldb, long long sB, int tb,
                                                float beta, float* C, int ldc, long long sC) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = va;
      const int gn = n0 + mm;
      float vb = 0.f;
      if (gn < N && gk < K) vb = tb ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][mm] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) {
        float* c = C + (long long)gm * ldc + gn;
        *c = alpha * acc[i][j] + (beta == 0.f ? 0.f : beta * *c);
      }
    }
}

// BF16 inference GEMM with FP32 accumulation: C (M x N) = A (M x K, row-major bf16) * W^T
// (W: N x K, row-major bf16), one 16 x 8 tensor-core tile (mma.sync m16n8k16) per warp step.
__global__ void __launch_bounds__(128) gemm_bf16_nt(int M, int N, int K, const __nv_bfloat16* A,
                                                    const __nv_bfloat16* W, float* C) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = (blockIdx.y * 4 + warp) * 16;
  const int n0 = blockIdx.x * 8;
  if (m0 >= M) return;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  const int g = lane / 4, q = lane % 4;
  for (int k0 = 0; k0 < K; k0 += 16) {
    auto ldA = [&](int r, int k) -> __nv_bfloat16 {
      return (r < M && k < K) ? A[(long long)r * K + k] : __float2bfloat16(0.f);
    };
    auto ldW = [&](int n, int k) -> __nv_bfloat16 {
      return (n < N && k < K) ? W[(long long)n * K + k] : __float2bfloat16(0.f);
    };
    // fragment layout of m16n8k16 (row.col): a0..a7, b0..b3 per thread
    __nv_bfloat162 a01 = __halves2bfloat162(ldA(m0 + g, k0 + 2 * q), ldA(m0 + g, k0 + 2 * q + 1));
    __nv_bfloat162 a23 = __halves2bfloat162(ldA(m0 + g + 8, k0 + 2 * q), ldA(m0 + g + 8, k0 + 2 * q + 1));
    __nv_bfloat162 a45 = __halves2bfloat162(ldA(m0 + g, k0 + 2 * q + 8), ldA(m0 + g, k0 + 2 * q + 9));
    __nv_bfloat162 a67 = __halves2bfloat162(ldA(m0 + g + 8, k0 + 2 * q + 8), ldA(m0 + g + 8, k0 + 2 * q + 9));
    __nv_bfloat162 b01 = __halves2bfloat162(ldW(n0 + g, k0 + 2 * q), ldW(n0 + g, k0 + 2 * q + 1));
    __nv_bfloat162 b23 = __halves2bfloat162(ldW(n0 + g, k0 + 2 * q + 8), ldW(n0 + g, k0 + 2 * q + 9));
    const unsigned ra0 = *reinterpret_cast<unsigned*>(&a01), ra1 = *reinterpret_cast<unsigned*>(&a23);
    const unsigned ra2 = *reinterpret_cast<unsigned*>(&a45), ra3 = *reinterpret_cast<unsigned*>(&a67);
    const unsigned rb0 = *reinterpret_cast<unsigned*>(&b01), rb1 = *reinterpret_cast<unsigned*>(&b23);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(ra0), "r"(ra1), "r"(ra2), "r"(ra3), "r"(rb0), "r"(rb1));
  }
  const int r0 = m0 + g, r1 = m0 + g + 8, cc = n0 + 2 * q;
  if (r0 < M && cc < N) C[(long long)r0 * N + cc] = c[0];
  if (r0 < M && cc + 1 < N) C[(long long)r0 * N + cc + 1] = c[1];
  if (r1 < M && cc < N) C[(long long)r1 * N + cc] = c[2];
  if (r1 < M && cc + 1 < N) C[(long long)r1 * N + cc + 1] = c[3];
}

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }

// BF16 inference layer with the bias and the activation fused: out = SiLU(A W^T + b), A (M x K) and
// W (N x K) row-major BF16 (16-byte aligned rows), b FP32, K % 32 == 0, N % 64 == 0.  Block tile
// 128 x 64; K tiles of 32 double-buffered in shared memory by cp.async (rows padded to 80 bytes:
// the fragment loads below hit 32 distinct banks); 8 warps of 32 x 32, each a 2 x 4 grid of
// mma.sync m16n8k16 tiles with FP32 accumulation, k16 steps in the same order as gemm_bf16_nt; the
// epilogue adds b, applies SiLU and writes BF16 (the same FP32 operations as bias_act_fwd).
__global__ void __launch_bounds__(256) gemm_bf16_silu(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                      const __nv_bfloat16* __restrict__ W,
                                                      const float* __restrict__ bias, __nv_bfloat16* out) {
  constexpr int BM = 128, BN = 64, BK = 32, LDS = BK + 8;
  __shared__ __align__(16) __nv_bfloat16 sA[2][BM * LDS];
  __shared__ __align__(16) __nv_bfloat16 sW[2][BN * LDS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 3, wn = warp >> 2;
  const int g = lane >> 2, q = lane & 3;
  const long long m0 = (long long)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  auto load_tile = [&](int buf, int k0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {  // A: 128 rows x 4 chunks of 16 bytes
      const int c = tid + i * 256;
      const int r = c >> 2, kc = (c & 3) * 8;
      const long long gr = m0 + r;
      const bool ok = gr < M;
      const __nv_bfloat16* src = A + (ok ? gr : 0LL) * K + k0 + kc;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&sA[buf][r * LDS + kc])),
                   "l"(src), "r"(ok ? 16 : 0)
                   : "memory");
    }
    {  // W: 64 rows x 4 chunks
      const int r = tid >> 2, kc = (tid & 3) * 8;
      const __nv_bfloat16* src = W + (long long)(n0 + r) * K + k0 + kc;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&sW[buf][r * LDS + kc])),
                   "l"(src)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto lds32 = [](const __nv_bfloat16* p) -> uint32_t { return *reinterpret_cast<const uint32_t*>(p); };
  float acc[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[mi][ni][j] = 0.f;
  const int nk = K / BK;
  load_tile(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      load_tile((kt + 1) & 1, (kt + 1) * BK);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const __nv_bfloat16* a = sA[kt & 1];
    const __nv_bfloat16* w = sW[kt & 1];
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + g;
        af[mi][0] = lds32(a + r * LDS + ks + 2 * q);
        af[mi][1] = lds32(a + (r + 8) * LDS + ks + 2 * q);
        af[mi][2] = lds32(a + r * LDS + ks + 2 * q + 8);
        af[mi][3] = lds32(a + (r + 8) * LDS + ks + 2 * q + 8);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn * 32 + ni * 8 + g;
        bf[ni][0] = lds32(w + c * LDS + ks + 2 * q);
        bf[ni][1] = lds32(w + c * LDS + ks + 2 * q + 8);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bf[ni][0]), "r"(bf[ni][1]));
    }
    __syncthreads();  // this buffer is refilled two tiles on
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int c = n0 + wn * 32 + ni * 8 + 2 * q;
      const float b0 = bias[c], b1 = bias[c + 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long r = m0 + wm * 32 + mi * 16 + g + 8 * h;
        if (r >= M) continue;
        const float z0 = acc[mi][ni][2 * h] + b0, z1 = acc[mi][ni][2 * h + 1] + b1;
        *reinterpret_cast<__nv_bfloat162*>(out + r * N + c) = __floats2bfloat162_rn(z0 * sigm(z0), z1 * sigm(z1));
      }
    }
}

// Z += b (row broadcast); A = SiLU(Z) (act = 1) or Z (act = 0).  Z kept for the backward pass.
__global__ void bias_act_fwd(int n, int w, float* Z, const float* b, float* A, int act, __nv_bfloat16* Abf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * w;
       i += (long long)gridDim.x * blockDim.x) {
    const float z = Z[i] + b[i % w];
    Z[i] = z;
    const float a = act ? z * sigm(z) : z;
    if (A) A[i] = a;
    if (Abf) Abf[i] = __float2bfloat16(a);
  }
}

// dZ = dA * SiLU'(Z)
__global__ void act_bwd(long long n, const float* Z, const float* dA, float* dZ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float z = Z[i], s = sigm(z);
    dZ[i] = dA[i] * s * (1.f + z * (1.f - s));
  }
}

// loss = mean (y - t)^2 (accumulated into *loss), dY = 2 (y - t) / n
__global__ void mse_fwd_bwd(int n, const float* y, const float* t, float* dy, float* loss) {
  float s = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    if (dy) dy[i] = 2.f * d / n;
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / n);
}

// db[j] = sum_i dZ[i][j]
__global__ void colsum(int n, int w, const float* dZ, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= w) return;
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += dZ[(long long)i * w + j];
  db[j] = s;
}

__global__ void adam_step(long long n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                          float c1, float c2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16(long long n, const float* x, __nv_bfloat16* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

int nblk(long long n) { return fhmg::grid_for(n, 16); }

}  // namespace

// Features of (lam, alpha, t), all O(1): log10(lam)/5, alpha, log10(t)/5 (t > 0), s/(1+s),
// log1p(s)/10 with s = lam t^alpha, t^alpha.
__device__ __forceinline__ void ws_features(double lam, double alpha, double t, float* f) {
  const double ta = pow(t, alpha), s = lam * ta;
  f[0] = (float)(log10(lam) / 5.0);
  f[1] = (float)alpha;
  f[2] = (float)(log10(t) / 5.0);
  f[3] = (float)(s / (1.0 + s));
  f[4] = (float)(log1p(s) / 10.0);
  f[5] = (float)ta;
}

__global__ void build_features(int nmodes, const double* lam, int M, const double* t, double alpha, float* X) {
  const long long total = (long long)nmodes * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / M), m = (int)(i % M);
    ws_features(lam[k], alpha, t[m + 1], X + i * kFeat);
  }
}

struct fhmg_wsnet_s {
  int hidden = 0, layers = 0;     // hidden width, number of hidden layers
  std::vector<int> width;         // n_0 = kFeat, ..., n_L = 1
  std::vector<long long> woff, boff;
  long long nparams = 0;
  float* P = nullptr;             // parameters
  float* G = nullptr;             // gradients
  float* Mo = nullptr;            // Adam moments
  float* Vo = nullptr;
  __nv_bfloat16* Pbf = nullptr;   // BF16 copy of the weights (inference)
  long long step = 0;
  // activations for a batch of up to cap rows
  int cap = 0;
  std::vector<float*> Z, A, dA;   // per layer
  float* dZ = nullptr;
  float* loss = nullptr;
  __nv_bfloat16* Abf[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
};

namespace {

template <typename T>
int nalloc(fhmg_wsnet net, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
  if (e != cudaSuccess) return fhmg_internal_fail(FHMG_ENOMEM, cudaGetErrorString(e));
  net->allocs.push_back(*p);
  return FHMG_OK;
}

int ensure_cap(fhmg_wsnet net, int n) {
  if (n <= net->cap) return FHMG_OK;
  const int L = (int)net->width.size() - 1;
  net->Z.assign(L, nullptr);
  net->A.assign(L + 1, nullptr);
  net->dA.assign(L + 1, nullptr);
  int maxw = 0;
  for (int w : net->width) maxw = w > maxw ? w : maxw;
  for (int l = 0; l < L; ++l) {
    int s = nalloc(net, &net->Z[l], (size_t)n * net->width[l + 1]);
    if (s) return s;
    if ((s = nalloc(net, &net->A[l + 1], (size_t)n * net->width[l + 1]))) return s;
    if ((s = nalloc(net, &net->dA[l + 1], (size_t)n * net->width[l + 1]))) return s;
  }
  int s = nalloc(net, &net->dZ, (size_t)n * maxw);
  if (s) return s;
  if ((s = nalloc(net, &net->Abf[0], (size_t)n * maxw))) return s;
  if ((s = nalloc(net, &net->Abf[1], (size_t)n * maxw))) return s;
  net->cap = n;
  return FHMG_OK;
}

int gemm(cudaStream_t st, int M, int N, int K, float alpha, const float* A, int lda, int ta, const float* B, int ldb,
         int tb, float beta, float* C, int ldc, int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm_f32<<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, ta, B, ldb, sB, tb, beta, C, ldc, sC);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  return FHMG_OK;
}

// FP32 forward of n rows X (n x kFeat) -> output A[L] (n x 1); activations kept.
int forward32(fhmg_wsnet net, cudaStream_t st, const float* X, int n) {
  const int L = (int)net->width.size() - 1;
  int s = ensure_cap(net, n);
  if (s) return s;
  const float* in = X;
  for (int l = 0; l < L; ++l) {
    const int wi = net->width[l], wo = net->width[l + 1];
    // Z = in W^T  (in: n x wi, W: wo x wi)
    if ((s = gemm(st, n, wo, wi, 1.f, in, wi, 0, net->P + net->woff[l], wi, 1, 0.f, net->Z[l], wo))) return s;
    bias_act_fwd<<<nblk((long long)n * wo), 256, 0, st>>>(n, wo, net->Z[l], net->P + net->boff[l], net->A[l + 1],
                                                        l < L - 1 ? 1 : 0, nullptr);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    in = net->A[l + 1];
  }
  return FHMG_OK;
}

// Backward of the MSE loss against targets Y; gradients into net->G (overwritten).
int backward32(fhmg_wsnet net, cudaStream_t st, const float* X, const float* Y, int n) {
  const int L = (int)net->width.size() - 1;
  NCK(cudaMemsetAsync(net->loss, 0, sizeof(float), st));
  mse_fwd_bwd<<<nblk(n), 256, 0, st>>>(n, net->A[L], Y, net->dA[L], net->loss);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  for (int l = L - 1; l >= 0; --l) {
    const int wi = net->width[l], wo = net->width[l + 1];
    const float* dz = net->dA[l + 1];
    if (l < L - 1) {
      act_bwd<<<nblk((long long)n * wo), 256, 0, st>>>((long long)n * wo, net->Z[l], net->dA[l + 1], net->dZ);
      ++g_nn_launches;
      NCK(cudaGetLastError());
      dz = net->dZ;
    }
    const float* in = l == 0 ? X : net->A[l];
    // dW = dz^T in  (wo x wi);  db = colsum(dz);  dA_l = dz W (n x wi)
    int s = gemm(st, wo, wi, n, 1.f, dz, wo, 1, in, wi, 0, 0.f, net->G + net->woff[l], wi);
    if (s) return s;
    colsum<<<(wo + 127) / 128, 128, 0, st>>>(n, wo, dz, net->G + net->boff[l]);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    if (l > 0 && (s = gemm(st, n, wi, wo, 1.f, dz, wo, 0, net->P + net->woff[l], wi, 0, 0.f, net->dA[l], wi))) return s;
  }
  return FHMG_OK;
}

}  // namespace

extern "C" {

int fhmg_wsnet_create(int hidden, int layers, unsigned long long seed, fhmg_wsnet* out) {
  if (!out || hidden < 8 || hidden > 4096 || layers < 1 || layers > 8)
    return fhmg_internal_fail(FHMG_EINVAL, "wsnet: hidden in [8, 4096], layers in [1, 8]");
  fhmg_wsnet net = new (std::nothrow) fhmg_wsnet_s;
  if (!net) return fhmg_internal_fail(FHMG_ENOMEM, "host allocation failed");
  net->hidden = hidden;
  net->layers = layers;
  net->width.push_back(kFeat);
  for (int l = 0; l < layers; ++l) net->width.push_back(hidden);
  net->width.push_back(1);
  const int L = (int)net->width.size() - 1;
  std::vector<float> host;
  std::mt19937_64 rng(seed);
  for (int l = 0; l < L; ++l) {
    const int wi = net->width[l], wo = net->width[l + 1];
    net->woff.push_back((long long)host.size());
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / wi));
    for (long long i = 0; i < (long long)wi * wo; ++i) host.push_back(nd(rng) * (l == L - 1 ? 0.1f : 1.f));
    net->boff.push_back((long long)host.size());
    for (int i = 0; i < wo; ++i) host.push_back(0.f);
  }
  net->nparams = (long long)host.size();
  int s = FHMG_OK;
  auto bail = [&](int st) {
    fhmg_wsnet_destroy(net);
    return st;
  };
  if ((s = nalloc(net, &net->P, host.size())) || (s = nalloc(net, &net->G, host.size())) ||
      (s = nalloc(net, &net->Mo, host.size())) || (s = nalloc(net, &net->Vo, host.size())) ||
      (s = nalloc(net, &net->Pbf, host.size())) || (s = nalloc(net, &net->loss, 1)))
    return bail(s);
  if (cudaMemcpy(net->P, host.data(), host.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->Mo, 0, host.size() * 4) != cudaSuccess || cudaMemset(net->Vo, 0, host.size() * 4) != cudaSuccess)
    return bail(fhmg_internal_fail(FHMG_ECUDA, "wsnet upload failed"));
  *out = net;
  return FHMG_OK;
}

int fhmg_wsnet_destroy(fhmg_wsnet net) {
  if (!net) return FHMG_OK;
  for (void* a : net->allocs) cudaFree(a);
  delete net;
  return FHMG_OK;
}

int fhmg_wsnet_num_params(fhmg_wsnet net, long long* n) {
  if (!net || !n) return fhmg_internal_fail(FHMG_EINVAL, "null argument");
  *n = net->nparams;
  return FHMG_OK;
}

int fhmg_wsnet_get_params(fhmg_wsnet net, float* host) {
  if (!net || !host) return fhmg_internal_fail(FHMG_EINVAL, "null argument");
  NCK(cudaMemcpy(host, net->P, net->nparams * 4, cudaMemcpyDeviceToHost));
  return FHMG_OK;
}

int fhmg_wsnet_set_params(fhmg_wsnet net, const float* host) {
  if (!net || !host) return fhmg_internal_fail(FHMG_EINVAL, "null argument");
  NCK(cudaMemcpy(net->P, host, net->nparams * 4, cudaMemcpyHostToDevice));
  return FHMG_OK;
}

int fhmg_wsnet_forward(fhmg_wsnet net, const float* X, int n, int bf16, float* Y, void* stream) {
  if (!net || !X || !Y || n < 1) return fhmg_internal_fail(FHMG_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int L = (int)net->width.size() - 1;
  int s = ensure_cap(net, n);
  if (s) return s;
  if (!bf16) {
    if ((s = forward32(net, st, X, n))) return s;
    NCK(cudaMemcpyAsync(Y, net->A[L], sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    return FHMG_OK;
  }
  // BF16 tensor-core inference (FP32 accumulation): weights and activations rounded to BF16
  to_bf16<<<nblk(net->nparams), 256, 0, st>>>(net->nparams, net->P, net->Pbf);
  ++g_nn_launches;
  to_bf16<<<nblk((long long)n * kFeat), 256, 0, st>>>((long long)n * kFeat, X, net->Abf[0]);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  int cur = 0;
  for (int l = 0; l < L; ++l) {
    const int wi = net->width[l], wo = net->width[l + 1];
    const bool last = l == L - 1;
    const __nv_bfloat16* Wl = net->Pbf + net->woff[l];
    if (!last && wi % 32 == 0 && wo % 64 == 0 && reinterpret_cast<uintptr_t>(Wl) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(net->Abf[cur]) % 16 == 0) {
      // hidden layers of the full width: one tiled launch, bias and SiLU fused (Z is not needed:
      // the backward pass runs on the FP32 forward's activations)
      dim3 grid(wo / 64, (n + 127) / 128);
      gemm_bf16_silu<<<grid, 256, 0, st>>>(n, wo, wi, net->Abf[cur], Wl, net->P + net->boff[l], net->Abf[1 - cur]);
      ++g_nn_launches;
      NCK(cudaGetLastError());
      cur = 1 - cur;
      continue;
    }
    dim3 grid((wo + 7) / 8, (n + 63) / 64);
    gemm_bf16_nt<<<grid, 128, 0, st>>>(n, wo, wi, net->Abf[cur], net->Pbf + net->woff[l], net->Z[l]);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    bias_act_fwd<<<nblk((long long)n * wo), 256, 0, st>>>(n, wo, net->Z[l], net->P + net->boff[l],
                                                        last ? Y : nullptr, last ? 0 : 1,
                                                        last ? nullptr : net->Abf[1 - cur]);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    cur = 1 - cur;
  }
  return FHMG_OK;
}

int fhmg_wsnet_loss_grad(fhmg_wsnet net, const float* X, const float* Y, int n, float* loss_host, float* grad_host,
                         void* stream) {
  if (!net || !X || !Y || n < 1) return fhmg_internal_fail(FHMG_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int s = forward32(net, st, X, n);
  if (s || (s = backward32(net, st, X, Y, n))) return s;
  if (loss_host) NCK(cudaMemcpyAsync(loss_host, net->loss, 4, cudaMemcpyDeviceToHost, st));
  if (grad_host) NCK(cudaMemcpyAsync(grad_host, net->G, net->nparams * 4, cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  return FHMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- spectral warm start

int fhmg_internal_problem_geom(fhmg_problem p, int* dim, int* N, int* M, double* Lx, void** stream,
                               const double** t_host);

namespace {

// S[n][p] = sin((p+1) pi (n+1) / (N+1)), n < N, p < K  (the discrete sine modes of A_h)
__global__ void sine_basis(int N, int K, float* S) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)N * K;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / K), p = (int)(i % K);
    S[i] = (float)sin((double)(p + 1) * (n + 1) * M_PI / (N + 1));
  }
}

__global__ void d2f(long long n, const double* x, float* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f2d(long long n, const float* x, double* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// eigenvalue of mode k (2D: k = p K + q) of the 3-/5-point negative Laplacian
__device__ __forceinline__ double mode_lambda(int dim, int N, double Lx, int K, int k) {
  const double h = Lx / (N + 1);
  const int p = dim == 1 ? k : k / K, q = dim == 1 ? -1 : k % K;
  auto e = [&](int j) {
    const double s = sin((j + 1) * M_PI / (2.0 * (N + 1)));
    return 4.0 / (h * h) * s * s;
  };
  return e(p) + (dim == 2 ? e(q) : 0.0);
}

__global__ void mode_lambdas(int dim, int N, double Lx, int K, int nm, double* lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nm) lam[k] = mode_lambda(dim, N, Lx, K, k);
}

// G[m][k] = c_k * y[k][m] / lam_k  (predicted mode amplitudes per time level)
__global__ void mode_amplitudes(int nm, int M, const float* c, const float* y, const double* lam, float* G) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nm * M;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / M), m = (int)(i % M);
    G[(long long)m * nm + k] = (float)((double)c[k] * y[i] / lam[k]);
  }
}

// training pairs: y = lam * uhat[m][k] / c[k] for modes with |c_k| >= thr (row order k-major)
__global__ void mode_targets(int nm, int M, const float* c, const float* uhat, const double* lam, float thr,
                             const int* keep, const int* kpos, float* Y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nm * M;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / M), m = (int)(i % M);
    if (!keep[k]) continue;
    Y[(long long)kpos[k] * M + m] = (float)(lam[k] * (double)uhat[(long long)m * nm + k] / (double)c[k]);
  }
}

__global__ void build_features_kept(int nm, const double* lam, int M, const double* t, double alpha, const int* keep,
                                    const int* kpos, float* X) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nm * M;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / M), m = (int)(i % M);
    if (!keep || keep[k]) {
      const long long row = (long long)(keep ? kpos[k] : k) * M + m;
      ws_features(lam[k], alpha, t[m + 1], X + row * kFeat);
    }
  }
}

// FP64 projection used for training targets (small sizes; accuracy over speed):
// T[l][p][x] = sum_y S[y][p] u[l][y][x];  out[l][p][q] = sc^2 sum_x T[l][p][x] S[x][q]  (2D)
// out[l][p] = sc sum_x u[l][x] S[x][p]  (1D)
__global__ void sine_basis64(int N, int K, double* S) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)N * K;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / K), p = (int)(i % K);
    S[i] = sin((double)(p + 1) * (n + 1) * M_PI / (N + 1));
  }
}

__global__ void project64_a(int dim, int N, int K, int nl, const double* u, const double* S, double* T) {
  const long long total = dim == 1 ? (long long)nl * K : (long long)nl * K * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    if (dim == 1) {
      const int l = (int)(i / K), p = (int)(i % K);
      double s = 0.0;
      for (int x = 0; x < N; ++x) s += u[(long long)l * N + x] * S[(long long)x * K + p];
      T[i] = s;
    } else {
      const int l = (int)(i / ((long long)K * N)), r = (int)(i % ((long long)K * N)), p = r / N, x = r % N;
      double s = 0.0;
      for (int y = 0; y < N; ++y) s += S[(long long)y * K + p] * u[((long long)l * N + y) * N + x];
      T[i] = s;
    }
  }
}
__global__ void project64_b(int dim, int N, int K, int nl, const double* T, const double* S, double sc, float* out) {
  const long long total = dim == 1 ? (long long)nl * K : (long long)nl * K * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    if (dim == 1) {
      out[i] = (float)(sc * T[i]);
    } else {
      const int l = (int)(i / ((long long)K * K)), r = (int)(i % ((long long)K * K)), p = r / K, q = r % K;
      double s = 0.0;
      for (int x = 0; x < N; ++x) s += T[((long long)l * K + p) * N + x] * S[(long long)x * K + q];
      out[i] = (float)(sc * sc * s);
    }
  }
}

struct Spectral {
  int dim, N, M, K, nm;
  double Lx;
  cudaStream_t st;
  const double* thost;
  std::vector<void*> mem;
  float* S = nullptr;   // N x K
  double* lam = nullptr;
  double* tdev = nullptr;
  ~Spectral() {
    for (void* p : mem) cudaFree(p);
  }
  template <typename T>
  int alloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) return fhmg_internal_fail(FHMG_ENOMEM, cudaGetErrorString(e));
    mem.push_back(*p);
    return FHMG_OK;
  }
  int init(fhmg_problem p, int K_) {
    void* sv;
    int s = fhmg_internal_problem_geom(p, &dim, &N, &M, &Lx, &sv, &thost);
    if (s) return s;
    st = (cudaStream_t)sv;
    K = K_ < N ? K_ : N;
    nm = dim == 1 ? K : K * K;
    if ((s = alloc(&S, (size_t)N * K)) || (s = alloc(&lam, nm)) || (s = alloc(&tdev, M + 1))) return s;
    sine_basis<<<nblk((long long)N * K), 256, 0, st>>>(N, K, S);
    ++g_nn_launches;
    mode_lambdas<<<(nm + 127) / 128, 128, 0, st>>>(dim, N, Lx, K, nm, lam);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    NCK(cudaMemcpyAsync(tdev, thost, sizeof(double) * (M + 1), cudaMemcpyHostToDevice, st));
    return FHMG_OK;
  }
  // FP64 coefficients (training targets): x is FP64, nl x N^dim; out FP32 nl x K^dim
  int project64(const double* x, int nl, float* out) {
    double *S64, *T;
    int s = alloc(&S64, (size_t)N * K);
    if (s || (s = alloc(&T, dim == 1 ? (size_t)nl * K : (size_t)nl * K * N))) return s;
    sine_basis64<<<nblk((long long)N * K), 256, 0, st>>>(N, K, S64);
    ++g_nn_launches;
    const long long na = dim == 1 ? (long long)nl * K : (long long)nl * K * N;
    project64_a<<<nblk(na), 256, 0, st>>>(dim, N, K, nl, x, S64, T);
    ++g_nn_launches;
    const long long nb_ = dim == 1 ? (long long)nl * K : (long long)nl * K * K;
    project64_b<<<nblk(nb_), 256, 0, st>>>(dim, N, K, nl, T, S64, 2.0 / (N + 1), out);
    ++g_nn_launches;
    NCK(cudaGetLastError());
    return FHMG_OK;
  }
  // coefficients of nl grid functions (time levels) of x (FP32, nl x N^dim) on the modes:
  // out[l][k], scaled by (2/(N+1))^dim so that x = sum_k out_k s_k exactly for a sine series
  int project(const float* x, int nl, float* out) {
    const float sc = 2.f / (N + 1);
    if (dim == 1) return gemm(st, nl, K, N, sc, x, N, 0, S, K, 0, 0.f, out, K);
    float* T1;
    int s = alloc(&T1, (size_t)nl * K * N);
    if (s) return s;
    // T1[l] = S^T (K x N) x[l] (N x N)  -> K x N
    if ((s = gemm(st, K, N, N, sc, S, K, 1, x, N, 0, 0.f, T1, N, nl, 0, (long long)N * N, (long long)K * N))) return s;
    // out[l] = T1[l] (K x N) S (N x K) -> K x K
    return gemm(st, K, K, N, sc, T1, N, 0, S, K, 0, 0.f, out, K, nl, (long long)K * N, 0, (long long)K * K);
  }
};

}  // namespace

extern "C" {

int fhmg_wsnet_launches(long long* n) {
  if (!n) return fhmg_internal_fail(FHMG_EINVAL, "n is NULL");
  *n = g_nn_launches.load();
  return FHMG_OK;
}

int fhmg_ws_predict(fhmg_wsnet net, fhmg_problem prob, const double* f, double alpha, int K, int bf16, double* u0) {
  if (!net || !prob || !f || !u0 || K < 1) return fhmg_internal_fail(FHMG_EINVAL, "bad arguments");
  Spectral sp;
  int s = sp.init(prob, K);
  if (s) return s;
  const int N = sp.N, M = sp.M, nm = sp.nm, dim = sp.dim;
  const long long npts = dim == 1 ? N : (long long)N * N;
  // coefficients of the source (constant in time: its last time level)
  float *f32, *c, *X, *Y, *G, *T1, *U;
  if ((s = sp.alloc(&f32, npts)) || (s = sp.alloc(&c, nm)) || (s = sp.alloc(&X, (size_t)nm * M * kFeat)) ||
      (s = sp.alloc(&Y, (size_t)nm * M)) || (s = sp.alloc(&G, (size_t)nm * M)))
    return s;
  d2f<<<nblk(npts), 256, 0, sp.st>>>(npts, f + (long long)(M - 1) * npts, f32);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  if ((s = sp.project(f32, 1, c))) return s;
  build_features_kept<<<nblk((long long)nm * M), 256, 0, sp.st>>>(nm, sp.lam, M, sp.tdev, alpha, nullptr, nullptr, X);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  if ((s = fhmg_wsnet_forward(net, X, nm * M, bf16, Y, sp.st))) return s;
  mode_amplitudes<<<nblk((long long)nm * M), 256, 0, sp.st>>>(nm, M, c, Y, sp.lam, G);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  // synthesis u0[m] = sum_k G[m][k] s_k, in FP32, then widened to FP64
  if ((s = sp.alloc(&U, (size_t)M * npts))) return s;
  if (dim == 1) {
    // U (M x N) = G (M x K) S^T (K x N)
    if ((s = gemm(sp.st, M, N, K, 1.f, G, K, 0, sp.S, K, 1, 0.f, U, N))) return s;
  } else {
    if ((s = sp.alloc(&T1, (size_t)M * K * N))) return s;
    // T1[m] = G[m] (K x K) S^T (K x N);  U[m] = S (N x K) T1[m] (K x N)
    if ((s = gemm(sp.st, K, N, K, 1.f, G, K, 0, sp.S, K, 1, 0.f, T1, N, M, (long long)K * K, 0, (long long)K * N)))
      return s;
    if ((s = gemm(sp.st, N, N, K, 1.f, sp.S, K, 0, T1, N, 0, 0.f, U, N, M, 0, (long long)K * N, (long long)N * N)))
      return s;
  }
  f2d<<<nblk((long long)M * npts), 256, 0, sp.st>>>((long long)M * npts, U, u0);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  NCK(cudaStreamSynchronize(sp.st));
  return FHMG_OK;
}

int fhmg_ws_dataset(fhmg_problem prob, const double* u, const double* f, double alpha, int K, float rel_thr,
                    float* X_out, float* Y_out, long long* nrows) {
  if (!prob || !u || !f || !X_out || !Y_out || !nrows || K < 1) return fhmg_internal_fail(FHMG_EINVAL, "bad arguments");
  Spectral sp;
  int s = sp.init(prob, K);
  if (s) return s;
  const int N = sp.N, M = sp.M, nm = sp.nm, dim = sp.dim;
  const long long npts = dim == 1 ? N : (long long)N * N;
  float *c, *uh;
  if ((s = sp.alloc(&c, nm)) || (s = sp.alloc(&uh, (size_t)M * nm))) return s;
  if ((s = sp.project64(f + (long long)(M - 1) * npts, 1, c)) || (s = sp.project64(u, M, uh))) return s;
  // modes kept: |c_k| >= rel_thr * max |c|
  std::vector<float> ch(nm);
  NCK(cudaMemcpyAsync(ch.data(), c, sizeof(float) * nm, cudaMemcpyDeviceToHost, sp.st));
  NCK(cudaStreamSynchronize(sp.st));
  float cmax = 0.f;
  for (float v : ch) cmax = std::fabs(v) > cmax ? std::fabs(v) : cmax;
  std::vector<int> keep(nm), kpos(nm);
  int nk = 0;
  for (int k = 0; k < nm; ++k) {
    keep[k] = std::fabs(ch[k]) >= rel_thr * cmax && cmax > 0.f;
    kpos[k] = nk;
    nk += keep[k];
  }
  int *dkeep, *dkpos;
  if ((s = sp.alloc(&dkeep, nm)) || (s = sp.alloc(&dkpos, nm))) return s;
  NCK(cudaMemcpyAsync(dkeep, keep.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, sp.st));
  NCK(cudaMemcpyAsync(dkpos, kpos.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, sp.st));
  build_features_kept<<<nblk((long long)nm * M), 256, 0, sp.st>>>(nm, sp.lam, M, sp.tdev, alpha, dkeep, dkpos, X_out);
  ++g_nn_launches;
  mode_targets<<<nblk((long long)nm * M), 256, 0, sp.st>>>(nm, M, c, uh, sp.lam, rel_thr, dkeep, dkpos, Y_out);
  ++g_nn_launches;
  NCK(cudaGetLastError());
  NCK(cudaStreamSynchronize(sp.st));
  *nrows = (long long)nk * M;
  return FHMG_OK;
}

int fhmg_wsnet_train(fhmg_wsnet net, const float* X, const float* Y, long long nsamples, int batch, int steps,
                     float lr, unsigned long long seed, float* last_loss, void* stream) {
  if (!net || !X || !Y || nsamples < batch || batch < 1 || steps < 0)
    return fhmg_internal_fail(FHMG_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  std::mt19937_64 rng(seed);
  std::uniform_int_distribution<long long> pick(0, nsamples - batch);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps; ++it) {
    // contiguous mini-batches at random offsets (the samples are stored shuffled)
    const long long o = pick(rng);
    const float* xb = X + o * kFeat;
    const float* yb = Y + o;
    int s = forward32(net, st, xb, batch);
    if (s || (s = backward32(net, st, xb, yb, batch))) return s;
    ++net->step;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    adam_step<<<nblk(net->nparams), 256, 0, st>>>(net->nparams, net->P, net->G, net->Mo, net->Vo, lr, b1, b2, c1, c2,
                                                 eps);
    ++g_nn_launches;
    NCK(cudaGetLastError());
  }
  if (last_loss) {
    NCK(cudaMemcpyAsync(last_loss, net->loss, 4, cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
  }
  return FHMG_OK;
}

}  // extern "C"
