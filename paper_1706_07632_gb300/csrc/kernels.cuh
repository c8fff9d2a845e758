// CUDA kernels (sm_103a) for multigrid waveform relaxation with an H-matrix time operator.
//
// Grid functions are time-major with space contiguous: value (m, p) at m * ld + p, m = 0..M-1
// standing for t_1..t_M, p the spatial index (1D: p = n - 1; 2D: p = iy * N + ix).
//
// The H-matrix walk over leaf rows (the hot path) is in panel.cuh; this file holds the
// geometry helpers and the stencil / transfer kernels around it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fhmg {

// Geometry of the columns a smoothing half-sweep updates.
struct Geo {
  int dim;       // 0: compact columns, no stencil; 1 or 2: colour of a grid
  int N;         // interior points per dimension (dim > 0)
  int colour;    // 0 or 1 (dim > 0)
  long long ld;  // elements per time level of the arrays addressed
  double inv_h2; // 1/h^2 (dim > 0)
};

// Number of points of a colour (dim 1: colour 0 = odd n (1-based), colour 1 = even n;
// dim 2: colour 0 = ix + iy even (0-based, same parity as 1-based i + j), colour 1 = odd).
__host__ __device__ inline long long colour_count(int dim, int N, int colour) {
  if (dim == 0) return N;
  if (dim == 1) return colour == 0 ? (N + 1) / 2 : N / 2;
  long long first = colour == 0 ? (N + 1) / 2 : N / 2;  // points in an even row
  return (long long)((N - 1) / 2) * N + first;
}

// Spatial index of the c-th point of a colour.
__host__ __device__ inline long long colour_pos(int dim, int N, int colour, long long c, int* iy_out,
                                                int* ix_out) {
  if (dim == 1) {
    long long p = 2 * c + colour;
    *iy_out = 0;
    *ix_out = (int)p;
    return p;
  }
  long long first = colour == 0 ? (N + 1) / 2 : N / 2;
  long long q = c / N, rem = c % N;
  int iy, ix;
  if (rem < first) {
    iy = (int)(2 * q);
    ix = (int)(colour + 2 * rem);
  } else {
    iy = (int)(2 * q + 1);
    ix = (int)((1 - colour) + 2 * (rem - first));
  }
  *iy_out = iy;
  *ix_out = ix;
  return (long long)iy * N + ix;
}

// ---------------------------------------------------------------- stencil / transfer kernels
//
// Launch shape of the grid-function kernels: blockIdx.x / threadIdx.x run along a grid row (x),
// blockIdx.y is the row (y; 0 in 1D), blockIdx.z strides over the time levels, so no index is
// recovered by a division.

// Restriction of the defect with the time operator commuted out:
//   Xc = FW(u)  and  Bc = FW(F - A_h u), so that the coarse right-hand side is Bc - R~ Xc
// (FW acts per time level and R~ per spatial point, so FW(R~ u) = R~ FW(u)).  One thread per
// coarse point (cx, cy) per time level.
template <typename T>
__global__ void restrict_pre_kernel(int dim, int Nf, double inv_h2, int M, const T* __restrict__ U,
                                    const T* __restrict__ F, T* __restrict__ Xc, T* __restrict__ Bc) {
  const int Nc = (Nf - 1) / 2;
  const int cx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y;
  if (cx >= Nc) return;
  const long long nc = dim == 1 ? Nc : (long long)Nc * Nc;
  const long long nf = dim == 1 ? Nf : (long long)Nf * Nf;
  const T ih2 = (T)inv_h2;
  for (int m = blockIdx.z; m < M; m += gridDim.z) {
    const T* u = U + (long long)m * nf;
    const T* f = F + (long long)m * nf;
    T xs = 0, bs = 0;
    if (dim == 1) {
      const int pc = 2 * cx + 1;
#pragma unroll
      for (int o = -1; o <= 1; ++o) {
        const int pp = pc + o;
        const T w = o == 0 ? (T)0.5 : (T)0.25;
        const T uc = u[pp];
        const T ul = pp > 0 ? u[pp - 1] : (T)0;
        const T ur = pp < Nf - 1 ? u[pp + 1] : (T)0;
        xs += w * uc;
        bs += w * (f[pp] - (2 * uc - ul - ur) * ih2);
      }
    } else {
      const int py = 2 * cy + 1, px = 2 * cx + 1;
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
          const int yy = py + oy, xx = px + ox;
          const T w = (T)((oy == 0 ? 2 : 1) * (ox == 0 ? 2 : 1)) * (T)0.0625;
          const long long pp = (long long)yy * Nf + xx;
          const T uc = u[pp];
          T s = 0;
          if (xx > 0) s += u[pp - 1];
          if (xx < Nf - 1) s += u[pp + 1];
          if (yy > 0) s += u[pp - Nf];
          if (yy < Nf - 1) s += u[pp + Nf];
          xs += w * uc;
          bs += w * (f[pp] - (4 * uc - s) * ih2);
        }
    }
    const long long c = (long long)cy * Nc + cx;
    Xc[(long long)m * nc + c] = xs;
    Bc[(long long)m * nc + c] = bs;
  }
}

// 1D weights of fine index x (0-based) on coarse indices: odd x -> coarse (x-1)/2 (1), even x ->
// coarse x/2 - 1 and x/2 (1/2 each; missing ones are boundary zeros)
template <typename T>
__device__ __forceinline__ void lin_weights(int x, int Nc, int& c0, T& w0, int& c1, T& w1) {
  if (x & 1) {
    c0 = (x - 1) / 2; w0 = 1; c1 = c0; w1 = 0;
  } else {
    c0 = x / 2 - 1; w0 = (T)0.5; c1 = x / 2; w1 = (T)0.5;
    if (c0 < 0) { c0 = 0; w0 = 0; }
    if (c1 >= Nc) { c1 = Nc - 1; w1 = 0; }
  }
}

// u_f += P e_c, linear (1D) / bilinear (2D) interpolation in space, per time level; one thread per
// fine point.
template <typename T>
__global__ void prolong_add_kernel(int dim, int Nf, int M, const T* __restrict__ E, T* __restrict__ U) {
  const int Nc = (Nf - 1) / 2;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= Nf) return;
  const long long nf = dim == 1 ? Nf : (long long)Nf * Nf;
  const long long nc = dim == 1 ? Nc : (long long)Nc * Nc;
  int ax0, ax1, ay0 = 0, ay1 = 0;
  T wx0, wx1, wy0 = 1, wy1 = 0;
  lin_weights<T>(x, Nc, ax0, wx0, ax1, wx1);
  if (dim == 2) lin_weights<T>(y, Nc, ay0, wy0, ay1, wy1);
  const long long pp = (long long)y * Nf + x;
  for (int m = blockIdx.z; m < M; m += gridDim.z) {
    const T* e = E + (long long)m * nc;
    T v;
    if (dim == 1) {
      v = wx0 * e[ax0] + wx1 * e[ax1];
    } else {
      v = wy0 * (wx0 * e[(long long)ay0 * Nc + ax0] + wx1 * e[(long long)ay0 * Nc + ax1]) +
          wy1 * (wx0 * e[(long long)ay1 * Nc + ax0] + wx1 * e[(long long)ay1 * Nc + ax1]);
    }
    U[(long long)m * nf + pp] += v;
  }
}

// Gathers, for the points of one colour, X = u and B = F - A_h u into compact arrays (the time
// product R~ X is then subtracted by the MATVEC walk).  colour < 0: all points, in place order.
// One thread per point of the row blockIdx.y (1D: the only row): the colour's points of row y are
// x = x0 + 2 j with compact indices c0 + j (colour_pos order), so nothing is divided.
template <typename T>
__global__ void gather_defect_kernel(int dim, int N, int colour, double inv_h2, int M, const T* __restrict__ U,
                                     const T* __restrict__ F, T* __restrict__ Xo, T* __restrict__ Bo) {
  const int y = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const long long nf = dim == 1 ? N : (long long)N * N;
  long long ncol, c;
  int x;
  if (colour < 0) {
    if (j >= N) return;
    x = j;
    ncol = nf;
    c = (long long)y * N + x;
  } else {
    ncol = colour_count(dim, N, colour);
    const int first = colour == 0 ? (N + 1) / 2 : N / 2;  // points of the colour in an even row
    const bool even_row = dim == 1 || (y & 1) == 0;
    const int n_row = even_row ? first : N - first;
    if (j >= n_row) return;
    x = (even_row ? colour : 1 - colour) + 2 * j;
    c = dim == 1 ? j : (long long)(y / 2) * N + (even_row ? 0 : first) + j;
  }
  const long long pp = (long long)y * N + x;
  const T ih2 = (T)inv_h2;
  const T diag = dim == 1 ? (T)2 : (T)4;
  for (int m = blockIdx.z; m < M; m += gridDim.z) {
    const T* u = U + (long long)m * nf;
    const T uc = u[pp];
    T s = 0;
    if (x > 0) s += u[pp - 1];
    if (x < N - 1) s += u[pp + 1];
    if (dim == 2) {
      if (y > 0) s += u[pp - N];
      if (y < N - 1) s += u[pp + N];
    }
    if (Xo) Xo[(long long)m * ncol + c] = uc;
    Bo[(long long)m * ncol + c] = F[(long long)m * nf + pp] - (diag * uc - s) * ih2;
  }
}

// F = f + d_{m,m} g  (initial data moved to the right-hand side); blockIdx.y unused (flat points)
template <typename T>
__global__ void add_initial_kernel(long long npts, int M, const T* __restrict__ f, const T* __restrict__ dmm,
                                   const T* __restrict__ g, T* __restrict__ F) {
  for (long long pp = blockIdx.x * (long long)blockDim.x + threadIdx.x; pp < npts;
       pp += (long long)gridDim.x * blockDim.x)
    for (int m = blockIdx.z; m < M; m += gridDim.z) {
      const long long idx = (long long)m * npts + pp;
      F[idx] = f[idx] + (g ? dmm[m] * g[pp] : (T)0);
    }
}

// Launch shape for a grid function with nx points per row and ny rows (1 in 1D) over M time levels:
// enough CTAs along the time levels for about 16 per SM, each CTA then strides over time.
inline dim3 plane_grid(long long nx, long long ny, int M, int sms, int threads = 256) {
  const long long bx = (nx + threads - 1) / threads;
  const long long per = bx * ny;
  long long bz = ((long long)sms * 16 + per - 1) / per;
  if (bz > M) bz = M;
  if (bz < 1) bz = 1;
  if (bz > 65535) bz = 65535;
  return dim3((unsigned)bx, (unsigned)ny, (unsigned)bz);
}

}  // namespace fhmg
