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

// Restriction of the defect with the time operator commuted out:
//   Xc = FW(u)  and  Bc = FW(F - A_h u), so that the coarse right-hand side is Bc - R~ Xc
// (FW acts per time level and R~ per spatial point, so FW(R~ u) = R~ FW(u)).
template <typename T>
__global__ void restrict_pre_kernel(int dim, int Nf, double inv_h2, int M, const T* __restrict__ U,
                                    const T* __restrict__ F, T* __restrict__ Xc, T* __restrict__ Bc) {
  const int Nc = (Nf - 1) / 2;
  const long long nc = dim == 1 ? Nc : (long long)Nc * Nc;
  const long long nf = dim == 1 ? Nf : (long long)Nf * Nf;
  const long long total = nc * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / nc, c = idx % nc;
    const T* u = U + m * nf;
    const T* f = F + m * nf;
    const T ih2 = (T)inv_h2;
    T xs = 0, bs = 0;
    if (dim == 1) {
      const int pc = 2 * (int)c + 1;
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
      const int cy = (int)(c / Nc), cx = (int)(c % Nc);
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
    Xc[m * nc + c] = xs;
    Bc[m * nc + c] = bs;
  }
}

// u_f += P e_c, linear (1D) / bilinear (2D) interpolation in space, per time level.
template <typename T>
__global__ void prolong_add_kernel(int dim, int Nf, int M, const T* __restrict__ E, T* __restrict__ U) {
  const int Nc = (Nf - 1) / 2;
  const long long nf = dim == 1 ? Nf : (long long)Nf * Nf;
  const long long nc = dim == 1 ? Nc : (long long)Nc * Nc;
  const long long total = nf * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / nf, pp = idx % nf;
    const T* e = E + m * nc;
    // 1D weights of fine index x (0-based) on coarse indices: odd x -> coarse (x-1)/2 (1),
    // even x -> coarse x/2 - 1 and x/2 (1/2 each, missing ones are boundary zeros)
    auto lin = [&](int x, int& c0, T& w0, int& c1, T& w1) {
      if (x & 1) {
        c0 = (x - 1) / 2; w0 = 1; c1 = -1; w1 = 0;
      } else {
        c0 = x / 2 - 1; w0 = (T)0.5; c1 = x / 2; w1 = (T)0.5;
        if (c0 < 0) w0 = 0;
        if (c1 >= Nc) w1 = 0;
      }
    };
    T v = 0;
    if (dim == 1) {
      int a0, a1; T w0, w1;
      lin((int)pp, a0, w0, a1, w1);
      if (w0 != (T)0) v += w0 * e[a0];
      if (w1 != (T)0) v += w1 * e[a1];
    } else {
      const int y = (int)(pp / Nf), x = (int)(pp % Nf);
      int ay[2], ax[2]; T wy[2], wx[2];
      lin(y, ay[0], wy[0], ay[1], wy[1]);
      lin(x, ax[0], wx[0], ax[1], wx[1]);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
          if (wy[a] != (T)0 && wx[b] != (T)0) v += wy[a] * wx[b] * e[(long long)ay[a] * Nc + ax[b]];
    }
    U[m * nf + pp] += v;
  }
}

// Gathers, for the points of one colour, X = u and B = F - A_h u into compact arrays
// (the time product R~ X is then subtracted by the MATVEC walk).  colour < 0: all points.
template <typename T>
__global__ void gather_defect_kernel(int dim, int N, int colour, double inv_h2, int M, const T* __restrict__ U,
                                     const T* __restrict__ F, T* __restrict__ Xo, T* __restrict__ Bo) {
  const long long nf = dim == 1 ? N : (long long)N * N;
  const long long ncol = colour < 0 ? nf : colour_count(dim, N, colour);
  const long long total = ncol * M;
  const T ih2 = (T)inv_h2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / ncol, c = idx % ncol;
    long long pp;
    int iy, ix;
    if (colour < 0) {
      pp = c;
      iy = dim == 1 ? 0 : (int)(c / N);
      ix = dim == 1 ? (int)c : (int)(c % N);
    } else {
      pp = colour_pos(dim, N, colour, c, &iy, &ix);
    }
    const T* u = U + m * nf;
    const T uc = u[pp];
    T s = 0;
    if (ix > 0) s += u[pp - 1];
    if (ix < N - 1) s += u[pp + 1];
    if (dim == 2) {
      if (iy > 0) s += u[pp - N];
      if (iy < N - 1) s += u[pp + N];
    }
    const T diag = dim == 1 ? (T)2 : (T)4;
    if (Xo) Xo[m * ncol + c] = uc;
    Bo[m * ncol + c] = F[m * nf + pp] - (diag * uc - s) * ih2;
  }
}

// F = f + d_{m,m} g  (initial data moved to the right-hand side)
template <typename T>
__global__ void add_initial_kernel(long long npts, int M, const T* __restrict__ f, const T* __restrict__ dmm,
                                   const T* __restrict__ g, T* __restrict__ F) {
  const long long total = npts * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / npts, pp = idx % npts;
    F[idx] = f[idx] + (g ? dmm[m] * g[pp] : (T)0);
  }
}

}  // namespace fhmg
