// Exact solve of a coarse level, (R~ (x) I + I (x) A_h) E = RC, used as the coarse-grid
// correction of the cycle below a chosen grid size (the paper recurses to one point; the
// solver on the coarsest grid is a free choice of the multigrid method).
//
// A_h (3-point / 5-point stencil, zero Dirichlet boundaries) has the sine eigenvectors
// sin(p pi n / (N+1)) with eigenvalues (4/h^2) sin^2(p pi / (2(N+1))) (sums of two in 2D), so
// with the orthonormal DST-I matrix S (symmetric, S^2 = I):
//   RC^ = RC S  (along x, then y)        sine_transform_kernel
//   (R~ + lam_p I) w_p = RC^_p           one H-matrix triangular walk per mode (MODE_SMOOTH on
//                                        compact columns, with the mode's own diagonal
//                                        inverses streamed as DIAG chunks)
//   E = W S                               sine_transform_kernel
// All of it runs in FP64.
#pragma once
#include <cuda_runtime.h>

namespace fhmg {

// (D_ii + lam_k I)^{-1} for every diagonal leaf i of R~ and every mode k, in the layout of the
// FP64 DIAG chunks: entry (c, r) of a leaf's inverse at ((c / 2) * L + r) * 2 + c % 2.
// One CTA per (i, k); thread c forward-substitutes (D_ii + lam I) x = e_c (column c).
// Dd: nb leaf blocks, L x L row-major; out: nmodes x nb x L x L.  Dynamic shared memory:
// 2 L^2 doubles.
__global__ void mode_inverse_kernel(const double* __restrict__ Dd, const double* __restrict__ lam, int L, int nb,
                                    double* __restrict__ out) {
  extern __shared__ double sh[];
  double* D = sh;          // D_ii, row-major
  double* X = sh + L * L;  // X[r * L + c], the inverse
  const int i = blockIdx.x, k = blockIdx.y, c = threadIdx.x;
  const double s = lam[k];
  for (int e = c; e < L * L; e += blockDim.x) D[e] = Dd[(size_t)i * L * L + e];
  __syncthreads();
  if (c < L) {
    for (int r = 0; r < c; ++r) X[r * L + c] = 0.0;
    X[c * L + c] = 1.0 / (D[c * L + c] + s);
    for (int r = c + 1; r < L; ++r) {
      double a = 0.0;
      for (int q = c; q < r; ++q) a = fma(D[r * L + q], X[q * L + c], a);
      X[r * L + c] = -a / (D[r * L + r] + s);
    }
  }
  __syncthreads();
  double* o = out + ((size_t)k * nb + i) * L * L;
  for (int e = c; e < L * L; e += blockDim.x) {
    const int g = e / (2 * L), rem = e % (2 * L);
    const int r = rem / 2, col = 2 * g + rem % 2;
    o[e] = X[r * L + col];
  }
}

// out = in multiplied along one spatial axis by the symmetric n x n matrix S (row-major), for
// arrays of M time levels of ny x nx points (space contiguous):
//   axis 0 (x, n = nx): out[m, y, p] = sum_j S[j, p] in[m, y, j]
//   axis 1 (y, n = ny): out[m, p, x] = sum_j S[j, p] in[m, j, x]
// Accumulation in FP64 whatever the storage types.
template <typename Tin, typename Tout>
__global__ void sine_transform_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, const double* __restrict__ S,
                                      long long M, int ny, int nx, int axis) {
  const long long plane = (long long)ny * nx;
  const long long total = M * plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / plane;
    const int rem = (int)(idx - m * plane);
    const int y = rem / nx, x = rem - (rem / nx) * nx;
    double a = 0.0;
    if (axis == 0) {
      const Tin* row = in + m * plane + (long long)y * nx;
      for (int j = 0; j < nx; ++j) a = fma(S[(long long)j * nx + x], (double)row[j], a);
    } else {
      const Tin* col = in + m * plane + x;
      for (int j = 0; j < ny; ++j) a = fma(S[(long long)j * ny + y], (double)col[(long long)j * nx], a);
    }
    out[idx] = (Tout)a;
  }
}

}  // namespace fhmg
