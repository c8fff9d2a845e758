// Exact solve of a coarse level, (R~ (x) I + I (x) A_h) E = RC, used as the coarse-grid
// correction of the cycle below a chosen grid size (the paper recurses to one point; the
// solver on the coarsest grid is a free choice of the multigrid method).
//
// A_h (3-point / 5-point stencil, zero Dirichlet boundaries) has the sine eigenvectors
// sin(p pi n / (N+1)) with eigenvalues (4/h^2) sin^2(p pi / (2(N+1))) (sums of two in 2D), so
// with the orthonormal DST-I matrix S (symmetric, S^2 = I):
//   RC^ = RC S  (along x, then y)        sine_fft_kernel
//   (R~ + lam_p I) w_p = RC^_p           one H-matrix triangular walk per mode (MODE_SMOOTH on
//                                        compact columns, with the mode's own diagonal
//                                        inverses streamed as DIAG chunks)
//   E = W S                               sine_fft_kernel
// All of it runs in FP64.
#pragma once
#include <cuda_runtime.h>

namespace fhmg {

// (D_ii + lam_k I)^{-1} for every diagonal leaf i of R~ and every mode k, in the layout of the
// FP64 DIAG chunks: entry (c, r) of a leaf's inverse at ((c / 2) * L + r) * 2 + c % 2.
// One CTA per (i, k); thread c forward-substitutes (D_ii + lam I) x = e_c (column c).
// Dd: nb leaf blocks, L x L row-major; out: nmodes x nb x L x L.  out_df (optional): the same
// inverses as float pairs in the layout of the double-float DIAG chunks (hi block: entry (c, r) at
// ((c / 4) * L + r) * 4 + c % 4; lo block L^2 floats later), nmodes x nb x 2 L^2 floats.
// Dynamic shared memory: 2 L^2 doubles.
__global__ void mode_inverse_kernel(const double* __restrict__ Dd, const double* __restrict__ lam, int L, int nb,
                                    double* __restrict__ out, float* __restrict__ out_df) {
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
  if (out_df) {
    float* od = out_df + ((size_t)k * nb + i) * 2 * L * L;
    for (int e = c; e < L * L; e += blockDim.x) {
      const int g = e / (4 * L), rem = e % (4 * L);
      const int r = rem / 4, col = 4 * g + rem % 4;
      const double v = X[r * L + col];
      const float hi = __double2float_rn(v);
      od[e] = hi;
      od[L * L + e] = __double2float_rn(v - (double)hi);
    }
  }
}

// out = in multiplied along one spatial axis by the orthonormal DST-I matrix S (symmetric,
// S_jk = sqrt(2/(n+1)) sin(pi j k / (n+1))), through a complex FFT (O(n log n) per line): for one
// line x_1..x_n (n + 1 = 2^p), the odd extension y of length P = 2(n+1)
// (y_0 = y_{n+1} = 0, y_j = x_j, y_{P-j} = -x_j) has DFT Y_k = -2i sum_j x_j sin(pi j k / (n+1)),
// so (S x)_k = sqrt(2/(n+1)) * (-Im Y_k / 2).  One CTA per line, radix-2 decimation in time in
// shared memory (3P doubles); tw holds the twiddles exp(-2 pi i j / P), j < P/2 (cos, sin), built
// once on the host (no FP64 sine evaluation on the device's 1/64-rate FP64 pipe).  Lines: axis 0 =
// the M * ny rows of length nx (contiguous), axis 1 = the M * nx columns of length ny (stride nx).
template <typename Tin, typename Tout>
__global__ void sine_fft_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, const double2* __restrict__ tw,
                                long long M, int ny, int nx, int axis, int log2P) {
  extern __shared__ double sf[];
  const int P = 1 << log2P;
  const int n = P / 2 - 1;
  double* re = sf;
  double* im = sf + P;
  double2* w = reinterpret_cast<double2*>(sf + 2 * P);
  for (int j = threadIdx.x; j < P / 2; j += blockDim.x) w[j] = tw[j];
  const long long line = blockIdx.x;
  long long base, stride;
  if (axis == 0) {
    base = line * nx;
    stride = 1;
  } else {
    const long long m = line / nx, x = line % nx;
    base = m * (long long)ny * nx + x;
    stride = nx;
  }
  // odd extension, stored at bit-reversed positions
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double v = 0.0;
    if (j >= 1 && j <= n) v = (double)in[base + (long long)(j - 1) * stride];
    else if (j >= n + 2) v = -(double)in[base + (long long)(P - j - 1) * stride];
    const int r = (int)(__brev((unsigned)j) >> (32 - log2P));
    re[r] = v;
    im[r] = 0.0;
  }
  __syncthreads();
  for (int len = 2, s = 1; len <= P; len <<= 1, ++s) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < P / 2; b += blockDim.x) {
      const int grp = b / half, pos = b % half;
      const int i0 = grp * len + pos, i1 = i0 + half;
      const double2 cw = w[pos << (log2P - s)];  // exp(-2 pi i pos / len)
      const double tr = re[i1] * cw.x - im[i1] * cw.y;
      const double ti = re[i1] * cw.y + im[i1] * cw.x;
      re[i1] = re[i0] - tr;
      im[i1] = im[i0] - ti;
      re[i0] += tr;
      im[i0] += ti;
    }
    __syncthreads();
  }
  const double sc = -0.5 * sqrt(2.0 / (n + 1));
  for (int k = threadIdx.x; k < n; k += blockDim.x) out[base + (long long)k * stride] = (Tout)(sc * im[k + 1]);
}

}  // namespace fhmg
