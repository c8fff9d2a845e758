// CUDA kernels (sm_103a) for multigrid waveform relaxation with an H-matrix time operator.
//
// Grid functions are time-major with space contiguous: value (m, p) at m * ld + p, m = 0..M-1
// standing for t_1..t_M, p the spatial index (1D: p = n - 1; 2D: p = iy * N + ix).
//
// The H-matrix walk (hwalk_kernel) is the hot path.  One CTA owns TC spatial columns
// (time lines) and walks the M/L leaf rows of the time matrix in order.  For leaf row i it
//   1. forms the right-hand side of its TC columns for the L time levels of the leaf,
//   2. subtracts the dense near-field blocks D_ij x_j (j < i) read back from its own output,
//   3. subtracts the low-rank contributions U_i Z_i, Z held per block in a shared-memory
//      pool of k-row vectors (z = V^T x_sigma accumulated while sigma is being produced),
//   4. SMOOTH: x_i = (D_ii + s I)^-1 y (inverse precomputed per level, Algorithm 4's
//      dense-leaf solve); MATVEC: y -= D_ii x_i (Algorithm 3's dense-leaf product),
//   5. stores the leaf and folds it into the pool: Z += V_i^T x_i (Algorithms 3/4's
//      low-rank factor B^T x, started on the first leaf of sigma).
// Every column is independent (red-black: the other colour is frozen), so there is no
// inter-CTA communication; the sequential dependency is only along time within a CTA.
//
// Matrices are stored column-major on the device (element (r, k) at k * rows + r) so that
// the threads of a warp, which own consecutive rows, read consecutive addresses.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fhmg {

template <typename T>
struct HDev {
  const T* dense;         // nd x (L x L), column-major blocks
  const int* dptr;        // nb+1
  const int* dblk;        // dense off-diagonal block ids per leaf row
  const int* dcol;        // their leaf-column index
  const int* diag;        // nb: block id of the diagonal block
  const int* uptr;        // nb+1
  const int* uz;          // pool row per U-panel column
  const long long* uoff;  // nb: offset of the L x K_i panel (column-major)
  const T* udata;
  const int* vptr;        // nb+1
  const int* vz;          // pool row per V-panel row
  const int* vinit;       // 1: assign (first leaf of sigma), 0: accumulate
  const long long* voff;  // nb: offset of the K'_i x L panel (column-major)
  const T* vdata;
  int M, L, nb, pool;
};

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

// Thread layout of a walk CTA: NT = 256 threads own the L x TC tile of one leaf row; every
// (row, column) output is split over S threads along its reduction (k) dimension, so that a
// CTA with a single column still spreads one leaf step over the whole block.  Thread t:
// column c = t % TC, split s = (t / TC) % S, row group rg = t / (TC S), rows rg + RG q.
// The S partial sums of an output sit in lanes TC apart inside one warp (TC S <= 32) and are
// combined with xor-shuffles.
template <int L, int TC>
struct Tile {
  static constexpr int NT = 256;
  static constexpr int S0 = (NT / L) / TC;
  static constexpr int S = S0 < 1 ? 1 : S0;
  static constexpr int RG = NT / (TC * S);
  static constexpr int Q = L / RG;  // rows per thread
  static_assert(RG <= L && L % RG == 0 && TC * S <= 32, "tile shape");
};

enum { MODE_SMOOTH = 0, MODE_MATVEC = 1 };

template <typename T, int TC, int S>
__device__ __forceinline__ T reduce_splits(T v) {
#pragma unroll
  for (int o = TC; o < TC * S; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

// MODE_SMOOTH: X (at geometry positions) = (R~ + s I)^{-1} (F + neighbour sum / h^2), with
//   Xw = X (grid array read for neighbours and written), Bsrc = F, Dinv the level inverses.
// MODE_MATVEC: OUT = B - R~ X on compact columns (ld = geo.ld); OUT may alias B; if
//   norm != nullptr the max |OUT| is folded into *norm (bit pattern of a non-negative double).
template <typename T, int L, int TC, int MODE>
__global__ void __launch_bounds__(256)
hwalk_kernel(HDev<T> H, Geo geo, long long ncols, T* X, const T* Bsrc, T* OUT, const T* Dinv,
             unsigned long long* norm) {
  using TL = Tile<L, TC>;
  constexpr int NT = TL::NT, Q = TL::Q, RG = TL::RG, S = TL::S;
  extern __shared__ unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);  // [L][TC]
  T* zp = ys + L * TC;                      // [pool][TC]

  const int t = threadIdx.x;
  const int cl = t % TC;
  const int sp = (t / TC) % S;
  const int rg = t / (TC * S);
  const long long cg = (long long)blockIdx.x * TC + cl;
  const bool valid = cg < ncols;
  const long long ld = geo.ld;

  long long p = 0;
  long long nbr[4] = {-1, -1, -1, -1};
  if (valid) {
    if (MODE == MODE_SMOOTH && geo.dim > 0) {
      int iy, ix;
      p = colour_pos(geo.dim, geo.N, geo.colour, cg, &iy, &ix);
      nbr[0] = ix > 0 ? p - 1 : -1;
      nbr[1] = ix < geo.N - 1 ? p + 1 : -1;
      if (geo.dim == 2) {
        nbr[2] = iy > 0 ? p - geo.N : -1;
        nbr[3] = iy < geo.N - 1 ? p + geo.N : -1;
      }
    } else {
      p = cg;
    }
  }
  const T inv_h2 = (T)geo.inv_h2;
  double local_max = 0.0;

  for (int i = 0; i < H.nb; ++i) {
    const int m0 = i * L;
    T acc[Q];
    // 1. right-hand side (split 0 only; the other splits start from zero)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int r = rg + RG * q;
      T b = 0;
      if (valid && sp == 0) {
        const long long base = (long long)(m0 + r) * ld;
        b = Bsrc[base + p];
        if (MODE == MODE_SMOOTH) {
          T s = 0;
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (nbr[e] >= 0) s += X[base + nbr[e]];
          b += s * inv_h2;
        }
      }
      acc[q] = b;
    }
    // 2. dense near-field blocks, x_j read back from this CTA's own output
    const int d1 = ldro(H.dptr + i + 1);
    for (int d = ldro(H.dptr + i); d < d1; ++d) {
      const T* D = H.dense + (long long)ldro(H.dblk + d) * L * L;
      const T* xj = X + (long long)ldro(H.dcol + d) * L * ld + p;
#pragma unroll 4
      for (int k = sp; k < L; k += S) {
        const T xv = valid ? xj[(long long)k * ld] : (T)0;
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] -= ldro(D + k * L + rg + RG * q) * xv;
      }
    }
    // 3. low-rank contributions U_i Z_i
    {
      const int k0 = ldro(H.uptr + i), K = ldro(H.uptr + i + 1) - k0;
      const T* U = H.udata + ldro(H.uoff + i);
#pragma unroll 2
      for (int kk = sp; kk < K; kk += S) {
        const T zv = zp[ldro(H.uz + k0 + kk) * TC + cl];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] -= ldro(U + kk * L + rg + RG * q) * zv;
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = reduce_splits<T, TC, S>(acc[q]);
    // 4. diagonal leaf
    if (MODE == MODE_SMOOTH) {
      const T* Dd = Dinv + (long long)i * L * L;
      if (sp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) ys[(rg + RG * q) * TC + cl] = acc[q];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = rg + RG * q;
        T s = 0;
        for (int k = sp; k <= r; k += S) s += ldro(Dd + k * L + r) * ys[k * TC + cl];
        acc[q] = reduce_splits<T, TC, S>(s);
      }
      __syncthreads();
      if (sp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int r = rg + RG * q;
          ys[r * TC + cl] = acc[q];
          if (valid) X[(long long)(m0 + r) * ld + p] = acc[q];
        }
      }
      __syncthreads();
    } else {
      const T* Dd = H.dense + (long long)ldro(H.diag + i) * L * L;
      if (sp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int r = rg + RG * q;
          ys[r * TC + cl] = valid ? X[(long long)(m0 + r) * ld + p] : (T)0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = rg + RG * q;
        T s = 0;
        for (int k = sp; k <= r; k += S) s += ldro(Dd + k * L + r) * ys[k * TC + cl];
        s = acc[q] - reduce_splits<T, TC, S>(s);
        if (valid && sp == 0) {
          if (OUT) OUT[(long long)(m0 + r) * ld + p] = s;
          const double a = fabs((double)s);
          local_max = (a > local_max || a != a) ? a : local_max;
        }
      }
    }
    // 5. Z += V_i^T x_i : Kv x TC outputs, each a length-L dot product split over Sv lanes
    {
      const int v0 = ldro(H.vptr + i), Kv = ldro(H.vptr + i + 1) - v0;
      if (Kv > 0) {
        const T* V = H.vdata + ldro(H.voff + i);
        const int O = Kv * TC;
        int Sv = 32;
        while (Sv > 1 && Sv * O > NT) Sv >>= 1;
        const int g = t / Sv, sv = t % Sv, G = NT / Sv;
        for (int base = 0; base < O; base += G) {
          const int o = base + g;
          T s = 0;
          if (o < O) {
            const int kk = o / TC, c = o % TC;
            for (int k = sv; k < L; k += Sv) s += ldro(V + k * Kv + kk) * ys[k * TC + c];
          }
          for (int w = Sv >> 1; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
          if (o < O && sv == 0) {
            const int kk = o / TC, c = o % TC;
            T* z = zp + ldro(H.vz + v0 + kk) * TC + c;
            *z = ldro(H.vinit + v0 + kk) ? s : *z + s;
          }
        }
      }
    }
    __syncthreads();
  }
  if (MODE == MODE_MATVEC && norm != nullptr) {
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, local_max, o);
      local_max = (other > local_max || other != other) ? other : local_max;
    }
    if ((t & 31) == 0) atomicMax(norm, (unsigned long long)__double_as_longlong(local_max));
  }
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
