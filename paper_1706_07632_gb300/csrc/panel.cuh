// The H-matrix panel walk (hot path): smoother half-sweeps (Algorithm 4 per time line) and
// defect products (Algorithm 3 per time line) over a panel of TC spatial columns.
//
// A CTA owns TC time lines (columns) at a time and walks the leaf rows i = 0..nb-1 of the time
// matrix in order; it is persistent over column tiles.  The H-matrix data arrive as a stream of
// chunks (near-field blocks, slabs of the low-rank factors U and V, the diagonal block or its
// level inverse), in exactly the order the walk consumes them.  Thread 0 keeps NS chunks in
// flight: each chunk is one cp.async.bulk (TMA bulk copy, global -> shared) into a ring slot,
// completing on that slot's mbarrier; every thread waits on the slot's mbarrier (bounded spin)
// before using it, and the slot is refilled after the block-wide barrier that ends the chunk.
// All columns of the tile reuse every staged chunk.
//
// Per leaf row i the accumulators start from the right-hand side (smoother: F + neighbour
// sum / h^2; product: B), then
//   DENSE(j): y -= D_ij x_j     x_j from the shared ring of recent leaf tiles
//   UPART   : y -= U_i[:, k] z_k  z from the shared pool of low-rank coefficients
//   DIAG    : smoother x_i = (D_ii + s I)^{-1} y; product OUT = y - D_ii x_i
//   VPART   : z_k (+)= V_i[k, :] x_i   (the low-rank B^T x of Algorithms 3 and 4)
// Columns are independent (red-black: the other colour is frozen), so CTAs never communicate.
//
// T is the type of the grid functions and of the accumulation, TM the type of the H-matrix
// products (double, or float for the mixed path -- see ddiag).  Every (row, column) output is
// split over S threads along its reduction, combined by xor-shuffles, so a CTA with one column
// still spreads a leaf step over the whole block (the coarse grids are latency-bound).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fhmg {

struct PanelDev {
  const unsigned char* pkg;  // chunk bytes
  const int4* chunks;        // type | count << 4, aux, bytes, offset / 16
  const int* cptr;           // nb + 1
  int nb, L, pool, W, slot_bytes, ns;
};

template <int L, int TC, int NT_>
struct PTile {
  static constexpr int NT = NT_;
  static constexpr int S0 = (NT / L) / TC;
  static constexpr int S = S0 < 1 ? 1 : S0;     // splits per output
  static constexpr int RG = NT / (TC * S);      // row groups
  static constexpr int Q = L / RG;              // rows per thread
  static_assert(RG <= L && L % RG == 0 && TC * S <= 32 && 32 % (TC * S) == 0, "tile shape");
};

enum { MODE_SMOOTH = 0, MODE_MATVEC = 1 };
enum { PK_DENSE = 0, PK_UPART = 1, PK_DIAG = 2, PK_VPART = 3 };

constexpr long long kSpinLimit = 1LL << 24;  // bounded mbarrier wait (then error flag + exit)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// one TMA bulk copy global -> shared, completing bytes on the slot's mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename T, int TC, int S>
__device__ __forceinline__ T reduce_splits(T v) {
#pragma unroll
  for (int o = TC; o < TC * S; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout, in bytes from the (16-byte aligned) dynamic base.
struct PanelSmem {
  size_t ys, ysm, ring, zp, bar, flag, total;
};
__host__ __device__ inline PanelSmem panel_smem(int L, int TC, int pool, int W, int slot_bytes, int ns, int bT,
                                                int bTM) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  PanelSmem s;
  s.ys = a16((size_t)ns * slot_bytes);
  s.ysm = a16(s.ys + (size_t)L * TC * bT);
  s.ring = a16(s.ysm + (size_t)L * TC * bTM);
  s.zp = a16(s.ring + (size_t)W * L * TC * bTM);
  s.bar = a16(s.zp + (size_t)pool * TC * bTM);
  s.flag = s.bar + 8 * (size_t)ns;
  s.total = a16(s.flag + 16);
  return s;
}

// One walk job: one instance (H-matrix, grid, arrays) of a batched launch.
//   MODE_SMOOTH: X (at geometry positions) = (R~ + s I)^{-1} (F + neighbour sum / h^2);
//     B = F; Dinv = the level's inverted diagonal leaves (streamed as the DIAG chunks).
//   MODE_MATVEC: OUT = B - R~ X on compact columns (ld = geo.ld); OUT may alias B or be NULL;
//     norm != NULL folds max |OUT| into *norm (bit pattern of a non-negative double).
//   ddiag (FP64-storage mixed path only): the FP64 diagonal of the streamed DIAG blocks, nb x L;
//     the streamed blocks' own diagonal is then skipped and the diagonal term applied in T.
constexpr int kMaxJobs = 64;

template <typename T, typename TM>
struct WalkJob {
  PanelDev P;       // the job's chunk stream (P.ns unused)
  Geo geo;
  long long ncols;
  long long tile0;  // first global tile of the job
  T* X;
  const T* B;
  T* OUT;
  const TM* Dinv;
  const T* ddiag;
  unsigned long long* norm;
};

// A launch: up to kMaxJobs jobs with the same leaf size, column tile and mode, passed by value
// (kernel parameter space).  The shared-memory layout uses the maxima over the jobs.
template <typename T, typename TM>
struct WalkBatch {
  int njobs;
  int ns, pool, W, slot_bytes;
  long long ntiles;  // tiles over all jobs
  int* err;          // set to 1 if an mbarrier wait exceeds kSpinLimit (the kernel then returns)
  WalkJob<T, TM> job[kMaxJobs];
};

template <typename T, typename TM>
__device__ __forceinline__ int job_of(const WalkBatch<T, TM>& B, long long g) {
  int j = 0;
  while (j + 1 < B.njobs && B.job[j + 1].tile0 <= g) ++j;
  return j;
}

template <typename T, typename TM, int L, int TC, int MODE, int NT_>
__global__ void __launch_bounds__(NT_) hpanel_kernel(const __grid_constant__ WalkBatch<T, TM> B) {
  using TL = PTile<L, TC, NT_>;
  constexpr int NT = TL::NT, Q = TL::Q, RG = TL::RG, S = TL::S;
  constexpr int KS = L / S;
  constexpr int NA = KS >= 4 ? 4 : KS;
  extern __shared__ __align__(16) unsigned char sm[];
  const PanelSmem lay = panel_smem(L, TC, B.pool, B.W, B.slot_bytes, B.ns, sizeof(T), sizeof(TM));
  unsigned char* slots = sm;
  T* ys = reinterpret_cast<T*>(sm + lay.ys);     // y / x of the current leaf (T)
  TM* ysm = reinterpret_cast<TM*>(sm + lay.ysm);  // the same in TM, converted once per leaf
  TM* ring = reinterpret_cast<TM*>(sm + lay.ring);
  TM* zp = reinterpret_cast<TM*>(sm + lay.zp);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + lay.bar);
  volatile int* sflag = reinterpret_cast<volatile int*>(sm + lay.flag);

  const int t = threadIdx.x;
  const int cl = t % TC;
  const int sp = (t / TC) % S;
  const int rg = t / (TC * S);
  const int ns = B.ns;
  const int W = B.W;

  // producer cursor (thread 0): the next (tile, chunk) to stage, in consumption order
  long long pg = blockIdx.x;
  int pj = pg < B.ntiles ? job_of(B, pg) : 0;
  int pc = 0;
  long long issued = 0;
  auto issue_next = [&]() {
    if (pg >= B.ntiles) return;
    const WalkJob<T, TM>& J = B.job[pj];
    const int4 cd = __ldg(J.P.chunks + pc);
    const int type = cd.x & 15;
    const void* src = (MODE == MODE_SMOOTH && type == PK_DIAG)
                          ? (const void*)(J.Dinv + (long long)cd.y * L * L)
                          : (const void*)(J.P.pkg + 16LL * (long long)cd.w);
    const int slot = (int)(issued % ns);
    bulk_load(slots + (size_t)slot * B.slot_bytes, src, (uint32_t)cd.z, bar + slot);
    ++issued;
    if (++pc == __ldg(J.P.cptr + J.P.nb)) {
      pc = 0;
      pg += gridDim.x;
      if (pg < B.ntiles) pj = job_of(B, pg);
    }
  };

  if (t == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(bar + s, 1);
    *sflag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0)
    for (int s = 0; s < ns; ++s) issue_next();

  long long pos = 0;
  for (long long g = blockIdx.x; g < B.ntiles; g += gridDim.x) {
    const WalkJob<T, TM>& J = B.job[job_of(B, g)];
    const long long cg = (g - J.tile0) * TC + cl;
    const bool valid = cg < J.ncols;
    const long long ld = J.geo.ld;
    const T inv_h2 = (T)J.geo.inv_h2;
    T* X = J.X;
    const T* Bsrc = J.B;
    const int nb = J.P.nb;
    long long p = 0;
    long long nbr[4] = {-1, -1, -1, -1};
    if (valid) {
      if (MODE == MODE_SMOOTH && J.geo.dim > 0) {
        int iy, ix;
        p = colour_pos(J.geo.dim, J.geo.N, J.geo.colour, cg, &iy, &ix);
        nbr[0] = ix > 0 ? p - 1 : -1;
        nbr[1] = ix < J.geo.N - 1 ? p + 1 : -1;
        if (J.geo.dim == 2) {
          nbr[2] = iy > 0 ? p - J.geo.N : -1;
          nbr[3] = iy < J.geo.N - 1 ? p + J.geo.N : -1;
        }
      } else {
        p = cg;
      }
    }
    double local_max = 0.0;
    // right-hand side (and, for the product, the x tile) of the next leaf, prefetched
    T bn[Q], xn[Q];
    auto load_rhs = [&](int leaf) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = rg + RG * q;
        T b = 0, x = 0;
        if (valid && sp == 0 && leaf < nb) {
          const long long base = (long long)(leaf * L + r) * ld;
          b = Bsrc[base + p];
          if (MODE == MODE_SMOOTH) {
            T s = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (nbr[e] >= 0) s += X[base + nbr[e]];
            b += s * inv_h2;
          } else {
            x = X[base + p];
          }
        }
        bn[q] = b;
        xn[q] = x;
      }
    };
    load_rhs(0);

    for (int i = 0; i < nb; ++i) {
      T acc[Q];
      TM part[Q][NA];
      T xcur[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        acc[q] = bn[q];
        xcur[q] = xn[q];
#pragma unroll
        for (int a = 0; a < NA; ++a) part[q][a] = 0;
      }
      const int c1 = __ldg(J.P.cptr + i + 1);
      for (int c = __ldg(J.P.cptr + i); c < c1; ++c, ++pos) {
        const int slot = (int)(pos % ns);
        if (!mbar_wait(bar + slot, (uint32_t)((pos / ns) & 1))) {
          *sflag = 1;
          atomicExch(B.err, 1);
        }
        const int4 cd = __ldg(J.P.chunks + c);
        const int type = cd.x & 15, cnt = cd.x >> 4;
        const unsigned char* buf = slots + (size_t)slot * B.slot_bytes;
        if (type == PK_DENSE) {
          const TM* D = reinterpret_cast<const TM*>(buf);
          const int j = cd.y;
          if (i - j < W) {
            const TM* xr = ring + (size_t)(j % W) * L * TC;
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
              const int k = sp + kk * S;
              const TM xv = xr[k * TC + cl];
#pragma unroll
              for (int q = 0; q < Q; ++q) part[q][kk % NA] += D[k * L + rg + RG * q] * xv;
            }
          } else {
            const T* xj = X + (long long)j * L * ld + p;
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
              const int k = sp + kk * S;
              const TM xv = valid ? (TM)xj[(long long)k * ld] : (TM)0;
#pragma unroll
              for (int q = 0; q < Q; ++q) part[q][kk % NA] += D[k * L + rg + RG * q] * xv;
            }
          }
        } else if (type == PK_UPART) {
          const TM* U = reinterpret_cast<const TM*>(buf);
          const int* uz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * sizeof(TM));
          int a = 0;
          for (int kk = sp; kk < cnt; kk += S) {
            const TM zv = zp[uz[kk] * TC + cl];
#pragma unroll
            for (int q = 0; q < Q; ++q) part[q][a] += U[kk * L + rg + RG * q] * zv;
            a = (a + 1 == NA) ? 0 : a + 1;
          }
        } else if (type == PK_DIAG) {
          const TM* Dd = reinterpret_cast<const TM*>(buf);
          const T* ddiag = J.ddiag;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            TM s = part[q][0];
#pragma unroll
            for (int a = 1; a < NA; ++a) s += part[q][a];
            acc[q] = reduce_splits<T, TC, S>(acc[q] - (T)s);
          }
          TM* xr_i = ring + (size_t)(i % W) * L * TC;
          if (MODE == MODE_SMOOTH) {
            if (sp == 0) {
#pragma unroll
              for (int q = 0; q < Q; ++q) {
                ys[(rg + RG * q) * TC + cl] = acc[q];
                ysm[(rg + RG * q) * TC + cl] = (TM)acc[q];
              }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              const int r = rg + RG * q;
              TM s[NA];
#pragma unroll
              for (int a = 0; a < NA; ++a) s[a] = 0;
#pragma unroll
              for (int kk = 0; kk < KS; ++kk) {
                const int k = sp + kk * S;
                if (ddiag ? k < r : k <= r) s[kk % NA] += Dd[k * L + r] * ysm[k * TC + cl];
              }
              TM s1 = s[0];
#pragma unroll
              for (int a = 1; a < NA; ++a) s1 += s[a];
              T x = reduce_splits<T, TC, S>((T)s1);
              if (ddiag) x += ddiag[(long long)i * L + r] * ys[r * TC + cl];
              acc[q] = x;
            }
            __syncthreads();
            if (sp == 0) {
#pragma unroll
              for (int q = 0; q < Q; ++q) {
                const int r = rg + RG * q;
                const TM xm = (TM)acc[q];
                ysm[r * TC + cl] = xm;
                xr_i[r * TC + cl] = xm;
                if (valid) X[(long long)(i * L + r) * ld + p] = acc[q];
              }
            }
          } else {
            if (sp == 0) {
#pragma unroll
              for (int q = 0; q < Q; ++q) {
                const int r = rg + RG * q;
                const TM xm = (TM)xcur[q];
                ys[r * TC + cl] = xcur[q];
                ysm[r * TC + cl] = xm;
                xr_i[r * TC + cl] = xm;
              }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              const int r = rg + RG * q;
              TM s[NA];
#pragma unroll
              for (int a = 0; a < NA; ++a) s[a] = 0;
#pragma unroll
              for (int kk = 0; kk < KS; ++kk) {
                const int k = sp + kk * S;
                if (ddiag ? k < r : k <= r) s[kk % NA] += Dd[k * L + r] * ysm[k * TC + cl];
              }
              TM s1 = s[0];
#pragma unroll
              for (int a = 1; a < NA; ++a) s1 += s[a];
              T o = acc[q] - reduce_splits<T, TC, S>((T)s1);
              if (ddiag) o -= ddiag[(long long)i * L + r] * ys[r * TC + cl];
              if (valid && sp == 0) {
                if (J.OUT) J.OUT[(long long)(i * L + r) * ld + p] = o;
                const double av = fabs((double)o);
                local_max = (av > local_max || av != av) ? av : local_max;
              }
            }
          }
          load_rhs(i + 1);  // the next leaf's loads overlap the V slabs and the next chunk waits
        } else {  // PK_VPART
          const TM* V = reinterpret_cast<const TM*>(buf);
          const int* vz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * sizeof(TM));
          const int O = cnt * TC;
          int Sv = 32;
          while (Sv > 1 && Sv * O > NT) Sv >>= 1;
          const int gq = t / Sv, sv = t % Sv, G = NT / Sv;
          for (int base = 0; base < O; base += G) {
            const int o = base + gq;
            TM s = 0;
            if (o < O) {
              const int kk = o / TC, cc = o % TC;
              for (int k = sv; k < L; k += Sv) s += V[kk * L + k] * ysm[k * TC + cc];
            }
            for (int w = Sv >> 1; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
            if (o < O && sv == 0) {
              const int kk = o / TC, cc = o % TC;
              const int code = vz[kk];
              TM* z = zp + (code >> 1) * TC + cc;
              *z = (code & 1) ? s : *z + s;
            }
          }
        }
        __syncthreads();  // the slot and every shared-memory write of this chunk are done
        if (*sflag) {
          // drain (bounded) the copies still in flight, then leave
          if (t == 0)
            for (long long q2 = pos + 1; q2 < issued; ++q2) mbar_wait(bar + (int)(q2 % ns), (uint32_t)((q2 / ns) & 1));
          return;
        }
        if (t == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_next();
        }
      }
    }
    if (MODE == MODE_MATVEC && J.norm != nullptr) {
      for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, local_max, o);
        local_max = (other > local_max || other != other) ? other : local_max;
      }
      if ((t & 31) == 0) atomicMax(J.norm, (unsigned long long)__double_as_longlong(local_max));
    }
  }
}

}  // namespace fhmg
