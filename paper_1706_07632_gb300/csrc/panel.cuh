// The H-matrix panel walk (hot path): smoother half-sweeps (Algorithm 4 per time line) and
// defect products (Algorithm 3 per time line) over a panel of TC spatial columns.
//
// A CTA owns TC time lines (columns) at a time and walks the leaf rows i = 0..nb-1 of the time
// matrix in order; it is persistent over column tiles.  The H-matrix data arrive as a stream of
// chunks (near-field blocks, slabs of the low-rank factors U and V, the diagonal block or its
// level inverse), in exactly the order the walk consumes them.  A producer warp keeps NS chunks
// in flight: each chunk is one cp.async.bulk (TMA bulk copy, global -> shared) into a ring slot,
// completing on that slot's "full" mbarrier; every consumer thread waits on it before using the
// slot, and each consumer warp arrives on the slot's "empty" mbarrier when done, which lets the
// producer refill it.  Consumer warps therefore run through near-field, low-rank and V chunks
// without block-wide barriers; they meet only in the diagonal step, where y is exchanged and x_i
// published (an mbarrier over the consumer warps).  Every wait is a bounded mbarrier poll that
// also watches a shared abort flag: a warp whose wait gives up sets the flag and the error word
// and leaves, and every other wait then ends too, so no thread can be left waiting.
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
// still spreads a leaf step over the whole block (the coarse grids are latency-bound).  The
// chunk matrices are vector-interleaved (16-byte vectors of consecutive reduction indices, one
// vector per row, rows consecutive): a thread reads its row's vectors with 16-byte loads and the
// eight lanes of a shared-memory wavefront read eight consecutive rows of one split, so matrix
// and x-tile reads are free of bank conflicts.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fhmg {

struct PanelDev {
  const unsigned char* pkg;  // chunk bytes
  const int4* chunks;        // type | count << 4 | last << 12, aux, bytes, offset / 16
  const int* cptr;           // nb + 1
  int nb, L, pool, W, slot_bytes, ns;
  int far;                   // 1: some near-field block lies beyond the ring of W leaf tiles
};

// 16-byte vectors of the chunk layout
template <typename TM>
struct VecOf;
template <>
struct VecOf<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct VecOf<double> {
  using type = double2;
  static constexpr int n = 2;
};

// a += d .* x into four independent accumulators (gg: the vector's place in a thread's sequence)
__device__ __forceinline__ void vfma(float (&a)[4], int, const float4 d, const float4 x) {
  a[0] = fmaf(d.x, x.x, a[0]);
  a[1] = fmaf(d.y, x.y, a[1]);
  a[2] = fmaf(d.z, x.z, a[2]);
  a[3] = fmaf(d.w, x.w, a[3]);
}
__device__ __forceinline__ void vfma(double (&a)[4], int gg, const double2 d, const double2 x) {
  const int o = (gg & 1) * 2;
  a[o] = fma(d.x, x.x, a[o]);
  a[o + 1] = fma(d.y, x.y, a[o + 1]);
}
template <typename TM>
__device__ __forceinline__ TM sum4(const TM (&a)[4]) {
  return (a[0] + a[1]) + (a[2] + a[3]);
}
// VE consecutive z-pool entries named by an index vector
__device__ __forceinline__ float4 gather_z(const float* zp, const int* idx, int TC, int cl) {
  const int4 k = *reinterpret_cast<const int4*>(idx);
  return make_float4(zp[k.x * TC + cl], zp[k.y * TC + cl], zp[k.z * TC + cl], zp[k.w * TC + cl]);
}
__device__ __forceinline__ double2 gather_z(const double* zp, const int* idx, int TC, int cl) {
  const int2 k = *reinterpret_cast<const int2*>(idx);
  return make_double2(zp[k.x * TC + cl], zp[k.y * TC + cl]);
}
// VE consecutive rows k0.. of one global column (stride ld), converted to TM
template <typename T>
__device__ __forceinline__ float4 load_col(const T* x, long long k0, long long ld, bool ok, float*) {
  if (!ok) return make_float4(0.f, 0.f, 0.f, 0.f);
  return make_float4((float)x[k0 * ld], (float)x[(k0 + 1) * ld], (float)x[(k0 + 2) * ld], (float)x[(k0 + 3) * ld]);
}
template <typename T>
__device__ __forceinline__ double2 load_col(const T* x, long long k0, long long ld, bool ok, double*) {
  if (!ok) return make_double2(0.0, 0.0);
  return make_double2((double)x[k0 * ld], (double)x[(k0 + 1) * ld]);
}

// Thread tile of the walk: TC columns, each (row, column) output split over S threads that
// take the reduction's 16-byte vectors round robin.  Lane = column + TC * (row + RL * split), so
// the xor-shuffles that combine the splits use lane offsets TC * RL, 2 TC * RL, ...  When the
// block has more threads than outputs x splits (small leaves), the surplus warps stay idle.
template <int L, int TC, int NT_, int VE>
struct PTile {
  static constexpr int NT = NT_;
  static constexpr int NV = L / VE;                // vectors along a full reduction
  static constexpr int S1 = (NT / L) / TC;
  static constexpr int S0 = S1 < 1 ? 1 : S1;
  static constexpr int S = S0 > NV ? NV : S0;      // splits per output
  static constexpr int RL = 32 / (TC * S);         // rows per warp
  static constexpr int RG0 = NT / (TC * S);
  static constexpr int RG = RG0 > L ? L : RG0;     // active row groups
  static constexpr int Q = L / RG;                 // rows per thread
  static constexpr int NVT = NV / S;               // vectors per thread of a full reduction
  static_assert(TC * S <= 32 && 32 % (TC * S) == 0 && L % RG == 0 && NV % S == 0 && RG % RL == 0,
                "tile shape");
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

// a consumer warp's release of a slot (one arrival per warp)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait (limit polls) that also gives up once *abort is set
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                   long long limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort) return false;
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

// sum over the S splits of an output (lane offsets STEP, 2 STEP, ... < 32)
template <typename T, int STEP>
__device__ __forceinline__ T reduce_splits(T v) {
#pragma unroll
  for (int o = STEP; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout, in bytes from the (16-byte aligned) dynamic base.  x tiles (the current
// leaf's y, the ring of recent leaves' x) are stored per column with a padded length L + VE, so
// that 16-byte reads of different columns fall in different banks.
struct PanelSmem {
  size_t ysm, ring, zp, bar, ebar, cbar, desc, flag, total;
};
__host__ __device__ inline PanelSmem panel_smem(int L, int TC, int pool, int W, int slot_bytes, int ns, int bTM) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t LP = (size_t)L + 16 / bTM;
  PanelSmem s;
  s.ysm = a16((size_t)ns * slot_bytes);
  s.ring = a16(s.ysm + (size_t)TC * LP * bTM);
  s.zp = a16(s.ring + (size_t)W * TC * LP * bTM);
  s.bar = a16(s.zp + (size_t)pool * TC * bTM);  // "full" mbarriers
  s.ebar = s.bar + 8 * (size_t)ns;                 // "empty" mbarriers
  s.cbar = s.ebar + 8 * (size_t)ns;                // the consumer warps' own barrier
  s.desc = a16(s.cbar + 8);                        // descriptor of the chunk in each slot
  s.flag = s.desc + 16 * (size_t)ns;
  s.total = a16(s.flag + 16);
  return s;
}

// One walk job: one instance (H-matrix, grid, arrays) of a batched launch.
//   MODE_SMOOTH: X (at geometry positions) = (R~ + s I)^{-1} (F + neighbour sum / h^2);
//     B = F; Dinv = the level's inverted diagonal leaves (streamed as the DIAG chunks).
//   MODE_MATVEC: OUT = B - R~ X on compact columns (ld = geo.ld); OUT may alias B or be NULL;
//     norm != NULL folds max |OUT| into *norm (bit pattern of a non-negative double).
//   ddiag (FP32 products, required): the diagonal of the streamed DIAG blocks, nb x L, in T; the
//     FP32 blocks are stored without it and the diagonal term is applied in T.
//   dinv_cstride (smoother, one column per tile only): column c streams its own inverse set
//     Dinv + c * dinv_cstride (a per-column shift, e.g. one spatial eigenmode per column).
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
  long long dinv_cstride;
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
  int* err;          // set to 1 if a bounded mbarrier wait gives up (the kernel then returns)
  long long spin;    // poll limit of the consumer warps' waits (the producer keeps kSpinLimit)
  long long withhold;  // > 0: every producer stops before issuing its chunk number withhold - 1
                       // (test hook: the consumers' waits then run out; nothing else changes)
  WalkJob<T, TM> job[kMaxJobs];
};

template <typename T, typename TM>
__device__ __forceinline__ int job_of(const WalkBatch<T, TM>& B, long long g) {
  int j = 0;
  while (j + 1 < B.njobs && B.job[j + 1].tile0 <= g) ++j;
  return j;
}

// NT_ consumer threads (the walk) + one producer warp (the chunk stream).
template <typename T, typename TM, int L, int TC, int MODE, int NT_>
__global__ void __launch_bounds__(NT_ + 32) hpanel_kernel(const __grid_constant__ WalkBatch<T, TM> B) {
  using VT = typename VecOf<TM>::type;
  constexpr int VE = VecOf<TM>::n;
  using TL = PTile<L, TC, NT_, VE>;
  constexpr int NT = NT_;
  constexpr int Q = TL::Q, RG = TL::RG, S = TL::S, RL = TL::RL, NVT = TL::NVT;
  constexpr int STEP = TC * RL;            // lane offset between splits
  constexpr int LP = L + VE;               // padded x-tile column
  constexpr bool SPLITD = sizeof(TM) < 8;  // FP32 products: diagonal from ddiag, in T
  extern __shared__ __align__(16) unsigned char sm[];
  const PanelSmem lay = panel_smem(L, TC, B.pool, B.W, B.slot_bytes, B.ns, sizeof(TM));
  unsigned char* slots = sm;
  TM* ysm = reinterpret_cast<TM*>(sm + lay.ysm);  // y of the current leaf (smoother), in TM
  TM* ring = reinterpret_cast<TM*>(sm + lay.ring);
  TM* zp = reinterpret_cast<TM*>(sm + lay.zp);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + lay.bar);
  uint64_t* empty = reinterpret_cast<uint64_t*>(sm + lay.ebar);
  uint64_t* cbar = reinterpret_cast<uint64_t*>(sm + lay.cbar);
  int4* sdesc = reinterpret_cast<int4*>(sm + lay.desc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + lay.flag);

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int ns = B.ns;
  const int W = B.W;

  if (t == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, NT / 32);
    }
    mbar_init(cbar, NT / 32);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the last block-wide barrier: from here on the roles run apart

  if (t >= NT) {
    // ---- producer: one lane streams every chunk of every tile of this CTA, in order ----
    if (t != NT) return;
    long long k = 0;  // chunks issued
    int slot = 0;
    bool ok = true, stop = false;
    for (long long g = blockIdx.x; g < B.ntiles && ok && !stop; g += gridDim.x) {
      const WalkJob<T, TM>& J = B.job[job_of(B, g)];
      const int nch = __ldg(J.P.cptr + J.P.nb);
      int4 cdn = __ldg(J.P.chunks);
      for (int c = 0; c < nch; ++c, ++k) {
        const int4 cd = cdn;
        if (c + 1 < nch) cdn = __ldg(J.P.chunks + c + 1);
        if (k + 1 == B.withhold) {
          stop = true;
          break;
        }
        if (k >= ns && !mbar_wait_or_abort(empty + slot, (uint32_t)(((k / ns) - 1) & 1), abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int type = cd.x & 15;
        const void* src = (MODE == MODE_SMOOTH && type == PK_DIAG)
                              ? (const void*)(J.Dinv + (g - J.tile0) * TC * J.dinv_cstride + (long long)cd.y * L * L)
                              : (const void*)(J.P.pkg + 16LL * (long long)cd.w);
        sdesc[slot] = cd;  // published by the mbarrier arrive below (release), read after the wait
        bulk_load(slots + (size_t)slot * B.slot_bytes, src, (uint32_t)cd.z, full + slot);
        if (++slot == ns) slot = 0;
      }
    }
    if (!ok && !*abort_flag) {  // timed out waiting for the consumers
      *abort_flag = 1;
      atomicExch(B.err, 1);
    }
    // every copy in flight lands before the CTA may retire (bounded, abort or not)
    for (int s = 0; s < ns && s < k; ++s) {
      const long long n_s = (k - 1 - s) / ns + 1;  // issues into slot s
      mbar_wait(full + s, (uint32_t)((n_s - 1) & 1));
    }
    return;
  }

  // ---- consumers ----
  const int cl = lane % TC;
  const int rl = (lane / TC) % RL;
  const int sp = lane / STEP;
  const int rb0 = (t >> 5) * RL + rl;
  const bool act = rb0 < RG;  // false only in the surplus warps of small leaves
  const int rb = act ? rb0 : 0;
  uint32_t cbphase = 0;  // phase of the consumer barrier
  // warp-uniform exit after a wait that gave up (its own timeout or another warp's abort)
  auto give_up = [&](bool ok) -> bool {
    if (__all_sync(0xffffffffu, ok)) return false;
    if (lane == 0) {
      *abort_flag = 1;
      atomicExch(B.err, 1);
    }
    return true;
  };
  // all consumer warps meet (bounded)
  auto consumer_sync = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const bool ok = mbar_wait_or_abort(cbar, cbphase, abort_flag, B.spin);
    cbphase ^= 1;
    return !give_up(ok);
  };

  int cslot = 0;  // slot and full-barrier phase of the next chunk
  uint32_t cphase = 0;
  for (long long g = blockIdx.x; g < B.ntiles; g += gridDim.x) {
    const WalkJob<T, TM>& J = B.job[job_of(B, g)];
    const long long cg = (g - J.tile0) * TC + cl;
    const bool valid = cg < J.ncols;
    const long long ld = J.geo.ld;
    const T inv_h2 = (T)J.geo.inv_h2;
    T* X = J.X;
    const T* Bsrc = J.B;
    const T* ddg = J.ddiag;
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
    // right-hand side, x tile (product) and diagonal term (FP32 products) of the next leaf,
    // prefetched a leaf ahead by the threads that use them (issued at the diagonal step: issuing
    // them a whole leaf ahead raised the register count past the two-CTA occupancy)
    T bn[Q], xn[Q], dn[Q];
    auto load_rhs = [&](int leaf) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int r = rb + RG * q;
        T b = 0, x = 0, d = 0;
        if (act && sp == 0 && leaf < nb) {
          if (SPLITD) d = ddg[(long long)leaf * L + r];
          if (valid) {
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
        }
        bn[q] = b;
        xn[q] = x;
        dn[q] = d;
      }
    };
    load_rhs(0);

    for (int i = 0; i < nb; ++i) {
      T acc[Q], xcur[Q], ddv[Q];
      TM part[Q][4];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        acc[q] = bn[q];
        xcur[q] = xn[q];
        ddv[q] = dn[q];
#pragma unroll
        for (int a = 0; a < 4; ++a) part[q][a] = 0;
      }
      TM* xr_i = ring + ((i % W) * TC + cl) * LP;  // x_i of this column, once computed
      for (bool leaf_done = false; !leaf_done;) {
        if (give_up(mbar_wait_or_abort(full + cslot, cphase, abort_flag, B.spin))) return;
        const int4 cd = sdesc[cslot];
        leaf_done = ((cd.x >> 12) & 1) != 0;
        const int type = cd.x & 15, cnt = (cd.x >> 4) & 0xff;
        const unsigned char* buf = slots + (size_t)cslot * B.slot_bytes;
        const VT* A = reinterpret_cast<const VT*>(buf);
        if (type == PK_DENSE) {
          const int j = cd.y;
          if (i - j < W) {
            const TM* xr = ring + ((j % W) * TC + cl) * LP;
#pragma unroll
            for (int gg = 0; gg < NVT; ++gg) {
              const int g = sp + gg * S;
              const VT xv = *reinterpret_cast<const VT*>(xr + g * VE);
#pragma unroll
              for (int q = 0; q < Q; ++q) vfma(part[q], gg, A[g * L + rb + RG * q], xv);
            }
          } else {
            const T* xj = X + (long long)j * L * ld + p;
#pragma unroll
            for (int gg = 0; gg < NVT; ++gg) {
              const int g = sp + gg * S;
              const VT xv = load_col(xj, (long long)g * VE, ld, valid, (TM*)nullptr);
#pragma unroll
              for (int q = 0; q < Q; ++q) vfma(part[q], gg, A[g * L + rb + RG * q], xv);
            }
          }
        } else if (type == PK_UPART) {
          const int* uz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * sizeof(TM));
          const int nvq = cnt / VE;
#pragma unroll
          for (int gg = 0; gg < NVT; ++gg) {
            const int g = sp + gg * S;
            if (g < nvq) {
              const VT zv = gather_z(zp, uz + g * VE, TC, cl);
#pragma unroll
              for (int q = 0; q < Q; ++q) vfma(part[q], gg, A[g * L + rb + RG * q], zv);
            }
          }
        } else if (type == PK_DIAG) {
#pragma unroll
          for (int q = 0; q < Q; ++q) acc[q] = reduce_splits<T, STEP>(acc[q] - (T)sum4(part[q]));
          // the operand of the diagonal product: y (smoother) or x_i (product), in TM
          TM* opnd = MODE == MODE_SMOOTH ? ysm + cl * LP : xr_i;
          if (sp == 0 && act) {
#pragma unroll
            for (int q = 0; q < Q; ++q) opnd[rb + RG * q] = (TM)(MODE == MODE_SMOOTH ? acc[q] : xcur[q]);
          }
          if (!consumer_sync()) return;  // the operand is complete
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int r = rb + RG * q;
            TM a4[4] = {0, 0, 0, 0};
#pragma unroll
            for (int gg = 0; gg < NVT; ++gg) {
              const int g = sp + gg * S;
              vfma(a4, gg, A[g * L + r], *reinterpret_cast<const VT*>(opnd + g * VE));
            }
            const T s = reduce_splits<T, STEP>((T)sum4(a4));
            if (MODE == MODE_SMOOTH) {
              T x = s;
              if (SPLITD) x += ddv[q] * acc[q];
              if (sp == 0 && act) {
                xr_i[r] = (TM)x;
                if (valid) X[(long long)(i * L + r) * ld + p] = x;
              }
            } else {
              T o = acc[q] - s;
              if (SPLITD) o -= ddv[q] * xcur[q];
              if (valid && sp == 0 && act) {
                if (J.OUT) J.OUT[(long long)(i * L + r) * ld + p] = o;
                const double av = fabs((double)o);
                local_max = (av > local_max || av != av) ? av : local_max;
              }
            }
          }
          load_rhs(i + 1);  // the next leaf's loads overlap the V slabs and the next chunks
          // smoother: x_i is published for the V slabs (the product wrote its x_i before the first
          // barrier; a warp can rewrite an operand only after every warp reached the next one)
          if (MODE == MODE_SMOOTH && !consumer_sync()) return;
        } else {  // PK_VPART: rows are z entries, the reduction runs over x_i
          const int* vz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * sizeof(TM));
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int r = rb + RG * q;
            const bool live = act && r < cnt;
            TM a4[4] = {0, 0, 0, 0};
            if (live) {
#pragma unroll
              for (int gg = 0; gg < NVT; ++gg) {
                const int g = sp + gg * S;
                vfma(a4, gg, A[g * cnt + r], *reinterpret_cast<const VT*>(xr_i + g * VE));
              }
            }
            const TM s = reduce_splits<TM, STEP>(sum4(a4));
            if (live && sp == 0) {
              const int code = vz[r];
              TM* z = zp + (code >> 1) * TC + cl;
              *z = (code & 1) ? s : *z + s;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + cslot);  // this warp is done with the slot
        if (++cslot == ns) {
          cslot = 0;
          cphase ^= 1;
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
