// Tensor-core variant of the panel walk for FP32 products (grid functions in T = double or
// float).  Same chunk stream, producer warp, bounded mbarrier protocol and arithmetic as
// hpanel_kernel (panel.cuh); the products of a chunk with the TC columns of the tile,
//   DENSE  Y += D_ij X_j      (64 x 64) x (64 x TC)
//   UPART  Y += U_i Z         (64 x K)  x (K x TC),  Z gathered from the z pool
//   DIAG   X_i = Dinv Y (smoother) / Y -= D_ii X_i (product)
//   VPART  Z (+)= V_i X_i     (K' x 64) x (64 x TC)
// run as mma.sync m16n8k8 TF32 with FP32 accumulation, each product split in three,
// hi*hi + hi*lo + lo*hi (hi = tf32(a), lo = tf32(a - hi)), which keeps FP32 accuracy; each term
// has its own accumulator.  The matrices arrive pre-split in the fragment layout of
// build_panel_mma; x tiles are split once when written (tiles of <= 16 columns) or on load.
//
// Warps: 8 consumer warps, warp w owns row tile rt = w % 4 (16 rows of the leaf) and column half
// w / 4 (TC / 2 columns = TC / 16 n-tiles of 8).  Lane (g, t) = (lane / 4, lane % 4) holds the
// accumulator entries (rows g, g + 8; columns 2t, 2t + 1) of each n-tile.  The reduction index of
// every 16-block is permuted (physical k = 4t + 2s + k'/4 for step s and logical k'), identically
// for both operands, so that each lane reads its A and B operands as 16-byte vectors.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "panel.cuh"

namespace fhmg {

constexpr int kMmaLP = 80;  // padded x-tile column (floats): 8 columns x 4 lanes of 16-byte reads hit distinct banks

struct MmaSmem {
  size_t ysm, ring, zp, bar, ebar, cbar, desc, flag, total;
};
// x tiles (y of the current leaf, the ring of recent x) of tiles up to 16 columns are kept as TF32
// hi/lo pairs ([hi: TC x LP][lo: TC x LP] per tile), split once when written; wider tiles keep
// one float per entry and split on every load (their shared memory would not hold the pairs).
__host__ __device__ inline int mma_xsplit(int TC) { return TC <= 16 ? 2 : 1; }
__host__ __device__ inline MmaSmem mma_smem(int TC, int pool, int W, int slot_bytes, int ns) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t tile = (size_t)mma_xsplit(TC) * TC * kMmaLP * 4;
  MmaSmem s;
  s.ysm = a16((size_t)ns * slot_bytes);
  s.ring = a16(s.ysm + tile);
  s.zp = a16(s.ring + (size_t)W * tile);
  s.bar = a16(s.zp + (size_t)pool * TC * 4);
  s.ebar = s.bar + 8 * (size_t)ns;
  s.cbar = s.ebar + 8 * (size_t)ns;
  s.desc = a16(s.cbar + 8);
  s.flag = s.desc + 16 * (size_t)ns;
  s.total = a16(s.flag + 16);
  return s;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One accumulator per product term (lo*hi, hi*lo, hi*hi): the mma chains of a chunk are then
// three independent ones; the terms are summed, small ones first, where the products are used.
struct Acc3 {
  float lh[4], hl[4], hh[4];
};
__device__ __forceinline__ void acc_zero(Acc3& a) {
#pragma unroll
  for (int j = 0; j < 4; ++j) a.lh[j] = a.hl[j] = a.hh[j] = 0.f;
}
__device__ __forceinline__ float acc_sum(const Acc3& a, int j) { return (a.lh[j] + a.hl[j]) + a.hh[j]; }

// TF32 hi/lo words of four values
__device__ __forceinline__ void split4(const float4 v, uint32_t (&bh)[4], uint32_t (&bl)[4]) {
  const float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    bh[e] = to_tf32(xs[e]);
    bl[e] = to_tf32(xs[e] - __uint_as_float(bh[e]));
  }
}

// c += A B over one 16-block of the reduction: A from four 16-byte vectors (hi/lo of rows g and
// g + 8), B as the hi/lo words of the lane's four reduction indices; two k-steps, three products
// each (step 0: k' = t -> e 0, k' = t + 4 -> e 1; step 1: e 2, e 3).
__device__ __forceinline__ void mma_block(Acc3& c, const float4 h0, const float4 h1, const float4 l0, const float4 l1,
                                          const uint32_t (&bh)[4], const uint32_t (&bl)[4]) {
  mma_tf32(c.lh, __float_as_uint(l0.x), __float_as_uint(l1.x), __float_as_uint(l0.y), __float_as_uint(l1.y), bh[0], bh[1]);
  mma_tf32(c.hl, __float_as_uint(h0.x), __float_as_uint(h1.x), __float_as_uint(h0.y), __float_as_uint(h1.y), bl[0], bl[1]);
  mma_tf32(c.hh, __float_as_uint(h0.x), __float_as_uint(h1.x), __float_as_uint(h0.y), __float_as_uint(h1.y), bh[0], bh[1]);
  mma_tf32(c.lh, __float_as_uint(l0.z), __float_as_uint(l1.z), __float_as_uint(l0.w), __float_as_uint(l1.w), bh[2], bh[3]);
  mma_tf32(c.hl, __float_as_uint(h0.z), __float_as_uint(h1.z), __float_as_uint(h0.w), __float_as_uint(h1.w), bl[2], bl[3]);
  mma_tf32(c.hh, __float_as_uint(h0.z), __float_as_uint(h1.z), __float_as_uint(h0.w), __float_as_uint(h1.w), bh[2], bh[3]);
}

// The four A vectors of (row tile rt, k-block kb) of a chunk matrix with nkb k-blocks.
__device__ __forceinline__ void load_a(const float4* A, int rt, int kb, int nkb, int lane, float4& h0, float4& h1,
                                       float4& l0, float4& l1) {
  const float4* p = A + (size_t)((rt * nkb + kb) * 4) * 32 + lane;
  h0 = p[0];
  h1 = p[32];
  l0 = p[64];
  l1 = p[96];
}

template <typename T, int TC, int MODE>
__global__ void __launch_bounds__(288) hmma_kernel(const __grid_constant__ WalkBatch<T, float> B) {
  constexpr int L = 64, NT = 256, NTL = TC / 16;  // n-tiles of 8 columns per warp
  constexpr int LP = kMmaLP;
  static_assert(TC == 16 || TC == 32, "tensor-core tile");
  extern __shared__ __align__(16) unsigned char sm[];
  const MmaSmem lay = mma_smem(TC, B.pool, B.W, B.slot_bytes, B.ns);
  unsigned char* slots = sm;
  float* ysm = reinterpret_cast<float*>(sm + lay.ysm);
  float* ring = reinterpret_cast<float*>(sm + lay.ring);
  float* zp = reinterpret_cast<float*>(sm + lay.zp);
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
  __syncthreads();

  if (t >= NT) {
    // ---- producer (as in hpanel_kernel; the level inverses hold hi/lo pairs: 2 L^2 floats) ----
    if (t != NT) return;
    long long k = 0;
    int slot = 0;
    bool ok = true, stop = false;
    for (long long g = blockIdx.x; g < B.ntiles && ok && !stop; g += gridDim.x) {
      const WalkJob<T, float>& J = B.job[job_of(B, g)];
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
                              ? (const void*)(J.Dinv + (long long)cd.y * 2 * L * L)
                              : (const void*)(J.P.pkg + 16LL * (long long)cd.w);
        sdesc[slot] = cd;
        bulk_load(slots + (size_t)slot * B.slot_bytes, src, (uint32_t)cd.z, full + slot);
        if (++slot == ns) slot = 0;
      }
    }
    if (!ok && !*abort_flag) {
      *abort_flag = 1;
      atomicExch(B.err, 1);
    }
    for (int s = 0; s < ns && s < k; ++s) {
      const long long n_s = (k - 1 - s) / ns + 1;
      mbar_wait(full + s, (uint32_t)((n_s - 1) & 1));
    }
    return;
  }

  // ---- consumers ----
  const int w = t >> 5;
  const int rt = w & 3;                 // row tile
  const int cb = (w >> 2) * (TC / 2);   // first column of this warp
  const int g = lane >> 2, tq = lane & 3;
  constexpr int XS = TC <= 16 ? 2 : 1;        // mma_xsplit(TC)
  constexpr int TS = XS * TC * LP;            // floats per x tile
  // B operand of column col, k-block kb from an x tile (pre-split, or split here)
  auto load_b = [&](const float* tile, int col, int kb, uint32_t(&bh)[4], uint32_t(&bl)[4]) {
    const float* p = tile + col * LP + kb * 16 + 4 * tq;
    if (XS == 2) {
      const float4 hv = *reinterpret_cast<const float4*>(p);
      const float4 lv = *reinterpret_cast<const float4*>(p + TC * LP);
      bh[0] = __float_as_uint(hv.x), bh[1] = __float_as_uint(hv.y), bh[2] = __float_as_uint(hv.z), bh[3] = __float_as_uint(hv.w);
      bl[0] = __float_as_uint(lv.x), bl[1] = __float_as_uint(lv.y), bl[2] = __float_as_uint(lv.z), bl[3] = __float_as_uint(lv.w);
    } else {
      split4(*reinterpret_cast<const float4*>(p), bh, bl);
    }
  };
  auto store_x = [&](float* tile, int col, int row, float v) {
    if (XS == 2) {
      const uint32_t h = to_tf32(v);
      tile[col * LP + row] = __uint_as_float(h);
      tile[TC * LP + col * LP + row] = __uint_as_float(to_tf32(v - __uint_as_float(h)));
    } else {
      tile[col * LP + row] = v;
    }
  };
  uint32_t cbphase = 0;
  auto give_up = [&](bool ok) -> bool {
    if (__all_sync(0xffffffffu, ok)) return false;
    if (lane == 0) {
      *abort_flag = 1;
      atomicExch(B.err, 1);
    }
    return true;
  };
  auto consumer_sync = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const bool ok = mbar_wait_or_abort(cbar, cbphase, abort_flag, B.spin);
    cbphase ^= 1;
    return !give_up(ok);
  };

  int cslot = 0;
  uint32_t cphase = 0;
  for (long long gt = blockIdx.x; gt < B.ntiles; gt += gridDim.x) {
    const WalkJob<T, float>& J = B.job[job_of(B, gt)];
    const long long ld = J.geo.ld;
    const T inv_h2 = (T)J.geo.inv_h2;
    T* X = J.X;
    const T* Bsrc = J.B;
    const T* ddg = J.ddiag;
    const int nb = J.P.nb;
    // the lane's accumulator columns: n-tile nt, e = 0, 1 -> column cb + nt*8 + 2 tq + e
    long long pcol[NTL][2];
    int nmask[NTL][2];  // bit d: neighbour d exists (1D: -1, +1; 2D: also -N, +N)
    bool vcol[NTL][2];
#pragma unroll
    for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const long long cg = (gt - J.tile0) * TC + cb + nt * 8 + 2 * tq + e;
        vcol[nt][e] = cg < J.ncols;
        pcol[nt][e] = cg;
        nmask[nt][e] = 0;
        if (vcol[nt][e] && MODE == MODE_SMOOTH && J.geo.dim > 0) {
          int iy, ix;
          pcol[nt][e] = colour_pos(J.geo.dim, J.geo.N, J.geo.colour, cg, &iy, &ix);
          nmask[nt][e] = (ix > 0 ? 1 : 0) | (ix < J.geo.N - 1 ? 2 : 0);
          if (J.geo.dim == 2) nmask[nt][e] |= (iy > 0 ? 4 : 0) | (iy < J.geo.N - 1 ? 8 : 0);
        }
      }
    const long long nstep[4] = {-1, 1, -(long long)J.geo.N, (long long)J.geo.N};
    double local_max = 0.0;
    T bn[NTL][4], xn[NTL][4], dn[2];
    auto load_rhs = [&](int leaf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) dn[h] = (leaf < nb) ? ddg[(long long)leaf * L + rt * 16 + g + 8 * h] : (T)0;
#pragma unroll
      for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int h = j >> 1, e = j & 1;
          T b = 0, x = 0;
          if (leaf < nb && vcol[nt][e]) {
            const long long base = (long long)(leaf * L + rt * 16 + g + 8 * h) * ld + pcol[nt][e];
            b = Bsrc[base];
            if (MODE == MODE_SMOOTH) {
              T s = 0;
#pragma unroll
              for (int d = 0; d < 4; ++d)
                if (nmask[nt][e] & (1 << d)) s += X[base + nstep[d]];
              b += s * inv_h2;
            } else {
              x = X[base];
            }
          }
          bn[nt][j] = b;
          xn[nt][j] = x;
        }
    };
    load_rhs(0);

    for (int i = 0; i < nb; ++i) {
      T rhs[NTL][4], xcur[NTL][4], ddv[2];
      Acc3 acc[NTL];
#pragma unroll
      for (int nt = 0; nt < NTL; ++nt) {
        acc_zero(acc[nt]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          rhs[nt][j] = bn[nt][j];
          xcur[nt][j] = xn[nt][j];
        }
      }
      ddv[0] = dn[0];
      ddv[1] = dn[1];
      load_rhs(i + 1);
      float* xr_i = ring + (size_t)(i % W) * TS;  // x_i tile [column][k]
      for (bool leaf_done = false; !leaf_done;) {
        if (give_up(mbar_wait_or_abort(full + cslot, cphase, abort_flag, B.spin))) return;
        const int4 cd = sdesc[cslot];
        leaf_done = ((cd.x >> 12) & 1) != 0;
        const int type = cd.x & 15, cnt = (cd.x >> 4) & 0xff;
        const unsigned char* buf = slots + (size_t)cslot * B.slot_bytes;
        const float4* A = reinterpret_cast<const float4*>(buf);
        if (type == PK_DENSE) {
          const float* xr = ring + (size_t)(cd.y % W) * TS;
#pragma unroll
          for (int kb = 0; kb < 4; ++kb) {
            float4 h0, h1, l0, l1;
            load_a(A, rt, kb, 4, lane, h0, h1, l0, l1);
#pragma unroll
            for (int nt = 0; nt < NTL; ++nt) {
              uint32_t bh[4], bl[4];
              load_b(xr, cb + nt * 8 + g, kb, bh, bl);
              mma_block(acc[nt], h0, h1, l0, l1, bh, bl);
            }
          }
        } else if (type == PK_UPART) {
          const int nkb = cnt / 16;
          const int* uz = reinterpret_cast<const int*>(buf + (size_t)nkb * 4 * 4 * 32 * 16);
#pragma unroll
          for (int kb = 0; kb < 4; ++kb) {
            if (kb < nkb) {
              float4 h0, h1, l0, l1;
              load_a(A, rt, kb, nkb, lane, h0, h1, l0, l1);
              const int4 zi = *reinterpret_cast<const int4*>(uz + kb * 16 + 4 * tq);
#pragma unroll
              for (int nt = 0; nt < NTL; ++nt) {
                const int c = cb + nt * 8 + g;
                uint32_t bh[4], bl[4];
                split4(make_float4(zp[zi.x * TC + c], zp[zi.y * TC + c], zp[zi.z * TC + c], zp[zi.w * TC + c]), bh, bl);
                mma_block(acc[nt], h0, h1, l0, l1, bh, bl);
              }
            }
          }
        } else if (type == PK_DIAG) {
          // y = right-hand side - sum of the products (in T); the diagonal product's operand
          float* opnd = MODE == MODE_SMOOTH ? ysm : xr_i;
#pragma unroll
          for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int h = j >> 1, e = j & 1;
              rhs[nt][j] -= (T)acc_sum(acc[nt], j);
              const int col = cb + nt * 8 + 2 * tq + e, row = rt * 16 + g + 8 * h;
              store_x(opnd, col, row, (float)(MODE == MODE_SMOOTH ? rhs[nt][j] : xcur[nt][j]));
            }
#pragma unroll
          for (int nt = 0; nt < NTL; ++nt) acc_zero(acc[nt]);
          if (!consumer_sync()) return;  // the operand is complete
#pragma unroll
          for (int kb = 0; kb < 4; ++kb) {
            float4 h0, h1, l0, l1;
            load_a(A, rt, kb, 4, lane, h0, h1, l0, l1);
#pragma unroll
            for (int nt = 0; nt < NTL; ++nt) {
              uint32_t bh[4], bl[4];
              load_b(opnd, cb + nt * 8 + g, kb, bh, bl);
              mma_block(acc[nt], h0, h1, l0, l1, bh, bl);
            }
          }
#pragma unroll
          for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int h = j >> 1, e = j & 1;
              const int col = cb + nt * 8 + 2 * tq + e, row = rt * 16 + g + 8 * h;
              const long long at = (long long)(i * L + row) * ld + pcol[nt][e];
              if (MODE == MODE_SMOOTH) {
                const T x = (T)acc_sum(acc[nt], j) + ddv[h] * rhs[nt][j];
                store_x(xr_i, col, row, (float)x);
                if (vcol[nt][e]) X[at] = x;
              } else {
                const T o = rhs[nt][j] - (T)acc_sum(acc[nt], j) - ddv[h] * xcur[nt][j];
                if (vcol[nt][e]) {
                  if (J.OUT) J.OUT[at] = o;
                  const double av = fabs((double)o);
                  local_max = (av > local_max || av != av) ? av : local_max;
                }
              }
            }
          if (MODE == MODE_SMOOTH && !consumer_sync()) return;  // x_i is published for the V slabs
        } else {  // PK_VPART: rows are z entries (cnt of them), the reduction runs over x_i
          const int nrt = (cnt + 15) / 16;
          const int* vz = reinterpret_cast<const int*>(buf + (size_t)nrt * 4 * 4 * 32 * 16);
          if (rt < nrt) {
            Acc3 zacc[NTL];
#pragma unroll
            for (int nt = 0; nt < NTL; ++nt) acc_zero(zacc[nt]);
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
              float4 h0, h1, l0, l1;
              load_a(A, rt, kb, 4, lane, h0, h1, l0, l1);
#pragma unroll
              for (int nt = 0; nt < NTL; ++nt) {
                uint32_t bh[4], bl[4];
                load_b(xr_i, cb + nt * 8 + g, kb, bh, bl);
                mma_block(zacc[nt], h0, h1, l0, l1, bh, bl);
              }
            }
#pragma unroll
            for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int h = j >> 1, e = j & 1;
                const int zr = rt * 16 + g + 8 * h;
                if (zr < cnt) {
                  const int code = vz[zr];
                  float* z = zp + (code >> 1) * TC + cb + nt * 8 + 2 * tq + e;
                  const float v = acc_sum(zacc[nt], j);
                  *z = (code & 1) ? v : *z + v;
                }
              }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + cslot);
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
      if (lane == 0) atomicMax(J.norm, (unsigned long long)__double_as_longlong(local_max));
    }
  }
}

}  // namespace fhmg
