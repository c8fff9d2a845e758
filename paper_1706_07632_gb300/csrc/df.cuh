// FP64-accurate H-matrix products (Algorithm 3 per column: OUT = B - R~ X) and triangular solves
// on compact columns (Algorithm 4: X = (R~ + s I)^{-1} B, one inverse set per column allowed) in
// double-float arithmetic on the FP32 pipe.  On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, and the
// defect that decides convergence must be accurate to FP64 level; a double-float multiply-add
// (pairs of floats, error-free transformations) costs 11 FP32 instructions instead of one
// 1/64-rate DFMA.
//
// Numbers: a matrix entry a = ah + al (ah = fl32(a), al = fl32(a - ah), |a - ah - al| <= 2^-48 |a|,
// stored by build_panel_df), x = xh + xl likewise (split here from the FP64 arrays).  A product
// adds ah*xh exactly (TwoProd by FMA) and ah*xl + al*xh into the low word; al*xl (2^-48) is
// dropped.  Sums keep (h, l) with TwoSum on h.  The error of a dot product is a few 2^-48 of
// sum |a_k x_k|; OUT = B - (h + l) is formed in FP64.
//
// Walk, chunk stream, producer warp and bounded mbarrier protocol are those of hpanel_kernel
// (panel.cuh); x tiles, y and the z pool are kept as (hi, lo) pairs in shared memory.  The smoother
// form streams the inverses (D_ii + s I)^{-1} as float pairs in place of the DIAG chunks.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "panel.cuh"

namespace fhmg {

// s + e = a + b exactly (round to nearest; the _rn forms keep the compiler from contracting)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += (ah + al)(xh + xl)
__device__ __forceinline__ void df_mac(float& h, float& l, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  float s, err;
  two_sum(h, p, s, err);
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, e));
}

// (h, l) += (bh, bl), renormalised so that |l| <= ulp(h) / 2
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

struct DfSmem {
  size_t ysm, ring, zp, bar, ebar, cbar, desc, flag, total;
};
// x-tile ring: W slots x {hi, lo} x TC columns x (L + 4) floats; z pool: {hi, lo} x pool x TC
__host__ __device__ inline DfSmem df_smem(int L, int TC, int pool, int W, int slot_bytes, int ns) {
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t LP = (size_t)L + 4;
  DfSmem s;
  s.ysm = a16((size_t)ns * slot_bytes);  // y of the current leaf (smoother): {hi, lo} x TC x LP
  s.ring = a16(s.ysm + 2 * (size_t)TC * LP * 4);
  s.zp = a16(s.ring + (size_t)W * 2 * TC * LP * 4);
  s.bar = a16(s.zp + 2 * (size_t)pool * TC * 4);
  s.ebar = s.bar + 8 * (size_t)ns;
  s.cbar = s.ebar + 8 * (size_t)ns;
  s.desc = a16(s.cbar + 8);
  s.flag = s.desc + 16 * (size_t)ns;
  s.total = a16(s.flag + 16);
  return s;
}

// four double-float multiply-adds of one 16-byte vector pair into four accumulators
__device__ __forceinline__ void df_vec(float (&h)[4], float (&l)[4], const float4 ah, const float4 al, const float4 xh,
                                       const float4 xl) {
  df_mac(h[0], l[0], ah.x, al.x, xh.x, xl.x);
  df_mac(h[1], l[1], ah.y, al.y, xh.y, xl.y);
  df_mac(h[2], l[2], ah.z, al.z, xh.z, xl.z);
  df_mac(h[3], l[3], ah.w, al.w, xh.w, xl.w);
}

// MODE_SMOOTH: compact columns only (geo.dim == 0, no stencil), B the right-hand side, Dinv the
// inverses as float pairs (2 L^2 floats per leaf), dinv_cstride floats between columns' sets.
template <int L, int TC, int MODE>
__global__ void __launch_bounds__(288) hdf_kernel(const __grid_constant__ WalkBatch<double, float> B) {
  constexpr int NT = 256, VE = 4;
  using TL = PTile<L, TC, NT, VE>;
  constexpr int Q = TL::Q, RG = TL::RG, S = TL::S, RL = TL::RL, NVT = TL::NVT;
  constexpr int STEP = TC * RL;
  constexpr int LP = L + VE;
  extern __shared__ __align__(16) unsigned char sm[];
  const DfSmem lay = df_smem(L, TC, B.pool, B.W, B.slot_bytes, B.ns);
  unsigned char* slots = sm;
  float* ring = reinterpret_cast<float*>(sm + lay.ring);
  float* ysh = reinterpret_cast<float*>(sm + lay.ysm);
  float* zph = reinterpret_cast<float*>(sm + lay.zp);
  float* zpl = zph + (size_t)B.pool * TC;
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
    // ---- producer (as in hpanel_kernel) ----
    if (t != NT) return;
    long long k = 0;
    int slot = 0;
    bool ok = true, stop = false;
    for (long long g = blockIdx.x; g < B.ntiles && ok && !stop; g += gridDim.x) {
      const WalkJob<double, float>& J = B.job[job_of(B, g)];
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
        const void* src = (MODE == MODE_SMOOTH && (cd.x & 15) == PK_DIAG)
                              ? (const void*)(J.Dinv + (g - J.tile0) * TC * J.dinv_cstride + (long long)cd.y * 2 * L * L)
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
  const int cl = lane % TC;
  const int rl = (lane / TC) % RL;
  const int sp = lane / STEP;
  const int rb0 = (t >> 5) * RL + rl;
  const bool act = rb0 < RG;
  const int rb = act ? rb0 : 0;
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
  // the hi / lo tile of ring slot s for this thread's column
  auto tile_h = [&](int s) { return ring + ((size_t)(s * 2) * TC + cl) * LP; };
  auto tile_l = [&](int s) { return ring + ((size_t)(s * 2 + 1) * TC + cl) * LP; };

  int cslot = 0;
  uint32_t cphase = 0;
  for (long long g = blockIdx.x; g < B.ntiles; g += gridDim.x) {
    const WalkJob<double, float>& J = B.job[job_of(B, g)];
    const long long cg = (g - J.tile0) * TC + cl;
    const bool valid = cg < J.ncols;
    const long long ld = J.geo.ld;
    const double* X = J.X;
    const double* Bsrc = J.B;
    const int nb = J.P.nb;
    const long long p = cg;
    double local_max = 0.0;
    double bn[Q], xn[Q];
    auto load_rhs = [&](int leaf) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        double b = 0, x = 0;
        if (act && sp == 0 && valid && leaf < nb) {
          const long long base = (long long)(leaf * L + rb + RG * q) * ld + p;
          b = Bsrc[base];
          if (MODE == MODE_MATVEC) x = X[base];
        }
        bn[q] = b;
        xn[q] = x;
      }
    };
    load_rhs(0);

    for (int i = 0; i < nb; ++i) {
      double rhs[Q], xcur[Q];
      float ph[Q][4], pl[Q][4];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        rhs[q] = bn[q];
        xcur[q] = xn[q];
#pragma unroll
        for (int a = 0; a < 4; ++a) ph[q][a] = pl[q][a] = 0.f;
      }
      const int si = i % W;
      for (bool leaf_done = false; !leaf_done;) {
        if (give_up(mbar_wait_or_abort(full + cslot, cphase, abort_flag, B.spin))) return;
        const int4 cd = sdesc[cslot];
        leaf_done = ((cd.x >> 12) & 1) != 0;
        const int type = cd.x & 15, cnt = (cd.x >> 4) & 0xff;
        const unsigned char* buf = slots + (size_t)cslot * B.slot_bytes;
        const float4* Ah = reinterpret_cast<const float4*>(buf);
        if (MODE == MODE_SMOOTH && type == PK_DIAG) {
          // y = B - (products so far) in FP64, then x_i = Dinv y in double-float
          const float4* Al = Ah + L * L / 4;
          float* yh = ysh + (size_t)cl * LP;
          float* yl = ysh + (size_t)(TC + cl) * LP;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            float h = ph[q][0], l = pl[q][0];
#pragma unroll
            for (int a = 1; a < 4; ++a) df_add(h, l, ph[q][a], pl[q][a]);
#pragma unroll
            for (int o = STEP; o < 32; o <<= 1) {
              const float oh = __shfl_xor_sync(0xffffffffu, h, o);
              const float ol = __shfl_xor_sync(0xffffffffu, l, o);
              df_add(h, l, oh, ol);
            }
            rhs[q] -= (double)h + (double)l;
            if (sp == 0 && act) {
              float a, b2;
              df_split(rhs[q], a, b2);
              yh[rb + RG * q] = a;
              yl[rb + RG * q] = b2;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) ph[q][a] = pl[q][a] = 0.f;
          }
          if (!consumer_sync()) return;  // y is complete
#pragma unroll 2  // full unrolling overflows the instruction cache
          for (int gg = 0; gg < NVT; ++gg) {
            const int g = sp + gg * S;
            const float4 vh = *reinterpret_cast<const float4*>(yh + g * VE);
            const float4 vl = *reinterpret_cast<const float4*>(yl + g * VE);
#pragma unroll
            for (int q = 0; q < Q; ++q) df_vec(ph[q], pl[q], Ah[g * L + rb + RG * q], Al[g * L + rb + RG * q], vh, vl);
          }
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            float h = ph[q][0], l = pl[q][0];
#pragma unroll
            for (int a = 1; a < 4; ++a) df_add(h, l, ph[q][a], pl[q][a]);
#pragma unroll
            for (int o = STEP; o < 32; o <<= 1) {
              const float oh = __shfl_xor_sync(0xffffffffu, h, o);
              const float ol = __shfl_xor_sync(0xffffffffu, l, o);
              df_add(h, l, oh, ol);
            }
            if (sp == 0 && act) {
              tile_h(si)[rb + RG * q] = h;  // (h, l) is already a float pair of x
              tile_l(si)[rb + RG * q] = l;
              if (valid) J.X[(long long)(i * L + rb + RG * q) * ld + p] = (double)h + (double)l;
            }
          }
          load_rhs(i + 1);
          if (!consumer_sync()) return;  // x_i is published for the V slabs
        } else if (type == PK_DENSE || type == PK_DIAG) {
          const float4* Al = Ah + L * L / 4;
          const float *xh, *xl;
          if (type == PK_DIAG) {
            // x_i joins the ring (hi / lo) before its own diagonal product
            if (sp == 0 && act) {
#pragma unroll
              for (int q = 0; q < Q; ++q) {
                float h, l;
                df_split(xcur[q], h, l);
                tile_h(si)[rb + RG * q] = h;
                tile_l(si)[rb + RG * q] = l;
              }
            }
            if (!consumer_sync()) return;
            xh = tile_h(si);
            xl = tile_l(si);
          } else {
            xh = tile_h(cd.y % W);
            xl = tile_l(cd.y % W);
          }
          const bool far = type == PK_DENSE && i - cd.y >= W;
          const double* xj = X + (long long)cd.y * L * ld + p;
#pragma unroll 2  // full unrolling overflows the instruction cache
          for (int gg = 0; gg < NVT; ++gg) {
            const int g = sp + gg * S;
            float4 vh, vl;
            if (!far) {
              vh = *reinterpret_cast<const float4*>(xh + g * VE);
              vl = *reinterpret_cast<const float4*>(xl + g * VE);
            } else {
              float e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
              if (valid)
#pragma unroll
                for (int u = 0; u < 4; ++u) df_split(xj[(long long)(g * VE + u) * ld], e[u], e[4 + u]);
              vh = make_float4(e[0], e[1], e[2], e[3]);
              vl = make_float4(e[4], e[5], e[6], e[7]);
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) df_vec(ph[q], pl[q], Ah[g * L + rb + RG * q], Al[g * L + rb + RG * q], vh, vl);
          }
          if (type == PK_DIAG) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              float h = ph[q][0], l = pl[q][0];
#pragma unroll
              for (int a = 1; a < 4; ++a) df_add(h, l, ph[q][a], pl[q][a]);
#pragma unroll
              for (int o = STEP; o < 32; o <<= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, h, o);
                const float ol = __shfl_xor_sync(0xffffffffu, l, o);
                df_add(h, l, oh, ol);
              }
              const double o = rhs[q] - ((double)h + (double)l);
              if (valid && sp == 0 && act) {
                if (J.OUT) J.OUT[(long long)(i * L + rb + RG * q) * ld + p] = o;
                const double av = fabs(o);
                local_max = (av > local_max || av != av) ? av : local_max;
              }
            }
            load_rhs(i + 1);
          }
        } else if (type == PK_UPART) {
          const float4* Al = Ah + L * cnt / 4;
          const int* uz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * 8);
          const int nvq = cnt / VE;
#pragma unroll 2  // full unrolling overflows the instruction cache
          for (int gg = 0; gg < NVT; ++gg) {
            const int g = sp + gg * S;
            if (g < nvq) {
              const int4 zi = *reinterpret_cast<const int4*>(uz + g * VE);
              const float4 vh =
                  make_float4(zph[zi.x * TC + cl], zph[zi.y * TC + cl], zph[zi.z * TC + cl], zph[zi.w * TC + cl]);
              const float4 vl =
                  make_float4(zpl[zi.x * TC + cl], zpl[zi.y * TC + cl], zpl[zi.z * TC + cl], zpl[zi.w * TC + cl]);
#pragma unroll
              for (int q = 0; q < Q; ++q) df_vec(ph[q], pl[q], Ah[g * L + rb + RG * q], Al[g * L + rb + RG * q], vh, vl);
            }
          }
        } else {  // PK_VPART: rows are z entries, the reduction runs over x_i
          const float4* Al = Ah + cnt * L / 4;
          const int* vz = reinterpret_cast<const int*>(buf + (size_t)cnt * L * 8);
          const float* xh = tile_h(si);
          const float* xl = tile_l(si);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int r = rb + RG * q;
            const bool live = act && r < cnt;
            float zh[4] = {0, 0, 0, 0}, zl[4] = {0, 0, 0, 0};
            if (live) {
#pragma unroll 2
              for (int gg = 0; gg < NVT; ++gg) {
                const int g = sp + gg * S;
                df_vec(zh, zl, Ah[g * cnt + r], Al[g * cnt + r], *reinterpret_cast<const float4*>(xh + g * VE),
                       *reinterpret_cast<const float4*>(xl + g * VE));
              }
            }
            float h = zh[0], l = zl[0];
#pragma unroll
            for (int a = 1; a < 4; ++a) df_add(h, l, zh[a], zl[a]);
#pragma unroll
            for (int o = STEP; o < 32; o <<= 1) {
              const float oh = __shfl_xor_sync(0xffffffffu, h, o);
              const float ol = __shfl_xor_sync(0xffffffffu, l, o);
              df_add(h, l, oh, ol);
            }
            if (live && sp == 0) {
              const int code = vz[r];
              const int zi = (code >> 1) * TC + cl;
              if (code & 1) {
                zph[zi] = h;
                zpl[zi] = l;
              } else {
                float a = zph[zi], b = zpl[zi];
                df_add(a, b, h, l);
                zph[zi] = a;
                zpl[zi] = b;
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
