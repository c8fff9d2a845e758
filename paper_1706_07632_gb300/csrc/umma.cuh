// tcgen05 variant of the panel walk for wide panels (2D grids): BF16 products with FP32
// accumulation in tensor memory, FP32 grid functions.
//
// The walk of panel.cuh transposed onto the 5th-generation tensor cores.  A CTA owns a tile of
// 128 spatial columns; thread c of the four consumer warps owns column c (TMEM lane c).  Every
// chunk product of a leaf row i becomes one tcgen05.mma with M = 128 (the columns), N = the chunk's
// output rows, K = its reduction index, A from shared memory (the columns' operand tile, 128 x K,
// K-major) and B = the chunk itself (N x K, K-major, streamed by TMA bulk copies in the canonical
// no-swizzle core-matrix layout of build_panel_umma):
//   DENSE(j)  acc[c, r] += sum_k x_j[c, k] D_ij[r, k]        A = ring tile of leaf j
//   UPART     acc[c, r] += sum_k z[c, k] U_i[r, k]           A = the columns' z values, staged
//   DIAG      smoother: res[c, r] = sum_k y[c, k] Dinv'[r, k], y = b - acc, x = res + dinv_rr y
//             product:  acc[c, r] += sum_k x_i[c, k] D'_ii[r, k], out = b - acc - d_rr x
//   VPART     v[c, q] = sum_k x_i[c, k] V_i[q, k], then z[c, code_q] (+)= v[c, q]
// (D', Dinv': without their diagonal, which is applied in FP32 by the threads).  One elected thread
// issues the MMAs; tcgen05.commit signals their completion on mbarriers: the slot's "empty" barrier
// (which also collects one arrival per consumer warp, so a slot is refilled only when the MMA and
// every warp are done with it) and the acc / res / v barriers that the threads wait on before they
// read tensor memory with tcgen05.ld.  Threads write the A tiles (x ring, y, z) with 16-byte stores
// in the core-matrix layout, then fence.proxy.async and meet on a consumer mbarrier before the MMA
// that reads them is issued.  Every wait is bounded and watches the shared abort flag; every exit
// path frees the tensor memory after the MMAs in flight completed.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "walk.h"

namespace fhmg {

constexpr int kUmmaCols = 128;                 // columns per tile = MMA M = TMEM lanes
constexpr int kUmmaBlock = kUmmaCols + 32;     // consumer threads + producer warp
constexpr uint32_t kUmmaTmemCols = 256;        // acc [0,64), res [64,128), v [128,192)

struct UmmaSmem {
  size_t ring, ystage, zstage, zpool, bar, ebar, cbar, xbar, desc, flag, tslot, total;
};
// x ring (W tiles), one staging tile (128 x 64 BF16 each) that holds the columns' z values for the
// U products and, later in the same leaf, y for the inverse's product (the U products have then
// completed), z pool (pool x 128 FP32), mbarriers, slot descriptors, abort flag, TMEM address.
// Operand tiles are 128-byte aligned.
__host__ __device__ inline UmmaSmem umma_smem(int pool, int W, int slot_bytes, int ns) {
  auto a128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
  const size_t tile = (size_t)kUmmaCols * kUmmaL * 2;
  UmmaSmem s;
  s.ring = a128((size_t)ns * slot_bytes);
  s.ystage = s.ring + (size_t)W * tile;
  s.zstage = s.ystage;
  s.zpool = s.ystage + tile;
  s.bar = a128(s.zpool + (size_t)pool * kUmmaCols * 4);
  s.ebar = s.bar + 8 * (size_t)ns;
  s.cbar = s.ebar + 8 * (size_t)ns;  // consumer warps' barrier
  s.xbar = s.cbar + 8;               // acc, res, v (MMA completion), exit (consumer warps), done
  s.desc = (s.xbar + 5 * 8 + 15) & ~(size_t)15;
  s.flag = s.desc + 16 * (size_t)ns;
  s.tslot = s.flag + 16;
  s.total = a128(s.tslot + 16);
  return s;
}

// byte offset of entry (r, k) of a K-major operand tile with K columns (core-matrix layout)
__device__ __forceinline__ uint32_t umma_off(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading (K) byte offset 128, stride (8-row
// group) byte offset, fixed bits 46-48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M = 128, N
__device__ __forceinline__ uint32_t umma_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kUmmaCols >> 4) << 24);
}

// D[tmem] (+)= A B^T over K = 16 * steps, A (128 x K) and B (N x K) K-major tiles at a_addr / b_addr
__device__ __forceinline__ void umma_product(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, int K, int N,
                                             bool accumulate) {
  const uint32_t idesc = umma_idesc(N);
  const uint32_t sbo = (uint32_t)(K / 8) * 128;
  for (int s = 0; s < K / 16; ++s) {
    const uint64_t ad = umma_desc(a_addr + 256u * s, sbo);
    const uint64_t bd = umma_desc(b_addr + 256u * s, sbo);
    const uint32_t acc = (accumulate || s > 0) ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane (the warp's lane quarter), as floats
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// row c of a K-major operand tile with K columns: 8 consecutive entries k0..k0+7 as one 16-byte store
__device__ __forceinline__ void put8(unsigned char* tile, int c, int k0, int K, const float* v) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + umma_off(c, k0, K)) = q;
}

// row c of a K-major operand tile: entries k0..k0+7 already packed as BF16 pairs
__device__ __forceinline__ void put8_packed(unsigned char* tile, int c, int k0, int K, const uint32_t* q) {
  *reinterpret_cast<uint4*>(tile + umma_off(c, k0, K)) = make_uint4(q[0], q[1], q[2], q[3]);
}

// T = float grid functions; the jobs' Dinv are the level inverses (without diagonal) in the
// build_panel_umma layout (BF16 bits), ddiag the diagonal applied in FP32.
template <int MODE>
__global__ void __maxnreg__(168) humma_kernel(const __grid_constant__ WalkBatch<float, uint16_t> B) {
  constexpr int L = kUmmaL, NT = kUmmaCols;
  extern __shared__ __align__(16) unsigned char sm[];
  const UmmaSmem lay = umma_smem(B.pool, B.W, B.slot_bytes, B.ns);
  unsigned char* slots = sm;
  unsigned char* ring = sm + lay.ring;
  unsigned char* ystage = sm + lay.ystage;
  unsigned char* zstage = sm + lay.zstage;
  float* zpool = reinterpret_cast<float*>(sm + lay.zpool);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + lay.bar);
  uint64_t* empty = reinterpret_cast<uint64_t*>(sm + lay.ebar);
  uint64_t* cbar = reinterpret_cast<uint64_t*>(sm + lay.cbar);
  uint64_t* accbar = reinterpret_cast<uint64_t*>(sm + lay.xbar);
  uint64_t* resbar = accbar + 1;
  uint64_t* vbar = accbar + 2;
  uint64_t* exitbar = accbar + 3;
  uint64_t* donebar = accbar + 4;
  int4* sdesc = reinterpret_cast<int4*>(sm + lay.desc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + lay.flag);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + lay.tslot);
  const size_t tile_bytes = (size_t)NT * L * 2;

  const int t = threadIdx.x;
  const int w = t >> 5;
  const int lane = t & 31;
  const int ns = B.ns;
  const int W = B.W;

  if (t == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, NT / 32 + 1);  // every consumer warp + the MMAs' commit
    }
    mbar_init(cbar, NT / 32);
    for (int b = 0; b < 5; ++b) mbar_init(accbar + b, b == 3 ? NT / 32 : 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kUmmaTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before_sync();
  __syncthreads();  // the last block-wide barrier: from here on the roles run apart
  tc_after_sync();
  const uint32_t tmem = *tslot;

  if (t >= NT) {
    // ---- producer: one lane streams every chunk of every tile of this CTA, in order ----
    if (t != NT) return;
    long long k = 0;
    int slot = 0;
    bool ok = true, stop = false;
    for (long long g = blockIdx.x; g < B.ntiles && ok && !stop; g += gridDim.x) {
      const WalkJob<float, uint16_t>& J = B.job[job_of(B, g)];
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
        const void* src = (MODE == MODE_SMOOTH && type == PK_DIAG) ? (const void*)(J.Dinv + (long long)cd.y * L * L)
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

  // ---- consumers: thread c owns column c of the tile ----
  const int c = t;
  const bool issuer = t == 0;
  const uint32_t t_acc = tmem, t_res = tmem + 64, t_v = tmem + 128;
  const uint32_t lane_base = (uint32_t)(32 * w) << 16;  // this warp's TMEM lane quarter
  uint32_t cbphase = 0, accph = 0, resph = 0, vph = 0;
  int cslot = 0;
  uint32_t cphase = 0;
  bool failed = false;
  auto give_up = [&](bool ok) -> bool {
    if (__all_sync(0xffffffffu, ok)) return false;
    if (lane == 0) {
      *abort_flag = 1;
      atomicExch(B.err, 1);
    }
    return true;
  };
  // all consumer warps meet (bounded); tensor-memory reads and shared writes before it are ordered
  // before the MMAs issued after it
  // arrive_wait: the same meeting without the fences, for callers that fenced already and issued
  // global loads since (a proxy fence would wait for those loads to complete)
  auto arrive_wait = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const bool ok = mbar_wait_or_abort(cbar, cbphase, abort_flag, B.spin);
    cbphase ^= 1;
    tc_after_sync();
    return !give_up(ok);
  };
  auto consumer_sync = [&]() -> bool {
    async_proxy_fence();
    tc_before_sync();
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const bool ok = mbar_wait_or_abort(cbar, cbphase, abort_flag, B.spin);
    cbphase ^= 1;
    tc_after_sync();
    return !give_up(ok);
  };
  auto wait_mma = [&](uint64_t* bar, uint32_t& ph) -> bool {
    const bool ok = mbar_wait_or_abort(bar, ph, abort_flag, B.spin);
    ph ^= 1;
    tc_after_sync();
    return !give_up(ok);
  };

  for (long long g = blockIdx.x; g < B.ntiles && !failed; g += gridDim.x) {
    const WalkJob<float, uint16_t>& J = B.job[job_of(B, g)];
    const long long cg = (g - J.tile0) * NT + c;
    const bool valid = cg < J.ncols;
    const long long ld = J.geo.ld;
    const float inv_h2 = (float)J.geo.inv_h2;
    float* X = J.X;
    const float* Bsrc = J.B;
    const float* ddg = J.ddiag;
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
    // right-hand side of a leaf (smoother: F + neighbour sum / h^2) and, for the product, its x;
    // loaded one leaf ahead (issued right after the previous leaf's diagonal step, the last use of
    // these registers), so the loads overlap that leaf's V products and this leaf's first MMAs.
    // Rows of leaf i + 1 are never written during leaf i (X, OUT alias B only row by row).
    // b: right-hand side (product: B - d_rr x, the diagonal term folded in at load time);
    // xq: the product's x_i as packed BF16 pairs for the ring
    float b[L];
    uint32_t xq[MODE == MODE_MATVEC ? L / 2 : 1];
    // columns past the panel's end read column 0 (any valid address) and are zeroed, so that the
    // loads carry no predicate; compact columns load their 64 values as independent loads, grid
    // columns in groups of 8 rows (5 loads per row: the point and its neighbours), which bounds
    // the registers the loads in flight hold
    const long long pa = valid ? p : 0;
    const float keep = valid ? 1.f : 0.f;
    const bool grid = MODE == MODE_SMOOTH && J.geo.dim > 0;
    auto load_leaf = [&](int leaf) {
      if (leaf >= nb) return;
      const float* Bl = Bsrc + (long long)leaf * L * ld + pa;
      if (!grid) {
#pragma unroll
        for (int r = 0; r < L; ++r) b[r] = Bl[(long long)r * ld] * keep;
        if (MODE == MODE_MATVEC) {
          const float* Xl = X + (long long)leaf * L * ld + pa;
          const float* dd = ddg + (long long)leaf * L;
#pragma unroll
          for (int r = 0; r < L; r += 2) {
            const float x0 = Xl[(long long)r * ld] * keep, x1 = Xl[(long long)(r + 1) * ld] * keep;
            b[r] -= __ldg(dd + r) * x0;
            b[r + 1] -= __ldg(dd + r + 1) * x1;
            xq[r / 2] = pack_bf16(x0, x1);
          }
        }
        return;
      }
      const float* Xl = X + (long long)leaf * L * ld;
      const long long n0 = nbr[0] >= 0 ? nbr[0] : pa, n1 = nbr[1] >= 0 ? nbr[1] : pa;
      const long long n2 = nbr[2] >= 0 ? nbr[2] : pa, n3 = nbr[3] >= 0 ? nbr[3] : pa;
      const float w0 = nbr[0] >= 0 ? inv_h2 : 0.f, w1 = nbr[1] >= 0 ? inv_h2 : 0.f;
      const float w2 = nbr[2] >= 0 ? inv_h2 : 0.f, w3 = nbr[3] >= 0 ? inv_h2 : 0.f;
#pragma unroll
      for (int r0 = 0; r0 < L; r0 += 8) {
        float v[8], a0[8], a1[8], a2[8], a3[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long o = (long long)(r0 + j) * ld;
          v[j] = Bl[o];
          a0[j] = Xl[o + n0];
          a1[j] = Xl[o + n1];
          a2[j] = Xl[o + n2];
          a3[j] = Xl[o + n3];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) b[r0 + j] = keep * (v[j] + w0 * a0[j] + w1 * a1[j] + w2 * a2[j] + w3 * a3[j]);
      }
    };
    load_leaf(0);
    for (int i = 0; i < nb && !failed; ++i) {
      unsigned char* xr_i = ring + (size_t)(i % W) * tile_bytes;
      if (MODE == MODE_MATVEC) {
        // x_i into the ring now (its slot's previous tile, x_{i-W}, was last read by leaf i-1's MMAs,
        // complete since this thread waited on their barriers)
#pragma unroll
        for (int r = 0; r < L; r += 8) put8_packed(xr_i, c, r, L, &xq[r / 2]);
      }
      bool acc_used = false;
      int nu = 0;  // UPART chunks of this leaf so far
      for (bool leaf_done = false; !leaf_done && !failed;) {
        if (give_up(mbar_wait_or_abort(full + cslot, cphase, abort_flag, B.spin))) {
          failed = true;
          break;
        }
        const int4 cd = sdesc[cslot];
        leaf_done = ((cd.x >> 12) & 1) != 0;
        const int type = cd.x & 15, cnt = (cd.x >> 4) & 0xff;
        unsigned char* buf = slots + (size_t)cslot * B.slot_bytes;
        const uint32_t b_addr = smem_u32(buf);
        if (type == PK_DENSE) {
          if (issuer) {
            tc_after_sync();
            umma_product(t_acc, smem_u32(ring + (size_t)(cd.y % W) * tile_bytes), b_addr, L, L, acc_used);
            umma_commit(empty + cslot);
          }
          acc_used = true;
        } else if (type == PK_UPART) {
          const int kp = cnt;  // padded to 16; padding columns of U are zero
          if (nu > 0) {  // the previous U product of this leaf has read the staging tile
            if (issuer) umma_commit(accbar);
            if (!wait_mma(accbar, accph)) {
              failed = true;
              break;
            }
          }
          const int* uz = reinterpret_cast<const int*>(buf + (size_t)L * kp * 2);
          for (int k0 = 0; k0 < kp; k0 += 8) {
            float zv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) zv[e] = zpool[uz[k0 + e] * NT + c];
            put8(zstage, c, k0, kp, zv);
          }
          if (!consumer_sync()) {
            failed = true;
            break;
          }
          if (issuer) {
            umma_product(t_acc, smem_u32(zstage), b_addr, kp, L, acc_used);
            umma_commit(empty + cslot);
          }
          acc_used = true;
          ++nu;
        } else if (type == PK_DIAG) {
          if (MODE == MODE_SMOOTH) {
            if (acc_used) {
              if (issuer) umma_commit(accbar);
              if (!wait_mma(accbar, accph)) {
                failed = true;
                break;
              }
#pragma unroll
              for (int r0 = 0; r0 < L; r0 += 16) {
                float a[16];
                tmem_ld16(t_acc + lane_base + r0, a);
#pragma unroll
                for (int j = 0; j < 16; ++j) b[r0 + j] -= a[j];
              }
            }
            // b now holds y; stage it as the A operand of the inverse's product
#pragma unroll
            for (int r = 0; r < L; r += 8) put8(ystage, c, r, L, &b[r]);
            if (!consumer_sync()) {
              failed = true;
              break;
            }
            if (issuer) {
              umma_product(t_res, smem_u32(ystage), b_addr, L, L, false);
              umma_commit(empty + cslot);
              umma_commit(resbar);
            }
            if (!wait_mma(resbar, resph)) {
              failed = true;
              break;
            }
            const float* dd = ddg + (long long)i * L;
#pragma unroll
            for (int r0 = 0; r0 < L; r0 += 16) {
              float a[16];
              tmem_ld16(t_res + lane_base + r0, a);
#pragma unroll
              for (int j = 0; j < 16; ++j) b[r0 + j] = a[j] + __ldg(dd + r0 + j) * b[r0 + j];  // b := x_i
              put8(xr_i, c, r0, L, &b[r0]);
              put8(xr_i, c, r0 + 8, L, &b[r0 + 8]);
            }
            async_proxy_fence();  // x_i in the ring, ordered before the V products ...
            tc_before_sync();     // ... and the reads of res before later MMAs
            // global stores and loads only after the fence, which would otherwise wait for them
            if (valid) {
#pragma unroll
              for (int r = 0; r < L; ++r) X[(long long)(i * L + r) * ld + p] = b[r];
            }
            load_leaf(i + 1);
            if (!arrive_wait()) {  // x_i complete in the ring before the V products read it
              failed = true;
              break;
            }
          } else {
            if (!consumer_sync()) {  // x_i staged by every thread
              failed = true;
              break;
            }
            if (issuer) {
              umma_product(t_acc, smem_u32(xr_i), b_addr, L, L, acc_used);
              umma_commit(empty + cslot);
              umma_commit(accbar);
            }
            if (!wait_mma(accbar, accph)) {
              failed = true;
              break;
            }
#pragma unroll
            for (int r0 = 0; r0 < L; r0 += 16) {
              float a[16];
              tmem_ld16(t_acc + lane_base + r0, a);
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const float o = b[r0 + j] - a[j];
                if (valid) {
                  if (J.OUT) J.OUT[(long long)(i * L + r0 + j) * ld + p] = o;
                  const double av = fabs((double)o);
                  local_max = (av > local_max || av != av) ? av : local_max;
                }
              }
            }
            tc_before_sync();  // the reads of acc ordered before the next leaf's MMAs
            load_leaf(i + 1);
            if (!arrive_wait()) {  // every thread has read acc before the next leaf's MMAs
              failed = true;
              break;
            }
          }
        } else {  // PK_VPART: z entries from x_i
          const int np = (cnt + 15) / 16 * 16;
          if (issuer) {
            umma_product(t_v, smem_u32(xr_i), b_addr, L, np, false);
            umma_commit(empty + cslot);
            umma_commit(vbar);
          }
          if (!wait_mma(vbar, vph)) {
            failed = true;
            break;
          }
          const int* codes = reinterpret_cast<const int*>(buf + (size_t)np * L * 2);
          for (int q0 = 0; q0 < cnt; q0 += 16) {
            float a[16];
            tmem_ld16(t_v + lane_base + q0, a);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (q0 + j < cnt) {
                const int code = codes[q0 + j];
                float* z = zpool + (code >> 1) * NT + c;
                *z = (code & 1) ? a[j] : *z + a[j];
              }
            }
          }
          if (!leaf_done && !consumer_sync()) {  // v is read before the next V product overwrites it
            failed = true;
            break;
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
    if (MODE == MODE_MATVEC && J.norm != nullptr && !failed) {
      for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, local_max, o);
        local_max = (other > local_max || other != other) ? other : local_max;
      }
      if (lane == 0) atomicMax(J.norm, (unsigned long long)__double_as_longlong(local_max));
    }
  }
  // exit (normal or after a wait gave up): the MMAs issued so far complete, every consumer warp is
  // done with tensor memory (a barrier used once, so its phase is 0 whatever happened before), then
  // the allocating warp frees it.  Every consumer wait is bounded, so every warp arrives.
  if (issuer) umma_commit(donebar);
  tc_before_sync();
  __syncwarp();
  if (lane == 0) mbar_arrive(exitbar);
  if (w == 0) {
    mbar_wait(exitbar, 0);
    mbar_wait(donebar, 0);
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmmaTmemCols));
  }
}

}  // namespace fhmg
