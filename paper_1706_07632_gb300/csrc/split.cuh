// FP64-accurate finest-grid defect  r = F - A_h u - (R~ (x) I) u  on the tcgen05 tensor cores, by
// error-free splitting of both factors of the time product into small-integer digits (the scheme of
// Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012, with BF16
// digits and FP32 accumulation).
//
// Splitting.  Every row m of the dense time matrix R~ (lower triangular, M <= 512) has an exponent
// E_m with max_k |R~_mk| < 2^E_m; every grid point c has an exponent F_c with max_k |u_kc| < 2^F_c.
// Rounded to 49 bits, the scaled entries are sums of G = 7 balanced base-2^7 digits,
//     R~_mk = 2^E_m sum_a d_a(m,k) 2^{-7(a+1)},   u_kc = 2^F_c sum_b e_b(k,c) 2^{-7(b+1)},
// |d_0|, |e_0| <= 129, every other digit in [-64, 64].  Digits are small integers, exact in BF16, and
// a digit product (<= 2^14.1) is exact in the FP32 accumulator.  The products of digit pairs with
// equal a + b = g share the unit 2^{-7(g+2)}, so the group sums
//     A_g(m,c) = sum_{a+b=g} sum_k d_a(m,k) e_b(k,c)
// are integers; with K <= 512 their magnitude stays below (g+3) 2^21 <= 2^24 for g <= 5, so the
// tensor core's FP32 accumulation of these integers is exact (g = 6 may exceed 2^24 by a fraction,
// which costs at most a unit 2^-56 of the scale per accumulation step).  Then
//     sum_k R~_mk u_kc = 2^{E_m + F_c - 14} sum_g 2^{-7g} A_g(m,c) + O((m+1) 2^{E_m + F_c - 46}),
// the truncation coming from the 49-bit rounding of both factors and from the dropped groups
// g >= 7.  The group sums are combined in double-float arithmetic and joined to FP64 with integer
// operations (the FP64 pipe runs at 1/64 of the FP32 rate on GB300); a pre-pass at full occupancy
// forms B = F - A_h u in FP64 and the exponents F_c, and the kernel's epilogue writes r = B - R~ u.
//
// Kernel.  A CTA owns tiles of 64 grid points (MMA N = 64) and walks the output blocks I of 128
// time rows (MMA M = 128; TMEM lane = time row).  For every K-block J <= 2I+1 of 64 time levels
// the consumer warps split u's block J of the tile into the G digit tiles (B operands, 64 x 64,
// K-major, 128-byte swizzle, double-buffered), one MMA thread multiplies them with the digit tiles of R~'s
// block (I, J) (A operands, 128 x 64, produced by build_split, all-zero digit tiles left out) into
// the G group accumulators (G x 64 TMEM columns), and after the last J the consumer warps read the
// groups back (tcgen05.ld) and form r.  A producer warp streams the R~ digit tiles through an
// mbarrier ring with cp.async.bulk.  Every wait is bounded and watches the shared abort flag; every
// exit frees the tensor memory after the issued MMAs completed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "panel.cuh"
#include "umma.cuh"
#include "walk.h"

namespace fhmg {

constexpr int kSpG = 7;                         // digits per factor = group accumulators
constexpr int kSpCols = 64;                     // grid points per tile (MMA N)
constexpr int kSpRows = kSplitRows;             // time rows per output block (MMA M)
constexpr int kSpK = 64;                        // time levels per K-block
constexpr int kSpConsumers = 256;               // 8 consumer warps
constexpr int kSpBlock = kSpConsumers + 64;     // + producer warp + MMA warp
constexpr uint32_t kSpTmemCols = 512;
constexpr int kSpAtile = kSpRows * kSpK * 2;    // bytes of one R~ digit tile
constexpr int kSpBtile = kSpCols * kSpK * 2;    // bytes of one u digit tile
constexpr int kSpPieceLd = kSpRows + 1;         // float pairs per point of the epilogue's piece (odd: no bank conflicts)
static_assert((size_t)32 * kSpPieceLd * 8 <= (size_t)kSpG * kSpBtile, "a piece fits a digit buffer");

struct SplitSmem {
  size_t ring, xbuf, stage, col, bar, total;
};
__host__ __device__ inline SplitSmem split_smem(int ns) {
  SplitSmem s;
  s.ring = 0;
  s.xbuf = (size_t)ns * kSpAtile;
  // the next K-block's u values ([64 levels][64 points] doubles); during an epilogue the same bytes hold
  // the transposed piece of points 0..31 ([32 points][kSpPieceLd] float pairs; points 32..63 go to
  // the free digit buffer, kSpG * kSpBtile bytes)
  s.stage = s.xbuf + 2 * (size_t)kSpG * kSpBtile;
  const size_t stage_bytes = (size_t)kSpK * kSpCols * 8, piece_bytes = (size_t)32 * kSpPieceLd * 8;
  s.col = s.stage + (stage_bytes > piece_bytes ? stage_bytes : piece_bytes);
  s.bar = s.col + (size_t)kSpCols * 16;
  // full[ns], empty[ns], xready[2], xfree[2], accdone, accfree, cbar, exitbar, donebar, then the
  // abort flag, the group mask and the TMEM address
  s.total = s.bar + 8 * ((size_t)2 * ns + 9) + 16;
  return s;
}

// ---- operand layout: K-major, 128-byte swizzle ----
// A tile row holds its 64 K entries (BF16) in 128 bytes; 8-row groups form 1024-byte atoms in which
// the 16-byte chunk c of row r sits at chunk position c ^ (r % 8) (the tensor core reads the atoms
// without bank conflicts).  Tiles start on 1024-byte boundaries.
__host__ __device__ inline uint32_t sp_sw128_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ r) & 7) << 4) + (k & 7) * 2);
}
// shared-memory descriptor of such a tile: start address, leading byte offset unused (1), 8-row
// groups 1024 bytes apart, fixed bits 46-48 = 0b001, swizzle mode 128B (2 in bits 61-63); a K step
// of 16 entries (32 bytes) advances the start address field by 2
__device__ __forceinline__ uint64_t sp_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// ---- integer views of FP64 values (no FP64 arithmetic) ----

// round(|x| * 2^-s) for the 53-bit significand mt of x, s >= -7 (left shift) .. (>= 64: 0)
__device__ __forceinline__ long long sp_shift_round(unsigned long long mt, int s) {
  if (s <= 0) return (long long)(mt << (-s));
  if (s >= 64) return 0;
  return (long long)((mt + (1ULL << (s - 1))) >> s);
}

// round(x 2^{1075 - shift_base}) for the FP64 value x given by its bits (biased exponent e,
// significand mt: x = mt 2^{e - 1075}, so the result is round(mt 2^{e - shift_base})); subnormals as 0
__device__ __forceinline__ long long sp_fixed(unsigned long long bits, int shift_base) {
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long mt = (bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const long long v = sp_shift_round(mt, shift_base - e);
  return (bits >> 63) ? -v : v;
}

// float 2^k (0 below the normal range, clamped at 2^127)
__device__ __forceinline__ float sp_pow2f(int k) {
  return k < -126 ? 0.f : __int_as_float((min(k, 127) + 127) << 23);
}

// FP64 value of float f times 2^k, exactly (integer operations; f normal or zero)
__device__ __forceinline__ double sp_f2d_scaled(float f, int k) {
  const uint32_t b = __float_as_uint(f);
  const int ef = (int)((b >> 23) & 0xFF);
  if (ef == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const long long ed = (long long)ef - 127 + 1023 + k;
  if (ed <= 0) return 0.0;  // below the FP64 normal range
  if (ed >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ULL));
  const unsigned long long mant = (unsigned long long)(b & 0x7FFFFF) << 29;
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | mant));
}

// FP64 nearest (up to one rounding of the smaller part) to (h + l) 2^k for a float pair, by integer
// operations: the 24-bit significand of the part with the larger exponent is widened to 53 bits and
// the other one's added at its offset (dropped below 2^-25 of its last place); zero: the other alone.
__device__ __forceinline__ double sp_join(float h, float l, int k) {
  uint32_t hb = __float_as_uint(h), lb = __float_as_uint(l);
  if (((lb >> 23) & 0xFF) > ((hb >> 23) & 0xFF)) {  // the larger exponent leads (then d <= 29 below)
    const uint32_t x = hb;
    hb = lb;
    lb = x;
  }
  const int eh = (int)((hb >> 23) & 0xFF), el = (int)((lb >> 23) & 0xFF);
  if (eh == 0) return sp_f2d_scaled(l, k);
  long long Mh = (long long)((hb & 0x7FFFFF) | 0x800000) << 29;  // units 2^{eh - 127 - 52}
  if (hb >> 31) Mh = -Mh;
  if (el != 0) {
    const int d = el - eh + 29;  // l's significand in units of Mh's last place: shift by d
    const long long ml = (long long)((lb & 0x7FFFFF) | 0x800000);
    long long Ml = d >= 0 ? (ml << d) : (d > -25 ? ((ml + (1LL << (-d - 1))) >> (-d)) : 0);
    if (lb >> 31) Ml = -Ml;
    Mh += Ml;
  }
  if (Mh == 0) return 0.0;
  const unsigned long long sign = Mh < 0 ? (1ULL << 63) : 0ULL;
  unsigned long long a = (unsigned long long)(Mh < 0 ? -Mh : Mh);
  int e = eh - 127 - 52 + k;  // value = a 2^e
  const int lz = __clzll((long long)a);  // normalise to 53 bits (bit 52 set)
  if (lz > 11) {
    a <<= (lz - 11);
    e -= lz - 11;
  } else if (lz < 11) {
    const int sh = 11 - lz;
    a = (a + (1ULL << (sh - 1))) >> sh;
    e += sh;
    if (a >> 53) {
      a >>= 1;
      ++e;
    }
  }
  const long long ed = (long long)e + 52 + 1023;
  if (ed <= 0) return 0.0;
  if (ed >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ULL));
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | (a & 0xFFFFFFFFFFFFFULL)));
}

// (h, l) = a + b exactly
__device__ __forceinline__ void sp_two_sum(float a, float b, float& h, float& l) {
  h = __fadd_rn(a, b);
  const float bb = __fsub_rn(h, a);
  l = __fadd_rn(__fsub_rn(a, __fsub_rn(h, bb)), __fsub_rn(b, bb));
}


// two digits as a BF16 pair (the first in the low half)
__device__ __forceinline__ uint32_t sp_bf16pair(int d0, int d1) {
  // small integers are exact in FP32 via the 1.5 * 2^23 offset; their BF16 is the high half
  const uint32_t f0 = __float_as_uint(__int_as_float(0x4B400000 + d0) - 12582912.0f);
  const uint32_t f1 = __float_as_uint(__int_as_float(0x4B400000 + d1) - 12582912.0f);
  return __byte_perm(f0, f1, 0x7632);
}

// the G balanced base-2^7 digits of an integer |X| <= 2^49 (X = sum_b d_b 2^{7(G-1-b)}), most
// significant first; 32-bit operations: the low 28 bits give digits G-1..G-4, the rest d_0..d_2
__device__ __forceinline__ void sp_digits(long long X, int (&d)[kSpG]) {
  uint32_t lo = (uint32_t)X & 0x0FFFFFFFu;
  int hi = (int)(X >> 28);
#pragma unroll
  for (int b = kSpG - 1; b >= kSpG - 4; --b) {
    const int v = (int)((lo + 64u) & 127u) - 64;
    d[b] = v;
    lo = (uint32_t)((int)lo - v) >> 7;
  }
  hi += (int)lo;  // carry
#pragma unroll
  for (int b = kSpG - 5; b >= 1; --b) {
    const int v = ((hi + 64) & 127) - 64;
    d[b] = v;
    hi = (hi - v) >> 7;
  }
  d[0] = hi;
}

// FP64 value of the integer D times 2^k (D exact up to 53 bits, else rounded half up), by integer
// operations; 0 below the FP64 normal range
__device__ __forceinline__ double sp_ll2d(long long D, int k) {
  if (D == 0) return 0.0;
  const unsigned long long sign = D < 0 ? (1ULL << 63) : 0ULL;
  unsigned long long a = (unsigned long long)(D < 0 ? -D : D);
  int msb = 63 - __clzll((long long)a);
  if (msb <= 52) {
    a <<= (52 - msb);
  } else {
    const int sh = msb - 52;
    a = (a + (1ULL << (sh - 1))) >> sh;
    if (a >> 53) {
      a >>= 1;
      ++msb;
    }
  }
  const long long ed = (long long)msb + k + 1023;
  if (ed <= 0) return 0.0;
  if (ed >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ULL));
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | (a & 0xFFFFFFFFFFFFFULL)));
}

// Pre-pass, one thread per grid point (grid-stride), over the M time levels: fe[p] = the largest
// biased exponent of u at p, and B = F - A_h u written to B -- the defect kernel then subtracts R~ u
// in place.  The stencil needs FP64 accuracy (at N = 4095 it cancels 2^24-fold).  Two time levels in
// three form it with FP64 FMAs and subtractions (a few 2^-53 of |A_h| |u|); the third exactly in
// 64-bit fixed point relative to the largest of its five values (59 bits), converted by integer
// operations -- so the FP64 pipe (1/64 of the FP32 rate on GB300) and the integer pipe share the work
// -- and both end with one FMA, B = F - S / h^2.  An Inf or NaN in u or F propagates.
__global__ void __launch_bounds__(256) split_prep_kernel(const double* __restrict__ U, const double* __restrict__ F,
                                                         double* __restrict__ B, int* __restrict__ fe, long long ld,
                                                         int M, int dim, int N, double ih) {
  const unsigned long long* u = reinterpret_cast<const unsigned long long*>(U);
  const double cdiag = dim == 2 ? 4.0 : 2.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < ld; p += (long long)gridDim.x * blockDim.x) {
    const int ix = dim == 2 ? (int)(p % N) : (int)p;
    const int iy = dim == 2 ? (int)(p / N) : 0;
    const long long o0 = ix > 0 ? p - 1 : p, o1 = ix < N - 1 ? p + 1 : p;
    const long long o2 = (dim == 2 && iy > 0) ? p - N : p, o3 = (dim == 2 && iy < N - 1) ? p + N : p;
    const unsigned long long k0 = ix > 0 ? ~0ULL : 0ULL, k1 = ix < N - 1 ? ~0ULL : 0ULL;
    const unsigned long long k2 = (dim == 2 && iy > 0) ? ~0ULL : 0ULL, k3 = (dim == 2 && iy < N - 1) ? ~0ULL : 0ULL;
    unsigned int mx = 0;
#pragma unroll 3
    for (int m = 0; m < M; ++m) {
      const long long r = (long long)m * ld;
      const unsigned long long bc = __ldg(u + r + p);
      const unsigned long long x0 = __ldg(u + r + o0) & k0, x1 = __ldg(u + r + o1) & k1;
      const unsigned long long x2 = __ldg(u + r + o2) & k2, x3 = __ldg(u + r + o3) & k3;
      auto ex = [](unsigned long long b) { return (int)((b >> 52) & 0x7FF); };
      mx = max(mx, (unsigned int)ex(bc));
      double S;
      if (m % 3 != 2) {
        auto d = [](unsigned long long b) { return __longlong_as_double((long long)b); };
        const double t = fma(cdiag, d(bc), -d(x0));
        S = (t - d(x1)) - (d(x2) + d(x3));
      } else {
        // X = round(u 2^{59 - (ql - 1022)}) = round(mt 2^{e - ql + 6}); |D| < 2^62
        const int ql = max(max(ex(bc), ex(x0)), max(max(ex(x1), ex(x2)), ex(x3)));
        const int sb = ql - 6;
        const long long D = (dim == 2 ? 4 : 2) * sp_fixed(bc, sb) - sp_fixed(x0, sb) - sp_fixed(x1, sb) -
                            sp_fixed(x2, sb) - sp_fixed(x3, sb);
        S = ql == 2047 ? __longlong_as_double(0x7FF8000000000000LL) : sp_ll2d(D, ql - 1022 - 59);
      }
      B[r + p] = fma(-ih, S, __ldg(F + r + p));
    }
    fe[p] = (int)mx;
  }
}

struct SpCol {
  int fe;     // the point's exponent (biased; 2047: an Inf or NaN in u at the point, r := NaN)
  int valid;
  int pad0, pad1;
};

__global__ void __launch_bounds__(kSpBlock, 1) split_defect_kernel(const __grid_constant__ SplitArgs A) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  // the swizzled operand tiles need 1024-byte aligned addresses (the launcher adds 1 KB)
  unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
  const SplitSmem lay = split_smem(A.ns);
  const int ns = A.ns;
  unsigned char* ring = sm + lay.ring;
  unsigned char* xbuf = sm + lay.xbuf;
  SpCol* col = reinterpret_cast<SpCol*>(sm + lay.col);
  unsigned long long* stage = reinterpret_cast<unsigned long long*>(sm + lay.stage);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + lay.bar);
  uint64_t* empty = full + ns;
  uint64_t* xready = empty + ns;  // [2]
  uint64_t* xfree = xready + 2;   // [2]
  uint64_t* accdone = xfree + 2;
  uint64_t* accfree = accdone + 1;
  uint64_t* cbar = accdone + 2;
  uint64_t* exitbar = accdone + 3;
  uint64_t* donebar = accdone + 4;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(accdone + 5);
  volatile int* gmask = abort_flag + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accdone + 5) + 2;

  const int t = threadIdx.x;
  const int w = t >> 5;
  const int lane = t & 31;
  const int nI = A.M / kSpRows;

  if (t == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);  // the MMAs' commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(xready + b, kSpConsumers / 32);
      mbar_init(xfree + b, 1);
    }
    mbar_init(accdone, 2);  // the MMAs' commit + the MMA thread's arrive after publishing the group mask
    mbar_init(accfree, kSpConsumers / 32);
    mbar_init(cbar, kSpConsumers / 32);
    mbar_init(exitbar, kSpConsumers / 32 + 1);
    mbar_init(donebar, 1);
    *abort_flag = 0;
    *gmask = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kSpTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before_sync();
  __syncthreads();  // the last block-wide barrier: from here on the roles run apart
  tc_after_sync();
  const uint32_t tmem = *tslot;

  auto raise = [&]() {
    if (!*abort_flag) {
      *abort_flag = 1;
      atomicExch(A.err, 1);
    }
  };

  if (w == kSpConsumers / 32) {
    // ---- producer: R~ digit tiles of every pair of every tile of this CTA, in order ----
    if (lane != 0) return;
    long long k = 0;
    int slot = 0;
    bool ok = true, stop = false;
    const int npairs = nI * (nI + 1);
    for (long long g = blockIdx.x; g < A.ntiles && ok && !stop; g += gridDim.x)
      for (int q = 0; q < npairs && ok && !stop; ++q) {
        const int4 pd = __ldg(A.pairs + q);
        int ti = pd.y;
        for (int a = 0; a < kSpG; ++a) {
          if (!((pd.x >> a) & 1)) continue;
          if (k + 1 == A.withhold) {
            stop = true;
            break;
          }
          if (k >= ns && !mbar_wait_or_abort(empty + slot, (uint32_t)(((k / ns) - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bulk_load(ring + (size_t)slot * kSpAtile, A.At + (size_t)ti * kSpAtile, kSpAtile, full + slot);
          ++ti;
          ++k;
          if (++slot == ns) slot = 0;
        }
      }
    if (!ok) raise();
    for (int s = 0; s < ns && s < k; ++s) {
      const long long n_s = (k - 1 - s) / ns + 1;
      mbar_wait(full + s, (uint32_t)((n_s - 1) & 1));
    }
    return;
  }

  if (w == kSpConsumers / 32 + 1) {
    // ---- MMA thread ----
    if (lane == 0) {
      long long k = 0, q = 0, nblk = 0;
      int slot = 0;
      bool failed = false;
      for (long long g = blockIdx.x; g < A.ntiles && !failed; g += gridDim.x)
        for (int I = 0; I < nI && !failed; ++I, ++nblk) {
          if (nblk > 0 && !mbar_wait_or_abort(accfree, (uint32_t)((nblk - 1) & 1), abort_flag, A.spin)) {
            failed = true;
            break;
          }
          tc_after_sync();
          int touched = 0;
          for (int J = 0; J <= 2 * I + 1 && !failed; ++J, ++q) {
            const int b = (int)(q & 1);
            if (!mbar_wait_or_abort(xready + b, (uint32_t)((q >> 1) & 1), abort_flag, A.spin)) {
              failed = true;
              break;
            }
            tc_after_sync();
            const int4 pd = __ldg(A.pairs + I * (I + 1) + J);
            const uint32_t xb = smem_u32(xbuf + (size_t)b * kSpG * kSpBtile);
            // operand descriptors (K-major, 128-byte swizzle); a K step of 16 adds 2
            uint64_t bdesc[kSpG];
#pragma unroll
            for (int bb = 0; bb < kSpG; ++bb) bdesc[bb] = sp_desc_sw128(xb + (uint32_t)bb * kSpBtile);
            const uint32_t idesc = umma_idesc(kSpCols);
            for (int a = 0; a < kSpG; ++a) {
              if (!((pd.x >> a) & 1)) continue;
              if (!mbar_wait_or_abort(full + slot, (uint32_t)((k / ns) & 1), abort_flag, A.spin)) {
                failed = true;
                break;
              }
              tc_after_sync();
              const uint64_t adesc = sp_desc_sw128(smem_u32(ring + (size_t)slot * kSpAtile));
#pragma unroll
              for (int bb = 0; bb < kSpG; ++bb) {
                if (bb + a >= kSpG) break;
                const int gg = a + bb;
                const uint32_t d = tmem + 64u * gg;
                const uint32_t acc0 = (touched >> gg) & 1;
#pragma unroll
                for (int st = 0; st < kSpK / 16; ++st)
                  asm volatile(
                      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                      "l"(adesc + 2ULL * st), "l"(bdesc[bb] + 2ULL * st), "r"(idesc), "r"(st > 0 ? 1u : acc0)
                      : "memory");
                touched |= 1 << gg;
              }
              umma_commit(empty + slot);
              ++k;
              if (++slot == ns) slot = 0;
            }
            if (failed) break;
            umma_commit(xfree + b);
          }
          if (failed) break;
          *gmask = touched;
          umma_commit(accdone);
          mbar_arrive(accdone);  // release: the group mask is visible to the consumers after their wait
        }
      if (failed) raise();
      umma_commit(donebar);  // completes when every MMA issued above has completed
    }
    __syncwarp();
    tc_before_sync();
    if (lane == 0) mbar_arrive(exitbar);
    return;
  }

  // ---- consumers: 8 warps ----
  uint32_t cbphase = 0;
  bool failed = false;
  auto give_up = [&](bool ok) -> bool {
    if (__all_sync(0xffffffffu, ok)) return false;
    if (lane == 0) raise();
    return true;
  };
  auto consumer_meet = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(cbar);
    const bool ok = mbar_wait_or_abort(cbar, cbphase, abort_flag, A.spin);
    cbphase ^= 1;
    return !give_up(ok);
  };
  const long long ld = A.ld;
  const unsigned long long* Ub = reinterpret_cast<const unsigned long long*>(A.U);
  // split: thread t owns point n = t & 63 of the tile and 16 time levels (t >> 6) * 16 .. of a K-block
  const int sn = t & 63, sk = (t >> 6) * 16;
  // epilogue: lane quarter (time rows) and column half
  const int wq = w & 3, ch = w >> 2;
  const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
  unsigned long long nmax = 0;
  long long q = 0, nblk = 0;
  const int npairs = nI * (nI + 1);

  // L2 prefetch of the B rows that block I's epilogue reads (this thread's time row, its 32 points):
  // issued when the block's first pair is split, so that their latency overlaps the block's MMAs
  auto prefetch_block = [&](long long p0, int I) {
    const int m = I * kSpRows + wq * 32 + lane;
    const long long pc = p0 + ch * 32;
    const double* orow = A.OUT + (long long)m * ld;
#pragma unroll
    for (int o = 0; o < 32; o += 16) {
      const long long i = pc + o < ld ? pc + o : ld - 1;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(orow + i));
    }
  };

  // epilogue of output block I of the tile at p0 (its accumulators complete: accdone waited).  Phase
  // 1: all eight warps fold the seven groups of their 32 time rows x 32 points into double-float sums
  // and write them transposed into the two pieces (points 0..31 in the staging bytes, points 32..63
  // in digit buffer bfree, whose pair's MMAs completed with the block's), then release tensor memory,
  // so that the next block's MMAs start while phase 2 runs.  Phase 2: thread per grid point, so that
  // every global access is a contiguous row segment.
  auto epilogue = [&](long long p0, int I, int bfree, auto&& mid) -> bool {
    const int mask = *gmask;
    float2* const piece0 = reinterpret_cast<float2*>(stage);
    float2* const piece1 = reinterpret_cast<float2*>(xbuf + (size_t)bfree * kSpG * kSpBtile);
    if (!consumer_meet()) return false;  // every warp has read its staged values (piece 0 reuses them)
    {
      float2* const pc = ch ? piece1 : piece0;
      const int ml = wq * 32 + lane;
#pragma unroll 1
      for (int c8 = 0; c8 < 4; ++c8) {
        const uint32_t n0 = (uint32_t)(ch * 32 + c8 * 8);
        uint32_t r[kSpG][8];
#pragma unroll
        for (int gg = 0; gg < kSpG; ++gg)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
              : "=r"(r[gg][0]), "=r"(r[gg][1]), "=r"(r[gg][2]), "=r"(r[gg][3]), "=r"(r[gg][4]), "=r"(r[gg][5]),
                "=r"(r[gg][6]), "=r"(r[gg][7])
              : "r"(tmem + lane_base + 64u * gg + n0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // the loaded registers are read only after the wait
#pragma unroll
        for (int gg = 0; gg < kSpG; ++gg)
          asm volatile("" : "+r"(r[gg][0]), "+r"(r[gg][1]), "+r"(r[gg][2]), "+r"(r[gg][3]), "+r"(r[gg][4]),
                       "+r"(r[gg][5]), "+r"(r[gg][6]), "+r"(r[gg][7]));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float ph = (mask & 1) ? __uint_as_float(r[0][j]) : 0.f, pl = 0.f;
#pragma unroll
          for (int gg = 1; gg < kSpG; ++gg) {
            const float a = ((mask >> gg) & 1) ? __uint_as_float(r[gg][j]) : 0.f;
            float s2, e;
            sp_two_sum(ph, a * sp_pow2f(-7 * gg), s2, e);
            ph = s2;
            pl = __fadd_rn(pl, e);
          }
          pc[(size_t)(c8 * 8 + j) * kSpPieceLd + ml] = make_float2(ph, pl);
        }
      }
      tc_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(accfree);  // this warp is done with block I's accumulators
    }
    if (!consumer_meet()) return false;  // the pieces are complete
    // thread: point n = half * 32 + lane, time rows w * 16 .. + 15 of the block, half 0 first:
    // r = B - (R~ u), B = F - A_h u from the pre-pass (in OUT).  Once every thread is done with piece
    // 0, mid() may reuse the staging bytes (the next K-block's copies overlap half 1)
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int n = half * 32 + lane;
      const float2* const pc = half ? piece1 : piece0;
      const SpCol c = col[n];
      const long long p = p0 + n;
      const long long pa = c.valid ? p : 0;
      double bv[16];
      const double* bsrc = A.OUT + (long long)(I * kSpRows + w * 16) * ld + pa;
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) bv[rr] = __ldcg(bsrc + (long long)rr * ld);
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const int ml = w * 16 + rr;
        const int m = I * kSpRows + ml;
        const int Em = __ldg(A.rexp + m);
        const float2 P = pc[(size_t)lane * kSpPieceLd + ml];
        // (R~ u)_{m,c} = 2^{E_m + F_c - 14} P, F_c = fe - 1022
        const double y = sp_join(P.x, P.y, Em + c.fe - 1036);
        const double r = c.fe == 2047 ? __longlong_as_double(0x7FF8000000000000LL) : bv[rr] - y;
        if (c.valid) {
          A.OUT[(long long)m * ld + p] = r;
          const unsigned long long ab = (unsigned long long)__double_as_longlong(r) & 0x7FFFFFFFFFFFFFFFULL;
          nmax = ab > nmax ? ab : nmax;
        }
      }
      if (half == 0) {
        if (!consumer_meet()) return false;  // every thread is done with piece 0
        mid();
      }
    }
    return consumer_meet();  // every thread is done with the pieces
  };

  for (long long g = blockIdx.x; g < A.ntiles && !failed; g += gridDim.x) {
    const long long p0 = g * kSpCols;
    if (!consumer_meet()) {  // the previous tile's epilogue is done with col[]
      failed = true;
      break;
    }
    if (t < kSpCols) {
      const long long p = p0 + t;
      SpCol c{0, 0, 0, 0};
      if (p < ld) {
        c.valid = 1;
        c.fe = __ldg(A.fe + p);
      }
      col[t] = c;
    }
    if (!consumer_meet()) {
      failed = true;
      break;
    }
    const SpCol mine = col[sn];
    const long long ps = mine.valid ? p0 + sn : 0;
    const int fshift = mine.fe + 4;  // X = round(u 2^{49 - F_c}) = round(mt 2^{e - fe - 4})
    // this thread's 16 values of K-block J, staged in shared memory by cp.async (the next block's
    // copies are issued once this one's digits are published); each thread reads back only its own
    unsigned long long* mystage = stage + (size_t)sk * kSpCols + sn;
    auto stage16 = [&](int J) {
      const unsigned long long* src = Ub + (long long)(J * kSpK + sk) * ld + ps;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(mystage + (size_t)j * kSpCols)),
                     "l"(src + (long long)j * ld)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    stage16(0);
    // the tile's pairs in order; block I's epilogue runs after the first pair of block I + 1 is
    // split (so that block I's last MMAs overlap that work), the last block's at the tile's end
    int I = 0, J = 0;
    for (int s = 0; s < npairs && !failed; ++s, ++q) {
      const int b = (int)(q & 1);
      if (q >= 2 && give_up(mbar_wait_or_abort(xfree + b, (uint32_t)(((q >> 1) - 1) & 1), abort_flag, A.spin))) {
        failed = true;
        break;
      }
      const int In = J + 1 <= 2 * I + 1 ? I : I + 1;
      const int Jn = J + 1 <= 2 * I + 1 ? J + 1 : 0;
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      unsigned long long v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = mine.valid ? mystage[(size_t)j * kSpCols] : 0ULL;
      unsigned char* xb = xbuf + (size_t)b * kSpG * kSpBtile;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t pk[kSpG][4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          int d0[kSpG], d1[kSpG];
          sp_digits(sp_fixed(v[8 * h + j], fshift), d0);
          sp_digits(sp_fixed(v[8 * h + j + 1], fshift), d1);
#pragma unroll
          for (int a = 0; a < kSpG; ++a) pk[a][j / 2] = sp_bf16pair(d0[a], d1[a]);
        }
#pragma unroll
        for (int a = 0; a < kSpG; ++a)
          *reinterpret_cast<uint4*>(xb + (size_t)a * kSpBtile + sp_sw128_off(sn, sk + 8 * h)) =
              make_uint4(pk[a][0], pk[a][1], pk[a][2], pk[a][3]);
      }
      async_proxy_fence();
      __syncwarp();
      if (lane == 0) mbar_arrive(xready + b);
      if (J == 0) prefetch_block(p0, I);
      const bool last = s + 1 == npairs;
      const bool epi = (J == 0 && I > 0) || last;
      // the next pair's copies only now (the proxy fence above waits for this thread's outstanding
      // memory operations) and, when an epilogue runs here, once it is done with the staging bytes
      if (!epi && s + 1 < npairs) stage16(Jn);
      if (epi) {
        // epilogue of block I - 1 (or, at the tile's end, of the last block)
        const int Ie = last ? I : I - 1;
        // the digit buffer of the pair split before this one: its MMAs completed with block Ie's
        const int bfree = b ^ 1;
        if (give_up(mbar_wait_or_abort(accdone, (uint32_t)(nblk & 1), abort_flag, A.spin))) {
          failed = true;
          break;
        }
        tc_after_sync();
        if (!epilogue(p0, Ie, bfree, [&]() {
              if (s + 1 < npairs) stage16(Jn);
            })) {
          failed = true;
          break;
        }
        ++nblk;
      }
      I = In;
      J = Jn;
    }
  }
  if (A.norm != nullptr && !failed) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, nmax, o);
      nmax = other > nmax ? other : nmax;
    }
    if (lane == 0) atomicMax(A.norm, nmax);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no staging copy outlives the thread
  // exit: every consumer warp and the MMA warp arrive (bounded waits everywhere, so all do), the
  // MMA thread's last commit signals that every issued MMA completed, then warp 0 frees TMEM
  tc_before_sync();
  __syncwarp();
  if (lane == 0) mbar_arrive(exitbar);
  if (w == 0) {
    mbar_wait(exitbar, 0);
    mbar_wait(donebar, 0);
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSpTmemCols));
  }
}

}  // namespace fhmg
