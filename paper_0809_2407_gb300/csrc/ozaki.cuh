// FP64 products on the tensor cores by error-free splitting (the scheme of Ozaki, Ogita, Oishi
// and Rump), for the compact-WY products of TSQR.
//
// Each FP64 operand row (A) or column (B) is written in fixed point against its largest
// exponent and cut into pieces that bf16 holds exactly; the piece products of one weight sum
// exactly in one FP32 tensor-core accumulator (a "group"), and an int64 epilogue recombines the
// groups.  Two forms are used:
//   - the digit form (the thin Q, Q^T B and Q B): 7 balanced base-256 digits of a 54-bit fixed
//     point rounded to nearest, 34 digit pairs in 8 groups; about 2^-51 relative to |A| |B|
//     (row and column maxima).  Its helpers are under "balanced base-256 digits" below.
//   - the 7-bit form (the factorization's Gram entries and its blocked step): v = sign * mag *
//     2^(E_max - 1078) with mag < 2^56, cut into 8 slices of 7 bits c_1 (most significant) ..
//     c_8, each in [0, 127] with the sign of v.  Slice products are below 2^14; summed over
//     K = 64 below 2^20, and the pairs of equal weight s + t = g (at most 8) below 2^23, so one
//     accumulator per weight group g = 2..9 holds its sum exactly.  The epilogue recombines
//       X = sum_{g<=8} G_g 2^(7(8-g)) + floor(G_9 / 2^7)   (|X| < 2^63),
//     and the product is X * 2^(E_A + E_B - 2100); the 36 pairs with s + t <= 9 give about
//     2^-49 relative to |A| |B| (magnitudes are truncated toward zero).
//
// tcgen05 use: one thread issues kind::f16 MMAs (bf16 in, FP32 out, M = 128, K = 16) from
// 128-byte-swizzled K-major shared-memory operands; the eight group accumulators of a 64-column
// product take all 512 TMEM columns of the SM, so those kernels run one block per SM.  The B
// pieces that one A piece meets lie one after another in shared memory, as do their groups in
// TMEM, so one MMA of N up to 256 takes several of them.  Completion is signalled by
// tcgen05.commit on an mbarrier; every wait on it is bounded.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tsqr {
namespace oz {

constexpr int kSlices = 8;        // 7-bit slices: 56 bits of each operand
constexpr int kTmemCols = 512;    // 8 groups x 64 columns
constexpr int kN = 64;            // N of every product (the padded column count)
constexpr int kM = 128;           // M of every MMA (rows beyond the operand are zero)
constexpr int kK = 64;            // K of every product
constexpr uint32_t kASliceBytes = kM * kK * 2;  // 16 KB
constexpr uint32_t kBSliceBytes = kN * kK * 2;  // 8 KB

// ---- tcgen05 wrappers -------------------------------------------------------------------------
// Shared-memory matrix descriptor of a K-major operand in 128-byte swizzled rows of 64 bf16:
// 8-row groups 1024 bytes apart (SBO), descriptor version 1, swizzle mode 128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t v[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- operand layout ---------------------------------------------------------------------------
// Byte offset of element (row r, k) of a K-major bf16 operand with 64 k per 128-byte row and the
// 128-byte swizzle (16-byte chunk index XOR row & 7); the operand base is 1024-byte aligned.
__device__ __forceinline__ uint32_t op_off(int r, int k) {
  const uint32_t byte = (uint32_t)k * 2u;
  return (uint32_t)r * 128u + ((((byte >> 4) ^ ((uint32_t)r & 7u))) << 4) + (byte & 15u);
}

// ---- error-free splitting ----------------------------------------------------------------------
// Biased exponent of v (0 for zero or subnormal).
__device__ __forceinline__ int bexp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}
// Fixed-point form against the row/column maximum biased exponent emax: bit 63 = sign,
// bits 0..55 = mag with |v| = mag * 2^(emax - 1078) (truncated below 2^(emax - 1078)).
__device__ __forceinline__ uint64_t to_fixed(double v, int emax) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int d = E - emax + 3;  // <= 3
  uint64_t mag;
  if (d >= 0)
    mag = m << d;
  else
    mag = (-d < 64) ? (m >> (-d)) : 0ull;
  return (b & 0x8000000000000000ull) | mag;
}
// The same for a double-float value (hi, lo) held in an 8-byte slot (hi in the low word), with
// integer operations only.  bexp_pair: hi's exponent in the FP64 bias (0 for zero or an FP32
// subnormal hi), an upper bound of the pair's (|lo| <= ulp(hi)/2 keeps hi + lo inside hi's
// binade or just below it).  to_fixed_pair: hi and lo each in fixed point against emax, summed
// (each term truncated, one unit of the fixed grid more than a single truncation).
__device__ __forceinline__ int bexp_pair(double raw) {
  const uint32_t hb = (uint32_t)(unsigned long long)__double_as_longlong(raw);
  const int E = (int)((hb >> 23) & 0xFF);
  return E == 0 ? 0 : E + (1023 - 127);
}
__device__ __forceinline__ long long fixed_f32(uint32_t b, int emax) {
  const int E = (int)((b >> 23) & 0xFF);
  if (E == 0) return 0;
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);  // |f| = m 2^(E - 150)
  const int sh = E - emax + 928;                               // 2^(1078 - emax) scaling: <= 32
  const uint64_t mag = (sh >= 0) ? (m << sh) : ((-sh < 64) ? (m >> (-sh)) : 0ull);
  return (b & 0x80000000u) ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ uint64_t to_fixed_pair(double raw, int emax) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(raw);
  const long long v = fixed_f32((uint32_t)u, emax) + fixed_f32((uint32_t)(u >> 32), emax);
  return v < 0 ? (0x8000000000000000ull | (uint64_t)(-v)) : (uint64_t)v;
}

// bf16 bits of slice s (1-based) of a fixed-point value: sign * ((mag >> (56 - 7 s)) & 127).
__device__ __forceinline__ uint32_t slice_bf16(uint64_t fx, int s) {
  const uint32_t c = (uint32_t)(fx >> (56 - 7 * s)) & 127u;
  const uint32_t sign = (uint32_t)(fx >> 48) & 0x8000u;
  if (c == 0) return 0;
  const int p = 31 - __clz(c);  // 0..6
  return sign | ((uint32_t)(127 + p) << 7) | ((c << (7 - p)) & 0x7Fu);
}
// X * 2^k as FP64 (X != 0 handled; k from E_A + E_B - 2100).
__device__ __forceinline__ double scale_int(long long X, int k) {
  if (X == 0) return 0.0;
  const double d = (double)X;
  const int E = (int)((__double_as_longlong(d) >> 52) & 0x7FF);
  const int En = E + k;
  if (En >= 1 && En <= 2046)
    return __longlong_as_double(__double_as_longlong(d) + ((long long)k << 52));
  return scalbn(d, k);
}

// X * 2^k as FP64 with integer operations only (round to nearest even), so the conversion does
// not occupy the FP64 pipe: for kernels bound by that pipe (the factorization's steps).  The
// thin-Q and apply kernels, bound by the integer ALU, keep scale_int.  X = 0 gives 0.  Falls back
// to scale_int outside the normal range.
__device__ __forceinline__ double int_to_f64_scaled(long long X, int k) {
  if (X == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)X & 0x8000000000000000ull;
  unsigned long long a = (X < 0) ? (unsigned long long)(-X) : (unsigned long long)X;
  const int lz = __clzll((long long)a);  // a < 2^63, so lz >= 1
  const int top = 63 - lz;                // a in [2^top, 2^(top+1))
  const int E = top + k + 1023;           // biased exponent of the result
  if (E < 1 || E > 2046) return scale_int(X, k);
  unsigned long long mant;
  if (top <= 52) {
    mant = a << (52 - top);
  } else {
    const int sh = top - 52;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    mant = a >> sh;
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;  // may carry into 2^53
  }
  // mant in [2^52, 2^53]; adding the exponent field absorbs a carry to 2^53 correctly
  const unsigned long long bits = sgn | (((unsigned long long)(E - 1) << 52) + mant);
  return __longlong_as_double((long long)bits);
}

// The int64 recombination X (this file's header) of the 8 weight groups of kCols accumulator
// columns of this warp's 32 TMEM lanes: group g (2..9) at TMEM column offset (g - 2) * stride.
template <int kCols>
__device__ __forceinline__ void load_groups(uint32_t taddr, uint32_t stride, long long acc[kCols]) {
#pragma unroll
  for (int c = 0; c < kCols; ++c) acc[c] = 0;
#pragma unroll 1
  for (int g = 2; g <= oz::kSlices + 1; ++g) {
    uint32_t v[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr + (uint32_t)(g - 2) * stride));
    oz::tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const long long G = (long long)__float2int_rn(__uint_as_float(v[c]));
      acc[c] += (g <= oz::kSlices) ? G * (1ll << (7 * (oz::kSlices - g))) : (G >> 7);
    }
  }
}

// ---- balanced base-256 digits ------------------------------------------------------------------
// A second form of the split, for the thin Q's recurrence and leaf-product kernels.  The value is
// written in 54-bit fixed point against its row/column's largest biased exponent emax,
// m = v 2^(1076 - emax) rounded to nearest (|m| < 2^54), and m + 0x0080808080808080 (0x80 in each
// of bytes 0..6, which keeps the sum in [0, 2^56)) is read byte by byte: byte j minus 128 is the
// digit of weight 2^(8 j), in [-128, 127], so m = sum_j d_j 2^(8 j) exactly.  Digit s = 1..7 is
// byte 7 - s (most significant first).  A digit is exact in bf16 (at most 8 significant bits), a
// product of two is at most 2^14 in magnitude, and the pairs of one weight g = s + t <= 9 (at most
// 8 of them) summed over K = 64 stay below 2^23: exact FP32 TMEM groups.  The 34 pairs with
// s + t <= 9 leave an error of about 2^-51 relative to |A| |B| (the 7-bit form's 36 pairs: 2^-49);
// the digits need no sign handling, and one byte permute and one FP32 add make each of them.
constexpr int kDigits = 7;
constexpr int kDigitGroups = 8;  // weights g = 2 .. 9
constexpr unsigned long long kDigitBias = 0x0080808080808080ull;

// The B operand carries an eighth digit slice of zeros, so that the first A slice meets
// t = 1 .. 8 and its MMAs (which start every accumulation) write all 8 groups; A slice s meets
// B slices t = 1 .. digit_t_max(s) = 9 - s.
constexpr int kDigitBSlices = 8;
__host__ __device__ constexpr int digit_t_max(int s) { return 9 - s; }

// Biased 54-bit fixed point of an FP64 value against emax (biased exponent, >= the value's).
__device__ __forceinline__ uint64_t to_biased54(double v, int emax) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return kDigitBias;
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // |v| = mant 2^(E - 1075)
  const int d = E + 1 - emax;                                      // <= 1: mag < 2^54
  const uint64_t mag = (d >= 0) ? (mant << d) : ((-d < 64) ? ((mant + (1ull << (-d - 1))) >> (-d)) : 0ull);
  return (b >> 63) ? kDigitBias - mag : kDigitBias + mag;
}
// The same for a double-float value (hi, lo) in an 8-byte slot (hi in the low word): each part in
// fixed point against emax (the exponent bound of bexp_pair), summed.
__device__ __forceinline__ long long fixed54_f32(uint32_t b, int emax) {
  const int E = (int)((b >> 23) & 0xFF);
  if (E == 0) return 0;
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);  // |f| = m 2^(E - 150)
  const int sh = E - emax + 926;                               // 2^(1076 - emax) scaling: <= 30
  const uint64_t mag = (sh >= 0) ? (m << sh) : ((-sh < 64) ? ((m + (1ull << (-sh - 1))) >> (-sh)) : 0ull);
  return (b & 0x80000000u) ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ uint64_t to_biased54_pair(double raw, int emax) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(raw);
  return kDigitBias + (uint64_t)(fixed54_f32((uint32_t)u, emax) + fixed54_f32((uint32_t)(u >> 32), emax));
}
// bf16 bits of digit s (1-based) of two biased fixed-point values, packed low | high.
__device__ __forceinline__ uint32_t digit_pair(uint64_t m0, uint64_t m1, int s) {
  const int byte = 7 - s;
  const uint32_t w0 = (byte >= 4) ? (uint32_t)(m0 >> 32) : (uint32_t)m0;
  const uint32_t w1 = (byte >= 4) ? (uint32_t)(m1 >> 32) : (uint32_t)m1;
  const uint32_t sel = 0x7540u | (uint32_t)(byte & 3);  // [the byte, 0, 0, 0x4B]: 2^23 + byte
  const float f0 = __fsub_rn(__uint_as_float(__byte_perm(w0, 0x4B000000u, sel)), 8388736.f);
  const float f1 = __fsub_rn(__uint_as_float(__byte_perm(w1, 0x4B000000u, sel)), 8388736.f);
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}
// The 8 weight groups G_2..G_9 (exact integers in FP32) of 8 accumulator columns of this warp's
// 32 TMEM lanes (group g at column offset (g - 2) stride), four groups' loads in flight per wait,
// recombined per column into X = sum_{g <= 7} G_g 2^(8 (7 - g)) + floor((G_8 2^8 + G_9) / 2^16)
// (|X| < 2^62; the product is X 2^(eA + eB - 2096)).  Pairs of groups meet in int32 first
// (|G_g 2^8 + G_{g+1}| < 2^31).
__device__ __forceinline__ void load_digit_groups8(uint32_t taddr, uint32_t stride, long long X[8]) {
  int p[4][8];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t v[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[u][0]), "=r"(v[u][1]), "=r"(v[u][2]), "=r"(v[u][3]), "=r"(v[u][4]), "=r"(v[u][5]),
                     "=r"(v[u][6]), "=r"(v[u][7])
                   : "r"(taddr + (uint32_t)(4 * half + u) * stride));
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      p[2 * half][c] = __float2int_rn(__uint_as_float(v[0][c])) * 256 + __float2int_rn(__uint_as_float(v[1][c]));
      p[2 * half + 1][c] = __float2int_rn(__uint_as_float(v[2][c])) * 256 + __float2int_rn(__uint_as_float(v[3][c]));
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    X[c] = ((long long)p[0][c] << 32) + ((long long)p[1][c] << 16) + (long long)p[2][c] + (long long)(p[3][c] >> 16);
}

// Bounded wait on an mbarrier phase (thread-level); false on timeout.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  return mbar_wait_bounded(bar, parity, kWaitCycles);
}

}  // namespace oz
}  // namespace tsqr
