// FP64 natural logarithm of the shower kernels: the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the logarithm function in
// IEEE floating-point arithmetic", ACM TOMS 16 (1990) 378-400, written here
// from the method's description.
//
// For a positive normal x = 2^e m with m in [sqrt(1/2), sqrt(2)):
//   F = j/128 is the breakpoint nearest to m (j = 90 .. 181), f = m - F is
//   exact (|f| <= 2^-8), r = f (1/F) with |r| < 0.0056, and
//     ln x = e ln 2 + ln F + ln(1 + r).
//   ln(1 + r) is its Taylor polynomial to r^7 (the first omitted term is
//   below 2^-56 relative); e ln2_hi + ln_hi is exact because both are
//   multiples of 2^-42 (log_table.inc); the small parts, then r, then that
//   exact sum are added, so that only the last two additions round.  r is
//   used only as a factor, so no compiler contraction can change a result.
// Every other input (zero, negative, subnormal, infinite, NaN) goes to the
// CUDA library's log.  The error stays below one ulp (checked against a
// 60-digit reference in the tests), the same class as the library function,
// at about half its FP64 cost: one log is taken per winning trial and four
// per accepted emission, the largest single FP64 item of a veto cycle.
//
// The same code compiles for the host (exported for the accuracy tests) and
// the device; every multiply-add that matters is an explicit fma, so both
// round alike.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "log_table.inc"

namespace gaps {

// double -> float, round to nearest even, with integer instructions for
// every result in the normal float range (the FP64 pipe's conversion costs
// as much as an FMA on this part; the ALU's instructions a small fraction of
// that); zeros, tiny, huge and non-finite values take the hardware
// conversion.  Bitwise the hardware result (tested against numpy's).
__host__ __device__ __forceinline__ float f32_from_f64(double x) {
#ifdef __CUDA_ARCH__
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t bits;
  std::memcpy(&bits, &x, sizeof bits);
#endif
  const uint64_t mag = bits & 0x7fffffffffffffffull;
  // exponent field 897 .. 1150: normal floats, before rounding
  if (mag - 0x3810000000000000ull >= 0x0fe0000000000000ull) {
#ifdef __CUDA_ARCH__
    return __double2float_rn(x);
#else
    return static_cast<float>(x);
#endif
  }
  const uint64_t rounded = mag + 0x0fffffffull + ((mag >> 29) & 1ull);  // ties to even at bit 29
  const uint32_t out = static_cast<uint32_t>((rounded >> 29) - (uint64_t{896} << 23)) |
                       static_cast<uint32_t>((bits >> 32) & 0x80000000u);
#ifdef __CUDA_ARCH__
  return __uint_as_float(out);
#else
  float f;
  std::memcpy(&f, &out, sizeof f);
  return f;
#endif
}

struct alignas(32) LogEntry {
  double f, inv_f, ln_hi, ln_lo;  // 32 bytes: one sector
};

static __device__ const LogEntry kLogTableDevice[] = {GAPS_LOG_TABLE};
static const LogEntry kLogTableHost[] = {GAPS_LOG_TABLE};

__host__ __device__ __forceinline__ double log_fp64(double x) {
#ifdef __CUDA_ARCH__
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t bits;
  std::memcpy(&bits, &x, sizeof bits);
#endif
  // positive normal x (tested on the bits: the FP64 pipe's compares cost as
  // much as its FMAs on this part)
  if (bits - 0x0010000000000000ull >= 0x7fe0000000000000ull) return log(x);
  constexpr uint64_t kFrac = (uint64_t{1} << 52) - 1;
  constexpr uint64_t kSqrt2Frac = 0x6a09e667f3bcdull;  // fraction bits of sqrt(2)
  const uint64_t frac = bits & kFrac;
  int e = static_cast<int>(bits >> 52) - 1023;
  uint64_t mbits;
  int j;
  if (frac >= kSqrt2Frac) {
    // m = 1.frac / 2 in [sqrt(1/2), 1): 128 m = 64 + frac / 2^46
    e += 1;
    mbits = frac | (uint64_t{1022} << 52);
    j = 64 + static_cast<int>((frac + (uint64_t{1} << 45)) >> 46);
  } else {
    // m = 1.frac in [1, sqrt(2)): 128 m = 128 + frac / 2^45
    mbits = frac | (uint64_t{1023} << 52);
    j = 128 + static_cast<int>((frac + (uint64_t{1} << 44)) >> 45);
  }
#ifdef __CUDA_ARCH__
  const double m = __longlong_as_double(static_cast<long long>(mbits));
  const LogEntry* t = &kLogTableDevice[j - GAPS_LOG_J_FIRST];
  const double big_f = __ldg(&t->f), inv_f = __ldg(&t->inv_f), ln_hi = __ldg(&t->ln_hi), ln_lo = __ldg(&t->ln_lo);
#else
  double m;
  std::memcpy(&m, &mbits, sizeof m);
  const LogEntry& t = kLogTableHost[j - GAPS_LOG_J_FIRST];
  const double big_f = t.f, inv_f = t.inv_f, ln_hi = t.ln_hi, ln_lo = t.ln_lo;
#endif
  const double f = m - big_f;  // exact
  const double r = f * inv_f;
  // ln(1 + r) = r + r^2 q(r), q(r) = -1/2 + r/3 - r^2/4 + r^3/5 - r^4/6 + r^5/7
  double q = fma(1.0 / 7.0, r, -1.0 / 6.0);
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -1.0 / 4.0);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double r2 = r * r;
  double ed = 0.0;  // (double) e, from its bits (|e| < 2^11, exact)
  if (e != 0) {
    const uint32_t a = static_cast<uint32_t>(e < 0 ? -e : e);
#ifdef __CUDA_ARCH__
    const int top = 31 - __clz(static_cast<int>(a));
#else
    const int top = 31 - __builtin_clz(a);
#endif
    const uint64_t ebits = (static_cast<uint64_t>(e < 0) << 63) | (static_cast<uint64_t>(top + 1023) << 52) |
                           ((static_cast<uint64_t>(a) << (52 - top)) & ((uint64_t{1} << 52) - 1));
#ifdef __CUDA_ARCH__
    ed = __longlong_as_double(static_cast<long long>(ebits));
#else
    std::memcpy(&ed, &ebits, sizeof ed);
#endif
  }
  const double hi = fma(ed, GAPS_LOG_LN2_HI, ln_hi);  // exact
  // the small parts first, r (the largest of them, unrounded) next, hi last
  const double small = fma(r2, q, fma(ed, GAPS_LOG_LN2_LO, ln_lo));
  return hi + fma(f, inv_f, small);
}

}  // namespace gaps
