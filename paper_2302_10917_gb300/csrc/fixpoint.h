// Fixed-point helpers shared by the fixed-point trace apply and the
// fixed-point Krylov basis: FP64 values of one set (a block row, a trace
// vector, a chunk of a basis vector) held as signed 56-bit integers at the
// common scale 2^(1077 - Eb), Eb the largest biased FP64 exponent of the set,
// split into a low 28-bit limb and a signed high limb; products of two such
// numbers summed exactly in 64-bit integers and rounded once to FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mehdg {

constexpr int FIX_LO_BITS = 28;

// v as a fixed-point number at scale 2^(1077 - Eb), where Eb (>= 1) is the
// largest biased exponent of the set v belongs to: |result| <= 2^55, rounded to
// nearest (ties away from zero) on the magnitude. Integer operations only.
__device__ __forceinline__ int2 fix_limbs(unsigned long long bits, int Eb) {
  int eb = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (eb == 0) eb = 1;
  else m |= 1ull << 52;
  const int sh = eb - Eb + 2;   // <= 2 since eb <= Eb
  unsigned long long a;
  if (sh >= 0) {
    a = m << sh;
  } else {
    const int r = -sh;
    a = r > 54 ? 0ull : (m + (1ull << (r - 1))) >> r;
  }
  const long long v = (bits >> 63) ? -(long long)a : (long long)a;
  return make_int2((int)(v & ((1ll << FIX_LO_BITS) - 1)), (int)(v >> FIX_LO_BITS));
}

__device__ __forceinline__ int fix_exp_field(unsigned long long bits) {
  const int eb = (int)((bits >> 52) & 0x7ff);
  return eb == 0 ? 1 : eb;
}

// the exact sum hh 2^56 + (m0 + m1) 2^28 + ll of the limb products
__device__ __forceinline__ __int128 fix_sum128(long long hh, long long m0, long long m1, unsigned long long ll) {
  return ((__int128)hh << 56) + (((__int128)m0 + (__int128)m1) << 28) + (__int128)ll;
}

// t 2^e2 rounded once to FP64 (to nearest, ties to even) with integer operations
// only: normalise the magnitude, keep 64 bits with a sticky bit for the rest,
// round at bit 11 and assemble sign, exponent and significand. Results outside
// the normal range take a slower exact path.
__device__ __forceinline__ double fix_round(__int128 t, int e2) {
  const bool neg = t < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
  if (a == 0) return 0.0;
  const unsigned long long ahi = (unsigned long long)(a >> 64), alo = (unsigned long long)a;
  const int lz = ahi ? __clzll(ahi) : 64 + __clzll(alo);
  const unsigned __int128 nrm = a << lz;                   // leading one at bit 127
  unsigned long long top = (unsigned long long)(nrm >> 64);
  if ((unsigned long long)nrm != 0ull) top |= 1ull;        // sticky
  int E = e2 + 127 - lz;                                    // exponent of the leading one
  unsigned long long mant = top >> 11;                      // 53 bits
  const unsigned long long rem = top & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++E;
    }
  }
  const int B = E + 1023;
  if (B <= 0 || B >= 2047) {
    const double r = scalbn(__ull2double_rn(top), E - 63);
    return neg ? -r : r;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)B << 52) |
                                  (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// (hh 2^56 + (m0 + m1) 2^28 + ll) 2^(Er + Ex - 2154), rounded once to FP64: the
// exact sum of limb products of two fixed-point sets with scales Er and Ex.
// NaN when either scale comes from a non-finite input.
__device__ __forceinline__ double fix_result(long long hh, long long m0, long long m1, unsigned long long ll, int Er,
                                             int Ex) {
  if (Er == 2047 || Ex == 2047) return __longlong_as_double(0x7FF8000000000000ll);   // Inf or NaN input
  return fix_round(fix_sum128(hh, m0, m1, ll), Er + Ex - 2154);
}

// v 2^k for a finite v, by exponent arithmetic when the result stays normal
__device__ __forceinline__ double fix_ldexp(double v, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((b >> 52) & 0x7ff);
  if (eb == 0 || eb == 2047 || eb + k <= 0 || eb + k >= 2047) return scalbn(v, k);
  return __longlong_as_double((long long)(b + ((unsigned long long)(long long)k << 52)));
}

// exact limb products of one pair of fixed-point numbers into the four sums
__device__ __forceinline__ void fix_mac(long long& hh, long long& m0, long long& m1, unsigned long long& ll, int2 a,
                                        int2 b) {
  hh += (long long)a.y * b.y;
  m0 += (long long)a.y * b.x;
  m1 += (long long)a.x * b.y;
  ll += (unsigned long long)(unsigned)a.x * (unsigned)b.x;
}

}  // namespace mehdg
