// Short binary64 dot products formed on the integer pipes, exactly up to one
// final rounding.
//
// GB300 issues binary64 FMAs at 2 per clock per SM (64 cycles per warp
// instruction on each sub-partition), while its integer pipes take a 32-bit
// IMAD or IADD3 every other clock per lane.  A binary64 product can be formed
// exactly enough from three 32x32 -> 64-bit integer multiplies, so kernels
// whose binary64 work would otherwise bind them can move part of it here.
//
// Representation: a binary64 v = (-1)^s M 2^(E - 1075) with the 53-bit
// significand M (hidden bit included; E the biased exponent, 1 for
// subnormals) is held as two signed limbs a = +-(M >> 22) (31 bits) and
// b = +-(M mod 2^22) (22 bits), both carrying v's sign, and e = max(E, 1):
// v = (a 2^22 + b) 2^(e - 1075) exactly.  Zero gives a = b = 0.
//
// Product: (a 2^22 + b)(c 2^22 + d) = ac 2^44 + (ad + bc) 2^22 + bd, and
// P = ac + floor((ad + bc) / 2^22) is the product divided by 2^44 with an
// error below 2 (|product| >= 2^104 for normal operands, so below 2^-59
// relative); |P| < 2^62 + 2^33.
//
// Sum: every P is aligned to the largest exponent sum Em of the dot product
// and shifted right by 3 more bits (room for eight terms in a signed 64-bit
// accumulator).  In units of 2^(Em - 2103), each aligned term is off by less
// than 1.25 (its product error / 8 plus the truncation of the shift), and the
// largest term of normal operands is at least 2^57 units: the sum of K terms
// is within 1.25 K 2^-57 of the largest |term| (below 0.6 ulp of it for
// K = 8) before to_binary64 rounds it once to nearest (ties to even).  A
// binary64 FMA chain of K terms is only bounded by K 2^-53 sum|terms|.
#pragma once

#include <stdint.h>

namespace sscg {

struct Limbs {
  int a, b, e;
};

// v (or -v with NEG, by the sign bit alone) split into limbs; `bad` collects a
// flag for Inf/NaN inputs (biased exponent 2047), which this arithmetic does
// not represent.
template <bool NEG = false>
__device__ __forceinline__ Limbs to_limbs(double v, unsigned& bad) {
  const unsigned hi = (unsigned)__double2hiint(v) ^ (NEG ? 0x80000000u : 0u), lo = (unsigned)__double2loint(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  bad |= (e + 1u) >> 11;
  const unsigned hm = (hi & 0xfffffu) | (e ? 0x100000u : 0u);
  const unsigned A = __funnelshift_l(lo, hm, 10);  // bits 52..22 of M
  const unsigned B = lo & 0x3fffffu;               // bits 21..0
  const int s = (int)hi >> 31;
  Limbs l;
  l.a = ((int)A ^ s) - s;
  l.b = ((int)B ^ s) - s;
  l.e = e ? (int)e : 1;
  return l;
}

// the product of two limb pairs divided by 2^44 (error below 2)
__device__ __forceinline__ long long limb_product(const Limbs& c, const Limbs& y) {
  long long v = (long long)c.a * y.b;
  v += (long long)c.b * y.a;
  return (long long)c.a * y.a + (v >> 22);
}

// x / 2^d toward -infinity for d >= 0 (PTX clamps shift amounts above 64 to
// 64, which leaves the sign: 0 or -1)
__device__ __forceinline__ long long shift_down(long long x, int d) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(d));
  return r;
}

// S 2^(Em - 2103) rounded to the nearest binary64 (ties to even); ok is
// cleared when the result is outside the normal range (zero excepted).
__device__ __forceinline__ double to_binary64(long long S, int Em, bool& ok) {
  if (S == 0) return 0.0;
  const unsigned long long sg = S < 0 ? 1ull : 0ull;
  unsigned long long m = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll(m);
  m <<= lz;  // leading bit at 63
  const int be = 63 - lz + Em - 1080;
  if (be <= 0 || be >= 2047) {
    ok = false;
    return 0.0;
  }
  const unsigned long long frac = (m >> 11) & 0xfffffffffffffull;
  const unsigned long long rest = m & 0x7ffull;
  const unsigned long long up = (rest > 0x400ull || (rest == 0x400ull && (frac & 1ull))) ? 1ull : 0ull;
  // a carry out of the fraction moves into the exponent field, as it should
  return __longlong_as_double((long long)((sg << 63) | (((unsigned long long)be << 52) + frac + up)));
}

// c y in units of 2^(Em - 2103), Em >= c.e + y.e the largest exponent sum of
// the dot product (truncated; see the sum bound above)
__device__ __forceinline__ long long aligned_product(const Limbs& c, const Limbs& y, int Em) {
  return shift_down(limb_product(c, y), Em - (c.e + y.e) + 3);
}


// x / 2^d rounded to nearest (ties toward +infinity), d >= 1
__device__ __forceinline__ long long shift_round(long long x, int d) { return shift_down(shift_down(x, d - 1) + 1, 1); }

// A running sum of up to 2^H products whose exponents are not known in
// advance (a long dot product streamed term by term).  The sum is held in
// units of 2^(E - 2106 + H), E the largest exponent sum seen so far: a product
// with a larger one first re-aligns the running sum, and each product is
// added at the current alignment; both roundings are to nearest.  Bound, for
// m terms of normal operands: each product is off by at most 1/2 + 2^(1-H)
// units and each re-alignment by 1/2 unit of the final alignment, while the
// largest |term| is at least 2^(60-H) units, so before the final rounding the
// sum is within m (1 + 2^(1-H)) 2^(H-60) of the largest |term| (2^-48.9 for
// m = 34, H = 6; a binary64 FMA chain is bounded by m 2^-53 sum|terms|).
// |S| stays below 2^H (2^(62-H) + 1) < 2^63.
template <int H>
struct OnlineSum {
  long long S;
  int E;
  __device__ __forceinline__ OnlineSum() : S(0), E(0) {}
  __device__ __forceinline__ void add(const Limbs& c, const Limbs& y) {
    const int Ej = c.e + y.e;
    if (Ej > E) {
      S = shift_round(S, Ej - E);
      E = Ej;
    }
    S += shift_round(limb_product(c, y), E - Ej + H);
  }
  // the sum rounded once to binary64; ok cleared outside the normal range
  __device__ __forceinline__ double result(bool& ok) const { return to_binary64(S, E + H - 3, ok); }
};

}  // namespace sscg
