// Error-free splitting of FP64 values into 8-bit slices and exact recombination (Ozaki scheme:
// Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012)).
//
// A row of FP64 values x_k (|x_k| < 2^(E-1022), E = the row's largest biased exponent) is
// written as x_k = 2^(E-1022-56) * X_k, X_k a signed 56-bit integer (truncated: error below
// 2^-56 of the row's scale), and X_k = sum_p d_pk 2^(48-8p), p = 0..6, with signed digits
// |d_pk| <= 255.  Digits are exact in FP16 and BF16, products of two digits are exact, and sums
// of up to 7 x 32 such products stay below 2^24, so a tensor core with FP32 accumulation
// computes every diagonal D_t = sum_{p+q=t} sum_k d_pk e_qk exactly.  The dot product is then
// 2^(Ea+Eb-2044-64) * sum_{t<=6} D_t 2^(8(6-t)) (terms with p+q > 6 are below 2^-56 of the
// scales and dropped), recombined in integers and rounded once to FP64.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace qec {
namespace oz {

constexpr int kSlices = 7;
constexpr int kPart = 16;   // reals (inputs) and outputs of one row that one thread of a pass holds

OZ_HD uint64_t d2u(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}

OZ_HD double u2d(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

OZ_HD uint32_t f2u(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}

OZ_HD float u2f(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}

// Biased exponent field of x (0 for zero and subnormals).
OZ_HD int bexp(double x) { return (int)((d2u(x) >> 52) & 0x7FF); }

// BF16 bit pattern of the signed integer d, |d| <= 255 (exact).
OZ_HD uint16_t bf16_of_int(int d) {
  if (d == 0) return 0;
  const uint32_t a = (uint32_t)(d < 0 ? -d : d);
  const float f = u2f(0x4B000000u | a) - 8388608.0f;   // exact: a < 2^23
  return (uint16_t)((f2u(f) >> 16) | (d < 0 ? 0x8000u : 0u));
}

// The 56-bit magnitude X of x relative to the row exponent E: x = 2^(E-1022-56) * (-1)^s * X.
OZ_HD uint64_t mag56(double x, int E) {
  const uint64_t u = d2u(x);
  const int ex = (int)((u >> 52) & 0x7FF);                                    // 0: zero or subnormal
  const uint64_t m = ((u & 0xFFFFFFFFFFFFFull) | ((uint64_t)(ex != 0) << 52)) << 3;   // 56 bits
  const unsigned k = (unsigned)(E - (ex ? ex : 1));                           // >= 0 when E >= 1
#if defined(__CUDA_ARCH__)
  uint64_t X;
  asm("shr.b64 %0, %1, %2;" : "=l"(X) : "l"(m), "r"(k));                     // amounts >= 64 give 0
  return X;
#else
  return k > 63 ? 0ull : (m >> k);
#endif
}

// The 7 signed digits of x relative to the row exponent E (x == 0 or E == 0: all zero).
OZ_HD void split7(double x, int E, int* d) {
  const uint64_t X = E ? mag56(x, E) : 0ull;
  const int neg = (int)(d2u(x) >> 63);
  for (int p = 0; p < kSlices; ++p) {
    const int v = (int)((X >> (48 - 8 * p)) & 0xFF);
    d[p] = neg ? -v : v;
  }
}

// Recombination: y = 2^(Ea + Eb - 2044 - 64) * sum_t D_t 2^(8(6-t)), D_t FP32 values holding exact
// integers (|D_t| <= (t+1) * 32 * 255^2 < 2^24), formed as Z = sum_t D_t 2^(8(6-t)) / 2^10 in 64-bit
// integers (|Z| < 2^60) and rounded once to FP64.
// Exact integer of a float holding an integer of magnitude below 2^22: in [2^23, 2^24) after adding
// 1.5 * 2^23 the float's ulp is 1, so its bit pattern minus that of 1.5 * 2^23 is the integer (and a
// float below 2^22 that is not an integer is rounded to the nearest one).
OZ_HD int32_t small_float_int(float v) { return (int32_t)(f2u(v + 12582912.0f) - 0x4B400000u); }

OZ_HD float fma_f32(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// Z = H 2^30 + M 2^14 + L with three 32-bit pieces and two widening multiply-adds:
//   H = D_0 2^8 + D_1             (|H| <= 256 * 2080800 + 4161600 < 2^29),
//   M = D_2 2^8 + D_3             (|M| <= 256 * 6242400 + 8323200 < 2^31),
//   L = D_4 2^6 + round(D_5 / 4 + D_6 / 1024)   (|L| < 2^30).
// D_0 and D_1 are below 2^22 and converted by the magic number.  The two lowest diagonals' share
// D_5 / 4 + D_6 / 1024 (below 2^22) is formed in FP32 with one rounding (error below 1/8) and
// rounded to an integer: within 1 unit of the exact quotient.
OZ_HD int64_t combine7(const float* D) {
  const int32_t H = small_float_int(D[0]) * 256 + small_float_int(D[1]);
  const int32_t M = (int32_t)D[2] * 256 + (int32_t)D[3];
  const int32_t L = (int32_t)D[4] * 64 + small_float_int(fma_f32(D[6], 0x1p-10f, D[5] * 0.25f));
  return (int64_t)H * (1 << 30) + ((int64_t)M * (1 << 14) + (int64_t)L);
}

OZ_HD double assemble7(const float* D, int Ea, int Eb) {
  if (Ea == 0 || Eb == 0) return 0.0;
  const int64_t Z = combine7(D);
  if (Z == 0) return 0.0;
  const uint64_t neg = Z < 0 ? 1ull : 0ull;
  const uint64_t mag = neg ? (uint64_t)(-Z) : (uint64_t)Z;
#if defined(__CUDA_ARCH__)
  int lead = 63 - __clzll((long long)mag);
#else
  int lead = 63 - __builtin_clzll(mag);
#endif
  uint64_t mant;
  if (lead <= 52) {
    mant = mag << (52 - lead);
  } else {
    const int s = lead - 52;
    mant = (mag + (1ull << (s - 1))) >> s;
    if (mant >> 53) {
      mant >>= 1;
      ++lead;
    }
  }
  const int be = lead + Ea + Eb - 2098 + 1023;       // value = mag * 2^(Ea + Eb - 2098)
  if (be <= 0) return neg ? -0.0 : 0.0;              // below the normal range: flush
  if (be >= 2047) return u2d((neg << 63) | 0x7FF0000000000000ull);
  return u2d((neg << 63) | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// The same value through one int64 -> FP64 conversion (round to nearest even) and an exact
// power-of-two scaling of the exponent field: fewer integer operations, one conversion.
// v * 2^s for a finite v by its exponent field (flush to zero below the normal range).
OZ_HD double scale2(double v, int s) {
  const uint64_t u = d2u(v);
  const int be = (int)((u >> 52) & 0x7FF) + s;
  if ((u << 1) == 0 || be <= 0) return 0.0;   // zero test on the bits: no FP64 comparison
  if (be >= 2047) return u2d((u & 0x8000000000000000ull) | 0x7FF0000000000000ull);
  return u2d(u + ((uint64_t)(int64_t)s << 52));
}

OZ_HD double assemble7_cvt(const float* D, int Ea, int Eb) {
  if (Ea == 0 || Eb == 0) return 0.0;
  const int64_t Z = combine7(D);
  return scale2((double)Z, Ea + Eb - 2098);          // one rounding (the conversion), exact scaling
}

// assemble7_cvt when the caller has checked that Z * 2^(Ea + Eb - 2098) stays in the normal range
// for any Z with |Z| < 2^60 (Ea + Eb >= 1076 and Ea + Eb <= 2980) or that Eb = 0 gives Z = 0.
OZ_HD double assemble7_cvt_inrange(const float* D, int Ea, int Eb) {
  const int64_t Z = combine7(D);
  return Z ? u2d(d2u((double)Z) + ((uint64_t)(int64_t)(Ea + Eb - 2098) << 52)) : 0.0;
}

// The bounded probability pass keeps 3 slices of each operand (the top 24 of the 56 bits) and every
// product of them: Z = sum_{t<=4} D_t 2^(8(4-t)) exactly, y^ = Z 2^(Ea + Eb - 2092).  Diagonal t holds
// 1, 2, 3, 2, 1 slice products, so D_0, D_1, D_3 and D_4 are below 2^22 (magic-number conversion)
// and D_2 below 3 * 2^21: Z = H 2^24 + M 2^8 + D_4 with H = D_0 2^8 + D_1 (< 2^29) and
// M = D_2 2^8 + D_3 (< 2^31), |Z| < 2^54.
OZ_HD int64_t combine5(const float* D) {
  const int32_t H = small_float_int(D[0]) * 256 + small_float_int(D[1]);
  const int32_t M = (int32_t)D[2] * 256 + small_float_int(D[3]);
  return (int64_t)H * (1 << 24) + ((int64_t)M * 256 + (int64_t)small_float_int(D[4]));
}

// The fused pass's probability inputs: the top 24 bits of |x|'s significand (implicit bit included)
// aligned to the tile's largest biased exponent Et (>= 24, so that zero and subnormal x give 0):
// |x| = 2^(Et - 1046) (a + rho) with a < 2^24 and 0 <= rho < 1.  Its 3 digits are its bytes 2, 1, 0.
OZ_HD uint32_t top24(uint64_t u, int Et) {
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
#if defined(__CUDA_ARCH__)
  const uint32_t m24 = __funnelshift_l(lo, mh, 3);
#else
  const uint32_t m24 = (mh << 3) | (lo >> 29);
#endif
  const int k = Et - ex;
  return m24 >> (k < 31 ? k : 31);
}

// The fused pass's probability recombination keeps 3 slices of each operand (24-bit integers a and
// b) and only the diagonals t <= 2: Zt = round((D_0 2^32 + D_1 2^24 + D_2 2^16) / 2^24)
// = D_0 2^8 + D_1 + round(D_2 / 2^8).  D_0 < 2^21 and D_1 < 2^22 convert exactly by the magic number,
// D_2 / 2^8 (< 2^15, exact in FP32) is rounded to nearest; |Zt| < 2^29.  Against the exact product a b
// / 2^24 it is off by the dropped diagonals 3 and 4 (below 32 * 255^2 * 513 < 2^30 units of 2^-24) and
// the rounding (1/2).
OZ_HD int32_t combine3(const float* D) {
  return small_float_int(D[0]) * 256 + small_float_int(D[1]) + small_float_int(D[2] * 0x1p-8f);
}

// ---- FP32 with directed rounding (the device's IEEE intrinsics; on the host an emulation through
// FP64 that the CPU tests use: FP32 products are exact in FP64, sums are checked against the FP64
// result) -------------------------------------------------------------------------------------------
#if defined(__CUDA_ARCH__)
OZ_HD float f_add_rd(float a, float b) { return __fadd_rd(a, b); }
OZ_HD float f_add_ru(float a, float b) { return __fadd_ru(a, b); }
OZ_HD float f_mul_rd(float a, float b) { return __fmul_rd(a, b); }
OZ_HD float f_mul_ru(float a, float b) { return __fmul_ru(a, b); }
OZ_HD float f_fma_rd(float a, float b, float c) { return __fmaf_rd(a, b, c); }
OZ_HD float f_fma_ru(float a, float b, float c) { return __fmaf_ru(a, b, c); }
OZ_HD float f_sqrt_ru(float a) { return __fsqrt_ru(a); }
OZ_HD float u2f_rd(uint32_t v) { return __uint2float_rd(v); }
OZ_HD float u2f_ru(uint32_t v) { return __uint2float_ru(v); }
#else
inline float f_down(double r) { float f = (float)r; return (double)f > r ? nextafterf(f, -INFINITY) : f; }
inline float f_up(double r) { float f = (float)r; return (double)f < r ? nextafterf(f, INFINITY) : f; }
inline float f_add_rd(float a, float b) { return f_down((double)a + (double)b); }
inline float f_add_ru(float a, float b) { return f_up((double)a + (double)b); }
inline float f_mul_rd(float a, float b) { return f_down((double)a * (double)b); }
inline float f_mul_ru(float a, float b) { return f_up((double)a * (double)b); }
inline float f_fma_rd(float a, float b, float c) { return f_down((double)a * (double)b + (double)c); }
inline float f_fma_ru(float a, float b, float c) { return f_up((double)a * (double)b + (double)c); }
inline float f_sqrt_ru(float a) { float f = sqrtf(a); return (double)f * (double)f < (double)a ? nextafterf(f, INFINITY) : f; }
inline float u2f_rd(uint32_t v) { return f_down((double)v); }
inline float u2f_ru(uint32_t v) { return f_up((double)v); }
#endif

// Per-thread sums of the fused pass's probability phase over its tiles, in units of 2^-64, as FP32
// intervals with directed rounding (no FP64 work per tile).  Per tile the thread adds
//   N_t = nacc 2^(2 Et - 2092)   (nacc = sum of its 16 inputs' squared 24-bit integers, < 2^52),
//   A_t = aacc 2^(2 (Et + EP) - 4136)   (aacc = sum of its 16 outputs' squared Zt, < 2^62),
// and their truncation bounds 8 d sqrt(N_t) + 16 d^2 with d = 2^(Et - 1045) (inputs off by less than
// 2^(Et - 1046) each) and 8 D sqrt(A_t) + 16 D^2 with D = 2^(Et + EP - 2060) (outputs), which in the
// same units are 16 s_N (sqrt(nacc) + 4) and 2^11 s_A (sqrt(aacc) + 512) with s_N = 2^(2 Et - 2028),
// s_A = 2^(2 (Et + EP) - 4072).  Scales below the FP32 normal range (tiles whose squares are below
// about 2^-138) count as 0 in the lower sums and as 2^-126 in the upper ones.
// SqSum24 is one sum of the N kind (the speculative pass keeps two: its inputs under their group's
// exponent and its outputs under the tile's); FusedSums adds the A kind beside it.
struct SqSum24 {
  float lo = 0.f, hi = 0.f, e = 0.f;
  OZ_HD void add(uint64_t nacc, int Et) {
    const int kN = 2 * Et - 2028;
    const float sN = kN >= -126 ? u2f(uint32_t(kN + 127) << 23) : 0.f;
    const float sNh = kN >= -126 ? sN : 0x1p-126f;
    const uint32_t nh = (uint32_t)(nacc >> 32), nl = (uint32_t)nacc;   // nh < 2^20: exact in FP32
    const float n_lo = f_fma_rd((float)nh, 4294967296.f, u2f_rd(nl)), n_hi = f_fma_ru((float)nh, 4294967296.f, u2f_ru(nl));
    lo = f_add_rd(lo, f_mul_rd(n_lo, sN));
    hi = f_add_ru(hi, f_mul_ru(n_hi, sNh));
    e = f_add_ru(e, f_mul_ru(f_add_ru(f_sqrt_ru(n_hi), 4.f), f_mul_ru(16.f, sNh)));
  }
  // Midpoint and radius in real units: the sum lies in [n - rn, n + rn].
  OZ_HD void finish(double& n, double& rn) const {
    const double u = 0x1p-64;
    n = 0.5 * ((double)lo + (double)hi) * u;
    rn = (0.5 * ((double)hi - (double)lo) + (double)e) * u;
  }
};

struct FusedSums {
  SqSum24 n;
  float alo = 0.f, ahi = 0.f, ea = 0.f;
  OZ_HD void add_tile(uint64_t nacc, uint64_t aacc, int Et, int EP) {
    const int kA = 2 * (Et + EP) - 4072;
    const float sA = EP && kA >= -126 ? u2f(uint32_t(kA + 127) << 23) : 0.f;
    const float sAh = EP ? (kA >= -126 ? sA : 0x1p-126f) : 0.f;
    const float two32 = 4294967296.f;
    const uint32_t ah = (uint32_t)(aacc >> 32), al = (uint32_t)aacc;
    const float a_lo = f_fma_rd(u2f_rd(ah), two32, u2f_rd(al)), a_hi = f_fma_ru(u2f_ru(ah), two32, u2f_ru(al));
    n.add(nacc, Et);
    alo = f_add_rd(alo, f_mul_rd(a_lo, sA));
    ahi = f_add_ru(ahi, f_mul_ru(a_hi, sAh));
    ea = f_add_ru(ea, f_mul_ru(f_add_ru(f_sqrt_ru(a_hi), 512.f), f_mul_ru(2048.f, sAh)));
  }
  // Midpoints and radii in real units: N in [n - rn, n + rn], A in [a - ra, a + ra].
  OZ_HD void finish(double& nn, double& rn, double& a, double& ra) const {
    const double u = 0x1p-64;
    n.finish(nn, rn);
    a = 0.5 * ((double)alo + (double)ahi) * u;
    ra = (0.5 * ((double)ahi - (double)alo) + (double)ea) * u;
  }
};

// 2^e1 + 2^e2 rounded up to an FP64 value, built in the exponent and mantissa fields (no FP64
// arithmetic); at least the smallest normal number, infinity above the range.
OZ_HD double pow2_sum_up(int e1, int e2) {
  const int hi = e1 > e2 ? e1 : e2, lo = e1 > e2 ? e2 : e1;
  int be = hi + 1023;
  uint64_t mant = 1;                                  // the smaller term below one unit: round up
  if (hi == lo) {
    be += 1;
    mant = 0;
  } else if (hi - lo <= 52) {
    mant = 1ull << (52 - (hi - lo));
  }
  if (be < 1) return u2d(1ull << 52);
  if (be > 2046) return u2d(0x7FF0000000000000ull);
  return u2d(((uint64_t)be << 52) | mant);
}

// Bound on |sum_n y_n^2 - y^_n^2| over at most kPart outputs of one row, given a = sum y^_n^2 over
// them and ee = Ea + Eb.  With x = 2^(Ea-1078)(X_hi + rho), b = 2^(Eb-1078)(Y_hi + sigma), X_hi,
// Y_hi < 2^56 and the dropped parts |rho|, |sigma| < 2^32 + 1 (low 32 bits plus the truncation below
// the 56-bit integer), each output over 32 terms is off by at most
// Delta = 2^(ee-2156) * 32 * (2 * 2^56 * 2^33 + 2^66) < 2^(ee-2060); then
// sum |y^2 - y^^2| <= Delta * (2 * sum |y^| + kPart Delta) and 2 sum |y^| <= 2 sqrt(kPart a) = 8 sqrt(a)
// (Cauchy-Schwarz).  a < 2^(be-1022) for a's biased exponent be, and a is the correctly rounded
// value of the exact sum, which is then below 2^(be-1022) too, so sqrt(a) <= 2^ceil((be-1022)/2).
// Both terms are powers of two; their sum is returned, rounded up.
OZ_HD double part_bound(double a, int ee) {
  static_assert(kPart == 16, "the bound's constants are those of 16 outputs");
  const int d = ee - 2060;                            // Delta = 2^d
  const uint64_t ua = d2u(a);
  const int e1 = ua ? d + 3 + (((int)((ua >> 52) & 0x7FF) - 1021) >> 1) : -100000;   // 8 Delta sqrt(a)
  return pow2_sum_up(e1, 2 * d + 4);                  // + kPart Delta^2
}

OZ_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// (hi 2^64 + lo) * 2^s as FP64 for a 128-bit value below 2^126: normalised to 64 significant bits
// with a sticky bit for the bits below them, so that the one int -> FP64 conversion rounds it
// correctly (to nearest); 2^s is applied to the exponent field.
OZ_HD double u128_to_double(uint64_t hi, uint64_t lo, int s) {
  if (hi == 0) return scale2((double)lo, s);
  const int lz = clz64(hi);
  const uint64_t top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
  return scale2((double)(top | ((lo << lz) != 0 ? 1u : 0u)), s + 64 - lz);
}

// Exact sums of squares of up to kPart integers below 2^60 without FP64 work per term:
// v = h 2^30 + l (h, l < 2^30), v^2 = h^2 2^60 + 2 h l 2^30 + l^2, the three partial sums each
// below 16 * 2^60 = 2^64.  take() adds them exactly in 128 bits and converts once: one rounding
// (to nearest), relative error at most 2^-53.
struct SqAcc {
  uint64_t hh = 0, hl = 0, ll = 0;
  OZ_HD void add(uint64_t v) {
    const uint64_t h = v >> 30, l = v & 0x3FFFFFFFull;
    hh += h * h;
    hl += h * l;
    ll += l * l;
  }
  // sum * 2^s as FP64, then the accumulators restart
  OZ_HD double take(int s) {
    uint64_t lo = hh << 60, hi = hh >> 4;
    const uint64_t m = hl << 31;
    lo += m;
    hi += (hl >> 33) + (lo < m ? 1u : 0u);
    lo += ll;
    hi += lo < ll ? 1u : 0u;
    hh = hl = ll = 0;
    return u128_to_double(hi, lo, s);
  }
};

// The same for signed integers below 2^56 in magnitude, without taking magnitudes:
// z = h 2^30 + l with h = floor(z / 2^30) (|h| < 2^26) and 0 <= l < 2^30, so
// z^2 = h^2 2^60 + 2 h l 2^30 + l^2 with a signed middle sum below 16 * 2^56 in magnitude.
struct SqAccS {
  uint64_t hh = 0, ll = 0;
  int64_t hl = 0;
  OZ_HD void add(int64_t z) {
    const int64_t h = z >> 30, l = z & 0x3FFFFFFFll;   // arithmetic shift: floor
    hh += (uint64_t)(h * h);
    hl += h * l;
    ll += (uint64_t)(l * l);
  }
  OZ_HD double take(int s) {   // the sum is a sum of squares: its 128-bit value is not negative
    uint64_t lo = hh << 60, hi = hh >> 4;
    const uint64_t m = (uint64_t)hl << 31;
    lo += m;
    hi += (uint64_t)(hl >> 33) + (lo < m ? 1u : 0u);
    lo += ll;
    hi += lo < ll ? 1u : 0u;
    hh = ll = 0;
    hl = 0;
    return u128_to_double(hi, lo, s);
  }
};

}  // namespace oz
}  // namespace qec
