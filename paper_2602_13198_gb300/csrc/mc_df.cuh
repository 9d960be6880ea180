// mc_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2), which carries a 48-bit significand on the FP32 pipes.  GB300 issues FP32 at
// ~74x its FP64 rate, so the mixed-precision transport keeps the geodesic at near-FP64 accuracy
// (~1e-14 relative) in this form instead of in FP64.
//
// Error-free transformations: two-sum (Knuth, TAOCP vol. 2, 4.2.2), the fast two-sum for |a| >= |b|
// (Dekker 1971), and the FMA form of the exact product (a b = p + e with e = fma(a, b, -p)).  The
// addition is Dekker's: two-sum of the high parts, the low parts added into its error term, one
// renormalisation (11 FP32 operations).  Its error is bounded normwise, by a few 2^-48 (|a| + |b|),
// the size of the error the operands already carry, so a cancellation loses no more than they hold.
// The product adds the cross terms to the exact product of the high parts.  The exponent range is
// FP32's.
#pragma once
#include <cuda_runtime.h>

namespace mcgb {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// by an FP32 number (exact constants such as 2 or 0.5 and FP32 data)
__device__ __forceinline__ df operator*(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df operator*(float b, df a) { return a * b; }

__device__ __forceinline__ df operator+(df a, float b) {
  df s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df operator+(float b, df a) { return a + b; }
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }
__device__ __forceinline__ df operator-(float b, df a) { return (-a) + b; }

__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }

// 1 / a: FP32 reciprocal refined by one Newton step in double-float (error ~2^-47)
__device__ __forceinline__ df df_rcp(df a) {
  const float q0 = __frcp_rn(a.hi);
  const df r = 1.0f - a * q0;   // residual 1 - a q0, of order 2^-24
  return df_fast_two_sum(q0, __fmul_rn(q0, r.hi));
}

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.0f ? -a : a; }

// conversions: split a double into its nearest FP32 and the FP32 remainder; join exactly
__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

// Compile-time split of a double constant (for constants that are not FP32 numbers, like pi)
__host__ __device__ constexpr df df_const(double x) {
  return {(float)x, (float)(x - (double)(float)x)};
}

// ---- scalar-generic helpers: the geodesic code is written once for S = double (plain FP64) and
// S = df (mixed precision); for double every helper is the identity or the plain operation.
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(df x) { return df_to(x); }
// FP64 -> FP32 on the integer pipes, truncating (within one FP32 ulp): sign, exponent re-biased by
// 1023 - 127 and the top 23 mantissa bits.  Zeros keep their sign; values beyond the FP32 normal range,
// infinities and NaN take the conversion instruction.  For the split precision form, whose FP32
// coefficient arithmetic reads the FP64 geodesic state: conversions take FP64-pipe slots on GB300.
__device__ __forceinline__ float narrow_f(double d) {
  const long long b = __double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  if (e > 0 && e < 255) return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29));
  if ((b & 0x7fffffffffffffffLL) == 0) return __uint_as_float(hi & 0x80000000u);
  return (float)d;
}
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(df x) { return __fadd_rn(x.hi, x.lo); }
// a geodesic scalar in FP32 without an FP64-pipe conversion: narrowed on the integer pipes, or hi + lo
__device__ __forceinline__ float step_f(double x) { return narrow_f(x); }
__device__ __forceinline__ float step_f(df x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ double sabs(double x) { return fabs(x); }
__device__ __forceinline__ df sabs(df x) { return df_abs(x); }
__device__ __forceinline__ double srcp(double x) { return 1.0 / x; }
__device__ __forceinline__ df srcp(df x) { return df_rcp(x); }
// ordering of normalised double-float values
__device__ __forceinline__ bool df_ge(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// a model constant held in both forms: the double for S = double, its df split for S = df
template <typename S> __device__ __forceinline__ S pick(double d, df f);
template <> __device__ __forceinline__ double pick<double>(double d, df) { return d; }
template <> __device__ __forceinline__ df pick<df>(double, df f) { return f; }
// a compile-time constant
template <typename S> __host__ __device__ constexpr S cst(double x);
template <> __host__ __device__ constexpr double cst<double>(double x) { return x; }
template <> __host__ __device__ constexpr df cst<df>(double x) { return df_const(x); }

// Sums of products a0 b0 + a1 b1 + ... in one pass.  Each high-part product is split exactly (FMA),
// the high parts are summed with two-sum, and every error term (product errors, cross terms, sum
// errors) collects in one FP32 accumulator; a single renormalisation closes the sum.  Per term 12
// FP32 operations, where a product and a Dekker sum take 18; the error is bounded normwise like the
// sum's, by a few 2^-48 sum |a_i b_i|.
struct DotAcc {
  float s, e;
};
__device__ __forceinline__ DotAcc dot_first(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ void dot_add(DotAcc &d, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df t = df_two_sum(d.s, p);
  d.s = t.hi;
  d.e = __fadd_rn(d.e, __fadd_rn(t.lo, e));
}
__device__ __forceinline__ void dot_add(DotAcc &d, df x) {   // a term that is already a df value
  const df t = df_two_sum(d.s, x.hi);
  d.s = t.hi;
  d.e = __fadd_rn(d.e, __fadd_rn(t.lo, x.lo));
}
__device__ __forceinline__ df dot_end(DotAcc d) { return df_fast_two_sum(d.s, d.e); }
// x / 2, exact (barring underflow)
__device__ __forceinline__ df df_half(df x) { return {__fmul_rn(x.hi, 0.5f), __fmul_rn(x.lo, 0.5f)}; }

// The scalar-generic forms: for double the plain expression as written (so the FP64 path keeps its
// arithmetic), for df the one-pass accumulation.
__device__ __forceinline__ double sdot(double a0, double b0, double a1, double b1) { return a0 * b0 + a1 * b1; }
__device__ __forceinline__ double sdot(double a0, double b0, double a1, double b1, double a2, double b2) {
  return a0 * b0 + a1 * b1 + a2 * b2;
}
__device__ __forceinline__ double sdot(double a0, double b0, double a1, double b1, double a2, double b2, double a3,
                                       double b3) {
  return a0 * b0 + a1 * b1 + a2 * b2 + a3 * b3;
}
// a0 b0 + a1 b1 - c / 2 and a0 b0 - c / 2
__device__ __forceinline__ double sdot_mh(double a0, double b0, double a1, double b1, double c) {
  return a0 * b0 + a1 * b1 - 0.5f * c;
}
__device__ __forceinline__ double sdot_mh(double a0, double b0, double c) { return a0 * b0 - 0.5f * c; }
__device__ __forceinline__ df sdot(df a0, df b0, df a1, df b1) {
  DotAcc d = dot_first(a0, b0);
  dot_add(d, a1, b1);
  return dot_end(d);
}
__device__ __forceinline__ df sdot(df a0, df b0, df a1, df b1, df a2, df b2) {
  DotAcc d = dot_first(a0, b0);
  dot_add(d, a1, b1);
  dot_add(d, a2, b2);
  return dot_end(d);
}
__device__ __forceinline__ df sdot(df a0, df b0, df a1, df b1, df a2, df b2, df a3, df b3) {
  DotAcc d = dot_first(a0, b0);
  dot_add(d, a1, b1);
  dot_add(d, a2, b2);
  dot_add(d, a3, b3);
  return dot_end(d);
}
__device__ __forceinline__ df sdot_mh(df a0, df b0, df a1, df b1, df c) {
  DotAcc d = dot_first(a0, b0);
  dot_add(d, a1, b1);
  dot_add(d, -df_half(c));
  return dot_end(d);
}
__device__ __forceinline__ df sdot_mh(df a0, df b0, df c) {
  DotAcc d = dot_first(a0, b0);
  dot_add(d, -df_half(c));
  return dot_end(d);
}

// Velocity-Verlet updates x + k dl + a dl^2 / 2, k + a dl and k + (a + a') dl / 2, as sums of
// products for df
__device__ __forceinline__ double verlet_x(double x, double k, double a, double dl) {
  return x + k * dl + 0.5f * a * dl * dl;
}
__device__ __forceinline__ double verlet_k(double k, double a, double dl) { return k + a * dl; }
__device__ __forceinline__ double verlet_k2(double k, double a, double a1, double dl) {
  return k + 0.5f * (a + a1) * dl;
}
__device__ __forceinline__ df verlet_x(df x, df k, df a, df dl) {
  DotAcc d{x.hi, x.lo};
  dot_add(d, k, dl);
  dot_add(d, df_half(a) * dl, dl);
  return dot_end(d);
}
__device__ __forceinline__ df verlet_k(df k, df a, df dl) {
  DotAcc d{k.hi, k.lo};
  dot_add(d, a, dl);
  return dot_end(d);
}
__device__ __forceinline__ df verlet_k2(df k, df a, df a1, df dl) {
  DotAcc d{k.hi, k.lo};
  dot_add(d, df_half(a + a1), dl);
  return dot_end(d);
}

template <typename S> __device__ __forceinline__ S from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ df from_d<df>(double x) { return df_from(x); }
// Terms of the Verlet convergence test sum |k_new - k_old| < tol sum |k_new|: FP64 for double, FP32 for
// df (the difference of two close df values is exact enough in FP32 once the high parts cancel).
__device__ __forceinline__ double vdiff(double a, double b) { return fabs(a - b); }
__device__ __forceinline__ float vdiff(df a, df b) {
  return fabsf(__fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ double vmag(double a) { return fabs(a); }
__device__ __forceinline__ float vmag(df a) { return fabsf(a.hi); }
// a, b >= 0 (sums of magnitudes): compared as bit patterns, off the FP64 pipe
__device__ __forceinline__ bool below_tol(double a, double tol, float, double b) {
  return __double_as_longlong(a) < __double_as_longlong(tol * b);
}
__device__ __forceinline__ bool below_tol(float a, double, float tolf, float b) { return a < tolf * b; }

// Nearest integer of |x| < 2^22 with FP32 additions only: adding 1.5 * 2^23 leaves the integer in the
// low mantissa bits (ties to even).  Returns it as a float and, in k, as an int; no conversion
// instruction (those share the narrow FP64 pipe on this GPU).
__device__ __forceinline__ float rint_shift(float x, int &k) {
  const float t = __fadd_rn(x, 12582912.0f);
  k = __float_as_int(t) - 0x4B400000;
  return __fsub_rn(t, 12582912.0f);
}
// Cell index of a fractional table or zone coordinate: floor in FP64; in FP32 the shifted rounding of
// f - 1/2, which at an exact integer may give the cell below with weight 1 on its upper corner (the
// same linear blend).
__device__ __forceinline__ int zone_floor(double f) { return (int)floor(f); }
__device__ __forceinline__ int zone_floor(float f) {
  int k;
  rint_shift(__fsub_rn(f, 0.5f), k);
  return k;
}
// cell index and the fraction within it, FP32 coordinates
__device__ __forceinline__ int zone_split(float f, float &frac) {
  const int k = zone_floor(f);
  frac = f - k;
  return k;
}

// 2^e for -126 <= e <= 127, from its bit pattern
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// ---- elementary functions in double-float (own range reductions and Taylor polynomials; the
// high-order terms, below 2^-24 of the leading one, in FP32).  Both use a table of double-float
// constants built on the host in FP64: entries [0, 32) hold 2^(j/32), entries [32, 96) sin(pi j/32).
constexpr int kDfTabExp = 0, kDfTabSin = 32, kDfTabN = 96;

__device__ __forceinline__ df df_tab(const df *T, int i) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(T) + i);
  return {v.x, v.y};
}

// e^x for |x| < 80: x = (32 e + j) ln2/32 + t with |t| <= ln2/64; e^x = 2^e 2^(j/32) e^t, and e^t by its
// Taylor series to t^6 (truncation below 2^-56 for |t| <= ln2/64).
__device__ __forceinline__ df df_exp(df x, const df *T) {
  constexpr df kLn2_32 = df_const(0.6931471805599453094172321 / 32.0);
  int k;
  const float kf = rint_shift(x.hi * 46.16624130844683f, k);   // 32 / ln 2
  const df t = x - kLn2_32 * kf;
  const int j = k & 31, e = (k - j) / 32;
  const float q = t.hi;
  const float tail = q * q * q * q * (1.0f / 24.0f + q * (1.0f / 120.0f + q * (1.0f / 720.0f)));
  const df t2 = t * t;
  constexpr df kSixth = df_const(1.0 / 6.0);
  df em1 = (t2 * t) * kSixth + tail;
  em1 = em1 + t2 * 0.5f;
  em1 = em1 + t;
  const df r = df_tab(T, kDfTabExp + j) * (em1 + 1.0f);
  const float p2 = exp2i(e);
  return {r.hi * p2, r.lo * p2};
}

// sin(pi x) and cos(pi x): x = j/32 + z with |z| <= 1/64, w = pi z, angle addition with the tabulated
// sin and cos of pi j/32 (cos(pi j/32) = sin(pi (j + 16)/32)); sin w and cos w by their Taylor series
// to w^7 and w^8 (truncation below 2^-57 for |w| <= pi/64).
__device__ __forceinline__ void df_sincospi(df x, const df *T, df &s, df &c) {
  constexpr df kPi = df_const(3.14159265358979323846264338);
  int j;
  const float jf = rint_shift(x.hi * 32.0f, j);
  const df z = x - jf * 0.03125f;   // exact: j/32 is an FP32 number
  const df w = z * kPi;
  const float q = w.hi, q2 = q * q;
  const df w2 = w * w;
  constexpr df kM6 = df_const(-1.0 / 6.0), k24 = df_const(1.0 / 24.0);
  // sin w = w - w^3/6 + w^5/120 - w^7/5040
  df sw = (w2 * w) * kM6 + q2 * q2 * q * (1.0f / 120.0f - q2 * (1.0f / 5040.0f));
  sw = sw + w;
  // cos w = 1 - w^2/2 + w^4/24 - w^6/720 + w^8/40320
  df cw = (w2 * w2) * k24 + q2 * q2 * q2 * (-1.0f / 720.0f + q2 * (1.0f / 40320.0f));
  cw = cw + w2 * -0.5f;
  cw = cw + 1.0f;
  const df sa = df_tab(T, kDfTabSin + (j & 63)), ca = df_tab(T, kDfTabSin + ((j + 16) & 63));
  s = sa * cw + ca * sw;
  c = ca * cw - sa * sw;
}

}  // namespace mcgb
