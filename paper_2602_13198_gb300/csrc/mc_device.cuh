// mc_device.cuh -- device-side arithmetic of the Monte Carlo transport hot path
// (GPUmonty, arXiv 2602.13198), written for sm_103a.
//
// Everything a superphoton needs per step lives here: the Kerr-Schild metric in modified
// Kerr-Schild coordinates with closed-form first derivatives (section 2.4), the geodesic
// acceleration -Gamma^mu_ab k^a k^b contracted without forming the 40 Christoffel symbols,
// the iterated velocity-Verlet step (section 2.4), fluid interpolation and the invariant
// synchrotron / Compton coefficients (sections 2.2, 2.5-2.7), Philox4x32-10 streams keyed
// per superphoton, tetrads, and the thermal Compton kinematics (section 2.7).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "mc_df.cuh"
#include "mc_mlp.cuh"

namespace mcgb {

// ---------------------------------------------------------------- physical constants (CGS, CODATA 2018)
constexpr double kEE = 4.803204712570263e-10;
constexpr double kME = 9.1093837015e-28;
constexpr double kMP = 1.67262192369e-24;
constexpr double kCL = 2.99792458e10;
constexpr double kHPL = 6.62607015e-27;
constexpr double kSIGT = 6.6524587321e-25;
constexpr double kPI = 3.14159265358979323846;

// Hot cross-section table domain: ln Theta in [ln 1e-3, ln 1e3] (121), ln eps in [ln 1e-12, ln 1e6] (181)
constexpr int kHotNT = 121, kHotNE = 181;
constexpr double kHotLT0 = -6.907755278982137, kHotLT1 = 6.907755278982137;
constexpr double kHotLE0 = -27.631021115928547, kHotLE1 = 13.815510557964274;
// Angle-integral table: ln F on ln K in [ln 1e-10, ln 1e8], spacing 0.005
constexpr double kFLnK0 = -23.025850929940457, kFLnK1 = 18.420680743952367, kFStep = 0.005;
// K2(1/Theta) table: ln K2 on ln Theta in [ln 0.01, ln 1e4], spacing 0.002
constexpr double kK2LnT0 = -4.605170185988091, kK2LnT1 = 9.210340371976184, kK2Step = 0.002;

// ---------------------------------------------------------------- FP64 work on the integer pipes
// GB300's FP64 pipe (~1.7 lanes per SM per clock) bounds the FP64 transport kernels, and it also
// executes FP64 compares, min/max and conversions.  Where the outcome is the same bit for bit, these
// helpers do that work with integer instructions instead.
//
// Exact float -> double widening: a finite normal float's sign, exponent (re-biased by 1023 - 127)
// and mantissa are re-packed as a double; zeros keep their sign; subnormal floats (below 1.2e-38)
// take the conversion instruction.  The value is the conversion's (widening is exact).  Not for
// infinities or NaNs (grid values are checked finite when the grid is set).
__device__ __forceinline__ double widen_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t mag = u & 0x7fffffffu;
  if (mag < 0x00800000u) return mag == 0u ? __hiloint2double((int)(u & 0x80000000u), 0) : (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(u << 29));
}
// Order key of a double: keys compare as signed 64-bit integers in the order of the values
// (-0 < +0; not for NaN).  For non-negative values the key is the bit pattern itself.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// a >= b, a <= b for doubles known to be non-negative (or b negative in dle_nn: then false)
__device__ __forceinline__ bool dge_nn(double a, double b) { return __double_as_longlong(a) >= __double_as_longlong(b); }
__device__ __forceinline__ bool dle_nn(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
// max(x, 0) for any non-NaN x (a negative x has a negative bit pattern), and min / max of
// non-negative doubles
__device__ __forceinline__ double dmax0(double x) {
  const long long b = __double_as_longlong(x);
  return __longlong_as_double(b > 0 ? b : 0);
}
__device__ __forceinline__ double dmin_nn(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x < y ? x : y);
}
__device__ __forceinline__ double dmax_nn(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// ---------------------------------------------------------------- table-driven FP64 exp, log, sin/cos(pi x)
// Elementary functions for the FP64 transport after Tang's table-driven method (ACM Trans. Math.
// Softw. 15 (1989) 144, the exponential; 16 (1990) 378, the logarithm): the range reduction works on
// the integer bits of the argument and a small table, and only a short polynomial remains on the
// FP64 pipe, which bounds the FP64 transport kernels.  The tables (kFtN doubles) are built on the
// host in extended precision (ftab_host).  Measured on GB300, in FP64-pipe FMA-equivalents per call:
// exp 10.9 against 15.1 for CUDA's, log 14.8 against 28.7.  Checked against CUDA's functions by
// mc_selftest_math.
constexpr int kFtExp = 0, kFtInvC = 32, kFtLogHi = 160, kFtLogLo = 288, kFtSin = 416, kFtCos = 480, kFtN = 544;
void ftab_host(double *t);

// e^x = 2^m 2^(j/32) e^r with x = (32 m + j) ln2/32 + r, |r| <= ln2/64 (n = 32 m + j by the 1.5 * 2^52
// shift, ln2/32 split into 32 significant bits + rest for an exact reduction); e^r - 1 by its Taylor
// series to r^6 (truncation below 4e-18); 2^m added to the exponent bits.  Arguments outside
// (-708, 708) (results near or beyond the FP64 range, and NaN) take CUDA's exp.
__device__ __forceinline__ double exp_t(const double *T, double x) {
  if (!((__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x4086200000000000LL)) return exp(x);   // |x| < 708
  const double sh = 6755399441055744.0;
  const double t = fma(x, 46.166241308446828, sh);   // 32 / ln2
  const int n = __double2loint(t);
  const double nd = t - sh;
  double r = fma(nd, -0.021660849386535119, x);
  r = fma(nd, -5.9631716539705866e-12, r);
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double pm1 = fma(q, r * r, r);
  const double tj = __ldg(T + kFtExp + (n & 31));
  const double y = fma(tj, pm1, tj);
  return __hiloint2double(__double2hiint(y) + ((n >> 5) << 20), __double2loint(y));
}

// e^x - 1: for |x| < 1/4 its Taylor series to x^12 (truncation below 1e-17 relative), by Horner in
// FP64; otherwise e^x - 1 from exp_t, where the subtraction costs at most ~2.2 bits (e^x / |e^x - 1|
// < 4.5 for |x| >= 1/4).  Outside (-708, 708) exp_t takes CUDA's exp, which gives -1 and +inf at the
// ends as expm1 does.
__device__ __forceinline__ double expm1_t(const double *T, double x) {
  if ((__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x3FD0000000000000LL) {   // |x| < 1/4 (NaN fails)
    double q = fma(x, 1.0 / 479001600.0, 1.0 / 39916800.0);   // 1/12!, 1/11!
    q = fma(q, x, 1.0 / 3628800.0);
    q = fma(q, x, 1.0 / 362880.0);
    q = fma(q, x, 1.0 / 40320.0);
    q = fma(q, x, 1.0 / 5040.0);
    q = fma(q, x, 1.0 / 720.0);
    q = fma(q, x, 1.0 / 120.0);
    q = fma(q, x, 1.0 / 24.0);
    q = fma(q, x, 1.0 / 6.0);
    q = fma(q, x, 0.5);
    return fma(q, x * x, x);
  }
  return exp_t(T, x) - 1.0;
}

// log x = e ln2 + log c + log(1 + r): x = 2^e m, m in [1, 2), c = 1 + j/128 from the top 7 mantissa bits
// (so m - c is exact), r = (m - c)/c with 1/c from the table, log(1 + r) by its series to r^9
// (|r| < 1/128).  Accurate to ~1 ulp away from x = 1 and to ~2e-16 absolute near it.  Non-positive,
// subnormal, infinite and NaN arguments take CUDA's log.
__device__ __forceinline__ double log_t(const double *T, double x) {
  const long long b = __double_as_longlong(x);
  if (!(b >= 0x0010000000000000LL && b < 0x7FF0000000000000LL)) return log(x);
  const int hi = (int)(b >> 32);
  const int e = (hi >> 20) - 1023;
  const int j = (hi >> 13) & 127;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, (int)b);
  const double c = __hiloint2double(0x3ff00000 | (j << 13), 0);
  const double r = (m - c) * __ldg(T + kFtInvC + j);
  double q = fma(r, 1.0 / 9.0, -1.0 / 8.0);
  q = fma(q, r, 1.0 / 7.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double l1p = fma(q, r * r, r);
  const double ed = __hiloint2double(0x43300000, (int)(0x80000000u + (unsigned)e)) - 4503601774854144.0;   // (double)e
  const double kLn2Hi = 0.69314718055920821, kLn2Lo = 7.3710025651677989e-13;   // ln2: 40 significant bits + rest
  return fma(ed, kLn2Hi, __ldg(T + kFtLogHi + j)) + (l1p + fma(ed, kLn2Lo, __ldg(T + kFtLogLo + j)));
}

// sin(pi x), cos(pi x): x = n/32 + r exactly (|r| <= 1/64, n by the 1.5 * 2^52 shift), the angle-addition
// formula with sin, cos(pi j/32) from the table (j = n mod 64) and the Taylor series of sin, cos(pi r)
// (|pi r| <= pi/64, truncation below 3e-20).
__device__ __forceinline__ void sincospi_t(const double *T, double x, double &s, double &c) {
  const double sh = 6755399441055744.0;
  const double t = fma(x, 32.0, sh);
  const int j = __double2loint(t) & 63;
  const double r = fma(t - sh, -0.03125, x);
  const double a = r * 3.141592653589793, a2 = a * a;
  double ps = fma(a2, 1.0 / 362880.0, -1.0 / 5040.0);
  ps = fma(ps, a2, 1.0 / 120.0);
  ps = fma(ps, a2, -1.0 / 6.0);
  const double sa = fma(a * a2, ps, a);
  double pc = fma(a2, 1.0 / 40320.0, -1.0 / 720.0);
  pc = fma(pc, a2, 1.0 / 24.0);
  pc = fma(pc, a2, -0.5);
  const double ca = fma(a2, pc, 1.0);
  const double sj = __ldg(T + kFtSin + j), cj = __ldg(T + kFtCos + j);
  s = fma(sj, ca, cj * sa);
  c = fma(cj, ca, -(sj * sa));
}

// floor(f) and f - floor(f) of an FP64 index coordinate.  For 0 <= f < 2^30 the integer part is cut from
// the mantissa bits (exact), leaving one FP64 subtraction for the fraction instead of a floor, two
// conversions and a subtraction on the FP64 pipe; other arguments take floor().
__device__ __forceinline__ int floor_frac(double f, double &frac) {
  const long long b = __double_as_longlong(f);
  const int e = (int)(b >> 52) - 1023;   // b >= 0 here: the unbiased exponent
  if (b >= 0 && e < 30) {
    if (e < 0) {
      frac = f;
      return 0;
    }
    const long long keep = ~((1LL << (52 - e)) - 1);
    frac = f - __longlong_as_double(b & keep);
    return (int)((((b & 0x000fffffffffffffLL) | 0x0010000000000000LL)) >> (52 - e));
  }
  const double fl = floor(f);
  frac = f - fl;
  return (int)fl;
}

// cell index and the fraction within it, FP64 coordinates
__device__ __forceinline__ int zone_split(double f, double &frac) { return floor_frac(f, frac); }

// ---------------------------------------------------------------- model view passed to kernels
struct DevModel {
  // metric and units
  double a, mass, hslope, r_h;
  double rho_unit, B_unit, Ne_unit, Ccoef, L3;   // Ccoef = h L / (m_e c^2), L3 = L_unit^3
  double R_high, R_low, gam, thetae_min, thetae_max;
  double ithetae_max, iB_unit;   // 1 / thetae_max, 1 / B_unit
  // emission band / weights
  double lnu_min, dlnu, dlntot;
  int n_nu;
  // transport
  double eps_geo, verlet_tol, r_record, r_capture;
  int verlet_maxit, bias_mode, n_sc_max, scatter, k2_mode;
  double bias_p0, bias_max, roulette_w, roulette_p;
  double bias_scale;   // multiplies the configured bias of the generation being transported
  int64_t max_steps;
  // record
  double lnu_lo, dlog_bin;
  int n_bins, n_incl;
  // grid (zone-major primitives prim[z*8 + f])
  int n1, n2, n3, prim_f32;
  int64_t nz;
  double x1_0, dx1, x2_0, dx2, x3_0, dx3, x1_hi;
  double idx1, idx2, idx3;   // 1 / dx_i
  const double *prim64;
  const float *prim32;
  const float *prim32x;   // FP32 primitives for the FP32 coefficient path (the grid or a copy), or NULL
  // tables
  const double *lnF;      // angle integral
  int nF;
  const double *lnK2;
  int nK2;
  const double *hot;      // ln(sigma_h / sigma_T) [kHotNT][kHotNE]
  // per-run generation data
  const int64_t *start;   // exclusive scan of zone counts
  const double *zpref;    // 4 pi A nu_c per zone (int dOmega j_nu = zpref F(nu/nu_c))
  int brems;              // thermal bremsstrahlung on
  df dmass, da, dx1_0, dx1_hi, dr_record, dr_capture;   // double-float splits for the mixed geodesic
  df dpi2hh, dhh_pi, dd2th;   // pi (1 - h), (1 - h) / (2 pi), -2 pi^2 (1 - h): the theta map in double-float
  const df *dtab;             // double-float function table (kDfTabN entries)
  float fidx1, fidx2, fidx3, fx2_0, fx3_0;   // FP32 grid constants for the double-float zone lookup
  // FP32 copies of model constants and tables read by the FP32 arithmetic (no FP64 conversions there)
  float fNe_unit, fB_unit, fgam, fR_low, fR_high, fthetae_max, fithetae_max, fthetae_min, fverlet_tol;
  df deps_geo;
  int hslope1, kappa_on;
  // FP32 copies for the split precision form's weight arithmetic
  float fCcoef, fbias_p0, fbias_max, fbias_scale, froulette_w, froulette_p;
  const float *lnK2f, *hotf;
  const double *ftab;     // tables of the FP64 exp_t, log_t, sincospi_t (kFtN doubles)
  double kappa;           // > 0: kappa-distributed electrons for the synchrotron terms
  const double *kapJ, *kapA, *kapI;   // ln J, ln A, ln I on the kappa grid [kKapNX][kKapNW]
  const double *kapH;     // ln(sigma_h / sigma_T) of the kappa population [kKapNW][kHotNE]
  const double *zlnw;     // per zone: ln w of the kappa population (kappa only)
  double *zbq, *zbnt;     // per zone: q / nu_T and nu_T = k T_e / h (bremsstrahlung only)
  const double *zlnuc;    // ln nu_c per zone
  const double *zgmax;    // max_j g_ij per zone
  const double *lnw;      // ln w_j (n_nu)
  const double *winv;     // 1 / w_j (n_nu)
  uint64_t seed;
  double *spec;           // spectrum sums [n_incl][n_bins][3] of this model
};

// ---------------------------------------------------------------- Philox4x32-10 (Salmon et al. 2011)
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Per-superphoton stream: key = seed, counter = (draw/2, 0, id_lo, id_hi); a double per half block.
struct Rng {
  uint64_t id;
  uint32_t n;
  uint32_t cache_blk;
  uint32_t cache[4];
};

__device__ __forceinline__ void rng_init(Rng &s, uint64_t id, uint32_t n) {
  s.id = id;
  s.n = n;
  s.cache_blk = 0xFFFFFFFFu;
}

__device__ __forceinline__ double rng_u(Rng &s, uint64_t seed) {
  uint32_t blk = s.n >> 1;
  if (blk != s.cache_blk) {
    s.cache[0] = blk;
    s.cache[1] = 0u;
    s.cache[2] = (uint32_t)s.id;
    s.cache[3] = (uint32_t)(s.id >> 32);
    philox(s.cache, (uint32_t)seed, (uint32_t)(seed >> 32));
    s.cache_blk = blk;
  }
  uint32_t a = (s.n & 1u) ? s.cache[2] : s.cache[0];
  uint32_t b = (s.n & 1u) ? s.cache[3] : s.cache[1];
  s.n++;
  uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
  return ((double)m + 0.5) * 1.1102230246251565e-16;   // 2^-53
}

// Child stream id: splitmix64 output (Steele, Lea & Flood 2014) of parent + (event+1) * golden gamma.
__host__ __device__ __forceinline__ uint64_t child_id(uint64_t parent, uint32_t ev) {
  uint64_t z = parent + 0x9E3779B97F4A7C15ull * (uint64_t)(ev + 1u);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kZoneTag = 0xC000000000000000ull;

// ---------------------------------------------------------------- metric (section 2.4)
// Nonzero components of the MKS Kerr-Schild metric (symmetric): 00 01 03 11 13 22 33; its
// inverse has 00 01 11 13 22 33.  d1 / d2: derivatives with respect to x1 and x2.  S is the
// scalar of the geodesic arithmetic: double (plain FP64) or df (double-float, mixed precision).
template <typename S>
struct GeoT {
  S g00, g01, g03, g11, g13, g22, g33;
  S G00, G01, G11, G13, G22, G33;
  S d100, d101, d103, d111, d113, d122, d133;
  S d200, d201, d203, d211, d213, d222, d233;
  S r, sth, cth;
};
using Geo = GeoT<double>;

// theta(x2) = pi x2 + (1-h)/2 sin(2 pi x2) and its first two derivatives.
__device__ __forceinline__ void theta_map(double h, double x2, double &th, double &dth, double &d2th) {
  if (h == 1.0) {
    th = kPI * x2;
    dth = kPI;
    d2th = 0.0;
    return;
  }
  double s2, c2;
  sincospi(2.0 * x2, &s2, &c2);
  th = kPI * x2 + 0.5 * (1.0 - h) * s2;
  dth = kPI * (1.0 + (1.0 - h) * c2);
  d2th = -2.0 * kPI * kPI * (1.0 - h) * s2;
}

// sin and cos of |d| < 1/2 by their Taylor series (truncation below 1e-20 relative).
__device__ __forceinline__ void sincos_small(double d, double &s, double &c) {
  constexpr double s3 = -1.0 / 6.0, s5 = 1.0 / 120.0, s7 = -1.0 / 5040.0, s9 = 1.0 / 362880.0,
                   s11 = -1.0 / 39916800.0, s13 = 1.0 / 6227020800.0, s15 = -1.0 / 1307674368000.0;
  constexpr double c2 = -0.5, c4 = 1.0 / 24.0, c6 = -1.0 / 720.0, c8 = 1.0 / 40320.0, c10 = -1.0 / 3628800.0,
                   c12 = 1.0 / 479001600.0, c14 = -1.0 / 87178291200.0, c16 = 1.0 / 20922789888000.0;
  const double d2 = d * d;
  s = d + d * d2 * (s3 + d2 * (s5 + d2 * (s7 + d2 * (s9 + d2 * (s11 + d2 * (s13 + d2 * s15))))));
  c = 1.0 + d2 * (c2 + d2 * (c4 + d2 * (c6 + d2 * (c8 + d2 * (c10 + d2 * (c12 + d2 * (c14 + d2 * c16)))))));
}

// The double-float form of the metric below (after r, sin, cos of theta and the theta map): the same
// quantities, with the shared factors formed once, the factors 2 and 4 applied exactly, and the sums of
// products as one-pass accumulations (sdot).  The grouping differs from the FP64 form's; the values
// agree to double-float accuracy.
__device__ __forceinline__ df df_twice(df x) { return {__fmul_rn(x.hi, 2.0f), __fmul_rn(x.lo, 2.0f)}; }
template <bool DERIV, bool KERR>
__device__ __forceinline__ void metric_rest_df(df r, df s, df c, df dth, df d2th, df a, df M, df a2, GeoT<df> &G) {
  const df zero = df_const(0.0);
  const df s2 = s * s, r2 = r * r;
  const df sig = KERR ? sdot(r, r, a2, c * c) : r2;   // r^2 + a^2 cos^2
  const df rs = r * s2;
  const df Q = df_rcp(sig * rs * dth);   // one division for 1/Sigma, 1/r, 1/sin^2 and 1/(dtheta/dx2)
  const df Qd = Q * dth, sigs2 = sig * s2;
  const df isig = Qd * rs, ir = Qd * sigs2, is2 = Qd * sig * r, idth = Q * sig * rs;
  const df M2 = df_twice(M), M2r = M2 * r;
  const df f = M2r * isig, opf = f + 1.0f;
  const df as2 = KERR ? a * s2 : zero, a2s2 = KERR ? a2 * s2 : zero;
  const df Grp = KERR ? -(as2 * opf) : zero;
  const df dth2 = dth * dth;
  G.r = r;
  G.sth = s;
  G.cth = c;
  G.g00 = f - 1.0f;
  G.g01 = f * r;
  G.g03 = KERR ? -(as2 * f) : zero;
  G.g11 = opf * r2;
  G.g13 = Grp * r;
  G.g22 = sig * dth2;
  if constexpr (KERR) {
    DotAcc d{sig.hi, sig.lo};
    dot_add(d, a2s2, opf);
    G.g33 = s2 * dot_end(d);   // sin^2 (Sigma + a^2 sin^2 (1 + f))
  } else {
    G.g33 = sigs2;
  }
  G.G00 = -opf;
  G.G01 = f * ir;
  {
    DotAcc d = dot_first(r, r - M2);   // Delta = r (r - 2M) + a^2
    if (KERR) dot_add(d, a2);
    G.G11 = dot_end(d) * isig * (ir * ir);
  }
  G.G13 = KERR ? a * isig * ir : zero;
  G.G22 = isig * (idth * idth);
  G.G33 = isig * is2;
  if (!DERIV) return;
  const df isig2 = isig * isig;
  const df dfr = M2 * (sig - df_twice(r2)) * isig2;   // d f / d r
  const df rdfr = r * dfr;
  G.d100 = rdfr;
  G.d101 = r * (rdfr + f);
  G.d111 = r2 * (rdfr + df_twice(opf));
  G.d122 = df_twice(r2) * dth2;
  if constexpr (!KERR) {
    G.d103 = G.d113 = zero;
    G.d133 = df_twice(r * rs);
    G.d200 = G.d201 = G.d203 = G.d211 = G.d213 = zero;
    G.d222 = df_twice(sig * dth) * d2th;
    G.d233 = dth * (df_twice(s * c) * sig);
    return;
  }
  const df sc2 = df_twice(s * c);   // 2 sin cos
  const df dft = df_twice(M2r * isig2 * (a2 * s * c));   // d f / d theta = 4 M r a^2 s c / Sigma^2
  const df dGp_r = -(as2 * dfr);   // d g_tphi / dr = d g_rphi / dr
  const df dGtp_t = -(a * sdot(dft, s2, f, sc2));
  const df dGrp_t = -(a * sdot(sc2, opf, s2, dft));
  DotAcc dr{df_twice(rs).hi, df_twice(rs).lo};   // d g_phph / dr = 2 r s^2 + a^2 s^4 df/dr
  dot_add(dr, a2s2 * s2, dfr);
  const df dGpp_r = dot_end(dr);
  // d g_phph / dtheta = 2 s c (Sigma - a^2 s^2) + a^2 s^2 (4 s c (1 + f) + s^2 df/dtheta)
  const df dGpp_t = sdot(sc2, sig - a2s2, a2s2, sdot(df_twice(sc2), opf, s2, dft));
  // d/dx1 = r d/dr
  G.d103 = r * dGp_r;
  {
    DotAcc d{Grp.hi, Grp.lo};
    dot_add(d, r, dGp_r);
    G.d113 = r * dot_end(d);
  }
  G.d133 = r * dGpp_r;
  // d/dx2 = dth d/dtheta
  const df d200 = dth * dft;
  G.d200 = d200;
  G.d201 = d200 * r;
  G.d203 = dth * dGtp_t;
  G.d211 = d200 * r2;
  G.d213 = dth * dGrp_t * r;
  G.d222 = dth * sdot(-df_twice(a2 * s * c), dth2, df_twice(sig), d2th);
  G.d233 = dth * dGpp_t;
}

// Metric, inverse metric and (DERIV) x1/x2 derivatives at (x1, x2).  theta = pi x2 + delta with
// delta = (1-h)/2 sin(2 pi x2): sin and cos of theta come from sincospi(x2) and the series of the
// small angle delta (|delta| < 1/2 for h in (0, 1]) by angle addition.
// KERR = false: the a = 0 (Schwarzschild) form, with the terms that vanish at a = 0 left out.
// For S = df, r = e^x1 and the angular functions come from the double-float exp and sincospi, and
// sin, cos of theta = pi (x2 + delta/pi) from a second sincospi in place of the series.
template <bool DERIV, bool KERR = true, typename S = double>
__device__ __forceinline__ void metric_eval(const DevModel &m, S x1s, S x2s, GeoT<S> &G) {
  constexpr S kZeroS = cst<S>(0.0), kPiS = cst<S>(kPI);   // compile-time constants (no conversions)
  const S a = KERR ? pick<S>(m.a, m.da) : kZeroS, M = pick<S>(m.mass, m.dmass), a2 = a * a;
  S r, dth, d2th, s, c;
  if constexpr (std::is_same<S, df>::value) {
    r = df_exp(x1s, m.dtab);
    df sp, cp;
    df_sincospi(x2s, m.dtab, sp, cp);
    if (m.hslope1) {
      dth = kPiS;
      d2th = kZeroS;
      s = sp;
      c = cp;
    } else {
      const df s2x = df_twice(sp * cp), c2x = (cp - sp) * (cp + sp);   // sin, cos of 2 pi x2
      dth = m.dpi2hh * c2x + kPiS;
      d2th = m.dd2th * s2x;
      df_sincospi(x2s + m.dhh_pi * s2x, m.dtab, s, c);
    }
    metric_rest_df<DERIV, KERR>(r, s, c, dth, d2th, a, M, a2, G);
    return;
  } else {
    const double x1 = x1s, x2 = x2s;
    r = exp_t(m.ftab, x1);
    double sp, cp;
    sincospi_t(m.ftab, x2, sp, cp);
    if (m.hslope == 1.0) {
      dth = kPI;
      d2th = 0.0;
      s = sp;
      c = cp;
    } else {
      const double hh = 0.5 * (1.0 - m.hslope);
      const double s2x = 2.0 * sp * cp, c2x = (cp - sp) * (cp + sp);   // sin, cos of 2 pi x2
      dth = kPI * (1.0 + 2.0 * hh * c2x);
      d2th = -4.0 * kPI * kPI * hh * s2x;
      double sd, cd;
      sincos_small(hh * s2x, sd, cd);
      s = sp * cd + cp * sd;
      c = cp * cd - sp * sd;
    }
  }
  S s2 = s * s, c2 = c * c;
  S sig = KERR ? r * r + a2 * c2 : r * r;
  // one division for 1/Sigma, 1/r, 1/sin^2 and 1/(dtheta/dx2)
  const S rs = r * s2;
  S Q = srcp(sig * rs * dth);
  S Qd = Q * dth;
  S isig = Qd * rs, ir = Qd * sig * s2, is2 = Qd * sig * r, idth = Q * sig * rs;
  S f = 2.0f * M * r * isig;
  S opf = 1.0f + f;
  // Kerr-Schild components (t, r, theta, phi)
  S Gtt = f - 1.0f, Gtr = f, Grr = opf, Ghh = sig;
  S Gtp = KERR ? -a * f * s2 : kZeroS, Grp = KERR ? -a * s2 * opf : kZeroS;
  S Gpp = KERR ? s2 * (sig + a2 * s2 * opf) : s2 * sig;
  G.r = r;
  G.sth = s;
  G.cth = c;
  G.g00 = Gtt;
  G.g01 = Gtr * r;
  G.g03 = Gtp;
  G.g11 = Grr * r * r;
  G.g13 = Grp * r;
  G.g22 = Ghh * dth * dth;
  G.g33 = Gpp;
  // inverse: g^tt = -(1+f), g^tr = f, g^rr = (r^2 - 2Mr + a^2)/Sigma, g^rphi = a/Sigma,
  // g^thth = 1/Sigma, g^phph = 1/(Sigma sin^2); divided by the Jacobian factors
  G.G00 = -opf;
  G.G01 = f * ir;
  G.G11 = (KERR ? r * r - 2.0f * M * r + a2 : r * r - 2.0f * M * r) * isig * ir * ir;
  G.G13 = KERR ? a * isig * ir : kZeroS;
  G.G22 = isig * idth * idth;
  G.G33 = isig * is2;
  if (!DERIV) return;
  // derivatives of the KS components with respect to r and theta
  S dfr = 2.0f * M * (sig - 2.0f * r * r) * isig * isig;
  if constexpr (!KERR) {
    // a = 0: f, g_tr, g_rr depend on r only; g_thth = r^2, g_phph = r^2 sin^2
    const S zero = kZeroS;
    G.d100 = r * dfr;
    G.d101 = r * (r * dfr + Gtr);
    G.d103 = zero;
    G.d111 = r * r * (r * dfr + 2.0f * Grr);
    G.d113 = zero;
    G.d122 = r * (2.0f * r) * dth * dth;
    G.d133 = r * (2.0f * r * s2);
    G.d200 = G.d201 = G.d203 = G.d211 = G.d213 = zero;
    G.d222 = Ghh * 2.0f * dth * d2th;
    G.d233 = dth * (2.0f * s * c * sig);
    return;
  }
  S dft = 4.0f * M * r * a2 * s * c * isig * isig;
  S dGtp_r = -a * s2 * dfr, dGtp_t = -a * (dft * s2 + 2.0f * f * s * c);
  S dGrp_r = -a * s2 * dfr, dGrp_t = -a * (2.0f * s * c * opf + s2 * dft);
  S dGhh_r = 2.0f * r, dGhh_t = -2.0f * a2 * s * c;
  S dGpp_r = 2.0f * r * s2 + a2 * s2 * s2 * dfr;
  S dGpp_t = 2.0f * s * c * sig + s2 * (-2.0f * a2 * s * c) + a2 * (4.0f * s2 * s * c * opf + s2 * s2 * dft);
  // d/dx1 = r d/dr (Jacobian factor r also varies with x1)
  G.d100 = r * dfr;
  G.d101 = r * (r * dfr + Gtr);
  G.d103 = r * dGtp_r;
  G.d111 = r * r * (r * dfr + 2.0f * Grr);
  G.d113 = r * (r * dGrp_r + Grp);
  G.d122 = r * dGhh_r * dth * dth;
  G.d133 = r * dGpp_r;
  // d/dx2 = dth d/dtheta (Jacobian factor dth also varies with x2)
  G.d200 = dth * dft;
  G.d201 = dth * dft * r;
  G.d203 = dth * dGtp_t;
  G.d211 = dth * dft * r * r;
  G.d213 = dth * dGrp_t * r;
  G.d222 = dth * dGhh_t * dth * dth + Ghh * 2.0f * dth * d2th;
  G.d233 = dth * dGpp_t;
}

__device__ __forceinline__ void lower(const Geo &G, const double v[4], double o[4]) {
  o[0] = G.g00 * v[0] + G.g01 * v[1] + G.g03 * v[3];
  o[1] = G.g01 * v[0] + G.g11 * v[1] + G.g13 * v[3];
  o[2] = G.g22 * v[2];
  o[3] = G.g03 * v[0] + G.g13 * v[1] + G.g33 * v[3];
}

__device__ __forceinline__ double dot(const Geo &G, const double a[4], const double b[4]) {
  double lb[4];
  lower(G, b, lb);
  return a[0] * lb[0] + a[1] * lb[1] + a[2] * lb[2] + a[3] * lb[3];
}

// dk^mu/dlambda = -Gamma^mu_ab k^a k^b = -g^{mu nu} (k^1 (d1 g k)_nu + k^2 (d2 g k)_nu - 1/2 d_nu g_ab k^a k^b)
template <bool KERR = true, typename S = double>
__device__ __forceinline__ void accel(const GeoT<S> &G, const S k[4], S A[4]) {
  // sdot: the plain sums of products for double, one-pass accumulations for df
  if constexpr (!KERR) {
    // a = 0: d103 = d113 = d2(0,1,3) = G13 = 0
    S p0 = sdot(G.d100, k[0], G.d101, k[1]);
    S p1 = sdot(G.d101, k[0], G.d111, k[1]);
    S p2 = G.d122 * k[2];
    S p3 = G.d133 * k[3];
    S q2 = G.d222 * k[2];
    S q3 = G.d233 * k[3];
    S kDk1 = sdot(k[0], p0, k[1], p1, k[2], p2, k[3], p3);
    S kDk2 = sdot(k[2], q2, k[3], q3);
    S w0 = k[1] * p0;
    S w1 = sdot_mh(k[1], p1, kDk1);
    S w2 = sdot_mh(k[1], p2, k[2], q2, kDk2);
    S w3 = sdot(k[1], p3, k[2], q3);
    A[0] = -sdot(G.G00, w0, G.G01, w1);
    A[1] = -sdot(G.G01, w0, G.G11, w1);
    A[2] = -(G.G22 * w2);
    A[3] = -(G.G33 * w3);
    return;
  }
  S p0 = sdot(G.d100, k[0], G.d101, k[1], G.d103, k[3]);
  S p1 = sdot(G.d101, k[0], G.d111, k[1], G.d113, k[3]);
  S p2 = G.d122 * k[2];
  S p3 = sdot(G.d103, k[0], G.d113, k[1], G.d133, k[3]);
  S q0 = sdot(G.d200, k[0], G.d201, k[1], G.d203, k[3]);
  S q1 = sdot(G.d201, k[0], G.d211, k[1], G.d213, k[3]);
  S q2 = G.d222 * k[2];
  S q3 = sdot(G.d203, k[0], G.d213, k[1], G.d233, k[3]);
  S kDk1 = sdot(k[0], p0, k[1], p1, k[2], p2, k[3], p3);
  S kDk2 = sdot(k[0], q0, k[1], q1, k[2], q2, k[3], q3);
  S w0 = sdot(k[1], p0, k[2], q0);
  S w1 = sdot_mh(k[1], p1, k[2], q1, kDk1);
  S w2 = sdot_mh(k[1], p2, k[2], q2, kDk2);
  S w3 = sdot(k[1], p3, k[2], q3);
  A[0] = -sdot(G.G00, w0, G.G01, w1);
  A[1] = -sdot(G.G01, w0, G.G11, w1, G.G13, w3);
  A[2] = -(G.G22 * w2);
  A[3] = -sdot(G.G13, w1, G.G33, w3);
}

// Step size (reading; the paper gives none): each internal coordinate moves at most eps_geo of
// its scale (1 for ln r and phi, the distance to the nearer pole for x2).
template <typename S = double>
__device__ __forceinline__ S stepsize(const DevModel &m, const S X[4], const S K[4]) {
  // 1 / (1/d1 + 1/d2 + 1/d3) with d1 = eps/(|k1|+S), d2 = eps x2n/(|k2|+S), d3 = eps/(|k3|+S)
  // = eps x2n / ((|k1| + |k3|) x2n + |k2|): one division
  const double SMALL = 1e-40;
  double x2n = dmin_nn(fabs(X[2]), fabs(1.0 - X[2]));
  double den = ((fabs(K[1]) + SMALL) + (fabs(K[3]) + SMALL)) * x2n + (fabs(K[2]) + SMALL);
  return m.eps_geo * x2n / den;
}

// Double-float step size: the same rule in double-float, so that the steps land where the FP64
// path's do (an FP32 step length would move every step end along the path by ~1e-7).
template <>
__device__ __forceinline__ df stepsize<df>(const DevModel &m, const df X[4], const df K[4]) {
  const df a = df_abs(X[2]), b = df_abs(1.0f - X[2]);
  const df x2n = df_le(a, b) ? a : b;
  const df den = ((df_abs(K[1]) + df_abs(K[3])) * x2n + df_abs(K[2])) + 1e-30f;
  return (m.deps_geo * x2n) * df_rcp(den);
}

// ---------------------------------------------------------------- tables
__device__ __forceinline__ double cubic_table(const double *t, int n, double x0, double inv_step, double x) {
  double f = (x - x0) * inv_step, fr;
  const int i0 = floor_frac(f, fr);
  const int i = max(1, min(i0, n - 3));
  const double u = (i == i0) ? fr : f - i;
  double y0 = t[i - 1], y1 = t[i], y2 = t[i + 1], y3 = t[i + 2];
  // 4-point Lagrange through nodes i-1 .. i+2 at offset u from node i
  double um1 = u + 1.0, u1 = u - 1.0, u2 = u - 2.0;
  return -y0 * u * u1 * u2 / 6.0 + y1 * um1 * u1 * u2 / 2.0 - y2 * um1 * u * u2 / 2.0 + y3 * um1 * u * u1 / 6.0;
}

// int_0^{pi/2} sin^2 G(K / sin) dth from the table (0 beyond the table's upper end)
__device__ __forceinline__ double F_of_lnK(const DevModel &m, double lnK) {
  if (lnK >= kFLnK1) return 0.0;
  if (lnK <= kFLnK0) {
    // small-K power law F ~ K^(1/3) continued from the first node
    return exp_t(m.ftab, m.lnF[0] + (lnK - kFLnK0) / 3.0);
  }
  return exp_t(m.ftab, cubic_table(m.lnF, m.nF, kFLnK0, 1.0 / kFStep, lnK));
}

__device__ __forceinline__ double K2_of(const DevModel &m, double thetae) {
  if (m.k2_mode == 1) return 2.0 * thetae * thetae;
  return exp(cubic_table(m.lnK2, m.nK2, kK2LnT0, 1.0 / kK2Step, log(thetae)));
}

__device__ __forceinline__ double K2_of_ln(const DevModel &m, double thetae, double lt) {
  if (m.k2_mode == 1) return 2.0 * thetae * thetae;
  return exp(cubic_table(m.lnK2, m.nK2, kK2LnT0, 1.0 / kK2Step, lt));
}

__device__ __forceinline__ double lnK2_of_ln(const DevModel &m, double lt) {
  if (m.k2_mode == 1) return 0.6931471805599453 + 2.0 * lt;   // ln(2 Theta^2)
  return cubic_table(m.lnK2, m.nK2, kK2LnT0, 1.0 / kK2Step, lt);
}

__device__ __forceinline__ float K2_of_f(const DevModel &m, float thetae) {
  if (m.k2_mode == 1) return 2.0f * thetae * thetae;
  float f = (__logf(thetae) - (float)kK2LnT0) * (float)(1.0 / kK2Step);
  int i = max(0, min(zone_floor(f), m.nK2 - 2));
  float u = f - i;
  float l = (1.0f - u) * m.lnK2f[i] + u * m.lnK2f[i + 1];
  return __expf(l);
}

__device__ __forceinline__ double hot_lookup_ln(const DevModel &m, double lt, double le) {
  constexpr double st = (kHotNT - 1) / (kHotLT1 - kHotLT0), se = (kHotNE - 1) / (kHotLE1 - kHotLE0);
  double ft = (lt - kHotLT0) * st;
  double fe = (le - kHotLE0) * se;
  ft = dmin_nn(dmax0(ft), (double)(kHotNT - 1));
  fe = dmin_nn(dmax0(fe), (double)(kHotNE - 1));
  double a, b;
  const int i0 = floor_frac(ft, a), j0 = floor_frac(fe, b);
  const int i = min(i0, kHotNT - 2), j = min(j0, kHotNE - 2);
  if (i != i0) a = 1.0;   // at the last node (ft = kHotNT - 1)
  if (j != j0) b = 1.0;
  const double *h = m.hot;
  double v00 = h[i * kHotNE + j], v01 = h[i * kHotNE + j + 1];
  double v10 = h[(i + 1) * kHotNE + j], v11 = h[(i + 1) * kHotNE + j + 1];
  double l = (1 - a) * (1 - b) * v00 + (1 - a) * b * v01 + a * (1 - b) * v10 + a * b * v11;
  return kSIGT * exp_t(m.ftab, l);
}

__device__ __forceinline__ double hot_lookup(const DevModel &m, double thetae, double eps) {
  return hot_lookup_ln(m, log(thetae), log(eps));
}

__device__ __forceinline__ float hot_lookup_f(const DevModel &m, float thetae, float eps) {
  float ft = (__logf(thetae) - (float)kHotLT0) * (float)((kHotNT - 1) / (kHotLT1 - kHotLT0));
  float fe = (__logf(eps) - (float)kHotLE0) * (float)((kHotNE - 1) / (kHotLE1 - kHotLE0));
  ft = fminf(fmaxf(ft, 0.0f), (float)(kHotNT - 1));
  fe = fminf(fmaxf(fe, 0.0f), (float)(kHotNE - 1));
  const int i = max(0, min(zone_floor(ft), kHotNT - 2)), j = max(0, min(zone_floor(fe), kHotNE - 2));
  float a = ft - i, b = fe - j;
  const float *h32 = m.hotf;
  float v00 = h32[i * kHotNE + j], v01 = h32[i * kHotNE + j + 1];
  float v10 = h32[(i + 1) * kHotNE + j], v11 = h32[(i + 1) * kHotNE + j + 1];
  float l = (1 - a) * (1 - b) * v00 + (1 - a) * b * v01 + a * (1 - b) * v10 + a * b * v11;
  return (float)kSIGT * __expf(l);
}

// X^(1/6) for X in (1e-30, 1e30): z = X^(-1/6) from an FP32 seed (relative error < 1e-5) refined by two
// division-free Newton steps on f(z) = z^-6 - X (z <- z + z (1 - X z^6) / 6, error ~3.5 e^2 per step),
// then X^(1/6) = X z^5.  Outside that range: cbrt(sqrt(X)).
__device__ __forceinline__ double pow_sixth(double X) {
  if (!(X > 1e-30 && X < 1e30)) return cbrt(sqrt(X));
  double z = (double)__expf(__logf((float)X) * (-1.0f / 6.0f));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double z2 = z * z;
    const double t = fma(-X, z2 * z2 * z2, 1.0);
    z = fma(z * t, 1.0 / 6.0, z);
  }
  const double z2 = z * z;
  return X * (z2 * z2 * z);
}

// ---------------------------------------------------------------- kappa electrons (future work in section 6)
// Synchrotron terms of kappa-distributed electrons from the single-electron spectrum: with
// X = nu / (nu_B sin), nu_B = e B / (2 pi m_e c) and F the synchrotron function,
//   j_nu = (sqrt3 e^3 n_e B sin / 4 pi m_e c^2) J(X, w),  J = int f F(2X / 3 gamma^2) dgamma,
//   nu alpha_nu = (c^2 / 8 pi nu) (sqrt3 e^3 n_e B sin / (m_e c^2)^2) A(X, w),
//   int dOmega j_nu = (sqrt3 e^3 n_e B / m_e c^2) I(nu / nu_B, w);
// ln J, ln A, ln I tabulated on this grid and interpolated bilinearly.
constexpr int kKapNX = 601, kKapNW = 61, kKapNF = 6001;
constexpr double kKapLX0 = -9.210340371976184, kKapLX1 = 36.841361487904734;   // ln X in [1e-4, 1e16]
constexpr double kKapLW0 = -6.907755278982137, kKapLW1 = 6.907755278982137;    // ln w in [1e-3, 1e3]
constexpr double kKapLF0 = -30.0, kKapLF1 = 5.298317366548036;                 // ln x of the F table
constexpr double kKapFloor = -700.0;
constexpr double kKapCj = 1.7320508075688772 * kEE * kEE * kEE / (kME * kCL * kCL);   // sqrt3 e^3 / m_e c^2
constexpr double kNuB1 = kEE / (2.0 * kPI * kME * kCL);                                // nu_B / B

__device__ __forceinline__ double kap_interp(const double *t, double lx, double lw) {
  constexpr double sx = (kKapNX - 1) / (kKapLX1 - kKapLX0), sw = (kKapNW - 1) / (kKapLW1 - kKapLW0);
  double fx = fmin(fmax((lx - kKapLX0) * sx, 0.0), (double)(kKapNX - 1));
  double fw = fmin(fmax((lw - kKapLW0) * sw, 0.0), (double)(kKapNW - 1));
  int i = min((int)fx, kKapNX - 2), j = min((int)fw, kKapNW - 2);
  double a = fx - i, b = fw - j;
  const double *r = t + i * kKapNW + j;
  double l = (1 - a) * (1 - b) * r[0] + (1 - a) * b * r[1] + a * (1 - b) * r[kKapNW] + a * b * r[kKapNW + 1];
  return exp(l);
}

// nu alpha_nu of the kappa population at angle sth to the field
__device__ __forceinline__ double kappa_nu_alpha(const DevModel &m, double ne, double thetae, double B, double sth,
                                                 double nu) {
  const double lx = log(nu / (kNuB1 * B * sth)), lw = log(thetae * (m.kappa - 3.0) / m.kappa);
  constexpr double kCa = kCL * kCL / (8.0 * kPI) * kKapCj / (kME * kCL * kCL);
  return kCa * ne * B * sth * kap_interp(m.kapA, lx, lw) / nu;
}

// Hot cross-section of the kappa population, bilinear in (ln w, ln eps) on the kappa w grid and the
// thermal table's eps grid (clamped to both)
__device__ __forceinline__ double kap_hot_lookup(const DevModel &m, double thetae, double eps) {
  constexpr double sw = (kKapNW - 1) / (kKapLW1 - kKapLW0), se = (kHotNE - 1) / (kHotLE1 - kHotLE0);
  double fw = (log(fmax(thetae, 1e-300) * (m.kappa - 3.0) / m.kappa) - kKapLW0) * sw;
  double fe = (log(eps) - kHotLE0) * se;
  fw = fmin(fmax(fw, 0.0), (double)(kKapNW - 1));
  fe = fmin(fmax(fe, 0.0), (double)(kHotNE - 1));
  int i = min((int)fw, kKapNW - 2), j = min((int)fe, kHotNE - 2);
  double a = fw - i, b = fe - j;
  const double *h = m.kapH;
  double v00 = h[i * kHotNE + j], v01 = h[i * kHotNE + j + 1];
  double v10 = h[(i + 1) * kHotNE + j], v11 = h[(i + 1) * kHotNE + j + 1];
  return kSIGT * exp((1 - a) * (1 - b) * v00 + (1 - a) * b * v01 + a * (1 - b) * v10 + a * b * v11);
}

// ---------------------------------------------------------------- bremsstrahlung (future work in section 6)
// Total thermal bremsstrahlung cooling rate of a hydrogen plasma [erg s^-1 cm^-3], electron-ion plus
// electron-electron, from the fits of Stepney & Guilbert (1983) in the form of Narayan & Yi (1995);
// the spectrum is 4 pi j_nu = q (h / k T) exp(-h nu / k T) and absorption follows Kirchhoff's law.
__device__ __forceinline__ double brems_q(double ne, double th) {
  constexpr double kAlphaF = 7.2973525693e-3, kRe = 2.8179403262e-13, kMc2 = kME * kCL * kCL;
  double fei, fee;
  if (th < 1.0) {
    fei = 4.0 * sqrt(2.0 * th / (kPI * kPI * kPI)) * (1.0 + 1.781 * pow(th, 1.34));
    fee = 20.0 / (9.0 * sqrt(kPI)) * (44.0 - 3.0 * kPI * kPI) * th * sqrt(th) *
          (1.0 + 1.1 * th + th * th - 1.25 * th * th * sqrt(th));
  } else {
    fei = 9.0 * th / (2.0 * kPI) * (log(1.123 * th + 0.48) + 1.5);
    fee = 24.0 * th * (log(1.1232 * th) + 1.28);
  }
  return ne * ne * kAlphaF * kMc2 * kCL * (1.25 * kSIGT * fei + kRe * kRe * fee);
}

// nu alpha_nu = nu j_nu / B_nu = q c^2 (1 - exp(-h nu / k T)) / (8 pi k T nu^2)
__device__ __forceinline__ double brems_nu_alpha(double ne, double th, double nu) {
  if (!(ne > 0.0 && th > 0.0)) return 0.0;
  const double kt = th * kME * kCL * kCL;
  return brems_q(ne, th) * kCL * kCL * (-expm1(-kHPL * nu / kt)) / (8.0 * kPI * kt * nu * nu);
}

// int dOmega j_nu of zone z at weight-table node j: synchrotron (pref F(nu/nu_c); 0 when the zone
// has no synchrotron) plus, when on, bremsstrahlung (q / nu_T) exp(-nu / nu_T).
__device__ __forceinline__ double F_of_lnK(const DevModel &m, double lnK);
__device__ __forceinline__ double kap_interp(const double *t, double lx, double lw);
__device__ __forceinline__ double zone_E(const DevModel &m, int64_t z, double pref, double lnuc, int j) {
  // kappa: lnuc holds ln nu_B and the zone's ln w sits in zlnw
  double e = (pref == 0.0) ? 0.0
             : (m.kappa > 0.0) ? pref * kap_interp(m.kapI, m.lnu_min + j * m.dlnu - lnuc, m.zlnw[z])
                               : pref * F_of_lnK(m, m.lnu_min + j * m.dlnu - lnuc);
  if (m.brems && m.zbq[z] > 0.0) e += m.zbq[z] * exp_t(m.ftab, -exp_t(m.ftab, m.lnu_min + j * m.dlnu) / m.zbnt[z]);
  return e;
}

// ---------------------------------------------------------------- synchrotron (section 2.2)
// G(X) = (X^1/2 + 2^11/12 X^1/6)^2 exp(-X^1/3)
__device__ __forceinline__ double Gsyn(double X) {
  double x6 = cbrt(sqrt(X));
  double x3 = x6 * x6;
  double t = x6 * x6 * x6 + 1.8877486253633870 * x6;   // 2^(11/12)
  return t * t * exp(-x3);
}
// the same in the emission sampler: the Newton sixth root and the table-driven exponential
__device__ __forceinline__ double Gsyn_t(const double *T, double X) {
  double x6 = pow_sixth(X);
  double x3 = x6 * x6;
  double t = x6 * x3 + 1.8877486253633870 * x6;   // 2^(11/12)
  return t * t * exp_t(T, -x3);
}

// ---------------------------------------------------------------- fluid (sections 2.5-2.7)
// model constant in the plasma arithmetic's type: the double, or its FP32 copy
template <typename T> __device__ __forceinline__ T mv(double d, float f);
template <> __device__ __forceinline__ double mv<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float mv<float>(double, float f) { return f; }

// metric component of scalar GS as the plasma arithmetic's type T
template <typename T> __device__ __forceinline__ T cvt(double x) { return (T)x; }
// FP32 from an FP64 value: truncated on the integer pipes in the split form's transport (NARROW), else
// the rounding conversion
template <bool NARROW> __device__ __forceinline__ float f32_of(double x) {
  if constexpr (NARROW) return narrow_f(x);
  else return (float)x;
}
template <bool NARROW> __device__ __forceinline__ float f32_of(df x) { return to_f(x); }
template <typename T, bool NARROW, typename V> __device__ __forceinline__ T cvtn(V x) {
  if constexpr (NARROW && sizeof(T) == 4) return f32_of<true>(x);
  else return cvt<T>(x);
}
template <typename T> __device__ __forceinline__ T cvt(df x);
template <> __device__ __forceinline__ float cvt<float>(df x) { return to_f(x); }
template <> __device__ __forceinline__ double cvt<double>(df x) { return to_d(x); }

template <typename T>
struct Plasma {
  T ne, thetae, B;
  T ucov[4], bcov[4];
  T bsq;
  T rb;    // 1 / sqrt(b^2) (0 without field); FP64 path only
  T ith;   // 1 / Theta_e (0 when Theta_e = 0); FP64 path only
  bool on;
};

// Primitives interpolated linearly in internal coordinates between zone centres (reading):
// clamped to the edge zones in x1 and x2, periodic in x3, no plasma outside the radial range.
// Zone-centred fractional indices of a point: FP64 for a double position, FP32 for a double-float one
// (the offset from the grid origin in double-float, then FP32).
__device__ __forceinline__ double zone_coord(const DevModel &m, const double X[4], int d) {
  return d == 1 ? (X[1] - m.x1_0) * m.idx1 - 0.5 : d == 2 ? (X[2] - m.x2_0) * m.idx2 - 0.5 : (X[3] - m.x3_0) * m.idx3 - 0.5;
}
__device__ __forceinline__ float zone_coord(const DevModel &m, const df X[4], int d) {
  return d == 1 ? to_f(X[1] - m.dx1_0) * m.fidx1 - 0.5f
                : d == 2 ? (to_f(X[2]) - m.fx2_0) * m.fidx2 - 0.5f : (to_f(X[3]) - m.fx3_0) * m.fidx3 - 0.5f;
}
// FP32 zone coordinates of an FP64 position (split form): the radial offset from the grid origin in
// FP64, then FP32, as the double-float form does.
__device__ __forceinline__ float zone_coord_f(const DevModel &m, const double X[4], int d) {
  return d == 1 ? narrow_f(X[1] - m.x1_0) * m.fidx1 - 0.5f
                : d == 2 ? (narrow_f(X[2]) - m.fx2_0) * m.fidx2 - 0.5f : (narrow_f(X[3]) - m.fx3_0) * m.fidx3 - 0.5f;
}
template <bool F32IDX, typename S>
__device__ __forceinline__ auto zone_coord_r(const DevModel &m, const S X[4], int d) {
  if constexpr (F32IDX && std::is_same<S, double>::value) return zone_coord_f(m, X, d);
  else return zone_coord(m, X, d);
}
__device__ __forceinline__ bool outside_radially(const DevModel &m, const double X[4]) {
  const long long k = dkey(X[1]);
  return k < dkey(m.x1_0) || k > dkey(m.x1_hi);
}
__device__ __forceinline__ bool outside_radially(const DevModel &m, const df X[4]) {
  return !(df_ge(X[1], m.dx1_0) && df_le(X[1], m.dx1_hi));
}

// F32IDX: FP32 index arithmetic for an FP64 position (the split form's transport); otherwise FP64 for
// FP64 positions and FP32 for double-float ones.
template <typename T, typename S, bool F32IDX = false>
__device__ __forceinline__ bool interp_prims(const DevModel &m, const S X[4], T pr[8]) {
  if (outside_radially(m, X)) return false;
  using R = typename std::conditional<F32IDX, float, decltype(vmag(X[0]))>::type;
  int i, j;
  R di, dj;
  {
    const R f1 = zone_coord_r<F32IDX>(m, X, 1);
    i = zone_split(f1, di);
    if (m.n1 == 1) { i = 0; di = 0; }
    else if (i < 0) { i = 0; di = 0; }
    else if (i > m.n1 - 2) { i = m.n1 - 2; di = 1; }
  }
  {
    const R f2 = zone_coord_r<F32IDX>(m, X, 2);
    j = zone_split(f2, dj);
    if (m.n2 == 1) { j = 0; dj = 0; }
    else if (j < 0) { j = 0; dj = 0; }
    else if (j > m.n2 - 2) { j = m.n2 - 2; dj = 1; }
  }
  int k0 = 0, k1 = 0;
  R dk = 0;
  if (m.n3 > 1) {
    const R f3 = zone_coord_r<F32IDX>(m, X, 3);
    const int ki = zone_split(f3, dk);
    long long kk = ki;
    k0 = (int)(((kk % m.n3) + m.n3) % m.n3);
    k1 = (k0 + 1) % m.n3;
  }
  int i1 = (m.n1 > 1) ? i + 1 : i, j1 = (m.n2 > 1) ? j + 1 : j;
  int64_t z00 = ((int64_t)i * m.n2 + j) * m.n3, z01 = ((int64_t)i * m.n2 + j1) * m.n3;
  int64_t z10 = ((int64_t)i1 * m.n2 + j) * m.n3, z11 = ((int64_t)i1 * m.n2 + j1) * m.n3;
  // FP32 output reads FP32 primitives when there are any (no per-corner conversions)
  constexpr bool kF32 = sizeof(T) == 4;
  const bool rd32 = kF32 ? (m.prim32x != nullptr) : (m.prim_f32 != 0);
  const float *p32 = kF32 ? m.prim32x : m.prim32;
  T w00, w01, w10, w11;
  if (kF32) {
    const T a = (T)di, b = (T)dj;
    w00 = (1 - a) * (1 - b); w01 = (1 - a) * b; w10 = a * (1 - b); w11 = a * b;
  } else {
    w00 = (T)((1 - di) * (1 - dj)); w01 = (T)((1 - di) * dj); w10 = (T)(di * (1 - dj)); w11 = (T)(di * dj);
  }
  T wk0 = (T)(1 - dk), wk1 = (T)dk;
#pragma unroll
  for (int f = 0; f < 8; ++f) pr[f] = (T)0;
  // FP32 fields into FP64 sums: widened on the integer pipes (the same values as the conversion)
  auto wide = [](float v) -> T {
    if constexpr (kF32) return v;
    else return widen_exact(v);
  };
  auto acc = [&](int64_t zb, T w) {
    if (rd32) {
      const float4 *p0 = reinterpret_cast<const float4 *>(p32 + (zb + k0) * 8);
      float4 a0 = __ldg(p0), a1 = __ldg(p0 + 1);
      T ww = w * wk0;
      pr[0] += ww * wide(a0.x); pr[1] += ww * wide(a0.y); pr[2] += ww * wide(a0.z); pr[3] += ww * wide(a0.w);
      pr[4] += ww * wide(a1.x); pr[5] += ww * wide(a1.y); pr[6] += ww * wide(a1.z); pr[7] += ww * wide(a1.w);
      if (m.n3 > 1) {
        const float4 *p1 = reinterpret_cast<const float4 *>(p32 + (zb + k1) * 8);
        float4 b0 = __ldg(p1), b1 = __ldg(p1 + 1);
        ww = w * wk1;
        pr[0] += ww * wide(b0.x); pr[1] += ww * wide(b0.y); pr[2] += ww * wide(b0.z); pr[3] += ww * wide(b0.w);
        pr[4] += ww * wide(b1.x); pr[5] += ww * wide(b1.y); pr[6] += ww * wide(b1.z); pr[7] += ww * wide(b1.w);
      }
    } else {
      const double2 *p0 = reinterpret_cast<const double2 *>(m.prim64 + (zb + k0) * 8);
      T ww = w * wk0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double2 v = __ldg(p0 + q);
        pr[2 * q] += ww * (T)v.x;
        pr[2 * q + 1] += ww * (T)v.y;
      }
      if (m.n3 > 1) {
        const double2 *p1 = reinterpret_cast<const double2 *>(m.prim64 + (zb + k1) * 8);
        ww = w * wk1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          double2 v = __ldg(p1 + q);
          pr[2 * q] += ww * (T)v.x;
          pr[2 * q + 1] += ww * (T)v.y;
        }
      }
    }
  };
  // same weights and order as a plain bilinear/trilinear blend
  acc(z00, w00);
  acc(z01, w01);
  acc(z10, w10);
  acc(z11, w11);
  return true;
}

// Fluid-frame quantities from primitives with metric G: 4-velocity from the normal-observer
// velocity, magnetic 4-vector b, n_e, |B| [G] and Theta_e from the R_high/R_low model.
template <typename T, typename GS = double, bool NARROW = false>
__device__ __forceinline__ void plasma_from_prims(const DevModel &m, const GeoT<GS> &G, const T pr[8], Plasma<T> &P,
                                                  T ucon_out[4], T bcon_out[4]) {
  T g00 = cvtn<T, NARROW>(G.g00), g01 = cvtn<T, NARROW>(G.g01), g03 = cvtn<T, NARROW>(G.g03),
    g11 = cvtn<T, NARROW>(G.g11), g13 = cvtn<T, NARROW>(G.g13), g22 = cvtn<T, NARROW>(G.g22),
    g33 = cvtn<T, NARROW>(G.g33);
  T rho = pr[0], uu = pr[1];
  T U1 = pr[5], U2 = pr[6], U3 = pr[7];
  constexpr bool kF64 = sizeof(T) == 8;
  T alpha = rsqrt(-cvtn<T, NARROW>(G.G00));
  T q = g11 * U1 * U1 + g22 * U2 * U2 + g33 * U3 * U3 + (T)2 * g13 * U1 * U3;
  T rg = rsqrt((T)1 + q);                   // 1 / gamma
  T gamma = kF64 ? ((T)1 + q) * rg : sqrt((T)1 + q);
  T u0 = gamma * (-cvtn<T, NARROW>(G.G00)) * alpha;   // gamma / alpha, alpha = (-g^tt)^(-1/2)
  T u1 = U1 - gamma * alpha * cvtn<T, NARROW>(G.G01);
  T u2 = U2, u3 = U3;
  T uc0 = g00 * u0 + g01 * u1 + g03 * u3;
  T uc1 = g01 * u0 + g11 * u1 + g13 * u3;
  T uc2 = g22 * u2;
  T uc3 = g03 * u0 + g13 * u1 + g33 * u3;
  T b0 = pr[2] * uc1 + pr[3] * uc2 + pr[4] * uc3;
  T iu0 = kF64 ? alpha * rg : (T)1 / u0;   // alpha / gamma
  T b1 = (pr[2] + b0 * u1) * iu0, b2 = (pr[3] + b0 * u2) * iu0, b3 = (pr[4] + b0 * u3) * iu0;
  T bc0 = g00 * b0 + g01 * b1 + g03 * b3;
  T bc1 = g01 * b0 + g11 * b1 + g13 * b3;
  T bc2 = g22 * b2;
  T bc3 = g03 * b0 + g13 * b1 + g33 * b3;
  P.ucov[0] = uc0; P.ucov[1] = uc1; P.ucov[2] = uc2; P.ucov[3] = uc3;
  P.bcov[0] = bc0; P.bcov[1] = bc1; P.bcov[2] = bc2; P.bcov[3] = bc3;
  if (ucon_out) { ucon_out[0] = u0; ucon_out[1] = u1; ucon_out[2] = u2; ucon_out[3] = u3; }
  if (bcon_out) { bcon_out[0] = b0; bcon_out[1] = b1; bcon_out[2] = b2; bcon_out[3] = b3; }
  P.bsq = b0 * bc0 + b1 * bc1 + b2 * bc2 + b3 * bc3;
  // sign tests of the FP64 instantiation on the bit patterns (x > 0 iff the pattern is positive)
  auto pos = [](T x) -> bool {
    if constexpr (kF64) return __double_as_longlong(x) > 0 && __double_as_longlong(x) < 0x7FF0000000000000LL;
    else return x > (T)0;
  };
  const bool rho_pos = pos(rho), bsq_pos = pos(P.bsq);
  P.ne = rho_pos ? rho * mv<T>(m.Ne_unit, m.fNe_unit) : (T)0;
  P.rb = (T)0;
  P.ith = (T)0;
  if (kF64) {
    // one reciprocal square root gives |b| (for B), 1/b^2 (for beta) and the 1/|b| of cos(theta_B)
    const T rb = bsq_pos ? rsqrt(P.bsq) : (T)0;
    P.rb = rb;
    P.B = P.bsq * rb * mv<T>(m.B_unit, m.fB_unit);
  } else {
    P.B = sqrt(fmax(P.bsq, (T)0)) * mv<T>(m.B_unit, m.fB_unit);
  }
  if (rho_pos && pos(uu)) {
    // Theta_e = (m_p/m_e)(gam-1)(u/rho)/(1 + T_i/T_e), T_i/T_e = (R_high beta^2 + R_low)/(1 + beta^2)
    T num, den;
    if (bsq_pos) {
      T beta = kF64 ? (T)2 * uu * (mv<T>(m.gam, m.fgam) - (T)1) * P.rb * P.rb : (T)2 * uu * (mv<T>(m.gam, m.fgam) - (T)1) / P.bsq;
      T b2x = beta * beta;
      num = (T)(kMP / kME) * (mv<T>(m.gam, m.fgam) - (T)1) * uu * ((T)1 + b2x);
      den = rho * ((T)1 + mv<T>(m.R_low, m.fR_low) + ((T)1 + mv<T>(m.R_high, m.fR_high)) * b2x);
    } else {
      num = (T)(kMP / kME) * (mv<T>(m.gam, m.fgam) - (T)1) * uu;
      den = rho * ((T)1 + mv<T>(m.R_high, m.fR_high));
    }
    T th, ith = (T)0;
    const T nd = num * den;
    bool nd_mid;
    if constexpr (kF64) {   // nd >= 0: 1e-300 < nd < 1e300 on the bit patterns
      const long long bnd = __double_as_longlong(nd);
      nd_mid = bnd > __double_as_longlong(1e-300) && bnd < __double_as_longlong(1e300);
    } else {
      nd_mid = false;
    }
    if (nd_mid) {
      // Theta_e and 1/Theta_e from one reciprocal
      const T inv = (T)1 / nd;
      th = num * (num * inv);
      ith = den * (den * inv);
    } else {
      th = num / den;
      if (kF64) ith = den / num;
    }
    bool over;
    if constexpr (kF64) over = __double_as_longlong(th) > __double_as_longlong(m.thetae_max);   // th >= 0
    else over = th > m.fthetae_max;
    if (over) {
      th = mv<T>(m.thetae_max, m.fthetae_max);
      ith = mv<T>(m.ithetae_max, m.fithetae_max);
    }
    P.thetae = th;
    P.ith = ith;
  } else {
    P.thetae = (T)0;
  }
  P.on = pos(P.ne);
}

// Invariant absorption nu alpha_nu (j/B_nu, section 2.5) and scattering nu n_e sigma_h (section 2.7), in
// the scalar W of the superphoton's weight arithmetic (FP64, or FP32 in the split precision form).
template <typename W>
struct CoefT {
  W ana, ans, thetae;
};
using Coef = CoefT<double>;

__device__ __forceinline__ void coefficients64(const DevModel &m, const Geo &G, const double X[4], const double K[4],
                                               bool want_s, Coef &c) {
  c.ana = c.ans = c.thetae = 0.0;
  double pr[8];
  if (!interp_prims<double>(m, X, pr)) return;
  Plasma<double> P;
  plasma_from_prims<double>(m, G, pr, P, nullptr, nullptr);
  c.thetae = P.thetae;
  if (!P.on) return;
  double eps = -(K[0] * P.ucov[0] + K[1] * P.ucov[1] + K[2] * P.ucov[2] + K[3] * P.ucov[3]);
  {
    const long long be = __double_as_longlong(eps);
    if (!(be > 0 && be < 0x7FF0000000000000LL)) return;   // eps > 0 (and finite) on the bit pattern
  }
  constexpr double kNuEps = kME * kCL * kCL / kHPL;   // nu / eps
  const double ieps = 1.0 / eps;
  double nu = eps * kNuEps;
  double lt = log_t(m.ftab, dmax_nn(P.thetae, 1e-300));
  // Theta_e >= Theta_min and a field (B > 0 implies b^2 > 0), as sign / order tests on bit patterns
  const bool emits = dge_nn(P.thetae, m.thetae_min) && __double_as_longlong(P.B) > 0;
  if (m.kappa_on && emits) {
    double kb = K[0] * P.bcov[0] + K[1] * P.bcov[1] + K[2] * P.bcov[2] + K[3] * P.bcov[3];
    double cth = fmin(1.0, fmax(-1.0, kb * P.rb * ieps));
    double s2 = 1.0 - cth * cth;
    if (s2 > 0.0) c.ana = kappa_nu_alpha(m, P.ne, P.thetae, P.B, s2 * rsqrt(s2), nu);
  } else if (emits) {
    double kb = K[0] * P.bcov[0] + K[1] * P.bcov[1] + K[2] * P.bcov[2] + K[3] * P.bcov[3];
    double cth = fmin(1.0, fmax(-1.0, kb * P.rb * ieps));
    double s2 = 1.0 - cth * cth;
    if (__double_as_longlong(s2) > 0) {   // s2 > 0 (s2 <= 1)
      constexpr double kNus = (2.0 / 9.0) * (kEE / (2.0 * kPI * kME * kCL));   // nu_s / (B Theta^2 sin)
      const double rs = rsqrt(s2);
      double nus = kNus * P.B * P.thetae * P.thetae * (s2 * rs);
      // X = nu / nu_s from the reciprocals at hand: 1/B = rb / B_unit, 1/Theta, 1/sin = rs
      double Xs = nu * (1.0 / kNus) * (P.rb * m.iB_unit) * (P.ith * P.ith) * rs;
      // G(X) / K2 with one exponential: G = t^2 exp(-X^1/3), t = X^1/2 + 2^(11/12) X^1/6
      double x6 = pow_sixth(Xs);
      double x3 = x6 * x6;
      if (!dge_nn(x3, 745.0)) {   // x3 < 745; beyond, exp(-X^1/3) underflows: no emission or absorption
        double t = x6 * x3 + 1.8877486253633870 * x6;
        double GoK = t * t * exp_t(m.ftab, -x3 - lnK2_of_ln(m, lt));
        // nu alpha_nu = nu j_nu / B_nu with j_nu = sqrt2 pi e^2 n_e nu_s G / (3 c K2) and
        // B_nu = 2 h nu^3 / (c^2 expm1(h nu / k T)), h nu / k T = eps / Theta_e:
        // nu alpha_nu = (sqrt2 pi e^2 c / 6h) n_e (G / K2) expm1(eps/Theta) nu_s / nu^2
        const double C1 = 1.4142135623730951 * kPI * kEE * kEE * kCL / (6.0 * kHPL) / (kNuEps * kNuEps);
        c.ana = C1 * P.ne * GoK * expm1_t(m.ftab, eps * P.ith) * nus * (ieps * ieps);
      }
    }
  }
  if (m.brems) c.ana += brems_nu_alpha(P.ne, P.thetae, nu);
  if (want_s) c.ans = nu * P.ne * (m.kappa > 0.0 ? kap_hot_lookup(m, P.thetae, eps) : hot_lookup_ln(m, lt, log_t(m.ftab, eps)));
}

// Mixed precision: the same quantities with FP32 plasma state and coefficient arithmetic.
template <typename S, typename W = double>
__device__ __forceinline__ void coefficients32(const DevModel &m, const GeoT<S> &G, const S X[4], const S K[4],
                                               bool want_s, CoefT<W> &c) {
  constexpr bool kSplit = std::is_same<W, float>::value;   // the split form's transport: narrow on integer pipes
  c.ana = c.ans = c.thetae = (W)0;
  float pr[8];
  if (!interp_prims<float, S, kSplit>(m, X, pr)) return;
  Plasma<float> P;
  plasma_from_prims<float, S, kSplit>(m, G, pr, P, nullptr, nullptr);
  c.thetae = P.thetae;
  if (!P.on) return;
  float kf[4] = {f32_of<kSplit>(K[0]), f32_of<kSplit>(K[1]), f32_of<kSplit>(K[2]), f32_of<kSplit>(K[3])};
  float eps = -(kf[0] * P.ucov[0] + kf[1] * P.ucov[1] + kf[2] * P.ucov[2] + kf[3] * P.ucov[3]);
  if (!(eps > 0.0f)) return;
  // frequencies and emissivities span ~1e-40..1e40: keep the products in ranges float holds
  float nu9 = eps * (float)(kME * kCL * kCL / kHPL * 1e-9);   // nu / 1e9 Hz
  float ana = 0.0f;
  if (P.thetae >= m.fthetae_min && P.B > 0.0f && P.bsq > 0.0f) {
    float kb = kf[0] * P.bcov[0] + kf[1] * P.bcov[1] + kf[2] * P.bcov[2] + kf[3] * P.bcov[3];
    float cth = fminf(1.0f, fmaxf(-1.0f, kb / (eps * sqrtf(P.bsq))));
    float s2 = 1.0f - cth * cth;
    if (s2 > 0.0f) {
      float sth = sqrtf(s2);
      // nu_s / 1e9 Hz
      float nus9 = (float)((2.0 / 9.0) * (kEE / (2.0 * kPI * kME * kCL)) * 1e-9) * P.B * P.thetae * P.thetae * sth;
      float X = nu9 / nus9;
      float x6 = cbrtf(sqrtf(X));
      float t = x6 * x6 * x6 + 1.887748625f * x6;
      float Gs = t * t * __expf(-x6 * x6);
      // nu alpha_nu = nu j / B_nu = j c^2 expm1(eps/Theta) / (2 h nu^2)
      //            = [sqrt2 pi e^2 n_e nus / (3 c K2) G] c^2 expm1 / (2 h nu^2)
      float em1 = expm1f(eps / P.thetae);
      float pre = (float)(1.4142135623730951 * kPI * kEE * kEE / (3.0 * kCL) * kCL * kCL / (2.0 * kHPL) * 1e-9);
      // units: n_e [cm^-3] * nus9 / nu9^2 carries the 1e9 scalings: nus/nu^2 = 1e-9 nus9/nu9^2
      ana = pre * P.ne * nus9 / (nu9 * nu9) / K2_of_f(m, P.thetae) * Gs * em1;
    }
  }
  c.ana = (W)ana;
  if (m.kappa_on) {
    // kappa population: its absorption integral (FP64 tables) in place of the thermal fit
    c.ana = (W)0;
    if (P.thetae >= m.fthetae_min && P.B > 0.0f && P.bsq > 0.0f) {
      double kb = to_d(K[0]) * P.bcov[0] + to_d(K[1]) * P.bcov[1] + to_d(K[2]) * P.bcov[2] + to_d(K[3]) * P.bcov[3];
      double cth = fmin(1.0, fmax(-1.0, kb / ((double)eps * sqrt((double)P.bsq))));
      double s2 = 1.0 - cth * cth;
      if (s2 > 0.0)
        c.ana = (W)kappa_nu_alpha(m, (double)P.ne, (double)P.thetae, (double)P.B, sqrt(s2), (double)nu9 * 1e9);
    }
  }
  // bremsstrahlung absorption in FP64 (n_e^2 leaves the FP32 range in dense plasma)
  if (m.brems) c.ana = (W)((double)c.ana + brems_nu_alpha((double)P.ne, (double)P.thetae, (double)nu9 * 1e9));
  if (want_s) {
    if (m.kappa_on) {
      c.ans = (W)((double)nu9 * 1e9 * (double)P.ne * kap_hot_lookup(m, (double)P.thetae, (double)eps));
    } else {
      float sh = hot_lookup_f(m, fmaxf(P.thetae, 1e-30f), eps);
      c.ans = (W)(nu9 * P.ne * (sh * 1e9f));
    }
  }
}

// Mixed precision with the coefficient surrogate, split around the network evaluation.
// Part A: plasma state at the new point, the absorption coefficient without its 1/K2 factor, and
// the normalised network inputs (ln Theta_e, ln(nu/nu_c), ln eps).
struct CoefA {
  bool on, emit;
  float thetae, ne, eps, nu9, ana_k2;   // ana = ana_k2 / K2
  float in[3];
};

template <typename S>
__device__ __forceinline__ void coefficients32_a(const DevModel &m, const GeoT<S> &G, const S X[4], const S K[4],
                                                 CoefA &a) {
  constexpr bool kSplit = std::is_same<S, double>::value;   // FP64 geodesic: the split form with the network
  a.on = a.emit = false;
  a.thetae = a.ne = a.eps = a.nu9 = a.ana_k2 = 0.0f;
  a.in[0] = a.in[1] = a.in[2] = 0.0f;
  float pr[8];
  if (!interp_prims<float, S, kSplit>(m, X, pr)) return;
  Plasma<float> P;
  plasma_from_prims<float, S, kSplit>(m, G, pr, P, nullptr, nullptr);
  a.thetae = P.thetae;
  if (!P.on) return;
  float kf[4] = {f32_of<kSplit>(K[0]), f32_of<kSplit>(K[1]), f32_of<kSplit>(K[2]), f32_of<kSplit>(K[3])};
  float eps = -(kf[0] * P.ucov[0] + kf[1] * P.ucov[1] + kf[2] * P.ucov[2] + kf[3] * P.ucov[3]);
  if (!(eps > 0.0f)) return;
  a.on = true;
  a.ne = P.ne;
  a.eps = eps;
  float nu9 = eps * (float)(kME * kCL * kCL / kHPL * 1e-9);
  a.nu9 = nu9;
  float lnK = 0.0f;
  if (P.thetae >= m.fthetae_min && P.B > 0.0f && P.bsq > 0.0f) {
    float kb = kf[0] * P.bcov[0] + kf[1] * P.bcov[1] + kf[2] * P.bcov[2] + kf[3] * P.bcov[3];
    float cth = fminf(1.0f, fmaxf(-1.0f, kb / (eps * sqrtf(P.bsq))));
    float s2 = 1.0f - cth * cth;
    if (s2 > 0.0f) {
      float sth = sqrtf(s2);
      float nuc9 = (float)((2.0 / 9.0) * (kEE / (2.0 * kPI * kME * kCL)) * 1e-9) * P.B * P.thetae * P.thetae;
      float nus9 = nuc9 * sth;
      float Xs = nu9 / nus9;
      float x6 = cbrtf(sqrtf(Xs));
      float t = x6 * x6 * x6 + 1.887748625f * x6;
      float Gs = t * t * __expf(-x6 * x6);
      float em1 = expm1f(eps / P.thetae);
      float pre = (float)(1.4142135623730951 * kPI * kEE * kEE / (3.0 * kCL) * kCL * kCL / (2.0 * kHPL) * 1e-9);
      a.ana_k2 = pre * P.ne * nus9 / (nu9 * nu9) * Gs * em1;
      a.emit = a.ana_k2 > 0.0f;
      lnK = __logf(nu9 / nuc9);
    }
  }
  a.in[0] = fminf(1.0f, fmaxf(-1.0f, __logf(fmaxf(P.thetae, 1e-30f)) * (float)(1.0 / kSurLT1)));
  a.in[1] = fminf(1.0f, fmaxf(-1.0f, lnK * (float)(1.0 / kSurLK1)));
  a.in[2] = fminf(1.0f, fmaxf(-1.0f, (__logf(eps) - (float)(0.5 * (kSurLE0 + kSurLE1))) *
                                             (float)(2.0 / (kSurLE1 - kSurLE0))));
}

// Part B: K2 and sigma_h from the network outputs inside the trained domain (table otherwise).
template <typename W = double>
__device__ __forceinline__ void coefficients32_b(const DevModel &m, const CoefA &a, const float out[3], bool want_s,
                                                 CoefT<W> &c) {
  c.ana = c.ans = (W)0;
  c.thetae = a.thetae;
  if (!a.on) return;
  const float th = a.thetae;
  if (a.emit) {
    float k2 = (th >= (float)kSurThetaK2Min && th <= 1e3f) ? 2.0f * th * th * __expf(out[1]) : K2_of_f(m, th);
    c.ana = (W)(a.ana_k2 / k2);
  }
  if (want_s) {
    bool in_dom = th >= 1e-3f && th <= 1e3f && a.eps >= 1e-12f && a.eps <= 1e6f;
    float sh = in_dom ? (float)kSIGT * __expf(out[0]) : hot_lookup_f(m, fmaxf(th, 1e-30f), a.eps);
    c.ans = (W)(a.nu9 * a.ne * (sh * 1e9f));
  }
}

// ---------------------------------------------------------------- bias (section 2.7)
__device__ __forceinline__ double bias_of(const DevModel &m, double thetae, int nsc) {
  double b;
  if (m.bias_mode == 1) b = m.bias_p0 * (nsc + 1.0) * (nsc + 1.0);
  else if (m.bias_mode == 2) b = m.bias_p0 * thetae * thetae;
  else b = m.bias_p0;
  // min / max on bit patterns: exact for the non-negative operands, and a negative b gives 1 as before
  const double b0 = dmax_nn(1.0, dmin_nn(b, m.bias_max));
  return dmax_nn(1.0, dmin_nn(m.bias_scale * b0, m.bias_max));   // = b0 at scale 1
}

// FP32 form (split precision): the same rule on FP32 copies of the parameters (bias_max beyond the FP32
// range becomes +inf, which bounds nothing, as before)
__device__ __forceinline__ float bias_of_f(const DevModel &m, float thetae, int nsc) {
  float b;
  if (m.bias_mode == 1) b = m.fbias_p0 * (nsc + 1.0f) * (nsc + 1.0f);
  else if (m.bias_mode == 2) b = m.fbias_p0 * thetae * thetae;
  else b = m.fbias_p0;
  const float b0 = fmaxf(1.0f, fminf(b, m.fbias_max));
  return fmaxf(1.0f, fminf(m.fbias_scale * b0, m.fbias_max));
}

// ---------------------------------------------------------------- tetrads (sections 2.1, 2.7)
__device__ __forceinline__ void gs_step(const Geo &G, double v[4], const double e[4], double sign) {
  double d = dot(G, v, e);
  // sign = +1 for the timelike e0 (e0.e0 = -1), -1 for spacelike unit vectors
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] += sign * d * e[q];
}

__device__ __forceinline__ bool normalize_space(const Geo &G, double v[4]) {
  double n2 = dot(G, v, v);
  if (!(n2 > 1e-30)) return false;
  double in = 1.0 / sqrt(n2);
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] *= in;
  return true;
}

__device__ __forceinline__ double gdiag(const Geo &G, int k) {
  return (k == 1) ? G.g11 : ((k == 2) ? G.g22 : G.g33);
}

// Emission tetrad: e0 = u, e3 = b/|b|, e1 and e2 from the coordinate directions keeping the
// largest part after projection (first index on ties).
static __device__ void tetrad_emission(const Geo &G, const double u[4], const double b[4], double bsq, double e[4][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) e[0][q] = u[q];
  double ib = 1.0 / sqrt(bsq);
#pragma unroll
  for (int q = 0; q < 4; ++q) e[3][q] = b[q] * ib;
  double best = -1.0;
  double t1[4] = {0, 0, 0, 0};
  int pick = 1;
  for (int k = 1; k < 4; ++k) {
    double t[4] = {0, 0, 0, 0};
    t[k] = 1.0;
    gs_step(G, t, e[0], 1.0);
    gs_step(G, t, e[3], -1.0);
    double fr = dot(G, t, t) / gdiag(G, k);
    if (fr > best) {
      best = fr;
      pick = k;
#pragma unroll
      for (int q = 0; q < 4; ++q) t1[q] = t[q];
    }
  }
  normalize_space(G, t1);
#pragma unroll
  for (int q = 0; q < 4; ++q) e[1][q] = t1[q];
  best = -1.0;
  double t2[4] = {0, 0, 0, 0};
  for (int k = 1; k < 4; ++k) {
    if (k == pick) continue;
    double t[4] = {0, 0, 0, 0};
    t[k] = 1.0;
    gs_step(G, t, e[0], 1.0);
    gs_step(G, t, e[3], -1.0);
    gs_step(G, t, e[1], -1.0);
    double fr = dot(G, t, t) / gdiag(G, k);
    if (fr > best) {
      best = fr;
#pragma unroll
      for (int q = 0; q < 4; ++q) t2[q] = t[q];
    }
  }
  normalize_space(G, t2);
#pragma unroll
  for (int q = 0; q < 4; ++q) e[2][q] = t2[q];
}

// Scattering tetrad: e0 = u, e1..e3 from the x1, x2, x3 directions by Gram-Schmidt.
static __device__ void tetrad_scatter(const Geo &G, const double u[4], double e[4][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) e[0][q] = u[q];
  for (int k = 1; k < 4; ++k) {
    double t[4] = {0, 0, 0, 0};
    t[k] = 1.0;
    gs_step(G, t, e[0], 1.0);
    for (int p = 1; p < k; ++p) gs_step(G, t, e[p], -1.0);
    normalize_space(G, t);
#pragma unroll
    for (int q = 0; q < 4; ++q) e[k][q] = t[q];
  }
}

// ---------------------------------------------------------------- Compton kinematics (section 2.7)
// The kinematics are written once for the real type R: double in the FP64 and double-float forms,
// float in the split precision form.  Uniforms come from the same counter-based stream in both.
__device__ __forceinline__ double r_log(double x) { return log(x); }
__device__ __forceinline__ float r_log(float x) { return logf(x); }
__device__ __forceinline__ double r_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float r_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float r_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double r_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float r_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double r_cospi(double x) { return cospi(x); }
__device__ __forceinline__ float r_cospi(float x) { return cospif(x); }
__device__ __forceinline__ void r_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void r_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
template <typename R>
__device__ __forceinline__ R rng_r(Rng &s, uint64_t seed) {
  return (R)rng_u(s, seed);
}

template <typename R>
__device__ __forceinline__ R sigma_kn_ratio(R e) {
  if (e < (R)1e-3) return (R)1 - (R)2 * e;
  R e2 = e * e, o2 = (R)1 + (R)2 * e;
  return (R)0.75 / e2 *
         ((R)2 + e2 * ((R)1 + e) / (o2 * o2) + (e2 - (R)2 * e - (R)2) / ((R)2 * e) * r_log1p((R)2 * e));
}

constexpr int kMaxTry = 10000;

// Maxwell-Juettner Lorentz factor: Sobol's method (Pozdnyakov, Sobol & Sunyaev 1983) for
// Theta >= 0.25; below, rejection from the Gamma(3/2, 5/2, 7/2) mixture bounding
// sqrt(t) (1+t) sqrt(t+2) e^{-t/Theta}, t = gamma - 1.
template <typename R>
static __device__ R sample_mj(R th, Rng &s, uint64_t seed) {
  if (th >= (R)0.25) {
    for (int it = 0; it < kMaxTry; ++it) {
      R u1 = rng_r<R>(s, seed), u2 = rng_r<R>(s, seed), u3 = rng_r<R>(s, seed), u4 = rng_r<R>(s, seed);
      R p = -th * r_log(u1 * u2 * u3);
      R eta = p - th * r_log(u4);
      if (eta * eta - p * p > (R)1 || it == kMaxTry - 1) return r_sqrt((R)1 + p * p);
    }
  }
  R c1 = (R)0.886226925452758 * r_pow(th, (R)1.5);
  R c2 = (R)(1.25 * 1.329340388179137) * r_pow(th, (R)2.5);
  R c3 = (R)(0.25 * 3.323350970447843) * r_pow(th, (R)3.5);
  R ct = c1 + c2 + c3;
  R t = 0;
  for (int it = 0; it < kMaxTry; ++it) {
    R uc = rng_r<R>(s, seed) * ct;
    int k = (uc < c1) ? 1 : ((uc < c1 + c2) ? 2 : 3);
    R prod = 1;
    for (int i = 0; i < k; ++i) prod *= rng_r<R>(s, seed);
    R ua = rng_r<R>(s, seed), ub = rng_r<R>(s, seed);
    R z = r_sqrt((R)-2 * r_log(ua)) * r_cospi((R)2 * ub);
    t = th * (-r_log(prod) + (R)0.5 * z * z);
    R acc = ((R)1 + t) * r_sqrt(t + (R)2) / ((R)1.4142135623730951 * ((R)1 + (R)1.25 * t + (R)0.25 * t * t));
    if (rng_r<R>(s, seed) < acc) break;
  }
  return (R)1 + t;
}

// Gamma(a) variate (Marsaglia & Tsang 2000), normals by Box-Muller from two uniforms; a < 1 through
// Gamma(a + 1) U^(1/a), the Gamma(a + 1) drawn first.
template <typename R>
static __device__ R gamma_mt(R a, Rng &s, uint64_t seed) {
  R boost = -1;
  if (a < (R)1) {
    boost = (R)1 / a;
    a += (R)1;
  }
  const R d = a - (R)1 / (R)3, c = r_rsqrt((R)9 * d);
  R g = d;
  for (int it = 0; it < kMaxTry; ++it) {
    const R u1 = rng_r<R>(s, seed), u2 = rng_r<R>(s, seed);
    const R x = r_sqrt((R)-2 * r_log((R)1 - u1)) * r_cospi((R)2 * u2);
    R v = (R)1 + c * x;
    if (v <= (R)0) continue;
    v = v * v * v;
    const R u = rng_r<R>(s, seed);
    if (u < (R)1 - (R)0.0331 * (x * x) * (x * x) || r_log(u) < (R)0.5 * x * x + d * ((R)1 - v + r_log(v))) {
      g = d * v;
      break;
    }
  }
  if (boost > (R)0) g *= r_pow(rng_r<R>(s, seed), boost);
  return g;
}

// Lorentz factor of a kappa electron: u = gamma - 1 has density (1 + u) sqrt(u (2 + u)) (1 + u/kw)^-(kappa+1),
// kw = kappa w.  Rejection from a three-term envelope, each term u^(a-1) (1 + u/kw)^-(kappa+1) drawn as
// u = kw G_a / G_(kappa+1-a): for w < 1 the envelope sqrt2 u^1/2 (1 + u)^2 (a = 3/2, 5/2, 7/2; acceptance
// sqrt(1 + u/2) / (1 + u)), otherwise (1 + u)^2 (a = 1, 2, 3; acceptance sqrt(1 - (1 + u)^-2)).  Term masses
// follow from B(a + 1, b - 1) / B(a, b) = a / (b - 1).
template <typename R>
static __device__ R sample_kappa(R kappa, R w, Rng &s, uint64_t seed, int &rejcap) {
  const R kw = kappa * w;
  const bool low = w < (R)1;
  const R a1 = low ? (R)1.5 : (R)1, b1 = kappa + (R)1 - a1;
  const R r2 = (R)2 * kw * a1 / (b1 - (R)1);
  const R r3 = r2 * ((R)0.5 * kw * (a1 + (R)1) / (b1 - (R)2));
  const R tot = (R)1 + r2 + r3;
  for (int it = 0; it < kMaxTry; ++it) {
    const R uc = rng_r<R>(s, seed) * tot;
    const R a = a1 + (uc < (R)1 ? (R)0 : (uc < (R)1 + r2 ? (R)1 : (R)2));
    const R ga = gamma_mt(a, s, seed);
    const R gb = gamma_mt(kappa + (R)1 - a, s, seed);
    const R u = kw * (ga / gb);
    const R acc = low ? r_sqrt((R)1 + (R)0.5 * u) / ((R)1 + u) : r_sqrt((R)1 - (R)1 / (((R)1 + u) * ((R)1 + u)));
    if (rng_r<R>(s, seed) < acc) return (R)1 + u;
  }
  rejcap++;
  return (R)1 + kw;
}

template <typename R>
__device__ __forceinline__ void perp_basis(const R n[3], R e1[3], R e2[3]) {
  R a0 = 1, a1 = 0;
  if (fabs(n[0]) >= (R)0.6) { a0 = 0; a1 = 1; }
  R d = a0 * n[0] + a1 * n[1];
  e1[0] = a0 - d * n[0];
  e1[1] = a1 - d * n[1];
  e1[2] = -d * n[2];
  R il = (R)1 / r_sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  e1[0] *= il; e1[1] *= il; e1[2] *= il;
  e2[0] = n[1] * e1[2] - n[2] * e1[1];
  e2[1] = n[2] * e1[0] - n[0] * e1[2];
  e2[2] = n[0] * e1[1] - n[1] * e1[0];
}

template <typename R>
__device__ __forceinline__ void boost3(R E, const R p[3], R beta, const R v[3], R &Eo, R po[3]) {
  R gam = (R)1 / r_sqrt((R)1 - beta * beta);
  R pv = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
  Eo = gam * (E - beta * pv);
  R ppar = gam * (pv - beta * E);
  po[0] = p[0] + (ppar - pv) * v[0];
  po[1] = p[1] + (ppar - pv) * v[1];
  po[2] = p[2] + (ppar - pv) * v[2];
}

// Scattered photon in the plasma frame for incoming energy eps along unit n; draws in the order
// [gamma (MJ), mu_e, accept]*, phi_e, [cos, accept]*, phi.
// kappa > 0: kappa-distributed electrons of temperature-like parameter w = th (kappa - 3) / kappa.
template <typename R>
static __device__ void compton_fluid(R kappa, R th, R eps, const R n[3], Rng &s, uint64_t seed, R &eo, R dir[3],
                                     int &rejcap) {
  R gam = 1, mue = 0, beta = 0;
  int it;
  for (it = 0; it < kMaxTry; ++it) {
    gam = kappa > (R)0 ? sample_kappa(kappa, th * (kappa - (R)3) / kappa, s, seed, rejcap) : sample_mj(th, s, seed);
    mue = (R)2 * rng_r<R>(s, seed) - (R)1;
    beta = r_sqrt((R)1 - (R)1 / (gam * gam));
    R om = (R)1 - beta * mue;
    R acc = om * sigma_kn_ratio(eps * gam * om) * (R)0.5;
    if (rng_r<R>(s, seed) < acc) break;
  }
  if (it == kMaxTry) rejcap++;
  R phie = (R)2 * rng_r<R>(s, seed);   // in units of pi
  R e1[3], e2[3];
  perp_basis(n, e1, e2);
  R se = r_sqrt(fmax((R)0, (R)1 - mue * mue));
  R sp, cp;
  r_sincospi(phie, &sp, &cp);
  R v[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = mue * n[i] + se * (cp * e1[i] + sp * e2[i]);
  R pin[3] = {eps * n[0], eps * n[1], eps * n[2]};
  R ee, pe[3];
  boost3(eps, pin, beta, v, ee, pe);
  R il = (R)1 / r_sqrt(pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]);
  R ne[3] = {pe[0] * il, pe[1] * il, pe[2] * il};
  R ct = 1, ep = ee;
  for (it = 0; it < kMaxTry; ++it) {
    ct = (R)2 * rng_r<R>(s, seed) - (R)1;
    ep = ee / ((R)1 + ee * ((R)1 - ct));
    R P;
    if (ee < (R)1e-4) {
      P = (R)0.5 * ((R)1 + ct * ct);
    } else {
      R r = ep / ee;
      P = (R)0.5 * r * r * (r + (R)1 / r - ((R)1 - ct * ct));
    }
    if (rng_r<R>(s, seed) < P) break;
  }
  if (it == kMaxTry) rejcap++;
  R phi = (R)2 * rng_r<R>(s, seed);
  R f1[3], f2[3];
  perp_basis(ne, f1, f2);
  R st = r_sqrt(fmax((R)0, (R)1 - ct * ct));
  r_sincospi(phi, &sp, &cp);
  R pp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) pp[i] = ep * (ct * ne[i] + st * (cp * f1[i] + sp * f2[i]));
  R Ef, pf[3];
  boost3(ep, pp, -beta, v, Ef, pf);
  eo = Ef;
  dir[0] = pf[0];
  dir[1] = pf[1];
  dir[2] = pf[2];
}

}  // namespace mcgb
