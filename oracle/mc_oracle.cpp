// mc_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, FP64 CPU oracle for the Monte Carlo radiative-transfer hot path of
// GPUmonty (arXiv 2602.13198).  Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark may load this library; the product path never does.
// It shares no source with the CUDA path.  Every function states the passage of the
// paper it follows; where the paper is silent the documented reading is used.
//
// Pins (tests/test_oracle_*.py): Philox known-answer vectors, Gauss-Legendre moments,
// libstdc++/scipy Bessel functions, numerical Klein-Nishina integrals, geodesic
// invariants (null condition, E, L, Carter Q), the Schwarzschild orbit equation,
// sampler histograms against their densities, the thermal Thomson-limit energy gain,
// and the analytic synchrotron sphere; for the later additions, the bremsstrahlung fits'
// continuity and classical limit, the kappa tables against scipy quadratures and their thermal
// limits, and the kappa sampler against its density.  The fluid state, the tetrads and the fluid
// interpolation are pinned at random points of spinning tori (both signs of the spin): u.u = -1
// and u's projection orthogonal to the normal observer equal to U^i; b^mu against an independent
// linear solve of b.u = 0, b^i u^t - b^t u^i = B^i; Theta_e at the beta -> infinity, beta = 1 and
// beta -> 0 points of the temperature model; e_a.e_b = eta_ab with e_0 = u and e_3 = b/|b|; and a
// primitive field linear in (x1, x2, x3) reproduced exactly, clamped and periodic as read.  The
// emission on those tori (weights, zone counts, frequency sampling) is pinned by its sums: the
// birth weights against the emitted photon number and weight x h nu against the emitted power,
// both computed from the zone volumes and the synchrotron fit outside the oracle.  No function is
// "parity unpinned".  The tori's recorded spectra, which add the transport, are built from these
// pinned parts and compared between the oracle and the CUDA path.
//
// Build: g++ -O2 -std=c++17 -fopenmp -shared -fPIC mc_oracle.cpp -o libmc_oracle.so

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <mutex>
#include <map>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- constants (CGS, CODATA 2018)
const double EE = 4.803204712570263e-10;   // electron charge [statC]
const double ME = 9.1093837015e-28;        // electron mass [g]
const double MP = 1.67262192369e-24;       // proton mass [g]
const double CL = 2.99792458e10;           // speed of light [cm/s]
const double HPL = 6.62607015e-27;         // Planck constant [erg s]
const double SIGMA_T = 6.6524587321e-25;   // Thomson cross-section [cm^2]
const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- Philox4x32-10 (Salmon et al. 2011)
// Counter-based generator: 10 rounds of the Philox S-box with two 32x32->64 multiplies,
// key schedule bumped by the Weyl constants between rounds.
void philox4x32_10(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// A per-superphoton random stream: key = Philox key (the run seed), stream id in the
// high counter words, draw index n in the low word.  Draw n uses block n/2, half n%2.
struct Stream {
  uint64_t seed;
  uint64_t id;
  uint32_t n;
};

double uniform(Stream &s) {
  uint32_t ctr[4] = {s.n >> 1, 0u, (uint32_t)s.id, (uint32_t)(s.id >> 32)};
  uint32_t key[2] = {(uint32_t)s.seed, (uint32_t)(s.seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  uint32_t a = (s.n & 1u) ? o[2] : o[0];
  uint32_t b = (s.n & 1u) ? o[3] : o[1];
  s.n++;
  uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
  return ((double)m + 0.5) * (1.0 / 9007199254740992.0);   // (m + 1/2) 2^-53, in (0,1)
}

// splitmix64 output function (Steele, Lea & Flood 2014): the stream id of the child
// created at a parent's e-th scattering event is splitmix64(parent_id + (e+1) * golden).
uint64_t splitmix64_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
uint64_t child_stream(uint64_t parent, uint32_t ev) {
  return splitmix64_out(parent + 0x9E3779B97F4A7C15ull * (uint64_t)(ev + 1u));
}
const uint64_t ZONE_STREAM_TAG = 0xC000000000000000ull;

// ---------------------------------------------------------------- Gauss-Legendre rule
// Newton iteration on P_n(x) from the three-term recurrence (textbook construction).
void gauss_legendre(int n, double a, double b, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(PI * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      pp = n * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = 0.0;
    for (int j = 1; j <= n; ++j) {
      double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
    }
    pp = n * (z * p0 - p1) / (z * z - 1.0);
    double wt = 2.0 / ((1.0 - z * z) * pp * pp);
    double h = 0.5 * (b - a), m = 0.5 * (b + a);
    x[i] = m - h * z;
    x[n - 1 - i] = m + h * z;
    w[i] = h * wt;
    w[n - 1 - i] = h * wt;
  }
}

}  // namespace

extern "C" {

// Parameters of one model (the problem statement: metric, units, frequency range,
// bias, bins).  Layout mirrored by the ctypes Structure in oracle/__init__.py.
struct or_params {
  double a;            // black-hole spin a/M
  double mass;         // 1: Kerr-Schild (M=1 in code units); 0: flat spacetime
  double hslope;       // MKS polar refinement, theta = pi x2 + (1-h)/2 sin(2 pi x2)
  double L_unit;       // code length [cm]
  double M_unit;       // mass unit [g]; rho_unit = M_unit / L_unit^3
  double R_high, R_low, gam;   // electron temperature model, adiabatic index
  double thetae_min, thetae_max;
  double nu_min, nu_max;       // emission band [Hz]
  double w_min;                // weight floor
  double n_s;                  // target number of superphotons N_s
  double eps_geo;              // step-size control
  double verlet_tol;           // relative error bound of the Verlet predictor loop
  double r_record;             // record radius [code units]
  double dh;                   // capture at r <= r_h (1 + dh)
  double bias_p0;              // bias parameter (meaning set by bias_mode)
  double lnu_lo, lnu_hi;       // spectrum range, log10(nu / Hz)
  double roulette_w, roulette_p;
  double bias_max;             // upper bound on b (reading: any b >= 1 keeps the estimate unbiased)
  double kappa;                // > 3: kappa-distributed electrons for synchrotron (reading), 0: thermal
  double bias_target;          // > 0: per-generation bias tuning (reading), 0: off
  int64_t max_steps;
  int32_t n_nu;                // weight-table nodes
  int32_t verlet_maxit;
  int32_t bias_mode;           // 0: b = max(1,p0); 1: b = max(1, p0 (n_sc+1)^2); 2: b = max(1, p0 Theta_e^2)
  int32_t n_sc_max;            // maximum scattering generation
  int32_t n_bins, n_incl;
  int32_t k2_mode;             // 0: exact K2(1/Theta); 1: K2 ~ 2 Theta^2
  int32_t scatter;             // 0: Compton scattering off
  int32_t brems;               // 1: thermal bremsstrahlung emission and absorption (reading)
};

struct or_grid {
  int32_t n1, n2, n3, pad;
  double x1_0, dx1, x2_0, dx2, x3_0, dx3;
  const double *prim;          // [8][n1*n2*n3]: rho, u, B1, B2, B3, U1, U2, U3; zone = (i*n2 + j)*n3 + k
};

struct or_stats {
  int64_t n_emit, n_child, n_rec, n_abs, n_capt, n_maxst;
  int64_t n_steps, n_iters, n_nonconv, n_roul_surv, n_rej_cap, n_events;
};

struct or_log {
  uint64_t id;
  int32_t gen, status;         // status: 1 recorded, 2 absorbed, 3 captured, 4 max steps
  double X[4], K[4];
  double w;
  int64_t nsteps;
  int32_t nev, pad;
};

}  // extern "C"

namespace {

// ---------------------------------------------------------------- metric (section 2.4)
// Kerr-Schild metric (mass 1 or 0) in modified Kerr-Schild internal coordinates
// x = (t, x1 = ln r, x2, x3 = phi), theta(x2) = pi x2 + (1-h)/2 sin(2 pi x2).
// Written once as a template so that it can be evaluated on dual numbers; the
// oracle obtains metric derivatives by forward-mode differentiation (exact up to
// rounding) and Christoffel symbols from their textbook definition.
struct D {
  double v, d1, d2;   // value, d/dx1, d/dx2
};
inline D operator+(D a, D b) { return {a.v + b.v, a.d1 + b.d1, a.d2 + b.d2}; }
inline D operator-(D a, D b) { return {a.v - b.v, a.d1 - b.d1, a.d2 - b.d2}; }
inline D operator*(D a, D b) { return {a.v * b.v, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2}; }
inline D operator/(D a, D b) {
  double iv = 1.0 / b.v;
  return {a.v * iv, (a.d1 * b.v - a.v * b.d1) * iv * iv, (a.d2 * b.v - a.v * b.d2) * iv * iv};
}
inline D operator*(double s, D a) { return {s * a.v, s * a.d1, s * a.d2}; }
inline D operator+(double s, D a) { return {s + a.v, a.d1, a.d2}; }
inline D operator-(double s, D a) { return {s - a.v, -a.d1, -a.d2}; }
inline D operator-(D a) { return {-a.v, -a.d1, -a.d2}; }
inline D Dexp(D a) { double e = std::exp(a.v); return {e, e * a.d1, e * a.d2}; }
inline D Dsin(D a) { double s = std::sin(a.v), c = std::cos(a.v); return {s, c * a.d1, c * a.d2}; }
inline D Dcos(D a) { double s = std::sin(a.v), c = std::cos(a.v); return {c, -s * a.d1, -s * a.d2}; }
inline double Dexp(double a) { return std::exp(a); }
inline double Dsin(double a) { return std::sin(a); }
inline double Dcos(double a) { return std::cos(a); }
template <class T> inline T cst(double v);
template <> inline double cst<double>(double v) { return v; }
template <> inline D cst<D>(double v) { return {v, 0.0, 0.0}; }

template <class T>
void metric_mks(const or_params &P, T x1, T x2, T g[4][4]) {
  const double a = P.a, m = P.mass, h = P.hslope;
  T r = Dexp(x1);
  T th = PI * x2 + (0.5 * (1.0 - h)) * Dsin((2.0 * PI) * x2);
  T dth = PI * (1.0 + (1.0 - h) * Dcos((2.0 * PI) * x2));
  T s = Dsin(th), c = Dcos(th);
  T s2 = s * s;
  T sig = r * r + (a * a) * (c * c);
  T f = (2.0 * m) * r / sig;
  // Kerr-Schild components in (t, r, theta, phi)
  T gtt = -(1.0 - f);
  T gtr = f;
  T gtp = -(a * (f * s2));
  T grr = 1.0 + f;
  T grp = -(a * (s2 * (1.0 + f)));
  T ghh = sig;
  T gpp = s2 * (sig + (a * a) * (s2 * (1.0 + f)));
  // Jacobian diag(1, dr/dx1 = r, dtheta/dx2, 1)
  T z = cst<T>(0.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) g[i][j] = z;
  g[0][0] = gtt;
  g[0][1] = g[1][0] = gtr * r;
  g[0][3] = g[3][0] = gtp;
  g[1][1] = grr * (r * r);
  g[1][3] = g[3][1] = grp * r;
  g[2][2] = ghh * (dth * dth);
  g[3][3] = gpp;
}

void gcov_at(const or_params &P, const double X[4], double g[4][4]) { metric_mks<double>(P, X[1], X[2], g); }

// Gauss-Jordan inverse with partial pivoting; returns the determinant.
double invert4(const double A[4][4], double Ai[4][4]) {
  double M[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      M[i][j] = A[i][j];
      M[i][j + 4] = (i == j) ? 1.0 : 0.0;
    }
  double det = 1.0;
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
    if (p != c) {
      for (int j = 0; j < 8; ++j) std::swap(M[p][j], M[c][j]);
      det = -det;
    }
    double piv = M[c][c];
    det *= piv;
    for (int j = 0; j < 8; ++j) M[c][j] /= piv;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double f = M[r][c];
      for (int j = 0; j < 8; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ai[i][j] = M[i][j + 4];
  return det;
}

// Christoffel symbols of the second kind (section 2.4, eq. geodesic-system):
// Gamma^mu_{ab} = 1/2 g^{mu n} (d_a g_{nb} + d_b g_{na} - d_n g_{ab}).
void christoffel(const or_params &P, const double X[4], double G[4][4][4]) {
  D x1 = {X[1], 1.0, 0.0}, x2 = {X[2], 0.0, 1.0};
  D gd[4][4];
  metric_mks<D>(P, x1, x2, gd);
  double g[4][4], gi[4][4], dg[4][4][4];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      g[m][n] = gd[m][n].v;
      dg[0][m][n] = 0.0;
      dg[1][m][n] = gd[m][n].d1;
      dg[2][m][n] = gd[m][n].d2;
      dg[3][m][n] = 0.0;
    }
  invert4(g, gi);
  for (int mu = 0; mu < 4; ++mu)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double s = 0.0;
        for (int n = 0; n < 4; ++n) s += gi[mu][n] * (dg[a][n][b] + dg[b][n][a] - dg[n][a][b]);
        G[mu][a][b] = 0.5 * s;
      }
}

// dk^mu/dlambda = -Gamma^mu_{ab} k^a k^b
void accel(const double G[4][4][4], const double K[4], double A[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    double s = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) s += G[mu][a][b] * K[a] * K[b];
    A[mu] = -s;
  }
}

double radius(const double X[4]) { return std::exp(X[1]); }
double theta_of(const or_params &P, double x2) {
  return PI * x2 + 0.5 * (1.0 - P.hslope) * std::sin(2.0 * PI * x2);
}

// Step size (the paper gives none; reading): the affine step that moves each internal
// coordinate by at most eps_geo of its natural scale: 1 for x1 = ln r and x3 = phi,
// the distance to the nearer pole for x2.
double stepsize(const or_params &P, const double X[4], const double K[4]) {
  const double SMALL = 1e-40;
  double x2n = std::min(std::fabs(X[2]), std::fabs(1.0 - X[2]));
  double d1 = P.eps_geo / (std::fabs(K[1]) + SMALL);
  double d2 = P.eps_geo * x2n / (std::fabs(K[2]) + SMALL);
  double d3 = P.eps_geo / (std::fabs(K[3]) + SMALL);
  return 1.0 / (1.0 / d1 + 1.0 / d2 + 1.0 / d3);
}

// Iterated velocity Verlet (section 2.4): position update with the acceleration at
// step n, predicted wavevector, acceleration at x_{n+1} with the predicted wavevector,
// corrected wavevector; the corrected value becomes the next prediction until the
// L1 relative change is below verlet_tol (or verlet_maxit passes).  The last
// acceleration evaluated is carried to the next step as (dk/dlambda)_n.
int verlet_step(const or_params &P, double X[4], double K[4], double A[4], double dl, bool *conv) {
  double Xn[4], Kp[4], Kn[4], An[4];
  for (int m = 0; m < 4; ++m) {
    Xn[m] = X[m] + K[m] * dl + 0.5 * A[m] * dl * dl;
    Kp[m] = K[m] + A[m] * dl;
  }
  double G[4][4][4];
  christoffel(P, Xn, G);
  int it = 0;
  *conv = false;
  while (true) {
    accel(G, Kp, An);
    double num = 0.0, den = 0.0;
    for (int m = 0; m < 4; ++m) {
      Kn[m] = K[m] + 0.5 * (A[m] + An[m]) * dl;
      num += std::fabs(Kn[m] - Kp[m]);
      den += std::fabs(Kn[m]);
    }
    ++it;
    for (int m = 0; m < 4; ++m) Kp[m] = Kn[m];
    if (num < P.verlet_tol * den) { *conv = true; break; }
    if (it >= P.verlet_maxit) break;
  }
  for (int m = 0; m < 4; ++m) {
    X[m] = Xn[m];
    K[m] = Kn[m];
    A[m] = An[m];
  }
  return it;
}

// ---------------------------------------------------------------- plasma (sections 2.2, 2.5)
struct Fluid {
  bool plasma;
  double ne, thetae, B;
  double ucon[4], ucov[4], bcon[4], bcov[4], bsq;
};

struct Units {
  double rho, U, B, Ne, C;   // rho_unit, U_unit, B_unit, n_e per code rho, C = h L / (m_e c^2)
};

Units make_units(const or_params &P) {
  Units u;
  u.rho = P.M_unit / (P.L_unit * P.L_unit * P.L_unit);
  u.U = u.rho * CL * CL;
  u.B = CL * std::sqrt(4.0 * PI * u.rho);
  u.Ne = u.rho / (MP + ME);
  u.C = HPL * P.L_unit / (ME * CL * CL);
  return u;
}

// Derived fluid-frame quantities from primitives (rho, u, B^i, U^i) at a point with
// metric g: 4-velocity from the normal-observer velocity U^i, magnetic 4-vector b,
// n_e, |B| in Gauss and Theta_e from the R_high/R_low temperature-ratio model.
void fluid_from_prims(const or_params &P, const Units &un, const double pr[8], const double g[4][4], Fluid &F) {
  double gi[4][4];
  invert4(g, gi);
  double rho = pr[0], uu = pr[1];
  double Bp[4] = {0.0, pr[2], pr[3], pr[4]};
  double Ut[4] = {0.0, pr[5], pr[6], pr[7]};
  double alpha = 1.0 / std::sqrt(-gi[0][0]);
  double q = 0.0;
  for (int i = 1; i < 4; ++i)
    for (int j = 1; j < 4; ++j) q += g[i][j] * Ut[i] * Ut[j];
  double gamma = std::sqrt(1.0 + q);
  F.ucon[0] = gamma / alpha;
  for (int i = 1; i < 4; ++i) F.ucon[i] = Ut[i] - gamma * alpha * gi[0][i];
  for (int m = 0; m < 4; ++m) {
    F.ucov[m] = 0.0;
    for (int n = 0; n < 4; ++n) F.ucov[m] += g[m][n] * F.ucon[n];
  }
  F.bcon[0] = 0.0;
  for (int i = 1; i < 4; ++i) F.bcon[0] += Bp[i] * F.ucov[i];
  for (int i = 1; i < 4; ++i) F.bcon[i] = (Bp[i] + F.bcon[0] * F.ucon[i]) / F.ucon[0];
  F.bsq = 0.0;
  for (int m = 0; m < 4; ++m) {
    F.bcov[m] = 0.0;
    for (int n = 0; n < 4; ++n) F.bcov[m] += g[m][n] * F.bcon[n];
    F.bsq += F.bcon[m] * F.bcov[m];
  }
  F.ne = (rho > 0.0) ? rho * un.Ne : 0.0;
  F.B = std::sqrt(std::max(F.bsq, 0.0)) * un.B;
  if (rho > 0.0 && uu > 0.0) {
    double trat;
    if (F.bsq > 0.0) {
      double beta = uu * (P.gam - 1.0) / (0.5 * F.bsq);
      double b2 = beta * beta;
      trat = P.R_high * b2 / (1.0 + b2) + P.R_low / (1.0 + b2);
    } else {
      trat = P.R_high;
    }
    F.thetae = (MP / ME) * (P.gam - 1.0) * uu / rho / (1.0 + trat);
    F.thetae = std::min(F.thetae, P.thetae_max);
  } else {
    F.thetae = 0.0;
  }
  F.plasma = F.ne > 0.0;
}

// Fluid at an arbitrary point (reading: primitives interpolated linearly in internal
// coordinates between zone centres, clamped to the edge zones in x1 and x2, periodic
// in x3; no plasma outside the radial extent of the grid).
struct Model;
void fluid_at(const Model &M, const double X[4], const double g[4][4], Fluid &F, bool clamp_radial = false);

// Synchrotron emissivity, eq. emissivity (Leung et al. 2011 fit), with
// nu_s = (2/9) (e B / 2 pi m_e c) Theta_e^2 sin(theta).
double K2_of(const or_params &P, double thetae) {
  if (P.k2_mode == 1) return 2.0 * thetae * thetae;   // large-temperature form, section 2.2
  return std::cyl_bessel_k(2.0, 1.0 / thetae);
}

// Gauss-Legendre rule on [a, b] with n nodes.
struct GL {
  int n;
  std::vector<double> x, w;
  GL(int n_, double a, double b) : n(n_), x(n_), w(n_) { gauss_legendre(n, a, b, x.data(), w.data()); }
};

// ---------------------------------------------------------------- kappa electrons (future work in section 6)
// Synchrotron emission and absorption of electrons with the kappa distribution
//   f(gamma) = N gamma (gamma^2 - 1)^1/2 (1 + (gamma - 1) / (kappa w))^-(kappa + 1),  w = Theta_e (kappa - 3) / kappa,
// from the single-electron spectrum in the ultrarelativistic limit (Rybicki & Lightman ch. 6):
//   j_nu = (sqrt3 e^3 n_e B sin / (4 pi m_e c^2)) J(X, w),       J = int f F(2X / 3 gamma^2) dgamma,
//   alpha_nu = (c^2 / 8 pi nu^2) (sqrt3 e^3 n_e B sin / (m_e c^2)^2) A(X, w),
//   A = - int F(2X / 3 gamma^2) gamma^2 d/dgamma(f / gamma^2) dgamma,
// X = nu / (nu_B sin), nu_B = e B / (2 pi m_e c), F(x) = x int_x^inf K_5/3 the synchrotron function; and
// int dOmega j_nu = 4 pi (sqrt3 e^3 n_e B / (4 pi m_e c^2)) I(nu / nu_B, w), I(Y, w) = int_0^1 sin J(Y / sin, w) dmu.
// ln J, ln A and ln I are tabulated on the grid below and interpolated bilinearly (reading).  The
// oracle computes F from the library Bessel function K_5/3 and the node integrals over
// t = ln(gamma - 1) by Gauss-Legendre panels.
const int KAP_NX = 601, KAP_NW = 61;
const double KAP_LX0 = -9.210340371976184, KAP_LX1 = 36.841361487904734;   // ln X in [1e-4, 1e16]
const double KAP_LW0 = -6.907755278982137, KAP_LW1 = 6.907755278982137;    // ln w in [1e-3, 1e3]
const double KAP_FLOOR = -700.0;

// synchrotron function by its definition (library K_5/3; t = x e^s, Gauss-Legendre panels in s on
// [0, ln(1 + 60 / x)], which resolves the t^-5/3 growth of K_5/3 near t = x)
double F_sync_direct(double x) {
  static const GL g(48, 0.0, 1.0);
  const double S = std::log1p(60.0 / x);
  const int np = std::max(8, (int)std::ceil(S / 0.125));
  const double h = S / np;
  double s = 0.0;
  for (int k = 0; k < np; ++k)
    for (int i = 0; i < g.n; ++i) {
      const double t = x * std::exp((k + g.x[i]) * h);
      s += g.w[i] * h * t * std::cyl_bessel_k(5.0 / 3.0, t);
    }
  return x * s;
}

struct KappaTables {
  double kappa = 0.0;
  std::vector<double> lnF;                 // ln F on ln x in [-30, ln 200], 6001 nodes (cubic)
  std::vector<double> lnJ, lnA, lnI;       // [KAP_NX][KAP_NW]
  double F(double x) const {
    const double l0 = -30.0, l1 = std::log(200.0);
    if (x >= 200.0) return 0.0;
    double lx = std::log(x);
    if (lx <= l0) return std::exp(lnF[0] + (lx - l0) / 3.0);   // F ~ x^1/3 below
    double f = (lx - l0) / (l1 - l0) * 6000.0;
    int i = std::max(1, std::min((int)std::floor(f), 6000 - 2));
    double u = f - i;
    double y0 = lnF[i - 1], y1 = lnF[i], y2 = lnF[i + 1], y3 = lnF[i + 2];
    double v = -y0 * u * (u - 1) * (u - 2) / 6.0 + y1 * (u + 1) * (u - 1) * (u - 2) / 2.0 -
               y2 * (u + 1) * u * (u - 2) / 2.0 + y3 * (u + 1) * u * (u - 1) / 6.0;
    return std::exp(v);
  }
};

double kap_interp(const std::vector<double> &t, double lx, double lw) {
  double fx = (lx - KAP_LX0) / (KAP_LX1 - KAP_LX0) * (KAP_NX - 1);
  double fw = (lw - KAP_LW0) / (KAP_LW1 - KAP_LW0) * (KAP_NW - 1);
  fx = std::min(std::max(fx, 0.0), (double)(KAP_NX - 1));
  fw = std::min(std::max(fw, 0.0), (double)(KAP_NW - 1));
  int i = std::min((int)fx, KAP_NX - 2), j = std::min((int)fw, KAP_NW - 2);
  double a = fx - i, b = fw - j;
  double l = (1 - a) * (1 - b) * t[i * KAP_NW + j] + (1 - a) * b * t[i * KAP_NW + j + 1] +
             a * (1 - b) * t[(i + 1) * KAP_NW + j] + a * b * t[(i + 1) * KAP_NW + j + 1];
  return std::exp(l);
}

void build_kappa(KappaTables &T, double kappa) {
  T.kappa = kappa;
  T.lnF.resize(6001);
  const double l0 = -30.0, l1 = std::log(200.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i <= 6000; ++i) T.lnF[i] = std::log(F_sync_direct(std::exp(l0 + (l1 - l0) * i / 6000.0)));
  T.lnJ.assign((size_t)KAP_NX * KAP_NW, KAP_FLOOR);
  T.lnA.assign((size_t)KAP_NX * KAP_NW, KAP_FLOOR);
  T.lnI.assign((size_t)KAP_NX * KAP_NW, KAP_FLOOR);
  static const GL gp(32, 0.0, 1.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int jw = 0; jw < KAP_NW; ++jw) {
    const double w = std::exp(KAP_LW0 + (KAP_LW1 - KAP_LW0) * jw / (KAP_NW - 1));
    const double kw = kappa * w;
    // t = ln(gamma - 1) over [ln(kappa w) - 25, ln(kappa w) + 45] in 280 panels of 32 nodes
    const double t0 = std::log(kw) - 25.0, h = 0.25;
    const int np = 280;
    std::vector<double> tt, ww;
    for (int k = 0; k < np; ++k)
      for (int i = 0; i < gp.n; ++i) { tt.push_back(t0 + (k + gp.x[i]) * h); ww.push_back(gp.w[i] * h); }
    const size_t nq = tt.size();
    std::vector<double> gam(nq), base(nq), aterm(nq);
    double norm = 0.0;
    for (size_t q = 0; q < nq; ++q) {
      const double e = std::exp(tt[q]), g = 1.0 + e, rt = std::sqrt(e * (2.0 + e));   // sqrt(gamma^2 - 1)
      const double lp = -(kappa + 1.0) * std::log1p(e / kw);
      gam[q] = g;
      base[q] = std::exp(lp + tt[q]);                       // P(gamma) dgamma/dt
      norm += ww[q] * g * rt * base[q];
      aterm[q] = g * rt * (kappa + 1.0) / (kw + e) - 1.0 / rt;   // gamma^2 d/dgamma(f/gamma^2) / (-f-free part)
    }
    for (int ix = 0; ix < KAP_NX; ++ix) {
      const double X = std::exp(KAP_LX0 + (KAP_LX1 - KAP_LX0) * ix / (KAP_NX - 1));
      double sj = 0.0, sa = 0.0;
      for (size_t q = 0; q < nq; ++q) {
        const double x = 2.0 * X / (3.0 * gam[q] * gam[q]);
        if (x >= 200.0) continue;
        const double Fq = T.F(x);
        const double rt = std::sqrt((gam[q] - 1.0) * (gam[q] + 1.0));
        sj += ww[q] * gam[q] * rt * base[q] * Fq;
        sa += ww[q] * aterm[q] * base[q] * Fq;
      }
      sj /= norm;
      sa /= norm;
      T.lnJ[(size_t)ix * KAP_NW + jw] = sj > 0.0 ? std::max(KAP_FLOOR, std::log(sj)) : KAP_FLOOR;
      T.lnA[(size_t)ix * KAP_NW + jw] = sa > 0.0 ? std::max(KAP_FLOOR, std::log(sa)) : KAP_FLOOR;
    }
  }
  // I(Y, w) = int_0^1 sin J(Y / sin, w) dmu = int_0^{pi/2} sin^2 J(Y / sin, w) dtheta over the interpolated
  // J, defined (reading) as the midpoint sum with 2048 points in theta
  const int M = 2048;
#pragma omp parallel for schedule(static)
  for (int ix = 0; ix < KAP_NX; ++ix) {
    const double lY = KAP_LX0 + (KAP_LX1 - KAP_LX0) * ix / (KAP_NX - 1);
    for (int jw = 0; jw < KAP_NW; ++jw) {
      const double lw = KAP_LW0 + (KAP_LW1 - KAP_LW0) * jw / (KAP_NW - 1);
      double s = 0.0;
      for (int k = 0; k < M; ++k) {
        const double st = std::sin((k + 0.5) * (0.5 * PI / M));
        s += st * st * kap_interp(T.lnJ, lY - std::log(st), lw);
      }
      s *= 0.5 * PI / M;
      T.lnI[(size_t)ix * KAP_NW + jw] = s > 0.0 ? std::max(KAP_FLOOR, std::log(s)) : KAP_FLOOR;
    }
  }
}

const KappaTables &kappa_tables(double kappa) {
  static std::mutex mu;
  static std::map<double, KappaTables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kappa);
  if (it == cache.end()) {
    KappaTables T;
    build_kappa(T, kappa);
    it = cache.emplace(kappa, std::move(T)).first;
  }
  return it->second;
}

double kappa_w(const or_params &P, double thetae) { return thetae * (P.kappa - 3.0) / P.kappa; }

double jnu_kappa(const or_params &P, double nu, double ne, double thetae, double B, double costh) {
  double s2 = 1.0 - costh * costh;
  if (s2 <= 0.0) return 0.0;
  const double sth = std::sqrt(s2), nuB = EE * B / (2.0 * PI * ME * CL);
  const KappaTables &T = kappa_tables(P.kappa);
  double Jv = kap_interp(T.lnJ, std::log(nu / (nuB * sth)), std::log(kappa_w(P, thetae)));
  return std::sqrt(3.0) * EE * EE * EE * ne * B * sth / (4.0 * PI * ME * CL * CL) * Jv;
}

// nu alpha_nu of the kappa population
double nu_alpha_kappa(const or_params &P, double nu, double ne, double thetae, double B, double costh) {
  double s2 = 1.0 - costh * costh;
  if (s2 <= 0.0) return 0.0;
  const double sth = std::sqrt(s2), nuB = EE * B / (2.0 * PI * ME * CL);
  const KappaTables &T = kappa_tables(P.kappa);
  double Av = kap_interp(T.lnA, std::log(nu / (nuB * sth)), std::log(kappa_w(P, thetae)));
  const double mc2 = ME * CL * CL;
  return CL * CL / (8.0 * PI * nu) * std::sqrt(3.0) * EE * EE * EE * ne * B * sth / (mc2 * mc2) * Av;
}

double jnu_angint_kappa(const or_params &P, double nu, double ne, double thetae, double B) {
  const double nuB = EE * B / (2.0 * PI * ME * CL);
  const KappaTables &T = kappa_tables(P.kappa);
  double Iv = kap_interp(T.lnI, std::log(nu / nuB), std::log(kappa_w(P, thetae)));
  return std::sqrt(3.0) * EE * EE * EE * ne * B / (ME * CL * CL) * Iv;   // 4 pi x (sqrt3 e^3 n_e B / 4 pi m_e c^2) I
}

double jnu(const or_params &P, double nu, double ne, double thetae, double B, double costh) {
  if (P.kappa > 0.0) {
    if (thetae < P.thetae_min || ne <= 0.0 || B <= 0.0) return 0.0;
    return jnu_kappa(P, nu, ne, thetae, B, costh);
  }
  if (thetae < P.thetae_min || ne <= 0.0 || B <= 0.0) return 0.0;
  double s2 = 1.0 - costh * costh;
  if (s2 <= 0.0) return 0.0;
  double sinth = std::sqrt(s2);
  double nus = (2.0 / 9.0) * (EE * B / (2.0 * PI * ME * CL)) * thetae * thetae * sinth;
  double X = nu / nus;
  double t = std::sqrt(X) + std::pow(2.0, 11.0 / 12.0) * std::pow(X, 1.0 / 6.0);
  return std::sqrt(2.0) * PI * EE * EE * ne * nus / (3.0 * CL * K2_of(P, thetae)) * t * t * std::exp(-std::cbrt(X));
}

// Planck function B_nu(T) with k T = Theta_e m_e c^2.
double bnu(double nu, double thetae) {
  return 2.0 * HPL * nu * nu * nu / (CL * CL) / std::expm1(HPL * nu / (thetae * ME * CL * CL));
}

// Angle integral F(K) = int_0^{pi/2} sin^2(th) G(K / sin th) dth, G(X) = (X^1/2 + 2^11/12 X^1/6)^2 e^{-X^1/3},
// so that int dOmega j_nu = 4 pi A nu_c F(nu / nu_c) with A = sqrt(2) pi e^2 n_e / (3 c K2).
// Gauss-Legendre with 64 nodes in theta (reading).

double Fang(double K) {
  static const GL gl(64, 0.0, PI / 2.0);
  double s = 0.0;
  for (int i = 0; i < gl.n; ++i) {
    double st = std::sin(gl.x[i]);
    double X = K / st;
    double t = std::sqrt(X) + std::pow(2.0, 11.0 / 12.0) * std::pow(X, 1.0 / 6.0);
    s += gl.w[i] * st * st * t * t * std::exp(-std::cbrt(X));
  }
  return s;
}

double nu_c_of(double thetae, double B) {
  return (2.0 / 9.0) * (EE * B / (2.0 * PI * ME * CL)) * thetae * thetae;
}

// int dOmega j_nu at frequency nu for a zone state.
double jnu_angint(const or_params &P, double nu, double ne, double thetae, double B) {
  if (thetae < P.thetae_min || ne <= 0.0 || B <= 0.0) return 0.0;
  if (P.kappa > 0.0) return jnu_angint_kappa(P, nu, ne, thetae, B);
  double nuc = nu_c_of(thetae, B);
  double A = std::sqrt(2.0) * PI * EE * EE * ne / (3.0 * CL * K2_of(P, thetae));
  return 4.0 * PI * A * nuc * Fang(nu / nuc);
}

// ---------------------------------------------------------------- bremsstrahlung (future work in section 6)
// Thermal bremsstrahlung of a hydrogen plasma (reading): total cooling rate q = q_ei + q_ee
// [erg s^-1 cm^-3] from the fits of Stepney & Guilbert (1983) in the form of Narayan & Yi (1995),
//   q_ei = 1.25 n_e n_i sigma_T c alpha_f m_e c^2 F_ei(Theta),
//     F_ei = 4 (2 Theta / pi^3)^1/2 (1 + 1.781 Theta^1.34)           (Theta < 1)
//          = 9 Theta / (2 pi) (ln(1.123 Theta + 0.48) + 1.5)          (Theta >= 1),
//   q_ee = n_e^2 c r_e^2 alpha_f m_e c^2 (20 / 9 sqrt(pi)) (44 - 3 pi^2) Theta^3/2
//          (1 + 1.1 Theta + Theta^2 - 1.25 Theta^5/2)                  (Theta < 1)
//        = n_e^2 c r_e^2 alpha_f m_e c^2 24 Theta (ln(1.1232 Theta) + 1.28)   (Theta >= 1),
// n_i = n_e, and an isotropic spectrum 4 pi j_nu = q (h / k T) exp(-h nu / k T) (a flat Gaunt shape
// normalised to q); absorption by Kirchhoff's law, alpha_nu = j_nu / B_nu.
const double ALPHA_F = 7.2973525693e-3;    // fine-structure constant
const double R_E = 2.8179403262e-13;       // classical electron radius [cm]

double brems_q(double ne, double th) {
  const double mc2 = ME * CL * CL;
  double fei = th < 1.0 ? 4.0 * std::sqrt(2.0 * th / (PI * PI * PI)) * (1.0 + 1.781 * std::pow(th, 1.34))
                        : 9.0 * th / (2.0 * PI) * (std::log(1.123 * th + 0.48) + 1.5);
  double qei = 1.25 * ne * ne * SIGMA_T * CL * ALPHA_F * mc2 * fei;
  double fee = th < 1.0 ? 20.0 / (9.0 * std::sqrt(PI)) * (44.0 - 3.0 * PI * PI) * std::pow(th, 1.5) *
                              (1.0 + 1.1 * th + th * th - 1.25 * std::pow(th, 2.5))
                        : 24.0 * th * (std::log(1.1232 * th) + 1.28);
  double qee = ne * ne * CL * R_E * R_E * ALPHA_F * mc2 * fee;
  return qei + qee;
}

// int dOmega j_nu = 4 pi j_nu of the bremsstrahlung (0 when off)
double brems_angint(const or_params &P, double nu, double ne, double th) {
  if (!P.brems || ne <= 0.0 || th <= 0.0) return 0.0;
  const double kt = th * ME * CL * CL;
  return brems_q(ne, th) * HPL / kt * std::exp(-HPL * nu / kt);
}

// nu alpha_nu = nu j_nu / B_nu = q c^2 (1 - exp(-h nu / k T)) / (8 pi k T nu^2)
double brems_nu_alpha(const or_params &P, double nu, double ne, double th) {
  if (!P.brems || ne <= 0.0 || th <= 0.0) return 0.0;
  const double kt = th * ME * CL * CL;
  return brems_q(ne, th) * CL * CL * (-std::expm1(-HPL * nu / kt)) / (8.0 * PI * kt * nu * nu);
}

// ---------------------------------------------------------------- Compton (section 2.7)
// Klein-Nishina total cross-section; sigma_T (1 - 2 eps) below eps = 1e-3.
double sigma_kn(double e) {
  if (e < 1e-3) return SIGMA_T * (1.0 - 2.0 * e);
  double e2 = e * e;
  return SIGMA_T * 0.75 / e2 *
         (2.0 + e2 * (1.0 + e) / ((1.0 + 2.0 * e) * (1.0 + 2.0 * e)) + (e2 - 2.0 * e - 2.0) / (2.0 * e) * std::log1p(2.0 * e));
}

// Hot cross-section sigma_h(Theta, eps) = <(1 - mu beta) sigma_KN(eps gamma (1 - mu beta))> over a
// Maxwell-Juettner electron population (section 2.7).  Quadrature (reading): gamma = 1 + Theta s^2,
// s in [0, 8] with 64 Gauss-Legendre nodes (the MJ density becomes gamma s^2 sqrt(Theta (2 + Theta s^2)) e^{-s^2}),
// mu in [-1, 1] with 32 nodes; the normalisation uses the same s rule.
double sigma_hot_quad(double thetae, double eps) {
  static const GL gs(64, 0.0, 8.0);
  static const GL gm(32, -1.0, 1.0);
  double num = 0.0, den = 0.0;
  for (int i = 0; i < gs.n; ++i) {
    double s = gs.x[i];
    double gam = 1.0 + thetae * s * s;
    double hs = gam * s * s * std::sqrt(thetae * (2.0 + thetae * s * s)) * std::exp(-s * s);
    double beta = std::sqrt(1.0 - 1.0 / (gam * gam));
    double q = 0.0;
    for (int j = 0; j < gm.n; ++j) {
      double om = 1.0 - gm.x[j] * beta;
      q += gm.w[j] * om * sigma_kn(eps * gam * om);
    }
    num += gs.w[i] * hs * 0.5 * q;
    den += gs.w[i] * hs;
  }
  return num / den;
}

// Lookup table (section 2.7: sigma_h precomputed): ln(sigma_h / sigma_T) on a grid
// uniform in ln Theta (121 nodes, 1e-3..1e3) and ln eps (181 nodes, 1e-12..1e6),
// bilinear in (ln Theta, ln eps), arguments clamped to the table range.
const int HT_NT = 121, HT_NE = 181;
const double HT_LT0 = -6.907755278982137, HT_LT1 = 6.907755278982137;   // ln 1e-3, ln 1e3
const double HT_LE0 = -27.631021115928547, HT_LE1 = 13.815510557964274;  // ln 1e-12, ln 1e6

struct HotTable {
  std::vector<double> v;   // [HT_NT][HT_NE]
  void build() {
    v.resize((size_t)HT_NT * HT_NE);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < HT_NT; ++i) {
      double th = std::exp(HT_LT0 + (HT_LT1 - HT_LT0) * i / (HT_NT - 1));
      for (int j = 0; j < HT_NE; ++j) {
        double e = std::exp(HT_LE0 + (HT_LE1 - HT_LE0) * j / (HT_NE - 1));
        v[(size_t)i * HT_NE + j] = std::log(sigma_hot_quad(th, e) / SIGMA_T);
      }
    }
  }
  double lookup(double thetae, double eps) const {
    double lt = std::log(thetae), le = std::log(eps);
    double ft = (lt - HT_LT0) / (HT_LT1 - HT_LT0) * (HT_NT - 1);
    double fe = (le - HT_LE0) / (HT_LE1 - HT_LE0) * (HT_NE - 1);
    ft = std::min(std::max(ft, 0.0), (double)(HT_NT - 1));
    fe = std::min(std::max(fe, 0.0), (double)(HT_NE - 1));
    int i = std::min((int)ft, HT_NT - 2), j = std::min((int)fe, HT_NE - 2);
    double a = ft - i, b = fe - j;
    double v00 = v[(size_t)i * HT_NE + j], v01 = v[(size_t)i * HT_NE + j + 1];
    double v10 = v[(size_t)(i + 1) * HT_NE + j], v11 = v[(size_t)(i + 1) * HT_NE + j + 1];
    double l = (1 - a) * (1 - b) * v00 + (1 - a) * b * v01 + a * (1 - b) * v10 + a * b * v11;
    return SIGMA_T * std::exp(l);
  }
};

HotTable &hot_table() {
  static HotTable t;
  static bool built = false;
#pragma omp critical(hot_table_build)
  {
    if (!built) { t.build(); built = true; }
  }
  return t;
}

// Maxwell-Juettner Lorentz factor, exact samplers (reading; the paper follows igrmonty):
//  Theta >= 0.25: Sobol's method (Pozdnyakov, Sobol & Sunyaev 1983): p = -Theta ln(u1 u2 u3),
//                 eta = p - Theta ln u4, accept if eta^2 - p^2 > 1;
//  Theta <  0.25: with t = gamma - 1, f(t) <= sqrt(2) sqrt(t) (1 + 5t/4 + t^2/4) e^{-t/Theta}; draw from
//                 that Gamma(3/2, 5/2, 7/2) mixture, accept with (1+t) sqrt(t+2) / (sqrt 2 (1 + 5t/4 + t^2/4)).
const int MAXTRY = 10000;

// ---------------------------------------------------------------- kappa electrons: scattering
// Hot cross-section of the kappa population, sigma_h(w, eps) = <(1 - mu beta) sigma_KN(eps gamma (1 - mu beta))>,
// tabulated as ln(sigma_h / sigma_T) on the kappa ln w grid x the thermal table's ln eps grid and
// interpolated bilinearly (reading); the oracle's nodes by Gauss-Legendre panels in t = ln(gamma - 1)
// (140 x 16) and, over mu, 24 Gauss-Legendre nodes in y = ln(1 - beta mu) (d mu = -e^y dy / beta), which
// resolves the Klein-Nishina turnover that ultrarelativistic electrons confine to mu -> 1.
struct KappaHot {
  std::vector<double> v;   // [KAP_NW][HT_NE]
  double lookup(double w, double eps) const {
    double fw = (std::log(w) - KAP_LW0) / (KAP_LW1 - KAP_LW0) * (KAP_NW - 1);
    double fe = (std::log(eps) - HT_LE0) / (HT_LE1 - HT_LE0) * (HT_NE - 1);
    fw = std::min(std::max(fw, 0.0), (double)(KAP_NW - 1));
    fe = std::min(std::max(fe, 0.0), (double)(HT_NE - 1));
    int i = std::min((int)fw, KAP_NW - 2), j = std::min((int)fe, HT_NE - 2);
    double a = fw - i, b = fe - j;
    double l = (1 - a) * (1 - b) * v[(size_t)i * HT_NE + j] + (1 - a) * b * v[(size_t)i * HT_NE + j + 1] +
               a * (1 - b) * v[(size_t)(i + 1) * HT_NE + j] + a * b * v[(size_t)(i + 1) * HT_NE + j + 1];
    return SIGMA_T * std::exp(l);
  }
};

const KappaHot &kappa_hot(double kappa) {
  static std::mutex mu;
  static std::map<double, KappaHot> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kappa);
  if (it != cache.end()) return it->second;
  KappaHot T;
  T.v.assign((size_t)KAP_NW * HT_NE, 0.0);
  static const GL gp(16, 0.0, 1.0);
  static const GL gm(24, -1.0, 1.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < KAP_NW; ++i) {
    const double w = std::exp(KAP_LW0 + (KAP_LW1 - KAP_LW0) * i / (KAP_NW - 1)), kw = kappa * w;
    const double t0 = std::log(kw) - 25.0, h = 0.5;
    std::vector<double> gam, bet, wt;
    double norm = 0.0;
    for (int k = 0; k < 140; ++k)
      for (int q = 0; q < gp.n; ++q) {
        const double t = t0 + (k + gp.x[q]) * h, e = std::exp(t), g = 1.0 + e, p = std::sqrt(e * (2.0 + e));
        const double f = g * p * std::exp(t - (kappa + 1.0) * std::log1p(e / kw));
        gam.push_back(g);
        bet.push_back(p / g);
        wt.push_back(gp.w[q] * h * f);
        norm += gp.w[q] * h * f;
      }
    for (int j = 0; j < HT_NE; ++j) {
      const double eps = std::exp(HT_LE0 + (HT_LE1 - HT_LE0) * j / (HT_NE - 1));
      double acc = 0.0;
      for (size_t q = 0; q < gam.size(); ++q) {
        // (1/2) int (1 - beta mu) sigma_KN dmu = (1 / 2 beta) int_{ln(1-beta)}^{ln(1+beta)} e^{2y} sigma_KN(eps gamma e^y) dy,
        // with ln(1 - beta) = -2 ln gamma - ln(1 + beta)
        const double y1 = std::log1p(bet[q]), y0 = -2.0 * std::log(gam[q]) - y1;
        double sm = 0.0;
        for (int r = 0; r < gm.n; ++r) {
          const double om = std::exp(0.5 * (y0 + y1) + 0.5 * (y1 - y0) * gm.x[r]);
          sm += gm.w[r] * om * om * sigma_kn(eps * gam[q] * om);
        }
        acc += wt[q] * 0.5 * (0.5 * (y1 - y0)) * sm / bet[q];
      }
      T.v[(size_t)i * HT_NE + j] = std::log(acc / norm / SIGMA_T);
    }
  }
  return cache.emplace(kappa, std::move(T)).first->second;
}

// Standard normal by the Box-Muller transform (two uniforms).
double normal_bm(Stream &s) {
  double u1 = 1.0 - uniform(s), u2 = uniform(s);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * PI * u2);
}

// Gamma(a) variate by the method of Marsaglia & Tsang (2000); for a < 1 from Gamma(a + 1) U^(1/a)
// (the Gamma(a + 1) draws first, then U).
double gamma_mt(double a, Stream &s) {
  if (a < 1.0) {
    const double g = gamma_mt(a + 1.0, s);
    return g * std::pow(uniform(s), 1.0 / a);
  }
  const double d = a - 1.0 / 3.0, c = 1.0 / std::sqrt(9.0 * d);
  for (int it = 0; it < MAXTRY; ++it) {
    double x = normal_bm(s), v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = uniform(s);
    if (u < 1.0 - 0.0331 * x * x * x * x) return d * v;
    if (std::log(u) < 0.5 * x * x + d * (1.0 - v + std::log(v))) return d * v;
  }
  return d;
}

// Lorentz factor of a kappa electron (reading).  In u = gamma - 1 the density is
// (1 + u) sqrt(u (2 + u)) (1 + u / (kappa w))^-(kappa+1).  It is bounded by an envelope whose terms are
// u^(a-1) (1 + u / (kappa w))^-(kappa+1), each a scaled beta-prime(a, kappa + 1 - a) density (x = u / (kappa w)
// = G_a / G_b, G ~ Gamma), mixed with weights from the beta-function integrals:
//   w < 1:  sqrt2 u^1/2 (1 + u)^2, terms a = 3/2, 5/2, 7/2 (ratio to the density sqrt(1 + u/2) / (1 + u));
//   w >= 1: (1 + u)^2,             terms a = 1, 2, 3       (ratio sqrt(1 - (1 + u)^-2)).
// Draws: component, Gamma(a), Gamma(kappa + 1 - a), acceptance; repeated until accepted.
double sample_kappa(double kappa, double w, Stream &s, int64_t *rejcap) {
  const double kw = kappa * w;
  const bool low = w < 1.0;
  const double a1 = low ? 1.5 : 1.0;
  // mass of each term: binomial coefficient x (kappa w)^a B(a, kappa + 1 - a), relative to the first;
  // B(a + 1, b - 1) / B(a, b) = a / (b - 1)
  const double b1 = kappa + 1.0 - a1;
  const double r2 = 2.0 * kw * a1 / (b1 - 1.0);                     // term 2 / term 1
  const double r3 = r2 * 0.5 * kw * (a1 + 1.0) / (b1 - 2.0);        // term 3 / term 1
  const double tot = 1.0 + r2 + r3;
  for (int it = 0; it < MAXTRY; ++it) {
    const double uc = uniform(s) * tot;
    const int k = uc < 1.0 ? 0 : (uc < 1.0 + r2 ? 1 : 2);
    const double a = a1 + k;
    const double ga = gamma_mt(a, s), gb = gamma_mt(kappa + 1.0 - a, s);
    const double u = kw * (ga / gb);
    const double acc = low ? std::sqrt(1.0 + 0.5 * u) / (1.0 + u) : std::sqrt(1.0 - 1.0 / ((1.0 + u) * (1.0 + u)));
    if (uniform(s) < acc) return 1.0 + u;
  }
  if (rejcap) (*rejcap)++;
  return 1.0 + kw;
}

double sample_mj(double thetae, Stream &s) {
  if (thetae >= 0.25) {
    for (int it = 0; it < MAXTRY; ++it) {
      double u1 = uniform(s), u2 = uniform(s), u3 = uniform(s), u4 = uniform(s);
      double p = -thetae * std::log(u1 * u2 * u3);
      double eta = p - thetae * std::log(u4);
      if (eta * eta - p * p > 1.0 || it == MAXTRY - 1) return std::sqrt(1.0 + p * p);
    }
  }
  double c1 = 0.886226925452758 * std::pow(thetae, 1.5);          // Gamma(3/2) Theta^3/2
  double c2 = 1.25 * 1.329340388179137 * std::pow(thetae, 2.5);   // 5/4 Gamma(5/2) Theta^5/2
  double c3 = 0.25 * 3.323350970447843 * std::pow(thetae, 3.5);   // 1/4 Gamma(7/2) Theta^7/2
  double ct = c1 + c2 + c3;
  double t = 0.0;
  for (int it = 0; it < MAXTRY; ++it) {
    double uc = uniform(s) * ct;
    int k = (uc < c1) ? 1 : ((uc < c1 + c2) ? 2 : 3);
    double prod = 1.0;
    for (int i = 0; i < k; ++i) prod *= uniform(s);
    double ua = uniform(s), ub = uniform(s);
    double z = std::sqrt(-2.0 * std::log(ua)) * std::cos(2.0 * PI * ub);
    t = thetae * (-std::log(prod) + 0.5 * z * z);
    double acc = (1.0 + t) * std::sqrt(t + 2.0) / (std::sqrt(2.0) * (1.0 + 1.25 * t + 0.25 * t * t));
    if (uniform(s) < acc) break;
  }
  return 1.0 + t;
}

// Two unit vectors completing an orthonormal basis with unit vector n (fixed construction).
void perp_basis(const double n[3], double e1[3], double e2[3]) {
  double a[3] = {1.0, 0.0, 0.0};
  if (std::fabs(n[0]) >= 0.6) { a[0] = 0.0; a[1] = 1.0; }
  double d = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
  for (int i = 0; i < 3; ++i) e1[i] = a[i] - d * n[i];
  double l = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int i = 0; i < 3; ++i) e1[i] /= l;
  e2[0] = n[1] * e1[2] - n[2] * e1[1];
  e2[1] = n[2] * e1[0] - n[0] * e1[2];
  e2[2] = n[0] * e1[1] - n[1] * e1[0];
}

// Lorentz boost of (E, p) into the frame moving with speed beta along unit v.
void boost(double E, const double p[3], double beta, const double v[3], double *Eo, double po[3]) {
  double gam = 1.0 / std::sqrt(1.0 - beta * beta);
  double pv = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
  *Eo = gam * (E - beta * pv);
  double ppar = gam * (pv - beta * E);
  for (int i = 0; i < 3; ++i) po[i] = p[i] + (ppar - pv) * v[i];
}

// Compton scattering in the plasma frame (section 2.7): photon energy eps, unit direction n;
// electron from the thermal population with pair acceptance (1 - beta mu) sigma_KN(eps_e) / (2 sigma_T);
// rest-frame angle from the Klein-Nishina differential cross-section (Thomson form below
// eps_e = 1e-4), eps' = eps_e / (1 + eps_e (1 - cos)); boosted back.  Random draws in fixed order:
// [gamma (MJ draws), mu_e, accept]*, phi_e, [cos, accept]*, phi.
void compton_fluid(double kappa, double thetae, double eps, const double n[3], Stream &s, double *eps_out,
                   double dir_out[3], int64_t *rejcap) {
  double gam = 1.0, mue = 0.0, beta = 0.0;
  int it = 0;
  for (it = 0; it < MAXTRY; ++it) {
    gam = kappa > 0.0 ? sample_kappa(kappa, thetae * (kappa - 3.0) / kappa, s, rejcap) : sample_mj(thetae, s);
    mue = 2.0 * uniform(s) - 1.0;
    beta = std::sqrt(1.0 - 1.0 / (gam * gam));
    double om = 1.0 - beta * mue;
    double acc = om * sigma_kn(eps * gam * om) / (2.0 * SIGMA_T);
    if (uniform(s) < acc) break;
  }
  if (it == MAXTRY && rejcap) (*rejcap)++;
  double phie = 2.0 * PI * uniform(s);
  double e1[3], e2[3];
  perp_basis(n, e1, e2);
  double se = std::sqrt(std::max(0.0, 1.0 - mue * mue));
  double v[3];
  for (int i = 0; i < 3; ++i) v[i] = mue * n[i] + se * (std::cos(phie) * e1[i] + std::sin(phie) * e2[i]);
  double pin[3] = {eps * n[0], eps * n[1], eps * n[2]};
  double ee, pe[3];
  boost(eps, pin, beta, v, &ee, pe);
  double lp = std::sqrt(pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]);
  double ne[3] = {pe[0] / lp, pe[1] / lp, pe[2] / lp};
  double ct = 1.0, ep = ee;
  for (it = 0; it < MAXTRY; ++it) {
    ct = 2.0 * uniform(s) - 1.0;
    ep = ee / (1.0 + ee * (1.0 - ct));
    double P;
    if (ee < 1e-4) {
      P = 0.5 * (1.0 + ct * ct);
    } else {
      double r = ep / ee;
      P = 0.5 * r * r * (r + 1.0 / r - (1.0 - ct * ct));
    }
    if (uniform(s) < P) break;
  }
  if (it == MAXTRY && rejcap) (*rejcap)++;
  double phi = 2.0 * PI * uniform(s);
  double f1[3], f2[3];
  perp_basis(ne, f1, f2);
  double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
  double np[3], pp[3];
  for (int i = 0; i < 3; ++i) {
    np[i] = ct * ne[i] + st * (std::cos(phi) * f1[i] + std::sin(phi) * f2[i]);
    pp[i] = ep * np[i];
  }
  double mv[3] = {v[0], v[1], v[2]};
  double Ef, pf[3];
  boost(ep, pp, -beta, mv, &Ef, pf);
  *eps_out = Ef;
  for (int i = 0; i < 3; ++i) dir_out[i] = pf[i];
}

// ---------------------------------------------------------------- tetrads (sections 2.1, 2.7)
double dot4(const double g[4][4], const double a[4], const double b[4]) {
  double s = 0.0;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) s += a[m] * g[m][n] * b[n];
  return s;
}

// Gram-Schmidt against e0 (timelike, e0.e0 = -1) and the given spacelike unit vectors.
void gs_orth(const double g[4][4], double v[4], const double e0[4], const double (*es)[4], int ns) {
  double d0 = dot4(g, v, e0);
  for (int m = 0; m < 4; ++m) v[m] += d0 * e0[m];
  for (int k = 0; k < ns; ++k) {
    double d = dot4(g, v, es[k]);
    for (int m = 0; m < 4; ++m) v[m] -= d * es[k][m];
  }
}
bool normalize_space(const double g[4][4], double v[4]) {
  double n2 = dot4(g, v, v);
  if (!(n2 > 1e-30)) return false;
  double n = std::sqrt(n2);
  for (int m = 0; m < 4; ++m) v[m] /= n;
  return true;
}

// Emission tetrad: e0 = u, e3 = b/|b|; e1 and e2 from the coordinate directions d_1, d_2, d_3
// (reading of "Gram-Schmidt"): after projecting out e0 and e3 (and e1 for e2), the direction
// keeping the largest fraction |t_perp|^2 / |t|^2 is taken (first index on ties), so the
// construction never degenerates whatever the field geometry.
void tetrad_emission(const double g[4][4], const Fluid &F, double e[4][4]) {
  for (int m = 0; m < 4; ++m) e[0][m] = F.ucon[m];
  double bn = std::sqrt(F.bsq);
  for (int m = 0; m < 4; ++m) e[3][m] = F.bcon[m] / bn;
  double es[2][4];
  for (int m = 0; m < 4; ++m) es[0][m] = e[3][m];
  double t[4][4];
  double frac[4] = {0, 0, 0, 0};
  int pick = 1;
  for (int k = 1; k < 4; ++k) {
    for (int m = 0; m < 4; ++m) t[k][m] = (m == k) ? 1.0 : 0.0;
    gs_orth(g, t[k], e[0], es, 1);
    frac[k] = dot4(g, t[k], t[k]) / g[k][k];
    if (frac[k] > frac[pick]) pick = k;
  }
  normalize_space(g, t[pick]);
  for (int m = 0; m < 4; ++m) { e[1][m] = t[pick][m]; es[1][m] = t[pick][m]; }
  int pick2 = -1;
  double best = -1.0;
  double t2[4][4];
  for (int k = 1; k < 4; ++k) {
    if (k == pick) continue;
    for (int m = 0; m < 4; ++m) t2[k][m] = (m == k) ? 1.0 : 0.0;
    gs_orth(g, t2[k], e[0], es, 2);
    double f = dot4(g, t2[k], t2[k]) / g[k][k];
    if (f > best) { best = f; pick2 = k; }
  }
  normalize_space(g, t2[pick2]);
  for (int m = 0; m < 4; ++m) e[2][m] = t2[pick2][m];
}

// Scattering tetrad: e0 = u, e1, e2, e3 from the x1, x2, x3 coordinate directions.
void tetrad_scatter(const double g[4][4], const Fluid &F, double e[4][4]) {
  for (int m = 0; m < 4; ++m) e[0][m] = F.ucon[m];
  double es[3][4];
  for (int k = 1; k < 4; ++k) {
    double t[4] = {0, 0, 0, 0};
    t[k] = 1.0;
    gs_orth(g, t, e[0], es, k - 1);
    normalize_space(g, t);
    for (int m = 0; m < 4; ++m) { e[k][m] = t[m]; es[k - 1][m] = t[m]; }
  }
}

// ---------------------------------------------------------------- model
struct Zone {
  double ne, thetae, B;
};

struct Model {
  or_params P;
  Units un;
  int n1, n2, n3;
  int64_t nz;
  double x1_0, dx1, x2_0, dx2, x3_0, dx3;
  std::vector<double> prim;          // [8][nz]
  // prepared per (N_s, seed)
  int nnu;
  double lnumin, dlnu, dlntot;
  std::vector<double> lnw;           // ln w_j
  std::vector<double> g;             // [nz][nnu]: (int dOmega j_nu(nu_j)) / w_j
  std::vector<double> gmax, nbar, vol;
  std::vector<int64_t> counts, start;
  int64_t total = 0;
  uint64_t seed = 0;
  double r_h = 0.0;
  std::vector<double> bscale;        // bias scale per scattering generation (last full run)
  double scale_of(int nsc) const {
    if (bscale.empty()) return 1.0;
    return bscale[std::min((size_t)nsc, bscale.size() - 1)];
  }
};

void zone_center(const Model &M, int64_t z, double X[4]) {
  int64_t i = z / ((int64_t)M.n2 * M.n3);
  int64_t j = (z / M.n3) % M.n2;
  int64_t k = z % M.n3;
  X[0] = 0.0;
  X[1] = M.x1_0 + (i + 0.5) * M.dx1;
  X[2] = M.x2_0 + (j + 0.5) * M.dx2;
  X[3] = M.x3_0 + (k + 0.5) * M.dx3;
}

void zone_prims(const Model &M, int64_t z, double pr[8]) {
  for (int f = 0; f < 8; ++f) pr[f] = M.prim[(size_t)f * M.nz + z];
}

void fluid_at(const Model &M, const double X[4], const double g[4][4], Fluid &F, bool clamp_radial) {
  double lo = M.x1_0, hi = M.x1_0 + M.n1 * M.dx1;
  if (!clamp_radial && (X[1] < lo || X[1] > hi)) {
    F.plasma = false;
    F.ne = F.thetae = F.B = 0.0;
    return;
  }
  auto idx = [](double x, double x0, double dx, int n, int *i0, double *d) {
    double f = (x - x0) / dx - 0.5;
    int i = (int)std::floor(f);
    double di = f - i;
    if (n == 1) { *i0 = 0; *d = 0.0; return; }
    if (i < 0) { i = 0; di = 0.0; }
    if (i > n - 2) { i = n - 2; di = 1.0; }
    *i0 = i;
    *d = di;
  };
  int i, j;
  double di, dj;
  idx(std::min(std::max(X[1], lo), hi), M.x1_0, M.dx1, M.n1, &i, &di);
  idx(X[2], M.x2_0, M.dx2, M.n2, &j, &dj);
  int k0 = 0, k1 = 0;
  double dk = 0.0;
  if (M.n3 > 1) {
    double f = (X[3] - M.x3_0) / M.dx3 - 0.5;
    double fl = std::floor(f);
    dk = f - fl;
    long long kk = (long long)fl;
    k0 = (int)(((kk % M.n3) + M.n3) % M.n3);
    k1 = (k0 + 1) % M.n3;
  }
  int i1 = (M.n1 > 1) ? i + 1 : i, j1 = (M.n2 > 1) ? j + 1 : j;
  double pr[8];
  for (int f = 0; f < 8; ++f) {
    const double *p = &M.prim[(size_t)f * M.nz];
    auto at = [&](int a, int b, int c) { return p[((int64_t)a * M.n2 + b) * M.n3 + c]; };
    double v = (1 - di) * (1 - dj) * ((1 - dk) * at(i, j, k0) + dk * at(i, j, k1)) +
               (1 - di) * dj * ((1 - dk) * at(i, j1, k0) + dk * at(i, j1, k1)) +
               di * (1 - dj) * ((1 - dk) * at(i1, j, k0) + dk * at(i1, j, k1)) +
               di * dj * ((1 - dk) * at(i1, j1, k0) + dk * at(i1, j1, k1));
    pr[f] = v;
  }
  fluid_from_prims(M.P, M.un, pr, g, F);
}

// Invariant absorption and scattering coefficients nu*alpha at a point (sections 2.5-2.7).
struct Coef {
  double ana, ans, thetae;
  Fluid F;
};

void coefficients(const Model &M, const double X[4], const double K[4], bool want_scatter, Coef &c) {
  double g[4][4];
  gcov_at(M.P, X, g);
  fluid_at(M, X, g, c.F);
  c.ana = c.ans = 0.0;
  c.thetae = c.F.thetae;
  if (!c.F.plasma) return;
  double eps = 0.0;
  for (int m = 0; m < 4; ++m) eps -= K[m] * c.F.ucov[m];
  if (!(eps > 0.0)) return;
  double nu = eps * ME * CL * CL / HPL;
  double cth = 0.0;
  if (c.F.bsq > 0.0) {
    double kb = 0.0;
    for (int m = 0; m < 4; ++m) kb += K[m] * c.F.bcov[m];
    cth = kb / (eps * std::sqrt(c.F.bsq));
    cth = std::min(1.0, std::max(-1.0, cth));
  }
  if (M.P.kappa > 0.0) {
    // a non-thermal population: alpha from its own integral, not Kirchhoff's law
    if (c.F.thetae >= M.P.thetae_min && c.F.ne > 0.0 && c.F.B > 0.0)
      c.ana = nu_alpha_kappa(M.P, nu, c.F.ne, c.F.thetae, c.F.B, cth);
  } else {
    double j = jnu(M.P, nu, c.F.ne, c.F.thetae, c.F.B, cth);
    if (j > 0.0) c.ana = nu * j / bnu(nu, c.F.thetae);
  }
  c.ana += brems_nu_alpha(M.P, nu, c.F.ne, c.F.thetae);
  if (want_scatter) {
    double th = std::max(c.F.thetae, 1e-300);
    c.ans = nu * c.F.ne * (M.P.kappa > 0.0 ? kappa_hot(M.P.kappa).lookup(th * (M.P.kappa - 3.0) / M.P.kappa, eps)
                                           : hot_table().lookup(th, eps));
  }
}

// Bias b >= 1 (section 2.7): the configured form b_0, clamped to [1, bias_max], times the scale of
// the superphoton's generation, clamped again.
double bias_of(const or_params &P, double thetae, int nsc, double scale) {
  double b;
  if (P.bias_mode == 1) b = P.bias_p0 * (nsc + 1.0) * (nsc + 1.0);
  else if (P.bias_mode == 2) b = P.bias_p0 * thetae * thetae;
  else b = P.bias_p0;
  const double b0 = std::max(1.0, std::min(b, P.bias_max));
  return std::max(1.0, std::min(scale * b0, P.bias_max));
}

// Bias tuning (reading; the paper names it as future work): the next generation's scale from this
// generation's scattered superphotons per superphoton carried, r: s' = s clamp(target / r, 1/8, 8),
// 8 when r = 0, at most 1e12.
double tune_next_scale(double s, int64_t carried, int64_t children, double target) {
  double r = carried > 0 ? (double)children / (double)carried : 0.0;
  double f = r > 0.0 ? target / r : 8.0;
  f = std::min(8.0, std::max(0.125, f));
  return std::min(1e12, s * f);
}

// ---------------------------------------------------------------- transport (sections 2.4-2.7, 3)
struct Photon {
  double X[4], K[4], A[4];
  double w, wb, ana, ans, acc, x1t;
  Stream s;
  int nsc;
  uint32_t nev;
  int64_t nsteps;
};

struct Child {
  double X[4], K[4], w;
  uint64_t id;
  uint32_t ctr;   // draws already taken from the child's stream by the scattering kinematics
  int nsc;
};

struct Acc {
  std::vector<double> spec;   // [n_incl][n_bins][3]
  or_stats st;
  std::vector<or_log> log;
  bool want_log = false;
};

void record(const Model &M, const Photon &p, Acc &acc) {
  double g[4][4];
  gcov_at(M.P, p.X, g);
  double kt = 0.0;
  for (int n = 0; n < 4; ++n) kt += g[0][n] * p.K[n];
  double E = -kt;   // energy at infinity in m_e c^2
  if (!(E > 0.0)) return;
  double nu = E * ME * CL * CL / HPL;
  double l = std::log10(nu);
  const or_params &P = M.P;
  double d = (P.lnu_hi - P.lnu_lo) / P.n_bins;
  int ib = (int)std::floor((l - P.lnu_lo) / d);
  if (ib < 0 || ib >= P.n_bins) return;
  double th = theta_of(P, p.X[2]);
  double thf = std::acos(std::fabs(std::cos(th)));
  int ii = (int)std::floor(thf / (0.5 * PI) * P.n_incl);
  ii = std::min(std::max(ii, 0), P.n_incl - 1);
  double we = p.w * E;
  double *sp = &acc.spec[((size_t)ii * P.n_bins + ib) * 3];
  sp[0] += we;
  sp[1] += we * we;
  sp[2] += 1.0;
}

void init_transport(const Model &M, Photon &p) {
  p.x1t = -std::log(uniform(p.s));
  p.acc = 0.0;
  bool scat = M.P.scatter && p.nsc < M.P.n_sc_max;
  Coef c;
  coefficients(M, p.X, p.K, scat, c);
  p.ana = c.ana;
  p.ans = c.ans;
  double G[4][4][4];
  christoffel(M.P, p.X, G);
  accel(G, p.K, p.A);
  p.nsteps = 0;
  p.nev = 0;
  p.wb = p.w;
}

void scatter_child(const Model &M, const double Xe[4], const double Ke[4], double wc, uint64_t cid, int nsc,
                   std::vector<Child> &stack, Acc &acc) {
  double g[4][4];
  gcov_at(M.P, Xe, g);
  Fluid F;
  // reading: an event located by linear fraction just outside the radial grid takes the plasma
  // of the nearest grid edge (the step's scattering depth came from inside the grid)
  fluid_at(M, Xe, g, F, true);
  Stream s{M.seed, cid, 0u};
  double e[4][4];
  tetrad_scatter(g, F, e);
  double kf[4];
  double kcov[4];
  for (int m = 0; m < 4; ++m) {
    kcov[m] = 0.0;
    for (int n = 0; n < 4; ++n) kcov[m] += g[m][n] * Ke[n];
  }
  for (int a = 0; a < 4; ++a) {
    double d = 0.0;
    for (int m = 0; m < 4; ++m) d += e[a][m] * kcov[m];
    kf[a] = (a == 0) ? -d : d;
  }
  double eps = kf[0];
  double ln = std::sqrt(kf[1] * kf[1] + kf[2] * kf[2] + kf[3] * kf[3]);
  double n[3] = {kf[1] / ln, kf[2] / ln, kf[3] / ln};
  double eo, dir[3];
  compton_fluid(M.P.kappa, std::max(F.thetae, 1e-8), eps, n, s, &eo, dir, &acc.st.n_rej_cap);
  Child c;
  for (int m = 0; m < 4; ++m) c.K[m] = eo * e[0][m] + dir[0] * e[1][m] + dir[1] * e[2][m] + dir[2] * e[3][m];
  for (int m = 0; m < 4; ++m) c.X[m] = Xe[m];
  c.w = wc;
  c.id = cid;
  c.ctr = s.n;
  c.nsc = nsc;
  stack.push_back(c);
  acc.st.n_child++;
}

// Transport one superphoton to completion; children are pushed on the stack.
void transport(const Model &M, Photon &p, std::vector<Child> &stack, Acc &acc) {
  const or_params &P = M.P;
  const double C = M.un.C;
  int status = 0;
  bool scat = P.scatter && p.nsc < P.n_sc_max;
  while (true) {
    double dl = stepsize(P, p.X, p.K);
    double X0[4], K0[4];
    for (int m = 0; m < 4; ++m) { X0[m] = p.X[m]; K0[m] = p.K[m]; }
    bool conv;
    int it = verlet_step(P, p.X, p.K, p.A, dl, &conv);
    acc.st.n_iters += it;
    if (!conv) acc.st.n_nonconv++;
    p.nsteps++;
    acc.st.n_steps++;
    Coef c;
    coefficients(M, p.X, p.K, scat, c);
    double tau_a = 0.5 * (p.ana + c.ana) * C * dl;
    double w0 = p.w;
    double wn = w0 * std::exp(-tau_a);
    if (scat) {
      double tau_s = 0.5 * (p.ans + c.ans) * C * dl;
      if (tau_s > 0.0) {
        double b = bias_of(P, c.thetae, p.nsc, M.scale_of(p.nsc));
        double d = b * tau_s;
        if (p.acc + d > p.x1t) {
          double f = (p.x1t - p.acc) / d;
          double Xe[4], Ke[4];
          for (int m = 0; m < 4; ++m) {
            Xe[m] = X0[m] + f * (p.X[m] - X0[m]);
            Ke[m] = K0[m] + f * (p.K[m] - K0[m]);
          }
          double we = w0 * std::exp(-f * tau_a);
          uint64_t cid = child_stream(p.s.id, p.nev);
          scatter_child(M, Xe, Ke, we / b, cid, p.nsc + 1, stack, acc);
          p.nev++;
          acc.st.n_events++;
          wn *= (1.0 - 1.0 / b);
          p.acc = 0.0;
          p.x1t = -std::log(uniform(p.s));
        } else {
          p.acc += d;
        }
      }
    }
    p.w = wn;
    p.ana = c.ana;
    p.ans = c.ans;
    double r = radius(p.X);
    if (r >= P.r_record) {
      record(M, p, acc);
      status = 1;
      acc.st.n_rec++;
      break;
    }
    if (P.mass > 0.0 && r <= M.r_h * (1.0 + P.dh)) {
      status = 3;
      acc.st.n_capt++;
      break;
    }
    if (!(p.w > 0.0)) {
      status = 2;
      acc.st.n_abs++;
      break;
    }
    if (p.w < P.roulette_w * p.wb) {
      if (uniform(p.s) < P.roulette_p) {
        p.w /= P.roulette_p;
        acc.st.n_roul_surv++;
      } else {
        status = 2;
        acc.st.n_abs++;
        break;
      }
    }
    if (p.nsteps >= P.max_steps) {
      status = 4;
      acc.st.n_maxst++;
      break;
    }
  }
  if (acc.want_log) {
    or_log L;
    L.id = p.s.id;
    L.gen = p.nsc;
    L.status = status;
    for (int m = 0; m < 4; ++m) { L.X[m] = p.X[m]; L.K[m] = p.K[m]; }
    L.w = p.w;
    L.nsteps = p.nsteps;
    L.nev = (int32_t)p.nev;
    L.pad = 0;
    acc.log.push_back(L);
  }
}

// Emission of primary superphoton uid (section 2.3): zone from the exclusive scan of counts,
// frequency proposed by rejection against the piecewise-linear interpolant (in ln nu) of the
// zone's dN/dln(nu) node values g_j, direction by rejection against j_nu(theta)/j_nu(pi/2),
// azimuth uniform, wavevector built in the emission tetrad at the zone centre.  The weight is
// w(nu) g(nu) / g_lin(nu) = int dOmega j_nu(nu) / g_lin(nu): with it the expected emitted spectrum
// is the zone's exact dN/dln(nu) (section 2.3 accepts against dN/dln(nu) at the drawn nu itself),
// and the trapezoid zone count cancels from the normalisation.
void emit(const Model &M, int64_t uid, Photon &p, int64_t *rejcap) {
  const or_params &P = M.P;
  int64_t z = (int64_t)(std::upper_bound(M.start.begin(), M.start.end(), uid) - M.start.begin()) - 1;
  p.s = Stream{M.seed, (uint64_t)uid, 0u};
  const double *gz = &M.g[(size_t)z * M.nnu];
  double gm = M.gmax[z];
  double lnu = M.lnumin, glin = 0.0;
  int it;
  for (it = 0; it < 100000; ++it) {
    double r1 = uniform(p.s);
    lnu = M.lnumin + r1 * M.dlntot;
    double fj = (lnu - M.lnumin) / M.dlnu;
    int j = std::min(std::max((int)std::floor(fj), 0), M.nnu - 2);
    double fr = fj - j;
    glin = (1.0 - fr) * gz[j] + fr * gz[j + 1];
    double r2 = uniform(p.s);
    if (r2 * gm < glin) break;
  }
  if (it == 100000) (*rejcap)++;
  double nu = std::exp(lnu);
  double pr[8];
  zone_prims(M, z, pr);
  double X[4];
  zone_center(M, z, X);
  double g[4][4];
  gcov_at(P, X, g);
  Fluid F;
  fluid_from_prims(P, M.un, pr, g, F);
  const double jsyn = jnu_angint(P, nu, F.ne, F.thetae, F.B), jbr = brems_angint(P, nu, F.ne, F.thetae);
  // with bremsstrahlung on, the emitting process is drawn in proportion to the two
  // angle-integrated emissivities; the bremsstrahlung direction is isotropic
  bool synchrotron = true;
  if (P.brems) synchrotron = uniform(p.s) * (jsyn + jbr) < jsyn;
  double cth = 0.0;
  if (synchrotron) {
    double jmax = jnu(P, nu, F.ne, F.thetae, F.B, 0.0);
    for (it = 0; it < 100000; ++it) {
      double r3 = uniform(p.s);
      cth = 2.0 * r3 - 1.0;
      double r4 = uniform(p.s);
      if (r4 * jmax < jnu(P, nu, F.ne, F.thetae, F.B, cth)) break;
    }
    if (it == 100000) (*rejcap)++;
  } else {
    cth = 2.0 * uniform(p.s) - 1.0;
  }
  double phi = 2.0 * PI * uniform(p.s);
  double sth = std::sqrt(std::max(0.0, 1.0 - cth * cth));
  double eps = HPL * nu / (ME * CL * CL);
  double e[4][4];
  // without a field (a bremsstrahlung-only plasma) the frame of the scattering tetrad serves
  if (F.bsq > 0.0) tetrad_emission(g, F, e);
  else tetrad_scatter(g, F, e);
  double kf[4] = {eps, eps * sth * std::cos(phi), eps * sth * std::sin(phi), eps * cth};
  for (int m = 0; m < 4; ++m) {
    p.X[m] = X[m];
    p.K[m] = kf[0] * e[0][m] + kf[1] * e[1][m] + kf[2] * e[2][m] + kf[3] * e[3][m];
  }
  // superphoton weight: int dOmega j_nu at the drawn nu over the interpolated target
  p.w = glin > 0.0 ? (jsyn + jbr) / glin : 0.0;
  p.nsc = 0;
}

// Weights (eq. weight_calc) and zone counts (section 2.3).
int prepare(Model &M, double n_s, uint64_t seed) {
  const or_params &P = M.P;
  M.seed = seed;
  M.nnu = P.n_nu;
  M.lnumin = std::log(P.nu_min);
  M.dlntot = std::log(P.nu_max / P.nu_min);
  M.dlnu = M.dlntot / (M.nnu - 1);
  const double dt = 1.0;
  M.vol.assign(M.nz, 0.0);
  M.g.assign((size_t)M.nz * M.nnu, 0.0);   // holds int dOmega j_nu first
  std::vector<Zone> zs(M.nz);
#pragma omp parallel
  {
    Zone last{-1.0, -1.0, -1.0};
    std::vector<double> row(M.nnu, 0.0);
#pragma omp for schedule(static)
    for (int64_t z = 0; z < M.nz; ++z) {
      double X[4], g[4][4], gi[4][4], pr[8];
      zone_center(M, z, X);
      gcov_at(P, X, g);
      double det = invert4(g, gi);
      M.vol[z] = std::sqrt(-det) * M.dx1 * M.dx2 * M.dx3 * P.L_unit * P.L_unit * P.L_unit;
      zone_prims(M, z, pr);
      Fluid F;
      fluid_from_prims(P, M.un, pr, g, F);
      Zone zz{F.ne, F.thetae, F.B};
      if (!(zz.ne == last.ne && zz.thetae == last.thetae && zz.B == last.B)) {
        for (int j = 0; j < M.nnu; ++j) {
          const double nuj = std::exp(M.lnumin + j * M.dlnu);
          row[j] = jnu_angint(P, nuj, zz.ne, zz.thetae, zz.B) + brems_angint(P, nuj, zz.ne, zz.thetae);
        }
        last = zz;
      }
      for (int j = 0; j < M.nnu; ++j) M.g[(size_t)z * M.nnu + j] = row[j];
    }
  }
  // w_j = dt dln(nu)_tot / (h N_s) sum_i V_i int dOmega j_nu(nu_j), floored at w_min (summed in zone order)
  M.lnw.assign(M.nnu, 0.0);
  std::vector<double> w(M.nnu);
  for (int j = 0; j < M.nnu; ++j) {
    double s = 0.0;
    for (int64_t z = 0; z < M.nz; ++z) s += M.vol[z] * M.g[(size_t)z * M.nnu + j];
    w[j] = std::max(P.w_min, dt * M.dlntot / (HPL * n_s) * s);
    M.lnw[j] = std::log(w[j]);
  }
  M.gmax.assign(M.nz, 0.0);
  M.nbar.assign(M.nz, 0.0);
  M.counts.assign(M.nz, 0);
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < M.nz; ++z) {
    double s = 0.0, gm = 0.0;
    for (int j = 0; j < M.nnu; ++j) {
      double gj = M.g[(size_t)z * M.nnu + j] / w[j];
      M.g[(size_t)z * M.nnu + j] = gj;
      double tj = (j == 0 || j == M.nnu - 1) ? 0.5 * M.dlnu : M.dlnu;
      s += tj * gj;
      gm = std::max(gm, gj);
    }
    double nb = dt * M.vol[z] * s / HPL;
    M.nbar[z] = nb;
    M.gmax[z] = gm;
    double fl = std::floor(nb);
    Stream st{seed, ZONE_STREAM_TAG | (uint64_t)z, 0u};
    double u = uniform(st);
    M.counts[z] = (int64_t)fl + ((u < nb - fl) ? 1 : 0);
  }
  M.start.assign(M.nz, 0);
  int64_t acc = 0;
  for (int64_t z = 0; z < M.nz; ++z) {
    M.start[z] = acc;
    acc += M.counts[z];
  }
  M.total = acc;
  return 0;
}

void merge_stats(or_stats &a, const or_stats &b) {
  a.n_emit += b.n_emit; a.n_child += b.n_child; a.n_rec += b.n_rec; a.n_abs += b.n_abs;
  a.n_capt += b.n_capt; a.n_maxst += b.n_maxst; a.n_steps += b.n_steps; a.n_iters += b.n_iters;
  a.n_nonconv += b.n_nonconv; a.n_roul_surv += b.n_roul_surv; a.n_rej_cap += b.n_rej_cap;
  a.n_events += b.n_events;
}

}  // namespace

// ================================================================= C interface
extern "C" {

void or_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }

void or_uniforms(uint64_t seed, uint64_t id, uint32_t n0, int64_t n, double *out) {
  Stream s{seed, id, n0};
  for (int64_t i = 0; i < n; ++i) out[i] = uniform(s);
}

uint64_t or_child_stream(uint64_t parent, uint32_t ev) { return child_stream(parent, ev); }

void or_gauss_legendre(int n, double a, double b, double *x, double *w) { gauss_legendre(n, a, b, x, w); }

void or_gcov(const or_params *P, const double *X, double *g16) {
  double g[4][4];
  gcov_at(*P, X, g);
  for (int i = 0; i < 16; ++i) g16[i] = g[i / 4][i % 4];
}

double or_sqrtmg(const or_params *P, const double *X) {
  double g[4][4], gi[4][4];
  gcov_at(*P, X, g);
  return std::sqrt(-invert4(g, gi));
}

void or_christoffel(const or_params *P, const double *X, double *G64) {
  double G[4][4][4];
  christoffel(*P, X, G);
  for (int i = 0; i < 64; ++i) G64[i] = G[i / 16][(i / 4) % 4][i % 4];
}

// Free geodesic (no plasma) from (X0, K0) until r >= r_out, r <= r_in or max_steps.
// Returns the number of steps; writes the end state and the largest |k.k|/(k^t)^2 seen.
int64_t or_geodesic(const or_params *P, const double *X0, const double *K0, double r_in, double r_out,
                    int64_t max_steps, double *Xe, double *Ke, double *max_null, int64_t *iters) {
  double X[4], K[4], A[4], G[4][4][4];
  for (int m = 0; m < 4; ++m) { X[m] = X0[m]; K[m] = K0[m]; }
  christoffel(*P, X, G);
  accel(G, K, A);
  double mx = 0.0;
  int64_t n = 0, its = 0;
  while (n < max_steps) {
    double dl = stepsize(*P, X, K);
    bool conv;
    its += verlet_step(*P, X, K, A, dl, &conv);
    ++n;
    double g[4][4];
    gcov_at(*P, X, g);
    double kk = dot4(g, K, K);
    mx = std::max(mx, std::fabs(kk) / (K[0] * K[0]));
    double r = radius(X);
    if (r >= r_out || r <= r_in) break;
  }
  for (int m = 0; m < 4; ++m) { Xe[m] = X[m]; Ke[m] = K[m]; }
  *max_null = mx;
  if (iters) *iters = its;
  return n;
}

double or_jnu(const or_params *P, double nu, double ne, double thetae, double B, double costh) {
  return jnu(*P, nu, ne, thetae, B, costh);
}
double or_bnu(double nu, double thetae) { return bnu(nu, thetae); }
double or_K2(const or_params *P, double thetae) { return K2_of(*P, thetae); }
double or_Fang(double K) { return Fang(K); }
double or_jnu_angint(const or_params *P, double nu, double ne, double thetae, double B) {
  return jnu_angint(*P, nu, ne, thetae, B);
}
double or_sigma_kn(double e) { return sigma_kn(e); }
double or_sigma_hot_quad(double thetae, double eps) { return sigma_hot_quad(thetae, eps); }
double or_sigma_hot_table(double thetae, double eps) { return hot_table().lookup(thetae, eps); }

void or_sample_mj(double thetae, uint64_t seed, uint64_t id, int64_t n, double *out) {
  Stream s{seed, id, 0u};
  for (int64_t i = 0; i < n; ++i) out[i] = sample_mj(thetae, s);
}

// Compton scatterings of photons of energy eps along +z in a plasma at rest; returns the
// scattered energy and direction for n independent streams id0 .. id0+n-1.
void or_compton(double thetae, double eps, uint64_t seed, uint64_t id0, int64_t n, double *eps_out, double *dir_out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    Stream s{seed, id0 + (uint64_t)i, 0u};
    double nz[3] = {0.0, 0.0, 1.0};
    double eo, d[3];
    compton_fluid(0.0, thetae, eps, nz, s, &eo, d, nullptr);
    eps_out[i] = eo;
    for (int k = 0; k < 3; ++k) dir_out[3 * i + k] = d[k];
  }
}

// Derived fluid quantities at a point (for tests of the set-up).
void or_fluid(void *h, const double *X, double *out) {
  Model &M = *(Model *)h;
  double g[4][4];
  gcov_at(M.P, X, g);
  Fluid F;
  fluid_at(M, X, g, F);
  out[0] = F.ne; out[1] = F.thetae; out[2] = F.B; out[3] = F.plasma ? 1.0 : 0.0;
  for (int m = 0; m < 4; ++m) { out[4 + m] = F.ucon[m]; out[8 + m] = F.bcon[m]; }
}

// Fluid state from primitives at a point (fluid_from_prims, sections 2.2 and 2.5), for the pins of
// the fluid frame: out = ne, thetae, |B| [G], b^2, u^mu[4], u_mu[4], b^mu[4], b_mu[4] (20 doubles).
void or_fluid_from_prims(const or_params *P, const double *X, const double *pr, double *out) {
  double g[4][4];
  gcov_at(*P, X, g);
  Fluid F;
  fluid_from_prims(*P, make_units(*P), pr, g, F);
  out[0] = F.ne; out[1] = F.thetae; out[2] = F.B; out[3] = F.bsq;
  for (int m = 0; m < 4; ++m) {
    out[4 + m] = F.ucon[m];
    out[8 + m] = F.ucov[m];
    out[12 + m] = F.bcon[m];
    out[16 + m] = F.bcov[m];
  }
}

// Plasma-frame tetrad at a point with the given primitives (sections 2.1 and 2.7): kind 0 the
// emission tetrad, 1 the scattering tetrad; e16[4 a + mu] = e_(a)^mu.
void or_tetrad(const or_params *P, const double *X, const double *pr, int kind, double *e16) {
  double g[4][4];
  gcov_at(*P, X, g);
  Fluid F;
  fluid_from_prims(*P, make_units(*P), pr, g, F);
  double e[4][4];
  if (kind == 0) tetrad_emission(g, F, e);
  else tetrad_scatter(g, F, e);
  for (int a = 0; a < 4; ++a)
    for (int m = 0; m < 4; ++m) e16[4 * a + m] = e[a][m];
}

void *or_create(const or_params *P, const or_grid *G) {
  Model *M = new Model();
  M->P = *P;
  M->un = make_units(*P);
  M->n1 = G->n1; M->n2 = G->n2; M->n3 = G->n3;
  M->nz = (int64_t)G->n1 * G->n2 * G->n3;
  M->x1_0 = G->x1_0; M->dx1 = G->dx1; M->x2_0 = G->x2_0; M->dx2 = G->dx2; M->x3_0 = G->x3_0; M->dx3 = G->dx3;
  M->prim.assign(G->prim, G->prim + (size_t)8 * M->nz);
  M->r_h = (P->mass > 0.0) ? 1.0 + std::sqrt(1.0 - P->a * P->a) : 0.0;
  if (P->scatter) hot_table();
  if (P->kappa > 0.0) {
    kappa_tables(P->kappa);
    if (P->scatter) kappa_hot(P->kappa);
  }
  return M;
}

void or_destroy(void *h) { delete (Model *)h; }

int or_prepare(void *h, double n_s, uint64_t seed) { return prepare(*(Model *)h, n_s, seed); }

int64_t or_total(void *h) { return ((Model *)h)->total; }
int64_t or_nzones(void *h) { return ((Model *)h)->nz; }

void or_get_zone(void *h, int64_t *counts, double *nbar, double *gmax, double *vol) {
  Model &M = *(Model *)h;
  for (int64_t z = 0; z < M.nz; ++z) {
    if (counts) counts[z] = M.counts[z];
    if (nbar) nbar[z] = M.nbar[z];
    if (gmax) gmax[z] = M.gmax[z];
    if (vol) vol[z] = M.vol[z];
  }
}

void or_get_weights(void *h, double *lnw) {
  Model &M = *(Model *)h;
  for (int j = 0; j < M.nnu; ++j) lnw[j] = M.lnw[j];
}

// Birth states of primaries [uid0, uid0 + n) (after or_prepare): the emission alone, without
// transport.  X, K: n x 4; w: n (test hook).
void or_emit(void *h, int64_t uid0, int64_t n, double *X, double *K, double *w) {
  Model &M = *(Model *)h;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t q = 0; q < n; ++q) {
    Photon p;
    int64_t rejcap = 0;
    emit(M, uid0 + q, p, &rejcap);
    for (int i = 0; i < 4; ++i) {
      X[4 * q + i] = p.X[i];
      K[4 * q + i] = p.K[i];
    }
    w[q] = p.w;
  }
}

// Run primaries [uid0, uid1) (or the explicit uid list when uids != NULL) with all their
// descendants; accumulate the spectrum sums [n_incl][n_bins][3] and counters.  With a log
// buffer, every finished superphoton appends its end state.  A range run resets the bias scales
// (and tunes them when bias_target > 0); a uid-list run scatters with the scales of the last
// range run.
int or_run(void *h, int64_t uid0, int64_t uid1, const int64_t *uids, int64_t nuids, double *spec, or_stats *st,
           or_log *logbuf, int64_t log_cap, int64_t *log_n, int nthreads) {
  Model &M = *(Model *)h;
  const or_params &P = M.P;
  size_t nspec = (size_t)P.n_incl * P.n_bins * 3;
  int64_t n = uids ? nuids : (uid1 - uid0);
  if (nthreads <= 0) nthreads = 1;
  std::vector<Acc> accs(nthreads);
  for (auto &a : accs) {
    a.spec.assign(nspec, 0.0);
    std::memset(&a.st, 0, sizeof(a.st));
    a.want_log = (logbuf != nullptr);
  }
  const bool tuning = P.bias_target > 0.0 && uids == nullptr;
  if (uids == nullptr) M.bscale.assign(P.n_sc_max + 1, 1.0);
  if (tuning) {
    // generation by generation (the bias of a generation depends on the previous ones), in
    // batches of 2^24 primaries as the device path runs them; the first batch sets the scales
    const int64_t kBatch = (int64_t)1 << 24;
    const int n_gen = P.n_sc_max + 1;
    for (int64_t b0 = 0; b0 < n; b0 += kBatch) {
      const int64_t nb = std::min(kBatch, n - b0);
      std::vector<Child> cur, next;
      for (int gen = 0;; ++gen) {
        const int64_t n_items = gen == 0 ? nb : (int64_t)cur.size();
        if (n_items == 0) break;
        next.clear();
#pragma omp parallel num_threads(nthreads)
        {
          int tid = 0;
#ifdef _OPENMP
          tid = omp_get_thread_num();
#endif
          Acc &acc = accs[tid];
          std::vector<Child> local;
#pragma omp for schedule(dynamic, 16)
          for (int64_t q = 0; q < n_items; ++q) {
            Photon p;
            if (gen == 0) {
              emit(M, uid0 + b0 + q, p, &acc.st.n_rej_cap);
              acc.st.n_emit++;
            } else {
              const Child &c = cur[q];
              for (int m = 0; m < 4; ++m) { p.X[m] = c.X[m]; p.K[m] = c.K[m]; }
              p.w = c.w;
              p.nsc = c.nsc;
              p.s = Stream{M.seed, c.id, c.ctr};
            }
            init_transport(M, p);
            transport(M, p, local, acc);
          }
#pragma omp critical
          next.insert(next.end(), local.begin(), local.end());
        }
        if (b0 == 0 && gen + 1 < n_gen)
          M.bscale[gen + 1] = tune_next_scale(M.bscale[gen], n_items, (int64_t)next.size(), P.bias_target);
        cur.swap(next);
      }
    }
  } else
#pragma omp parallel num_threads(nthreads)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    Acc &acc = accs[tid];
    std::vector<Child> stack;
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; ++q) {
      int64_t uid = uids ? uids[q] : uid0 + q;
      Photon p;
      emit(M, uid, p, &acc.st.n_rej_cap);
      acc.st.n_emit++;
      init_transport(M, p);
      transport(M, p, stack, acc);
      while (!stack.empty()) {
        Child c = stack.back();
        stack.pop_back();
        Photon ch;
        for (int m = 0; m < 4; ++m) { ch.X[m] = c.X[m]; ch.K[m] = c.K[m]; }
        ch.w = c.w;
        ch.nsc = c.nsc;
        ch.s = Stream{M.seed, c.id, c.ctr};
        init_transport(M, ch);
        transport(M, ch, stack, acc);
      }
    }
  }
  std::memset(st, 0, sizeof(*st));
  for (size_t i = 0; i < nspec; ++i) spec[i] = 0.0;
  int64_t nl = 0;
  for (auto &a : accs) {
    for (size_t i = 0; i < nspec; ++i) spec[i] += a.spec[i];
    merge_stats(*st, a.st);
    if (logbuf)
      for (auto &L : a.log)
        if (nl < log_cap) logbuf[nl++] = L;
  }
  if (log_n) *log_n = nl;
  return 0;
}

double or_brems_q(double ne, double thetae) { return brems_q(ne, thetae); }
double or_F_sync(double x) { return F_sync_direct(x); }
double or_sigma_hot_kappa(double kappa, double w, double eps) { return kappa_hot(kappa).lookup(w, eps); }
void or_sample_kappa(double kappa, double w, uint64_t seed, uint64_t stream, int64_t n, double *out) {
  Stream s{seed, stream, 0u};
  for (int64_t i = 0; i < n; ++i) out[i] = sample_kappa(kappa, w, s, nullptr);
}
void or_compton_kappa(double kappa, double thetae, double eps, uint64_t seed, uint64_t stream0, int64_t n,
                      double *eps_out, double *mu_out) {
  const double nz[3] = {0.0, 0.0, 1.0};
  for (int64_t i = 0; i < n; ++i) {
    Stream s{seed, stream0 + (uint64_t)i, 0u};
    double eo, d[3];
    compton_fluid(kappa, thetae, eps, nz, s, &eo, d, nullptr);
    eps_out[i] = eo;
    mu_out[i] = d[2] / std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  }
}
double or_jnu_kappa(const or_params *P, double nu, double ne, double thetae, double B, double costh) {
  return jnu(*P, nu, ne, thetae, B, costh);
}
double or_nu_alpha_kappa(const or_params *P, double nu, double ne, double thetae, double B, double costh) {
  return nu_alpha_kappa(*P, nu, ne, thetae, B, costh);
}
double or_brems_angint(const or_params *P, double nu, double ne, double thetae) {
  return brems_angint(*P, nu, ne, thetae);
}
double or_brems_nu_alpha(const or_params *P, double nu, double ne, double thetae) {
  return brems_nu_alpha(*P, nu, ne, thetae);
}

int or_get_bias_scales(void *h, double *out, int n) {
  Model &M = *(Model *)h;
  for (int g = 0; g < n; ++g) out[g] = M.scale_of(g);
  return 0;
}

}  // extern "C"
