// mc_push.cuh -- per-superphoton transport arithmetic shared by the transport kernels
// (mc_transport.cu) and the batched persistent kernel (mc_batch.cu): state, emission (section 2.3),
// initialisation, the in-grid step (sections 2.4-2.7), the free-streaming step, recording and the
// Compton child (section 2.7), and the surrogate-split in-grid step.
#pragma once
#include <type_traits>

#include "mc_internal.h"

namespace mcgb {


// Precision forms of the transport.  S: the geodesic scalar; W: the weight, optical-depth and
// coefficient scalar; C32: FP32 plasma coefficients; K32: FP32 Compton kinematics.
//   0 plain FP64: every step in FP64;
//   1 mixed: geodesic in double-float (FP64-level accuracy on the FP32 pipes); FP32 coefficients,
//     optical depths, weights (relative to the FP64 birth weight) and scattering decision; FP64
//     Compton kinematics;
//   2 split: FP64 geodesic and step size, FP32 coefficients, optical depths, weights (relative to the
//     superphoton's FP64 birth weight), scattering decision and Compton kinematics.
template <int PREC> struct Form;
template <> struct Form<0> { using S = double; using W = double; static constexpr bool C32 = false, K32 = false; };
template <> struct Form<1> { using S = df; using W = float; static constexpr bool C32 = true, K32 = false; };
template <> struct Form<2> { using S = double; using W = float; static constexpr bool C32 = true, K32 = true; };

// Superphoton state.  The pool between phases holds FP64 (absolute weights); a transport kernel
// converts at load and save.  With W = float the weight is carried relative to the birth weight wb
// (weights reach 1e45, beyond FP32; the relative weight stays within [1e-13, ~10]).
template <typename S, typename W = double>
struct PhT {
  S X[4], K[4], A[4];
  W w, ana, ans, acc, x1t;
  double wb;
  Rng s;
  int nsc;
  uint32_t nev;
  int nsteps;
  int model;     // index of the superphoton's model in a batched run (0 otherwise)
  W wthr;        // roulette threshold: roulette_w * wb (W = float: roulette_w, relative); set at load
  double *raddr; // spectrum bin of a record made in this loop iteration (NULL: none), flushed per warp
  double rwe;    // its w E
};
using Ph = PhT<double>;
template <int PREC>
using PhF = PhT<typename Form<PREC>::S, typename Form<PREC>::W>;

// absolute weight of a superphoton state
template <typename S, typename W>
__device__ __forceinline__ double abs_w(const PhT<S, W> &p) {
  if constexpr (std::is_same<W, float>::value) return (double)p.w * p.wb;
  else return p.w;
}

struct LocalStats {
  unsigned long long emit, child, rec, abs, capt, maxst, steps, iters, nonconv, roul, rejcap, events, gsteps, giters;
};

template <bool C32, typename S, typename W>
__device__ __forceinline__ void coefs(const DevModel &m, const GeoT<S> &G, const S X[4], const S K[4], bool ws,
                                      CoefT<W> &c) {
  if constexpr (C32) coefficients32(m, G, X, K, ws, c);
  else coefficients64(m, G, X, K, ws, c);
}

template <bool C32, bool KERR = true>
static __device__ void init_transport(const DevModel &m, Ph &p) {
  p.x1t = -log(rng_u(p.s, m.seed));
  p.acc = 0.0;
  bool scat = m.scatter && p.nsc < m.n_sc_max;
  Geo G;
  metric_eval<true, KERR>(m, p.X[1], p.X[2], G);
  Coef c;
  coefs<C32>(m, G, p.X, p.K, scat, c);
  p.ana = c.ana;
  p.ans = c.ans;
  accel<KERR>(G, p.K, p.A);
  p.nsteps = 0;
  p.nev = 0;
  p.wb = p.w;
}

// Emission of primary uid (section 2.3) at the centre of its zone: frequency proposed from the
// piecewise-linear interpolant of the zone's dN/dln(nu) node values, weighted back to the exact one.
// In three parts: the zone and its emission data, the frequency rejection (run warp-cooperatively,
// emit_nu_warp), and the rest (direction, tetrad, wavevector, weight; emit_finish).
constexpr int kMaxRej = 100000;   // proposals per rejection loop before the draw is taken as it stands

struct EmitZone {
  int64_t z;
  double pref, lnuc, gm;
};

__device__ __forceinline__ EmitZone emit_zone(const DevModel &m, int64_t uid) {
  int64_t lo = 0, hi = m.nz - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(m.start + mid) <= uid) lo = mid;
    else hi = mid - 1;
  }
  return {lo, m.zpref[lo], m.zlnuc[lo], m.zgmax[lo]};
}

// Warp-cooperative rejection sampling.  Sequentially (as the method states it, and as a lane alone
// would run it), a superphoton evaluates proposals k = 0, 1, ... of a rejection loop, proposal k from
// its own stream positions n0 + 2k and n0 + 2k + 1, and takes the first accepted one.  coop_reject
// runs the loops of the 32 superphotons of a warp at once: each round hands the next proposals of the
// p pending superphotons to all 32 lanes (lane L evaluates proposal k0 + L/p of the (L mod p)-th
// pending superphoton, whose inputs and stream it reads by shuffles), and each superphoton takes its
// lowest accepted proposal of the round.  The draws, the accepted proposal, its values and the stream
// position afterwards are those of the sequential loop (the stream is counter based), with its cap of
// kMaxRej proposals (the last one then stands); the lanes no longer wait for a warp's slowest
// acceptance, and proposals past the first accepted one are evaluated and dropped.  Every lane of the
// warp calls it (have = false: no loop for this lane).  Pol supplies the inputs Par, the result Val,
// their shuffles and one proposal, eval(model, Par, stream, Val) -> accepted.  BATCH: the superphotons
// of a warp may belong to different models of a batched run (sm[model]); otherwise every one belongs
// to m.
template <bool BATCH, typename Pol>
static __device__ void coop_reject(const DevModel &m, const DevModel *sm, bool have, int model,
                                   const typename Pol::Par &par, uint64_t id, uint32_t &n, typename Pol::Val &out,
                                   LocalStats &ls) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool done = !have;
  int it = 0;   // proposals of this lane's superphoton evaluated so far
  while (true) {
    const unsigned P = __ballot_sync(FULL, !done);
    if (!P) break;
    const int np = __popc(P);
    const int rank = lane % np, k = lane / np;
    unsigned rest = P;   // the lane of the rank-th pending superphoton: drop the rank lowest set bits
    for (int i = 0; i < rank; ++i) rest &= rest - 1u;
    const int owner = __ffs(rest) - 1;
    const typename Pol::Par po = Pol::shfl(par, owner);
    const uint64_t ido = __shfl_sync(FULL, id, owner);
    const uint32_t no = __shfl_sync(FULL, n, owner);
    const int ito = __shfl_sync(FULL, it, owner);
    const int mo = BATCH ? __shfl_sync(FULL, model, owner) : 0;
    const bool valid = ito + k < kMaxRej;
    bool acc = false;
    typename Pol::Val v = Pol::zero();
    if (valid) {
      Rng s;
      rng_init(s, ido, no + 2u * (uint32_t)k);
      if constexpr (BATCH) acc = Pol::eval(sm[mo], po, s, v);
      else acc = Pol::eval(m, po, s, v);
    }
    // lanes working for the same superphoton; its proposals rise with the lane index
    const unsigned grp = __match_any_sync(FULL, owner);
    const unsigned A = __ballot_sync(FULL, acc) & grp, V = __ballot_sync(FULL, valid) & grp;
    const int win = A ? __ffs(A) - 1 : -1;
    const int last = V ? 31 - __clz(V) : -1;
    const int cnt = __popc(V);
    // the pending lane of rank r reads the result of its group, whose first lane is lane r
    const int myrank = __popc(P & ((1u << lane) - 1u));
    const int src = (!done) ? myrank : lane;
    const int win_o = __shfl_sync(FULL, win, src);
    const int last_o = __shfl_sync(FULL, last, src);
    const int cnt_o = __shfl_sync(FULL, cnt, src);
    const int pick = win_o >= 0 ? win_o : (last_o >= 0 ? last_o : lane);
    const typename Pol::Val vp = Pol::shfl(v, pick);
    if (!done) {
      if (win_o >= 0) {
        const int kw = (win_o - myrank) / np;
        n += 2u * (uint32_t)(kw + 1);
        out = vp;
        done = true;
      } else {
        n += 2u * (uint32_t)cnt_o;
        it += cnt_o;
        if (it >= kMaxRej) {   // the sequential loop's cap: its last proposal stands
          out = vp;
          ls.rejcap++;
          done = true;
        }
      }
    }
  }
}

// Frequency proposal: ln nu uniform over the table (r1), accepted when r2 gm < g_lin(ln nu).
struct NuPol {
  using Par = EmitZone;
  struct Val {
    double lnu, glin;
  };
  __device__ static Val zero() { return {0.0, 0.0}; }
  __device__ static Par shfl(const Par &p, int src) {
    return {__shfl_sync(0xffffffffu, p.z, src), __shfl_sync(0xffffffffu, p.pref, src),
            __shfl_sync(0xffffffffu, p.lnuc, src), __shfl_sync(0xffffffffu, p.gm, src)};
  }
  __device__ static Val shfl(const Val &v, int src) {
    return {__shfl_sync(0xffffffffu, v.lnu, src), __shfl_sync(0xffffffffu, v.glin, src)};
  }
  __device__ static bool eval(const DevModel &m, const Par &Z, Rng &s, Val &v) {
    double r1 = rng_u(s, m.seed);
    v.lnu = m.lnu_min + r1 * m.dlntot;
    double fj = (v.lnu - m.lnu_min) / m.dlnu;
    int j = min(max((int)floor(fj), 0), m.n_nu - 2);
    double fr = fj - j;
    double g0 = zone_E(m, Z.z, Z.pref, Z.lnuc, j) * m.winv[j];
    double g1 = zone_E(m, Z.z, Z.pref, Z.lnuc, j + 1) * m.winv[j + 1];
    v.glin = (1.0 - fr) * g0 + fr * g1;
    double r2 = rng_u(s, m.seed);
    return r2 * Z.gm < v.glin;
  }
};

// Direction relative to b, thermal synchrotron: cos(theta) uniform (r3), accepted with
// j(theta)/j(pi/2) = sin(th) G(K/sin th) / G(K), K = nu/nu_c (r4 jmax < sin th G(K0 / sin th)).
struct ThPol {
  struct Par {
    double K0, jmax;
  };
  struct Val {
    double cth;
  };
  __device__ static Val zero() { return {0.0}; }
  __device__ static Par shfl(const Par &p, int src) {
    return {__shfl_sync(0xffffffffu, p.K0, src), __shfl_sync(0xffffffffu, p.jmax, src)};
  }
  __device__ static Val shfl(const Val &v, int src) { return {__shfl_sync(0xffffffffu, v.cth, src)}; }
  __device__ static bool eval(const DevModel &m, const Par &q, Rng &s, Val &v) {
    double r3 = rng_u(s, m.seed);
    v.cth = 2.0 * r3 - 1.0;
    double r4 = rng_u(s, m.seed);
    double sth = sqrt(1.0 - v.cth * v.cth);
    return r4 * q.jmax < sth * Gsyn_t(m.ftab, q.K0 / sth);
  }
};

// Direction relative to b, kappa electrons: accepted with sin(th) J(X / sin th, w) / J(X, w), X = nu/nu_B.
struct ThKPol {
  struct Par {
    double lX, lw, jmax;
  };
  struct Val {
    double cth;
  };
  __device__ static Val zero() { return {0.0}; }
  __device__ static Par shfl(const Par &p, int src) {
    return {__shfl_sync(0xffffffffu, p.lX, src), __shfl_sync(0xffffffffu, p.lw, src),
            __shfl_sync(0xffffffffu, p.jmax, src)};
  }
  __device__ static Val shfl(const Val &v, int src) { return {__shfl_sync(0xffffffffu, v.cth, src)}; }
  __device__ static bool eval(const DevModel &m, const Par &q, Rng &s, Val &v) {
    double r3 = rng_u(s, m.seed);
    v.cth = 2.0 * r3 - 1.0;
    double r4 = rng_u(s, m.seed);
    double sth = sqrt(1.0 - v.cth * v.cth);
    double jt = sth > 0.0 ? sth * kap_interp(m.kapJ, q.lX - log(sth), q.lw) : 0.0;
    return r4 * q.jmax < jt;
  }
};

static __device__ void emit_post(const DevModel &m, const EmitZone &Z, double lnu, double glin, double jsum,
                                 double cth, Ph &p);

// Emission for the 32 lanes of a warp (every lane calls it; have = false: no superphoton).
// BATCH: lane's superphoton belongs to model `model` of the batch descriptors sm (m is not read).
template <bool BATCH = false>
static __device__ void emit_warp(const DevModel &m, const DevModel *sm, bool have, int model, int64_t uid, Ph &p,
                                 LocalStats &ls) {
  const DevModel &mine = BATCH ? sm[have ? model : 0] : m;
  EmitZone Z = {0, 0.0, 0.0, 1.0};
  if (have) Z = emit_zone(mine, uid);
  uint32_t n = 0u;
  NuPol::Val nv = NuPol::zero();
  coop_reject<BATCH, NuPol>(m, sm, have, model, Z, (uint64_t)uid, n, nv, ls);
  const double lnu = nv.lnu, glin = nv.glin;
  // the zone's emissivities at that frequency; with bremsstrahlung on, the process is drawn in
  // proportion to the two angle-integrated emissivities (bremsstrahlung is isotropic)
  double jsyn = 0.0, jbr = 0.0;
  int kind = 0;   // direction: 0 isotropic, 1 thermal synchrotron, 2 kappa synchrotron
  ThPol::Par tp = {1.0, 1.0};
  ThKPol::Par kp = {0.0, 0.0, 1.0};
  if (have) {
    const int64_t z = Z.z;
    const double pref = Z.pref, lnuc = Z.lnuc;
    jsyn = (pref == 0.0) ? 0.0
           : (mine.kappa > 0.0) ? pref * kap_interp(mine.kapI, lnu - lnuc, mine.zlnw[z])
                                : pref * F_of_lnK(mine, lnu - lnuc);
    jbr = (mine.brems && mine.zbq[z] > 0.0) ? mine.zbq[z] * exp_t(mine.ftab, -exp_t(mine.ftab, lnu) / mine.zbnt[z])
                                            : 0.0;
    bool synchrotron = true;
    if (mine.brems) {
      Rng s;
      rng_init(s, (uint64_t)uid, n);
      synchrotron = rng_u(s, mine.seed) * (jsyn + jbr) < jsyn;
      n += 1u;
    }
    if (synchrotron && mine.kappa > 0.0) {
      const double lX = lnu - lnuc, lw = mine.zlnw[z];
      kp = {lX, lw, kap_interp(mine.kapJ, lX, lw)};
      kind = 2;
    } else if (synchrotron) {
      const double K0 = exp_t(mine.ftab, lnu - lnuc);
      tp = {K0, Gsyn_t(mine.ftab, K0)};
      kind = 1;
    }
  }
  ThPol::Val tv = ThPol::zero();
  coop_reject<BATCH, ThPol>(m, sm, have && kind == 1, model, tp, (uint64_t)uid, n, tv, ls);
  ThKPol::Val kv = ThKPol::zero();
  coop_reject<BATCH, ThKPol>(m, sm, have && kind == 2, model, kp, (uint64_t)uid, n, kv, ls);
  if (!have) return;
  rng_init(p.s, (uint64_t)uid, n);
  double cth = kind == 1 ? tv.cth : kind == 2 ? kv.cth : 2.0 * rng_u(p.s, mine.seed) - 1.0;
  emit_post(mine, Z, lnu, glin, jsyn + jbr, cth, p);
}

static __device__ void emit_post(const DevModel &m, const EmitZone &Z, double lnu, double glin, double jsum,
                                 double cth, Ph &p) {
  const int64_t z = Z.z;
  double phi = 2.0 * rng_u(p.s, m.seed);   // units of pi
  double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
  double eps = exp_t(m.ftab, lnu) * (kHPL / (kME * kCL * kCL));
  // plasma at the zone centre
  int64_t iz = z / ((int64_t)m.n2 * m.n3), jz = (z / m.n3) % m.n2, kz = z % m.n3;
  double X[4] = {0.0, m.x1_0 + (iz + 0.5) * m.dx1, m.x2_0 + (jz + 0.5) * m.dx2, m.x3_0 + (kz + 0.5) * m.dx3};
  Geo G;
  metric_eval<false>(m, X[1], X[2], G);
  double pr[8];
  if (m.prim_f32) {
    for (int f = 0; f < 8; ++f) pr[f] = (double)m.prim32[z * 8 + f];
  } else {
    for (int f = 0; f < 8; ++f) pr[f] = m.prim64[z * 8 + f];
  }
  Plasma<double> P;
  double ucon[4], bcon[4];
  plasma_from_prims<double>(m, G, pr, P, ucon, bcon);
  double e[4][4];
  // without a field (a bremsstrahlung-only plasma) the frame of the scattering tetrad serves
  if (P.bsq > 0.0) tetrad_emission(G, ucon, bcon, P.bsq, e);
  else tetrad_scatter(G, ucon, e);
  double sp, cp;
  sincospi(phi, &sp, &cp);
  double kf[4] = {eps, eps * sth * cp, eps * sth * sp, eps * cth};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p.X[q] = X[q];
    p.K[q] = kf[0] * e[0][q] + kf[1] * e[1][q] + kf[2] * e[2][q] + kf[3] * e[3][q];
  }
  // weight w(nu) g(nu) / g_lin(nu) = int dOmega j_nu(nu) / g_lin(nu): the proposal follows the
  // piecewise-linear target, the weight restores the zone's exact dN/dln(nu) (section 2.3)
  p.w = glin > 0.0 ? jsum / glin : 0.0;
  p.nsc = 0;
}

// Compton kinematics of a scattered superphoton (section 2.7): at the event point Xe with the
// pre-event wavevector Ke, in the plasma frame there (radial lookup clamped to the grid), drawing from
// the child's own stream (cid from its start).  Returns the child's wavevector and the stream
// position after the draws.  Run when the child is loaded for the next generation, not inside the
// push: the child's stream is its own, so the result is the same as at the event itself.
// Scattering tetrad in FP32 from the FP64 metric at the point (split precision form).
static __device__ void tetrad_scatter_f(const Geo &G, const float u[4], float e[4][4]) {
  const float g00 = (float)G.g00, g01 = (float)G.g01, g03 = (float)G.g03, g11 = (float)G.g11, g13 = (float)G.g13,
              g22 = (float)G.g22, g33 = (float)G.g33;
  auto dotf = [&](const float a[4], const float b[4]) {
    return a[0] * (g00 * b[0] + g01 * b[1] + g03 * b[3]) + a[1] * (g01 * b[0] + g11 * b[1] + g13 * b[3]) +
           a[2] * (g22 * b[2]) + a[3] * (g03 * b[0] + g13 * b[1] + g33 * b[3]);
  };
#pragma unroll
  for (int q = 0; q < 4; ++q) e[0][q] = u[q];
  for (int k = 1; k < 4; ++k) {
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    t[k] = 1.0f;
    const float d0 = dotf(t, e[0]);
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] += d0 * e[0][q];
    for (int j = 1; j < k; ++j) {
      const float d = dotf(t, e[j]);
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] -= d * e[j][q];
    }
    const float n2 = dotf(t, t);
    const float in = n2 > 1e-30f ? rsqrtf(n2) : 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) e[k][q] = t[q] * in;
  }
}

// FP32 Compton kinematics (split precision form): the plasma frame, electron and Klein-Nishina draws
// in FP32 from the same stream; the child's wavevector is null to FP32 rounding (~1e-7 relative),
// far below the geodesic integrator's own drift of the null condition.
static __device__ void child_kinematics_f(const DevModel &m, const double Xe[4], const double Ke[4], uint64_t cid,
                                          double Kc[4], uint32_t &ctr, LocalStats &ls) {
  Geo G;
  metric_eval<false>(m, Xe[1], Xe[2], G);
  double Xc[4] = {Xe[0], fmin(fmax(Xe[1], m.x1_0), m.x1_hi), Xe[2], Xe[3]};
  float pr[8];
  interp_prims<float, double, true>(m, Xc, pr);
  Plasma<float> P;
  float ucon[4];
  plasma_from_prims<float, double, true>(m, G, pr, P, ucon, nullptr);
  float e[4][4];
  tetrad_scatter_f(G, ucon, e);
  const float k0 = (float)Ke[0], k1 = (float)Ke[1], k2 = (float)Ke[2], k3 = (float)Ke[3];
  const float kc[4] = {(float)G.g00 * k0 + (float)G.g01 * k1 + (float)G.g03 * k3,
                       (float)G.g01 * k0 + (float)G.g11 * k1 + (float)G.g13 * k3, (float)G.g22 * k2,
                       (float)G.g03 * k0 + (float)G.g13 * k1 + (float)G.g33 * k3};
  float kf[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float d = e[a][0] * kc[0] + e[a][1] * kc[1] + e[a][2] * kc[2] + e[a][3] * kc[3];
    kf[a] = (a == 0) ? -d : d;
  }
  const float eps = kf[0];
  const float il = rsqrtf(kf[1] * kf[1] + kf[2] * kf[2] + kf[3] * kf[3]);
  const float n[3] = {kf[1] * il, kf[2] * il, kf[3] * il};
  Rng s;
  rng_init(s, cid, 0u);
  float eo, dir[3];
  int rej = 0;
  compton_fluid<float>(m.kappa_on ? (float)m.kappa : 0.0f, fmaxf(P.thetae, 1e-8f), eps, n, s, m.seed, eo, dir, rej);
  ls.rejcap += rej;
#pragma unroll
  for (int q = 0; q < 4; ++q) Kc[q] = (double)(eo * e[0][q] + dir[0] * e[1][q] + dir[1] * e[2][q] + dir[2] * e[3][q]);
  ctr = s.n;
}

static __device__ void child_kinematics(const DevModel &m, const double Xe[4], const double Ke[4], uint64_t cid,
                                        double Kc[4], uint32_t &ctr, LocalStats &ls) {
  Geo G;
  metric_eval<false>(m, Xe[1], Xe[2], G);
  double Xc[4] = {Xe[0], fmin(fmax(Xe[1], m.x1_0), m.x1_hi), Xe[2], Xe[3]};
  double pr[8];
  interp_prims<double>(m, Xc, pr);
  Plasma<double> P;
  double ucon[4];
  plasma_from_prims<double>(m, G, pr, P, ucon, nullptr);
  double e[4][4];
  tetrad_scatter(G, ucon, e);
  double kc[4];
  lower(G, Ke, kc);
  double kf[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double d = e[a][0] * kc[0] + e[a][1] * kc[1] + e[a][2] * kc[2] + e[a][3] * kc[3];
    kf[a] = (a == 0) ? -d : d;
  }
  double eps = kf[0];
  double il = 1.0 / sqrt(kf[1] * kf[1] + kf[2] * kf[2] + kf[3] * kf[3]);
  double n[3] = {kf[1] * il, kf[2] * il, kf[3] * il};
  Rng s;
  rng_init(s, cid, 0u);
  double eo, dir[3];
  int rej = 0;
  compton_fluid(m.kappa, fmax(P.thetae, 1e-8), eps, n, s, m.seed, eo, dir, rej);
  ls.rejcap += rej;
#pragma unroll
  for (int q = 0; q < 4; ++q) Kc[q] = eo * e[0][q] + dir[0] * e[1][q] + dir[1] * e[2][q] + dir[2] * e[3][q];
  ctr = s.n;
}

// Compton event at Xe with pre-event wavevector Ke: the child (weight wc, stream cid, generation nsc)
// goes to the next generation's queue with stream position 0, which marks its kinematics as pending.
static __device__ void scatter_child(const PushIO &io, const double Xe[4], const double Ke[4], double wc, uint64_t cid,
                                     int nsc, int model, LocalStats &ls) {
  unsigned long long slot = atomicAdd(io.cnt + CNT_OUT, 1ull);
  ls.child++;
  if ((int64_t)slot >= io.out_cap) {
    atomicOr(io.cnt + CNT_ERR, 1ull);
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    io.out.X[q][slot] = Xe[q];
    io.out.K[q][slot] = Ke[q];
  }
  io.out.w[slot] = wc;
  io.out.id[slot] = cid;
  io.out.ctr[slot] = 0u;
  io.out.nsc[slot] = nsc;
  if (io.out.model) io.out.model[slot] = (int16_t)model;
}

// Loads child idx of a queue into p, running its pending Compton kinematics (FP32 with K32).
template <bool K32 = false>
static __device__ void load_child(const DevModel &m, const ChildBuf &q, int64_t idx, Ph &p, LocalStats &ls) {
  double Ke[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    p.X[k] = q.X[k][idx];
    Ke[k] = q.K[k][idx];
  }
  p.w = q.w[idx];
  const uint64_t id = q.id[idx];
  uint32_t ctr = q.ctr[idx];
  if (ctr == 0u) {
    if constexpr (K32) child_kinematics_f(m, p.X, Ke, id, p.K, ctr, ls);
    else child_kinematics(m, p.X, Ke, id, p.K, ctr, ls);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) p.K[k] = Ke[k];
  }
  rng_init(p.s, id, ctr);
  p.nsc = q.nsc[idx];
}

template <typename S>
__device__ __forceinline__ bool in_grid(const DevModel &m, const S X[4]) {
  if constexpr (std::is_same<S, df>::value) {
    return df_ge(X[1], m.dx1_0) && df_le(X[1], m.dx1_hi);
  } else {   // order keys of the doubles: the same test on the integer pipes
    const long long k = dkey(X[1]);
    return k >= dkey(m.x1_0) && k <= dkey(m.x1_hi);
  }
}
// Weight tests of the termination logic, on the bit patterns of the (non-negative) doubles compared
// as integers, which order them the same way, so that they take no FP64-pipe slot: w > 0 (NaN
// fails, as in FP64) and w < roulette_w * wb (the threshold is formed once, at load).
template <typename S, typename W>
__device__ __forceinline__ bool w_positive(const PhT<S, W> &p) {
  if constexpr (std::is_same<W, float>::value) {
    return p.w > 0.0f;
  } else {
    const long long b = __double_as_longlong(p.w);
    return b > 0 && b <= 0x7FF0000000000000LL;
  }
}
template <typename S, typename W>
__device__ __forceinline__ bool w_roulette(const DevModel &m, const PhT<S, W> &p) {
  if constexpr (std::is_same<W, float>::value) return p.w < p.wthr;
  else return __double_as_longlong(p.w) < __double_as_longlong(p.wthr);
}
// Russian roulette survival draw (survival roulette_p, weight / roulette_p)
template <typename S, typename W>
__device__ __forceinline__ bool roulette_survives(const DevModel &m, PhT<S, W> &p) {
  if constexpr (std::is_same<W, float>::value) {
    if (rng_r<float>(p.s, m.seed) < m.froulette_p) {
      p.w /= m.froulette_p;
      return true;
    }
  } else {
    if (rng_u(p.s, m.seed) < m.roulette_p) {
      p.w /= m.roulette_p;
      return true;
    }
  }
  return false;
}

// termination radii (recording sphere, capture near the horizon) in the geodesic's scalar; r > 0,
// so the FP64 tests compare bit patterns (a negative r_capture, the flat metric's, never captures)
__device__ __forceinline__ bool at_record(const DevModel &m, double r) { return dge_nn(r, m.r_record); }
__device__ __forceinline__ bool at_record(const DevModel &m, df r) { return df_ge(r, m.dr_record); }
__device__ __forceinline__ bool at_capture(const DevModel &m, double r) { return dle_nn(r, m.r_capture); }
__device__ __forceinline__ bool at_capture(const DevModel &m, df r) { return df_le(r, m.dr_capture); }

// Binning of a superphoton at the recording sphere (section 3): E_inf = -k_t, log-frequency bin x
// inclination bin.  The sums are not added here: the bin and w E wait in the state until the warp's
// flush_record, which adds each bin's share of the warp once.
template <typename GS, typename S, typename W>
static __device__ void record(const DevModel &m, const PushIO &io, const GeoT<GS> &G, PhT<S, W> &p) {
  double E = -(to_d(G.g00) * to_d(p.K[0]) + to_d(G.g01) * to_d(p.K[1]) + to_d(G.g03) * to_d(p.K[3]));
  if (!(E > 0.0)) return;
  double nu = E * (kME * kCL * kCL / kHPL);
  double l = log10(nu);
  int ib = (int)floor((l - m.lnu_lo) / m.dlog_bin);
  if (ib < 0 || ib >= m.n_bins) return;
  double thf = acos(fabs(to_d(G.cth)));
  int ii = (int)floor(thf / (0.5 * kPI) * m.n_incl);
  ii = min(max(ii, 0), m.n_incl - 1);
  p.raddr = m.spec + ((int64_t)ii * m.n_bins + ib) * 3;
  p.rwe = abs_w(p) * E;
}

// Warp-aggregated spectrum accumulation.  All 32 lanes call it at a converged point of their
// persistent loop (the loop's exit is warp-uniform); lanes whose superphoton was recorded in this
// iteration and that hit the same bin (of the same model) add sum w E, sum (w E)^2 and the count
// through their lowest lane, so a bin takes one set of FP64 atomics per warp and iteration.
template <typename S, typename W>
__device__ __forceinline__ void flush_record(PhT<S, W> &p) {
  const unsigned pend = __ballot_sync(0xffffffffu, p.raddr != nullptr);
  if (pend == 0u) return;
  const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)p.raddr);
  double s1 = 0.0, s2 = 0.0, n = 0.0;
  for (unsigned rem = pend; rem; rem &= rem - 1u) {   // pend is the same on every lane
    const int src = __ffs(rem) - 1;
    const double v = __shfl_sync(0xffffffffu, p.rwe, src);
    if ((peers >> src) & 1u) {
      s1 += v;
      s2 += v * v;
      n += 1.0;
    }
  }
  if (p.raddr && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    atomicAdd(p.raddr, s1);
    atomicAdd(p.raddr + 1, s2);
    atomicAdd(p.raddr + 2, n);
  }
  p.raddr = nullptr;
}

template <typename S, typename W>
static __device__ void write_log(const PushIO &io, const PhT<S, W> &p, int status) {
  if (!io.log) return;
  unsigned long long slot = atomicAdd(io.cnt + CNT_LOG, 1ull);
  if ((int64_t)slot >= io.log_cap) {
    atomicOr(io.cnt + CNT_ERR, 2ull);
    return;
  }
  mc_log_rec &L = io.log[slot];
  L.id = p.s.id;
  L.gen = p.nsc;
  L.status = status;
  for (int q = 0; q < 4; ++q) {
    L.X[q] = to_d(p.X[q]);
    L.K[q] = to_d(p.K[q]);
  }
  L.w = abs_w(p);
  L.nsteps = p.nsteps;
  L.nev = (int32_t)p.nev;
  L.pad = 0;
}

// Absorption, biased scattering (event located by linear fraction within the step) and the weight
// update of one in-grid step, in the weight scalar W of the precision form.  X0, K0: the step's start.
template <typename S, typename W>
__device__ __forceinline__ void absorb_scatter(const DevModel &m, const PushIO &io, PhT<S, W> &p, const S X0[4],
                                               const S K0[4], S dls, const CoefT<W> &c, bool scat, LocalStats &ls) {
  if constexpr (std::is_same<W, float>::value) {
    // the step length in FP32: narrowed on the integer pipes (FP64), or hi + lo (double-float)
    const float C = m.fCcoef, dl = step_f(dls);
    const float tau_a = 0.5f * (p.ana + c.ana) * C * dl;
    const float w0 = p.w;
    float wn = w0 * expf(-tau_a);
    if (scat) {
      const float tau_s = 0.5f * (p.ans + c.ans) * C * dl;
      if (tau_s > 0.0f) {
        const float b = bias_of_f(m, c.thetae, p.nsc);
        const float d = b * tau_s;
        if (p.acc + d > p.x1t) {
          const float f = (p.x1t - p.acc) / d;
          const double fd = f;
          double Xe[4], Ke[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Xe[q] = to_d(X0[q]) + fd * (to_d(p.X[q]) - to_d(X0[q]));
            Ke[q] = to_d(K0[q]) + fd * (to_d(p.K[q]) - to_d(K0[q]));
          }
          const float we = w0 * expf(-f * tau_a) / b;   // relative to the birth weight
          uint64_t cid = child_id(p.s.id, p.nev);
          scatter_child(io, Xe, Ke, (double)we * p.wb, cid, p.nsc + 1, p.model, ls);
          p.nev++;
          ls.events++;
          wn *= 1.0f - 1.0f / b;
          p.acc = 0.0f;
          p.x1t = -logf(rng_r<float>(p.s, m.seed));
        } else {
          p.acc += d;
        }
      }
    }
    p.w = wn;
  } else {
    const double C = m.Ccoef, dld = to_d(dls);
    double tau_a = 0.5 * (p.ana + c.ana) * C * dld;
    double w0 = p.w;
    double wn = w0 * exp_t(m.ftab, -tau_a);
    if (scat) {
      double tau_s = 0.5 * (p.ans + c.ans) * C * dld;
      if (__double_as_longlong(tau_s) > 0) {   // tau_s > 0 (tau_s >= 0)
        double b = bias_of(m, c.thetae, p.nsc);
        double d = b * tau_s;
        if (__double_as_longlong(p.acc + d) > __double_as_longlong(p.x1t)) {   // both >= 0
          double f = (p.x1t - p.acc) / d;
          double Xe[4], Ke[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Xe[q] = to_d(X0[q]) + f * (to_d(p.X[q]) - to_d(X0[q]));
            Ke[q] = to_d(K0[q]) + f * (to_d(p.K[q]) - to_d(K0[q]));
          }
          double we = w0 * exp(-f * tau_a);
          uint64_t cid = child_id(p.s.id, p.nev);
          scatter_child(io, Xe, Ke, we / b, cid, p.nsc + 1, p.model, ls);
          p.nev++;
          ls.events++;
          wn *= (1.0 - 1.0 / b);
          p.acc = 0.0;
          p.x1t = -log(rng_u(p.s, m.seed));
        } else {
          p.acc += d;
        }
      }
    }
    p.w = wn;
  }
  p.ana = c.ana;
  p.ans = c.ans;
}

// Termination tests after a step (recording at r >= r_record, capture, absorption, roulette, step
// cap); returns the status (0: continue) and writes the log record of a finished superphoton.
template <typename GS, typename S, typename W>
__device__ __forceinline__ int terminate(const DevModel &m, const PushIO &io, const GeoT<GS> &G, PhT<S, W> &p,
                                         int radius_term, LocalStats &ls) {
  int status = 0;
  if (radius_term == 1) {
    record(m, io, G, p);
    status = 1;
    ls.rec++;
  } else if (radius_term == 3) {
    status = 3;
    ls.capt++;
  } else if (!w_positive(p)) {
    status = 2;
    ls.abs++;
  } else {
    if (w_roulette(m, p)) {
      if (roulette_survives(m, p)) {
        ls.roul++;
      } else {
        status = 2;
        ls.abs++;
      }
    }
    if (status == 0 && p.nsteps >= m.max_steps) {
      status = 4;
      ls.maxst++;
    }
  }
  if (status) write_log(io, p, status);
  return status;
}

// One geodesic step with absorption, scattering and the termination tests; false when finished.
template <int PREC, bool KERR = true>
static __device__ bool step(const DevModel &m, const PushIO &io, PhF<PREC> &p, LocalStats &ls) {
  using S = typename Form<PREC>::S;
  using W = typename Form<PREC>::W;
  const bool scat = m.scatter && p.nsc < m.n_sc_max;
  S dl = stepsize(m, p.X, p.K);
  S X0[4], K0[4], Kp[4], An[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    X0[q] = p.X[q];
    K0[q] = p.K[q];
    p.X[q] = verlet_x(X0[q], K0[q], p.A[q], dl);
    Kp[q] = verlet_k(K0[q], p.A[q], dl);
  }
  GeoT<S> G;
  metric_eval<true, KERR>(m, p.X[1], p.X[2], G);
  int it = 0;
  bool conv = false;
  S Kn[4];
  while (true) {
    accel<KERR>(G, Kp, An);
    decltype(vmag(dl)) num = 0, den = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Kn[q] = verlet_k2(K0[q], p.A[q], An[q], dl);
      num += vdiff(Kn[q], Kp[q]);
      den += vmag(Kn[q]);
    }
    ++it;
#pragma unroll
    for (int q = 0; q < 4; ++q) Kp[q] = Kn[q];
    if (below_tol(num, m.verlet_tol, m.fverlet_tol, den)) {
      conv = true;
      break;
    }
    if (it >= m.verlet_maxit) break;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p.K[q] = Kn[q];
    p.A[q] = An[q];
  }
  ls.iters += it;
  ls.giters += it;
  ls.gsteps++;
  if (!conv) ls.nonconv++;
  p.nsteps++;
  ls.steps++;
  CoefT<W> c;
  coefs<Form<PREC>::C32>(m, G, p.X, p.K, scat, c);
  absorb_scatter(m, io, p, X0, K0, dl, c, scat, ls);
  const int rt = at_record(m, G.r) ? 1 : (at_capture(m, G.r) ? 3 : 0);
  return terminate(m, io, G, p, rt, ls) == 0;
}

// Free-streaming step (both end points outside the grid: no plasma, so tau_a = tau_s = 0 and the
// weight is unchanged): the same Verlet arithmetic and termination tests as step().  If the new
// point lies inside the grid the step is discarded (state untouched) and 2 is returned, so the
// in-grid phase redoes it with the coefficients.  Returns 0 to continue, 1 when finished.
template <int PREC, bool KERR = true>
static __device__ int step_free(const DevModel &m, const PushIO &io, PhF<PREC> &p, LocalStats &ls) {
  using S = typename Form<PREC>::S;
  S dl = stepsize(m, p.X, p.K);
  S Xn[4], Kp[4], An[4], Kn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Xn[q] = verlet_x(p.X[q], p.K[q], p.A[q], dl);
    Kp[q] = verlet_k(p.K[q], p.A[q], dl);
  }
  if (in_grid(m, Xn)) return 2;
  GeoT<S> G;
  metric_eval<true, KERR>(m, Xn[1], Xn[2], G);
  int it = 0;
  bool conv = false;
  while (true) {
    accel<KERR>(G, Kp, An);
    decltype(vmag(dl)) num = 0, den = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Kn[q] = verlet_k2(p.K[q], p.A[q], An[q], dl);
      num += vdiff(Kn[q], Kp[q]);
      den += vmag(Kn[q]);
    }
    ++it;
#pragma unroll
    for (int q = 0; q < 4; ++q) Kp[q] = Kn[q];
    if (below_tol(num, m.verlet_tol, m.fverlet_tol, den)) {
      conv = true;
      break;
    }
    if (it >= m.verlet_maxit) break;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p.X[q] = Xn[q];
    p.K[q] = Kn[q];
    p.A[q] = An[q];
  }
  ls.iters += it;
  if (!conv) ls.nonconv++;
  p.nsteps++;
  ls.steps++;
  p.ana = 0;
  p.ans = 0;
  const int rt = at_record(m, G.r) ? 1 : (at_capture(m, G.r) ? 3 : 0);
  return terminate(m, io, G, p, rt, ls) ? 1 : 0;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void flush_stats(const LocalStats &ls, unsigned long long *cnt) {
  const int lane = threadIdx.x & 31;
  unsigned long long v[14] = {ls.emit, ls.child, ls.rec, ls.abs, ls.capt, ls.maxst,
                              ls.steps, ls.iters, ls.nonconv, ls.roul, ls.rejcap, ls.events, ls.gsteps, ls.giters};
#pragma unroll
  for (int q = 0; q < 14; ++q) {
    unsigned long long s = warp_sum(v[q]);
    if (lane == 0 && s) atomicAdd(cnt + CNT_EMIT + q, s);
  }
}

template <typename S, typename W>
__device__ __forceinline__ void save_ph(const Pool &P, int64_t i, const PhT<S, W> &p) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    P.X[q][i] = to_d(p.X[q]);
    P.K[q][i] = to_d(p.K[q]);
    P.A[q][i] = to_d(p.A[q]);
  }
  P.w[i] = abs_w(p);
  P.wb[i] = p.wb;
  P.ana[i] = p.ana;
  P.ans[i] = p.ans;
  P.acc[i] = p.acc;
  P.x1t[i] = p.x1t;
  P.id[i] = p.s.id;
  P.ctr[i] = p.s.n;
  P.nev[i] = p.nev;
  P.nsc[i] = p.nsc;
  P.nsteps[i] = p.nsteps;
  if (P.model) P.model[i] = (int16_t)p.model;
}

template <typename S, typename W>
__device__ __forceinline__ void load_ph(const Pool &P, int64_t i, PhT<S, W> &p) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p.X[q] = from_d<S>(P.X[q][i]);
    p.K[q] = from_d<S>(P.K[q][i]);
    p.A[q] = from_d<S>(P.A[q][i]);
  }
  p.wb = P.wb[i];
  if constexpr (std::is_same<W, float>::value) p.w = (float)(P.w[i] / p.wb);
  else p.w = P.w[i];
  p.ana = (W)P.ana[i];
  p.ans = (W)P.ans[i];
  p.acc = (W)P.acc[i];
  p.x1t = (W)P.x1t[i];
  rng_init(p.s, P.id[i], P.ctr[i]);
  p.nev = P.nev[i];
  p.nsc = P.nsc[i];
  p.nsteps = P.nsteps[i];
  p.model = P.model ? (int)P.model[i] : 0;
  p.wthr = 0;
  p.raddr = nullptr;
}

// roulette threshold of model m: roulette_w * wb (relative weights: roulette_w)
template <typename S, typename W>
__device__ __forceinline__ void set_wthr(const DevModel &m, PhT<S, W> &p) {
  if constexpr (std::is_same<W, float>::value) p.wthr = m.froulette_w;
  else p.wthr = m.roulette_w * p.wb;
}

// load for a transport kernel of model m: also the roulette threshold
template <typename S, typename W>
__device__ __forceinline__ void load_ph(const Pool &P, int64_t i, PhT<S, W> &p, const DevModel &m) {
  load_ph(P, i, p);
  set_wthr(m, p);
}

// ---------------------------------------------------------------- surrogate in-grid push
// The mixed-precision in-grid step with the coefficient network: part A (geodesic, plasma state,
// network inputs), one tensor-core evaluation for the CTA's 128 superphotons, part B (optical
// depths, scattering, termination).  Identical to step<true> except for where K2 and sigma_h
// come from.
template <typename S>
struct SurCarry {
  S X0[4], K0[4];
  S dl;
  int term;   // radius test at the step end: 1 recording sphere reached, 3 captured, 0 neither
  CoefA a;
};

template <typename S, typename W>
static __device__ void step_sur_a(const DevModel &m, PhT<S, W> &p, SurCarry<S> &sc, LocalStats &ls) {
  S dl = stepsize(m, p.X, p.K);
  S Kp[4], An[4], Kn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    sc.X0[q] = p.X[q];
    sc.K0[q] = p.K[q];
    p.X[q] = verlet_x(sc.X0[q], sc.K0[q], p.A[q], dl);
    Kp[q] = verlet_k(sc.K0[q], p.A[q], dl);
  }
  GeoT<S> G;
  metric_eval<true>(m, p.X[1], p.X[2], G);
  int it = 0;
  bool conv = false;
  while (true) {
    accel(G, Kp, An);
    decltype(vmag(dl)) num = 0, den = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Kn[q] = verlet_k2(sc.K0[q], p.A[q], An[q], dl);
      num += vdiff(Kn[q], Kp[q]);
      den += vmag(Kn[q]);
    }
    ++it;
#pragma unroll
    for (int q = 0; q < 4; ++q) Kp[q] = Kn[q];
    if (below_tol(num, m.verlet_tol, m.fverlet_tol, den)) {
      conv = true;
      break;
    }
    if (it >= m.verlet_maxit) break;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p.K[q] = Kn[q];
    p.A[q] = An[q];
  }
  ls.iters += it;
  ls.giters += it;
  ls.gsteps++;
  if (!conv) ls.nonconv++;
  p.nsteps++;
  ls.steps++;
  sc.dl = dl;
  // only the radius tests cross the network evaluation (the metric is re-evaluated to record)
  sc.term = at_record(m, G.r) ? 1 : (at_capture(m, G.r) ? 3 : 0);
  coefficients32_a(m, G, p.X, p.K, sc.a);
}

template <int PREC>
static __device__ bool step_sur_b(const DevModel &m, const PushIO &io, PhF<PREC> &p,
                                  const SurCarry<typename Form<PREC>::S> &sc, const float out[3], LocalStats &ls) {
  using W = typename Form<PREC>::W;
  const bool scat = m.scatter && p.nsc < m.n_sc_max;
  CoefT<W> c;
  coefficients32_b(m, sc.a, out, scat, c);
  absorb_scatter(m, io, p, sc.X0, sc.K0, sc.dl, c, scat, ls);
  if (sc.term == 1) {
    GeoT<typename Form<PREC>::S> G;
    metric_eval<false>(m, p.X[1], p.X[2], G);
    return terminate(m, io, G, p, 1, ls) == 0;
  }
  const Geo Gd{};   // not read: recording needs the metric only when sc.term == 1
  return terminate(m, io, Gd, p, sc.term, ls) == 0;
}

}  // namespace mcgb
