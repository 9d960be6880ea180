// mc_tables.cu -- lookup tables and per-run superphoton generation (sections 2.1-2.3, 2.7).
//
// Tables built once per context on the device:
//   * ln F(K), F(K) = int_0^{pi/2} sin^2(th) G(K/sin th) dth, G(X) = (X^1/2 + 2^11/12 X^1/6)^2 e^{-X^1/3}:
//     the angle-integrated emissivity is int dOmega j_nu = 4 pi A nu_c F(nu/nu_c) (64-node Gauss-Legendre);
//   * ln K2(1/Theta) from K_2(x) = int_0^inf exp(-x cosh t) cosh 2t dt (trapezoid rule, which converges
//     geometrically for this entire integrand);
//   * ln(sigma_h / sigma_T) on the (Theta_e, eps) grid: Maxwell-Juettner average of (1 - mu beta)
//     sigma_KN with gamma = 1 + Theta s^2 (64 nodes, s in [0, 8]) and mu (32 nodes).
// Per run: zone volumes and emission prefactors, the weight table w(nu_j) (eq. weight_calc, a
// deterministic two-pass reduction over zones), expected zone counts, their stochastic rounding
// with the zone's Philox stream, and an exclusive scan giving each zone's first superphoton uid.
#include "mc_internal.h"

namespace mcgb {

// ---------------------------------------------------------------- tables
__global__ void k_table_F(double *lnF, int n, const double *glx, const double *glw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double K = exp(kFLnK0 + i * kFStep);
  double s = 0.0;
  for (int q = 0; q < 64; ++q) {
    double st = sin(glx[q]);
    s += glw[q] * st * st * Gsyn(K / st);
  }
  lnF[i] = log(s);
}

__global__ void k_table_K2(double *lnK2, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = exp(-(kK2LnT0 + i * kK2Step));   // x = 1 / Theta
  const double h = 1.0 / 64.0;
  double s = 0.5 * exp(-x);
  for (int q = 1; q < 4096; ++q) {
    double t = q * h;
    double ch = cosh(t);
    if (x * ch > 800.0) break;
    s += exp(-x * ch) * cosh(2.0 * t);
  }
  lnK2[i] = log(s * h);
}

__global__ void k_table_hot(double *hot, const double *gsx, const double *gsw, const double *gmx, const double *gmw) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kHotNT * kHotNE) return;
  int i = idx / kHotNE, j = idx % kHotNE;
  double th = exp(kHotLT0 + (kHotLT1 - kHotLT0) * i / (kHotNT - 1));
  double e = exp(kHotLE0 + (kHotLE1 - kHotLE0) * j / (kHotNE - 1));
  double num = 0.0, den = 0.0;
  for (int a = 0; a < 64; ++a) {
    double s = gsx[a];
    double gam = 1.0 + th * s * s;
    double hs = gam * s * s * sqrt(th * (2.0 + th * s * s)) * exp(-s * s);
    double beta = sqrt(1.0 - 1.0 / (gam * gam));
    double q = 0.0;
    for (int b = 0; b < 32; ++b) {
      double om = 1.0 - gmx[b] * beta;
      q += gmw[b] * om * sigma_kn_ratio(e * gam * om);
    }
    num += gsw[a] * hs * 0.5 * q;
    den += gsw[a] * hs;
  }
  hot[idx] = log(num / den);
}

void launch_tables(const DevModel &m, double *lnF, double *lnK2, double *hot, const double *gl_ang, const double *gl_s,
                   const double *gl_mu, cudaStream_t st) {
  k_table_F<<<(m.nF + 127) / 128, 128, 0, st>>>(lnF, m.nF, gl_ang, gl_ang + 64);
  k_table_K2<<<(m.nK2 + 127) / 128, 128, 0, st>>>(lnK2, m.nK2);
  k_table_hot<<<(kHotNT * kHotNE + 127) / 128, 128, 0, st>>>(hot, gl_s, gl_s + 64, gl_mu, gl_mu + 32);
}

// ---------------------------------------------------------------- kappa electrons
// ln F of the synchrotron function F(x) = x int_0^inf cosh(5u/3) / cosh(u) e^{-x cosh u} du (the integral
// representation of K_5/3 integrated over [x, inf)), by the trapezoid rule in u (even integrand).
__global__ void k_kap_F(double *lnF) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kKapNF) return;
  const double x = exp(kKapLF0 + (kKapLF1 - kKapLF0) * i / (kKapNF - 1));
  const double U = acosh(fmax(1.0, 760.0 / x)) + 2.0;
  const int n = (int)ceil(U / 0.004);
  const double h = U / n;
  double s = 0.0;
  for (int k = 0; k <= n; ++k) {
    const double u = k * h;
    const double v = exp(-x * cosh(u) + u * (2.0 / 3.0)) * (1.0 + exp(-u * (10.0 / 3.0))) / (1.0 + exp(-2.0 * u));
    s += (k == 0 || k == n) ? 0.5 * v : v;
  }
  lnF[i] = log(x * s * h);
}

__device__ __forceinline__ double kap_F(const double *lnF, double x) {
  if (x >= 200.0) return 0.0;
  const double lx = log(x);
  if (lx <= kKapLF0) return exp(lnF[0] + (lx - kKapLF0) / 3.0);   // F ~ x^1/3 below the table
  return exp(cubic_table(lnF, kKapNF, kKapLF0, (kKapNF - 1) / (kKapLF1 - kKapLF0), lx));
}

// ln J and ln A at one (X, w) node: trapezoid rule in t = ln(gamma - 1) over
// [ln(kappa w) - 25, ln(kappa w) + 45] with step 0.01, normalised by the same rule.
__global__ void k_kap_JA(const double *lnF, double kappa, double *lnJ, double *lnA) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= kKapNX * kKapNW) return;
  const int ix = node / kKapNW, jw = node % kKapNW;
  const double X = exp(kKapLX0 + (kKapLX1 - kKapLX0) * ix / (kKapNX - 1));
  const double w = exp(kKapLW0 + (kKapLW1 - kKapLW0) * jw / (kKapNW - 1));
  const double kw = kappa * w;
  const double t0 = log(kw) - 25.0, h = 0.01;
  const int n = 7000;
  double sn = 0.0, sj = 0.0, sa = 0.0;
  for (int k = 0; k <= n; ++k) {
    const double t = t0 + k * h, e = exp(t), g = 1.0 + e, rt = sqrt(e * (2.0 + e));
    const double base = exp(t - (kappa + 1.0) * log1p(e / kw));   // P(gamma) dgamma/dt
    const double wt = (k == 0 || k == n) ? 0.5 : 1.0;
    sn += wt * g * rt * base;
    const double x = 2.0 * X / (3.0 * g * g);
    if (x >= 200.0) continue;
    const double Fx = kap_F(lnF, x);
    sj += wt * g * rt * base * Fx;
    sa += wt * (g * rt * (kappa + 1.0) / (kw + e) - 1.0 / rt) * base * Fx;
  }
  sj /= sn;
  sa /= sn;
  lnJ[node] = sj > 0.0 ? fmax(kKapFloor, log(sj)) : kKapFloor;
  lnA[node] = sa > 0.0 ? fmax(kKapFloor, log(sa)) : kKapFloor;
}

// ln I(Y, w): I = int_0^{pi/2} sin^2 J(Y / sin, w) dtheta over the interpolated J, the midpoint sum with
// 2048 points in theta.
__global__ void k_kap_I(const double *lnJ, double *lnI) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= kKapNX * kKapNW) return;
  const int ix = node / kKapNW, jw = node % kKapNW;
  const double lY = kKapLX0 + (kKapLX1 - kKapLX0) * ix / (kKapNX - 1);
  const double lw = kKapLW0 + (kKapLW1 - kKapLW0) * jw / (kKapNW - 1);
  const int M = 2048;
  double s = 0.0;
  for (int k = 0; k < M; ++k) {
    const double st = sin((k + 0.5) * (0.5 * kPI / M));
    s += st * st * kap_interp(lnJ, lY - log(st), lw);
  }
  s *= 0.5 * kPI / M;
  lnI[node] = s > 0.0 ? fmax(kKapFloor, log(s)) : kKapFloor;
}

// ln(sigma_h / sigma_T) of the kappa population at one (w, eps) node, one warp per node: the average of
// (1 - beta mu) sigma_KN(eps gamma (1 - beta mu)) / sigma_T over the population (trapezoid rule in
// t = ln(gamma - 1) over [ln(kappa w) - 25, ln(kappa w) + 45] with step 0.02, normalised by the same rule)
// and over mu, as 32-point Gauss-Legendre in y = ln(1 - beta mu) on [ln(1 - beta), ln(1 + beta)]
// (d mu = -e^y dy / beta; the Klein-Nishina turnover of fast electrons sits at mu -> 1, where y spreads
// it out); lanes take every 32nd t, then a shuffle reduction.
__global__ void k_kap_hot(double kappa, const double *gmx, const double *gmw, double *lnH) {
  const int node = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (node >= kKapNW * kHotNE) return;   // whole warps leave together
  const int iw = node / kHotNE, je = node % kHotNE;
  const double w = exp(kKapLW0 + (kKapLW1 - kKapLW0) * iw / (kKapNW - 1));
  const double e = exp(kHotLE0 + (kHotLE1 - kHotLE0) * je / (kHotNE - 1));
  const double kw = kappa * w, t0 = log(kw) - 25.0, h = 0.02;
  const int n = 3500;
  double num = 0.0, den = 0.0;
  for (int k = lane; k <= n; k += 32) {
    const double t = t0 + k * h, x = exp(t), g = 1.0 + x, p = sqrt(x * (2.0 + x));
    const double f = ((k == 0 || k == n) ? 0.5 : 1.0) * g * p * exp(t - (kappa + 1.0) * log1p(x / kw));
    const double beta = p / g;
    const double y1 = log1p(beta), y0 = -2.0 * log(g) - y1;   // 1 - beta = 1 / (gamma^2 (1 + beta))
    const double ym = 0.5 * (y0 + y1), yh = 0.5 * (y1 - y0);
    double q = 0.0;
    for (int b = 0; b < 32; ++b) {
      const double om = exp(ym + yh * gmx[b]);
      q += gmw[b] * om * om * sigma_kn_ratio(e * g * om);
    }
    num += f * 0.5 * q * yh / beta;
    den += f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (lane == 0) lnH[node] = log(num / den);
}

void launch_kappa_tables(double kappa, double *lnF, double *lnJ, double *lnA, double *lnI, double *lnH,
                         const double *gl_mu, cudaStream_t st) {
  k_kap_F<<<(kKapNF + 127) / 128, 128, 0, st>>>(lnF);
  const int nn = kKapNX * kKapNW;
  k_kap_JA<<<(nn + 127) / 128, 128, 0, st>>>(lnF, kappa, lnJ, lnA);
  k_kap_I<<<(nn + 127) / 128, 128, 0, st>>>(lnJ, lnI);
  const int nh = kKapNW * kHotNE;   // one warp per node, four per block
  k_kap_hot<<<(nh + 3) / 4, 128, 0, st>>>(kappa, gl_mu, gl_mu + 32, lnH);
}

// ---------------------------------------------------------------- grid layout
__global__ void k_grid_to_aos(const void *src, int src_f32, void *dst, int dst_f32, int64_t nz, int *bad) {
  int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  for (int f = 0; f < 8; ++f) {
    double v = src_f32 ? (double)((const float *)src)[f * nz + z] : ((const double *)src)[f * nz + z];
    if (!isfinite(v)) atomicOr(bad, 1);
    if (dst_f32) ((float *)dst)[z * 8 + f] = (float)v;
    else ((double *)dst)[z * 8 + f] = v;
  }
}

void launch_grid_to_aos(const void *src, int src_f32, void *dst, int dst_f32, int64_t nz, int *bad, cudaStream_t st) {
  k_grid_to_aos<<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(src, src_f32, dst, dst_f32, nz, bad);
}

// ---------------------------------------------------------------- zones
__device__ __forceinline__ void zone_centre(const DevModel &m, int64_t z, double X[4]) {
  int64_t i = z / ((int64_t)m.n2 * m.n3);
  int64_t j = (z / m.n3) % m.n2;
  int64_t k = z % m.n3;
  X[0] = 0.0;
  X[1] = m.x1_0 + (i + 0.5) * m.dx1;
  X[2] = m.x2_0 + (j + 0.5) * m.dx2;
  X[3] = m.x3_0 + (k + 0.5) * m.dx3;
}

__device__ __forceinline__ void zone_prims(const DevModel &m, int64_t z, double pr[8]) {
  if (m.prim_f32) {
    for (int f = 0; f < 8; ++f) pr[f] = (double)m.prim32[z * 8 + f];
  } else {
    for (int f = 0; f < 8; ++f) pr[f] = m.prim64[z * 8 + f];
  }
}

// Zone volume sqrt(-g) d^3x L^3 (sqrt(-g) = Sigma sin(theta) r dtheta/dx2 for MKS Kerr-Schild) and the
// emission prefactor 4 pi A nu_c, A = sqrt(2) pi e^2 n_e / (3 c K2(1/Theta_e)), from the zone-centre state.
__global__ void k_zone_prep(DevModel m, double *zvol, double *zpref, double *zlnuc, int *bad) {
  int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= m.nz) return;
  double X[4];
  zone_centre(m, z, X);
  Geo G;
  metric_eval<false>(m, X[1], X[2], G);
  double th, dth, d2th;
  theta_map(m.hslope, X[2], th, dth, d2th);
  double sig = G.r * G.r + m.a * m.a * G.cth * G.cth;
  zvol[z] = sig * G.sth * G.r * dth * m.dx1 * m.dx2 * m.dx3 * m.L3;
  double pr[8];
  zone_prims(m, z, pr);
  Plasma<double> P;
  plasma_from_prims<double>(m, G, pr, P, nullptr, nullptr);
  if (!isfinite(P.thetae) || !isfinite(P.B) || !isfinite(P.ne)) atomicOr(bad, 2);
  double pref = 0.0, lnuc = 0.0;
  if (m.kappa > 0.0) {
    // kappa: int dOmega j_nu = (sqrt3 e^3 n_e B / m_e c^2) I(nu / nu_B, w); lnuc holds ln nu_B
    double lw = 0.0;
    if (P.thetae >= m.thetae_min && P.ne > 0.0 && P.B > 0.0) {
      pref = kKapCj * P.ne * P.B;
      lnuc = log(kNuB1 * P.B);
      lw = log(P.thetae * (m.kappa - 3.0) / m.kappa);
    }
    ((double *)m.zlnw)[z] = lw;
  } else if (P.thetae >= m.thetae_min && P.ne > 0.0 && P.B > 0.0) {
    double nuc = (2.0 / 9.0) * (kEE * P.B / (2.0 * kPI * kME * kCL)) * P.thetae * P.thetae;
    double A = 1.4142135623730951 * kPI * kEE * kEE * P.ne / (3.0 * kCL * K2_of(m, P.thetae));
    pref = 4.0 * kPI * A * nuc;
    lnuc = log(nuc);
  }
  zpref[z] = pref;
  zlnuc[z] = lnuc;
  if (m.brems) {
    // int dOmega j_nu = (q / nu_T) exp(-nu / nu_T), nu_T = k T_e / h
    const double nut = P.thetae * (kME * kCL * kCL / kHPL);
    const bool on = P.ne > 0.0 && P.thetae > 0.0;
    m.zbnt[z] = on ? nut : 1.0;
    m.zbq[z] = on ? brems_q(P.ne, P.thetae) / nut : 0.0;
  }
}

void launch_zone_prep(const DevModel &m, double *zvol, double *zpref, double *zlnuc, int *bad, cudaStream_t st) {
  k_zone_prep<<<(unsigned)((m.nz + 127) / 128), 128, 0, st>>>(m, zvol, zpref, zlnuc, bad);
}


constexpr int kChunk = 2048;

// partial[j][chunk] = sum over the chunk's zones of V_i int dOmega j_nu(nu_j): fixed assignment and a
// fixed reduction tree, so the weights are bit-reproducible run to run.
__global__ void k_weight_partial(DevModel m, const double *zvol, const double *zpref, const double *zlnuc,
                                 double *partial, int nchunks) {
  __shared__ double red[256];
  int chunk = blockIdx.x, j = blockIdx.y;
  int64_t z0 = (int64_t)chunk * kChunk;
  double s = 0.0;
  for (int q = threadIdx.x; q < kChunk; q += blockDim.x) {
    int64_t z = z0 + q;
    if (z < m.nz) s += zvol[z] * zone_E(m, z, zpref[z], zlnuc[z], j);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)j * nchunks + chunk] = red[0];
}

// w_j = max(w_min, dt dln(nu)_tot / (h N_s) sum_i V_i int dOmega j_nu(nu_j)), dt = 1 (cancels in nu L_nu)
__global__ void k_weight_final(DevModel m, const double *partial, int nchunks, double n_s, double w_min, double *lnw,
                               double *winv) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m.n_nu) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)j * nchunks + c];
  double w = fmax(w_min, m.dlntot / (kHPL * n_s) * s);
  lnw[j] = log(w);
  winv[j] = 1.0 / w;
}

void launch_weights(const DevModel &m, const double *zvol, const double *zpref, const double *zlnuc, double *partial,
                    int nchunks, double n_s, double w_min, double *lnw, double *winv, cudaStream_t st) {
  dim3 grid(nchunks, m.n_nu);
  k_weight_partial<<<grid, 256, 0, st>>>(m, zvol, zpref, zlnuc, partial, nchunks);
  k_weight_final<<<(m.n_nu + 127) / 128, 128, 0, st>>>(m, partial, nchunks, n_s, w_min, lnw, winv);
}

// Expected count nbar_i = V_i sum_j T_j g_ij / h (trapezoid in ln nu, g_ij = int dOmega j_nu / w_j), its
// maximum g over nodes (rejection bound), and N_i = floor(nbar) + [u_i < frac(nbar)], u_i the first
// uniform of the zone's stream.
__global__ void k_zone_counts(DevModel m, const double *zvol, const double *zpref, const double *zlnuc, double *zgmax,
                              double *znbar, int64_t *counts) {
  int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= m.nz) return;
  double pref = zpref[z], lnuc = zlnuc[z];
  double s = 0.0, gm = 0.0;
  if (pref != 0.0 || (m.brems && m.zbq[z] > 0.0)) {
    for (int j = 0; j < m.n_nu; ++j) {
      double g = zone_E(m, z, pref, lnuc, j) * m.winv[j];
      double t = (j == 0 || j == m.n_nu - 1) ? 0.5 * m.dlnu : m.dlnu;
      s += t * g;
      gm = fmax(gm, g);
    }
  }
  double nb = zvol[z] * s / kHPL;
  znbar[z] = nb;
  zgmax[z] = gm;
  double fl = floor(nb);
  Rng r;
  rng_init(r, kZoneTag | (uint64_t)z, 0u);
  double u = rng_u(r, m.seed);
  counts[z] = (int64_t)fl + ((u < nb - fl) ? 1 : 0);
}

void launch_counts(const DevModel &m, const double *zvol, const double *zpref, const double *zlnuc, double *zgmax,
                   double *znbar, int64_t *counts, cudaStream_t st) {
  k_zone_counts<<<(unsigned)((m.nz + 127) / 128), 128, 0, st>>>(m, zvol, zpref, zlnuc, zgmax, znbar, counts);
}

// ---------------------------------------------------------------- exclusive scan (int64)
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int64_t w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += sh[wid - 1];
  return v;
}

__global__ void k_scan_local(const int64_t *in, int64_t *out, int64_t *bsum, int64_t n) {
  __shared__ int64_t sh[32];
  int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int64_t v = (i < n) ? in[i] : 0;
  int64_t inc = block_incl_scan(v, sh);
  if (i < n) out[i] = inc - v;
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = inc;
}

__global__ void k_scan_sums(int64_t *bsum, int64_t nb, int64_t *total) {
  __shared__ int64_t sh[32];
  // each thread owns a contiguous run of block sums
  int64_t per = (nb + kScanBlock - 1) / kScanBlock;
  int64_t b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  int64_t loc = 0;
  for (int64_t b = b0; b < b1; ++b) loc += bsum[b];
  int64_t inc = block_incl_scan(loc, sh);
  int64_t run = inc - loc;
  for (int64_t b = b0; b < b1; ++b) {
    int64_t v = bsum[b];
    bsum[b] = run;
    run += v;
  }
  if (threadIdx.x == kScanBlock - 1) *total = inc;
}

__global__ void k_scan_add(int64_t *out, const int64_t *bsum, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

void launch_scan(const int64_t *counts, int64_t *start, int64_t *bsum, int64_t n, int64_t *total_dev, cudaStream_t st) {
  int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  k_scan_local<<<(unsigned)nb, kScanBlock, 0, st>>>(counts, start, bsum, n);
  k_scan_sums<<<1, kScanBlock, 0, st>>>(bsum, nb, total_dev);
  k_scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(start, bsum, n);
}

// ---------------------------------------------------------------- pipe peak (FMA chains)
// Eight independent FMA chains per thread keep the pipe busy without memory traffic; the result
// is stored only under a data-dependent condition that never holds, so nothing is optimised away.
template <typename T>
__global__ void k_fma_chain(T *sink, int iters, T seed) {
  T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  const T m = (T)0.999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
      a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
    }
  }
  T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

template <typename T>
static cudaError_t fma_peak_t(double *flops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 1024 * sizeof(T));
  if (e != cudaSuccess) return e;
  const int block = 256, grid = sms * 8;
  const int iters = sizeof(T) == 8 ? 256 : 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chain<T><<<grid, block>>>(sink, iters / 8, (T)1);   // warm-up
  double best = 0.0;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    k_fma_chain<T><<<grid, block>>>(sink, iters, (T)1);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8.0 * 16.0 * (double)iters * (double)grid * block;
    best = fmax(best, fl / (ms * 1e-3));
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *flops = best;
  return e;
}

cudaError_t fma_peak(bool fp64, double *flops) { return fp64 ? fma_peak_t<double>(flops) : fma_peak_t<float>(flops); }

// ---------------------------------------------------------------- special-function self-test
__global__ void k_to_f32(const double *src, float *dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

void launch_to_f32(const double *src, float *dst, int n, cudaStream_t st) {
  if (n > 0) k_to_f32<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
}

// Double-float function table: 2^(j/32) for j < 32, then sin(pi j/32) for j < 64 (by quadrant from the
// first-quadrant sine and cosine, so that 0 and +-1 are exact), split from FP64 values.
void df_table_host(df *t) {
  for (int j = 0; j < 32; ++j) t[kDfTabExp + j] = df_const(std::exp2(j / 32.0));
  for (int j = 0; j < 64; ++j) {
    const int q = j / 16, r = j % 16;
    double v = (q % 2 == 0) ? std::sin(kPI * r / 32.0) : std::cos(kPI * r / 32.0);
    if (q >= 2) v = -v;
    t[kDfTabSin + j] = df_const(v);
  }
}

__global__ void k_selftest_math(int which, const double *x, double *y, double *ref, int64_t n, const df *T,
                                const double *F) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  // table-driven FP64 functions against CUDA's
  if (which == 6) {
    y[i] = exp_t(F, v);
    ref[i] = exp(v);
    return;
  }
  if (which == 7) {
    y[i] = log_t(F, v);
    ref[i] = log(v);
    return;
  }
  if (which == 10) {
    y[i] = expm1_t(F, v);
    ref[i] = expm1(v);
    return;
  }
  if (which == 8 || which == 9) {
    double s, c, rs, rc;
    sincospi_t(F, v, s, c);
    sincospi(v, &rs, &rc);
    y[i] = which == 8 ? s : c;
    ref[i] = which == 8 ? rs : rc;
    return;
  }
  // double-float functions: the reference takes the input as split to double-float
  const df vd = df_from(v);
  if (which == 3) {
    y[i] = df_to(df_exp(vd, T));
    ref[i] = exp(df_to(vd));
    return;
  }
  if (which == 4 || which == 5) {
    df s, c;
    df_sincospi(vd, T, s, c);
    y[i] = df_to(which == 4 ? s : c);
    double rs, rc;
    sincospi(df_to(vd), &rs, &rc);
    ref[i] = which == 4 ? rs : rc;
    return;
  }
  if (which == 2) {
    y[i] = pow_sixth(v);
    ref[i] = cbrt(sqrt(v));
    return;
  }
  double s, c, rs, rc;
  sincos_small(v, s, c);
  sincos(v, &rs, &rc);
  y[i] = (which == 0) ? s : c;
  ref[i] = (which == 0) ? rs : rc;
}

// Tables of exp_t, log_t and sincospi_t, in extended precision: 2^(j/32); 1/c_j, log c_j split into its
// double and the remainder (c_j = 1 + j/128); sin and cos (pi j/32), exact at multiples of pi/2.
void ftab_host(double *t) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j < 32; ++j) t[kFtExp + j] = (double)exp2l((long double)j / 32.0L);
  for (int j = 0; j < 128; ++j) {
    const long double c = 1.0L + (long double)j / 128.0L;
    t[kFtInvC + j] = (double)(1.0L / c);
    const long double L = logl(c);
    const double hi = (double)L;
    t[kFtLogHi + j] = hi;
    t[kFtLogLo + j] = (double)(L - (long double)hi);
  }
  for (int j = 0; j < 64; ++j) {
    long double sv = sinl(pi * j / 32.0L), cv = cosl(pi * j / 32.0L);
    if (j % 16 == 0) {
      const int q = j / 16;
      sv = (q == 1) ? 1.0L : (q == 3) ? -1.0L : 0.0L;
      cv = (q == 0) ? 1.0L : (q == 2) ? -1.0L : 0.0L;
    }
    t[kFtSin + j] = (double)sv;
    t[kFtCos + j] = (double)cv;
  }
}

cudaError_t selftest_math(int which, const double *x_dev, double *y_dev, double *ref_dev, int64_t n) {
  df host[kDfTabN];
  df_table_host(host);
  double fhost[kFtN];
  ftab_host(fhost);
  df *tab = nullptr;
  double *ftab = nullptr;
  cudaError_t e = cudaMalloc(&tab, sizeof(host));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&ftab, sizeof(fhost));
  if (e != cudaSuccess) {
    cudaFree(tab);
    return e;
  }
  e = cudaMemcpy(tab, host, sizeof(host), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ftab, fhost, sizeof(fhost), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) {
    k_selftest_math<<<(unsigned)((n + 255) / 256), 256>>>(which, x_dev, y_dev, ref_dev, n, tab, ftab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tab);
  cudaFree(ftab);
  return e;
}

}  // namespace mcgb
