// mc_api.cu -- host side of the C ABI declared in include/mc.h.
//
// Owns the context: device tables, the zone-major copy of the fluid grid, per-run generation
// buffers, the two scattered-superphoton queues and the spectrum sums.  mc_run orchestrates one
// whole pass of the hot path on the caller's stream: weights and zone counts (a handful of small
// kernels), then the persistent transport kernel once per scattering generation, batching the
// primaries so the queues stay within their capacity (the paper's memory batching, section 3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mc_internal.h"
#include "mc_mlp.cuh"

using namespace mcgb;

static std::string g_init_err;

static int fail(mc_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  else g_init_err = msg;
  return code;
}

static void *dev_alloc(mc_ctx *c, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void *ptr = nullptr;
  if (c->p.alloc) {
    ptr = c->p.alloc(bytes, c->p.alloc_user);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) c->allocs.push_back(ptr);
  return ptr;
}

static void dev_free(mc_ctx *c, void *ptr) {
  if (!ptr) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), ptr);
  if (it != c->allocs.end()) c->allocs.erase(it);
  if (c->p.free) c->p.free(ptr, c->p.alloc_user);
  else cudaFree(ptr);
}

void *dev_alloc_ext(mc_ctx *c, size_t bytes) { return dev_alloc(c, bytes); }
void dev_free_ext(mc_ctx *c, void *ptr) { dev_free(c, ptr); }
int set_err(mc_ctx *c, int code, const char *msg) { return fail(c, code, msg); }

#define CU(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(c, MC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// Gauss-Legendre nodes and weights on [a, b] by Newton iteration on P_n (three-term recurrence).
static void gauss_legendre(int n, double a, double b, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int iter = 0; iter < 100; ++iter) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      dp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p1 = 1.0, p2 = 0.0;
    for (int k = 1; k <= n; ++k) {
      double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
    }
    dp = n * (z * p1 - p2) / (z * z - 1.0);
    double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    double h = 0.5 * (b - a), mid = 0.5 * (b + a);
    x[i] = mid - h * z;
    x[n - 1 - i] = mid + h * z;
    w[i] = w[n - 1 - i] = h * wt;
  }
}

DevModel make_model(const mc_ctx *c) {
  const mc_model_params &p = c->p;
  DevModel m;
  std::memset(&m, 0, sizeof(m));
  m.a = p.a;
  m.mass = p.mass;
  m.hslope = p.hslope;
  m.r_h = (p.mass > 0.0) ? 1.0 + std::sqrt(1.0 - p.a * p.a) : 0.0;
  double L = p.L_unit;
  m.L3 = L * L * L;
  m.rho_unit = p.M_unit / m.L3;
  m.B_unit = kCL * std::sqrt(4.0 * kPI * m.rho_unit);
  m.Ne_unit = m.rho_unit / (kMP + kME);
  m.Ccoef = kHPL * L / (kME * kCL * kCL);
  m.fCcoef = (float)m.Ccoef;
  m.R_high = p.R_high;
  m.R_low = p.R_low;
  m.gam = p.gam;
  m.thetae_min = p.thetae_min;
  m.thetae_max = p.thetae_max;
  m.n_nu = p.n_nu;
  m.lnu_min = std::log(p.nu_min);
  m.dlntot = std::log(p.nu_max / p.nu_min);
  m.dlnu = m.dlntot / (p.n_nu - 1);
  m.eps_geo = p.eps_geo;
  m.verlet_tol = p.verlet_tol;
  m.verlet_maxit = p.verlet_maxit;
  m.r_record = p.r_record;
  m.r_capture = (p.mass > 0.0) ? m.r_h * (1.0 + p.dh) : -1.0;
  m.bias_mode = p.bias_mode;
  m.bias_p0 = p.bias_p0;
  m.bias_max = p.bias_max;
  m.bias_scale = 1.0;
  m.fbias_scale = 1.0f;
  m.fbias_p0 = (float)p.bias_p0;
  m.fbias_max = (float)p.bias_max;   // beyond the FP32 range: +inf, no bound
  m.froulette_w = (float)p.roulette_w;
  m.froulette_p = (float)p.roulette_p;
  m.n_sc_max = p.n_sc_max;
  m.scatter = p.scatter;
  m.k2_mode = p.k2_mode;
  m.roulette_w = p.roulette_w;
  m.roulette_p = p.roulette_p;
  m.max_steps = p.max_steps;
  m.lnu_lo = p.lnu_lo;
  m.dlog_bin = (p.lnu_hi - p.lnu_lo) / p.n_bins;
  m.n_bins = p.n_bins;
  m.n_incl = p.n_incl;
  m.n1 = c->n1;
  m.n2 = c->n2;
  m.n3 = c->n3;
  m.nz = c->nz;
  m.prim_f32 = c->prim_f32;
  m.x1_0 = c->x1_0;
  m.dx1 = c->dx1;
  m.x2_0 = c->x2_0;
  m.dx2 = c->dx2;
  m.x3_0 = c->x3_0;
  m.dx3 = c->dx3;
  m.x1_hi = c->x1_0 + c->n1 * c->dx1;
  m.ithetae_max = 1.0 / p.thetae_max;
  m.iB_unit = 1.0 / m.B_unit;
  m.idx1 = 1.0 / c->dx1;
  m.idx2 = 1.0 / c->dx2;
  m.idx3 = 1.0 / c->dx3;
  m.prim64 = c->prim_f32 ? nullptr : (const double *)c->prim;
  m.prim32 = c->prim_f32 ? (const float *)c->prim : nullptr;
  m.prim32x = c->prim_f32 ? (const float *)c->prim : c->prim_x32;
  m.brems = p.brems;
  m.kappa = p.kappa;
  m.kapJ = c->kapJ;
  m.kapA = c->kapA;
  m.kapI = c->kapI;
  m.kapH = c->kapH;
  m.dmass = df_const(m.mass);
  m.da = df_const(m.a);
  m.dx1_0 = df_const(m.x1_0);
  m.dx1_hi = df_const(m.x1_hi);
  m.dr_record = df_const(m.r_record);
  m.dr_capture = df_const(m.r_capture);
  m.dpi2hh = df_const(kPI * (1.0 - p.hslope));
  m.dhh_pi = df_const((1.0 - p.hslope) / (2.0 * kPI));
  m.dd2th = df_const(-2.0 * kPI * kPI * (1.0 - p.hslope));
  m.dtab = c->dtab;
  m.ftab = c->ftab;
  m.fidx1 = (float)m.idx1;
  m.fidx2 = (float)m.idx2;
  m.fidx3 = (float)m.idx3;
  m.fx2_0 = (float)m.x2_0;
  m.fx3_0 = (float)m.x3_0;
  m.fNe_unit = (float)m.Ne_unit;
  m.fB_unit = (float)m.B_unit;
  m.fgam = (float)m.gam;
  m.fR_low = (float)m.R_low;
  m.fR_high = (float)m.R_high;
  m.fthetae_max = (float)m.thetae_max;
  m.fithetae_max = (float)m.ithetae_max;
  m.fthetae_min = (float)m.thetae_min;
  m.deps_geo = df_const(m.eps_geo);
  m.fverlet_tol = (float)m.verlet_tol;
  m.hslope1 = m.hslope == 1.0;
  m.kappa_on = m.kappa > 0.0;
  m.lnK2f = c->lnK2f;
  m.hotf = c->hotf;
  m.zlnw = c->zlnw;
  m.zbq = c->zbq;
  m.zbnt = c->zbnt;
  m.lnF = c->lnF;
  m.nF = c->nF;
  m.lnK2 = c->lnK2;
  m.nK2 = c->nK2;
  m.hot = c->hot;
  m.start = c->start;
  m.zpref = c->zpref;
  m.zlnuc = c->zlnuc;
  m.zgmax = c->zgmax;
  m.lnw = c->lnw;
  m.winv = c->winv;
  m.spec = c->spec;
  return m;
}

static int check_params(const mc_model_params *p, std::string &why) {
  auto bad = [&](const char *s) { why = s; return MC_ERR_INVALID_ARG; };
  if (!(p->mass == 0.0 || p->mass == 1.0)) return bad("mass must be 0 (flat) or 1 (Kerr-Schild)");
  if (!(std::fabs(p->a) < 1.0)) return bad("|a| must be < 1");
  if (!(p->hslope > 0.0 && p->hslope <= 1.0)) return bad("hslope must be in (0, 1]");
  if (!(p->L_unit > 0.0 && p->M_unit > 0.0)) return bad("L_unit and M_unit must be positive");
  if (!(p->nu_min > 0.0 && p->nu_max > p->nu_min)) return bad("need 0 < nu_min < nu_max");
  if (p->n_nu < 2 || p->n_nu > 100000) return bad("n_nu must be in [2, 100000]");
  if (!(p->w_min > 0.0)) return bad("w_min must be positive");
  if (!(p->eps_geo > 0.0 && p->eps_geo < 1.0)) return bad("eps_geo must be in (0, 1)");
  if (!(p->verlet_tol > 0.0) || p->verlet_maxit < 1) return bad("verlet_tol > 0 and verlet_maxit >= 1 required");
  if (!(p->r_record > 0.0)) return bad("r_record must be positive");
  if (p->n_bins < 1 || p->n_incl < 1 || !(p->lnu_hi > p->lnu_lo)) return bad("bad spectrum bins");
  if (p->n_incl * (int64_t)p->n_bins > (1 << 24)) return bad("too many spectrum bins");
  if (p->bias_mode < 0 || p->bias_mode > 2) return bad("bias_mode must be 0, 1 or 2");
  if (!(p->bias_max >= 1.0)) return bad("bias_max must be >= 1");
  if (!(p->bias_target >= 0.0 && p->bias_target < 1e30)) return bad("bias_target must be >= 0");
  if (p->brems != 0 && p->brems != 1) return bad("brems must be 0 or 1");
  if (p->brems && p->surrogate) return bad("the coefficient surrogate does not model bremsstrahlung");
  if (!(p->kappa == 0.0 || (p->kappa > 3.0 && p->kappa <= 1e8))) return bad("kappa must be 0 or in (3, 1e8]");
  if (p->kappa > 0.0 && p->surrogate) return bad("the coefficient surrogate does not model kappa electrons");
  if (p->n_sc_max < 0 || p->n_sc_max > 1000) return bad("n_sc_max out of range");
  if (!(p->roulette_p > 0.0 && p->roulette_p <= 1.0) || !(p->roulette_w >= 0.0)) return bad("bad roulette");
  if (p->max_steps < 1 || p->max_steps > 2000000000LL) return bad("max_steps out of range");
  if (p->precision != MC_PREC_FP64 && p->precision != MC_PREC_MIXED && p->precision != MC_PREC_SPLIT)
    return bad("unknown precision");
  if (p->surrogate != 0 && p->surrogate != 1) return bad("surrogate must be 0 or 1");
  if (p->surrogate == 1 && p->precision == MC_PREC_FP64) return bad("the surrogate runs in the mixed or split form");
  if (p->block != 0 && (p->block < 32 || p->block > 128 || p->block % 32)) return bad("block must be 32..128, multiple of 32");
  if (!(p->thetae_min >= 0.0 && p->thetae_max > 0.0)) return bad("bad Theta_e bounds");
  if (!(p->gam > 1.0)) return bad("gam must exceed 1");
  return MC_OK;
}

extern "C" {

const char *mc_version(void) { return "mcgb 0.1 (sm_103a)"; }

const char *mc_last_error(const mc_ctx *c) { return c ? c->err.c_str() : g_init_err.c_str(); }

void mc_free(mc_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->p.device);
  cudaDeviceSynchronize();
  mc_batch_release(c);
  std::vector<void *> a = c->allocs;
  for (void *ptr : a) dev_free(c, ptr);
  if (c->cnt_host) cudaFreeHost(c->cnt_host);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

int mc_init_model(mc_ctx **out, const mc_model_params *p) {
  if (!out || !p) return fail(nullptr, MC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  std::string why;
  int rc = check_params(p, why);
  if (rc) return fail(nullptr, rc, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, MC_ERR_NO_DEVICE, "no CUDA device");
  }
  if (p->device < 0 || p->device >= ndev) return fail(nullptr, MC_ERR_NO_DEVICE, "device ordinal out of range");
  mc_ctx *c = new (std::nothrow) mc_ctx();
  if (!c) return fail(nullptr, MC_ERR_OOM, "host allocation failed");
  c->p = *p;
  if (cudaSetDevice(p->device) != cudaSuccess) {
    delete c;
    return fail(nullptr, MC_ERR_CUDA, "cudaSetDevice failed");
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, p->device);
  c->nF = (int)std::floor((kFLnK1 - kFLnK0) / kFStep + 0.5) + 1;
  c->nK2 = (int)std::floor((kK2LnT1 - kK2LnT0) / kK2Step + 0.5) + 1;
  c->lnF = (double *)dev_alloc(c, sizeof(double) * c->nF);
  c->lnK2 = (double *)dev_alloc(c, sizeof(double) * c->nK2);
  c->lnK2f = (float *)dev_alloc(c, sizeof(float) * c->nK2);
  c->hotf = (float *)dev_alloc(c, sizeof(float) * kHotNT * kHotNE);
  c->hot = (double *)dev_alloc(c, sizeof(double) * kHotNT * kHotNE);
  c->gl = (double *)dev_alloc(c, sizeof(double) * (128 + 128 + 64));
  c->dtab = (df *)dev_alloc(c, sizeof(df) * kDfTabN);
  c->ftab = (double *)dev_alloc(c, sizeof(double) * kFtN);
  c->cnt = (unsigned long long *)dev_alloc(c, sizeof(unsigned long long) * CNT_N);
  c->total_dev = (int64_t *)dev_alloc(c, sizeof(int64_t));
  size_t nspec = (size_t)p->n_incl * p->n_bins * 3;
  c->spec = (double *)dev_alloc(c, sizeof(double) * nspec);
  c->lnw = (double *)dev_alloc(c, sizeof(double) * p->n_nu);
  c->winv = (double *)dev_alloc(c, sizeof(double) * p->n_nu);
  c->bad = (int *)dev_alloc(c, sizeof(int));
  if (!c->lnF || !c->lnK2 || !c->hot || !c->gl || !c->cnt || !c->total_dev || !c->spec || !c->lnw || !c->winv || !c->bad) {
    mc_free(c);
    return fail(nullptr, MC_ERR_OOM, "device allocation failed");
  }
  if (cudaMallocHost(&c->cnt_host, sizeof(unsigned long long) * (2 * CNT_N + 8)) != cudaSuccess) {
    cudaGetLastError();
    c->cnt_host = nullptr;
    mc_free(c);
    return fail(nullptr, MC_ERR_OOM, "pinned host allocation failed");
  }
  for (int k = 0; k < 4; ++k) {
    if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
      mc_free(c);
      return fail(nullptr, MC_ERR_CUDA, "event creation failed");
    }
  }
  std::vector<double> gl(320);
  gauss_legendre(64, 0.0, 0.5 * kPI, gl.data(), gl.data() + 64);      // angle integral
  gauss_legendre(64, 0.0, 8.0, gl.data() + 128, gl.data() + 192);     // hot cross-section, s
  gauss_legendre(32, -1.0, 1.0, gl.data() + 256, gl.data() + 288);    // hot cross-section, mu
  df dft[kDfTabN];
  df_table_host(dft);
  if (!c->dtab || cudaMemcpy(c->dtab, dft, sizeof(dft), cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_free(c);
    return fail(nullptr, MC_ERR_CUDA, "table upload failed");
  }
  std::vector<double> ft(kFtN);
  ftab_host(ft.data());
  if (!c->ftab || cudaMemcpy(c->ftab, ft.data(), sizeof(double) * kFtN, cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_free(c);
    return fail(nullptr, MC_ERR_CUDA, "table upload failed");
  }
  if (cudaMemcpy(c->gl, gl.data(), sizeof(double) * 320, cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_free(c);
    return fail(nullptr, MC_ERR_CUDA, "table upload failed");
  }
  if (p->kappa > 0.0) {
    c->kapF = (double *)dev_alloc(c, sizeof(double) * kKapNF);
    c->kapJ = (double *)dev_alloc(c, sizeof(double) * kKapNX * kKapNW);
    c->kapA = (double *)dev_alloc(c, sizeof(double) * kKapNX * kKapNW);
    c->kapI = (double *)dev_alloc(c, sizeof(double) * kKapNX * kKapNW);
    c->kapH = (double *)dev_alloc(c, sizeof(double) * kKapNW * kHotNE);
    if (!c->kapF || !c->kapJ || !c->kapA || !c->kapI || !c->kapH) {
      mc_free(c);
      return fail(nullptr, MC_ERR_OOM, "device allocation failed");
    }
    launch_kappa_tables(p->kappa, c->kapF, c->kapJ, c->kapA, c->kapI, c->kapH, c->gl + 256, 0);
  }
  DevModel m = make_model(c);
  launch_tables(m, c->lnF, c->lnK2, c->hot, c->gl, c->gl + 128, c->gl + 256, 0);
  if (!c->lnK2f || !c->hotf) {
    mc_free(c);
    return fail(nullptr, MC_ERR_OOM, "device allocation failed");
  }
  launch_to_f32(c->lnK2, c->lnK2f, c->nK2, 0);
  launch_to_f32(c->hot, c->hotf, kHotNT * kHotNE, 0);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    std::string msg = std::string("table build failed: ") + cudaGetErrorString(e);
    mc_free(c);
    return fail(nullptr, MC_ERR_CUDA, msg);
  }
  *out = c;
  return MC_OK;
}

int mc_set_grid(mc_ctx *c, const mc_grid_desc *g) {
  if (!c || !g || !g->prim) return fail(c, MC_ERR_INVALID_ARG, "null argument");
  if (g->n1 < 1 || g->n2 < 1 || g->n3 < 1) return fail(c, MC_ERR_INVALID_ARG, "grid dimensions must be >= 1");
  if (g->dtype != MC_DTYPE_F64 && g->dtype != MC_DTYPE_F32) return fail(c, MC_ERR_INVALID_ARG, "bad dtype");
  if (g->location != MC_LOC_HOST && g->location != MC_LOC_DEVICE) return fail(c, MC_ERR_INVALID_ARG, "bad location");
  if (!(g->dx1 > 0 && g->dx2 > 0 && g->dx3 > 0)) return fail(c, MC_ERR_INVALID_ARG, "grid spacings must be positive");
  if (!(g->x2_0 >= 0.0 && g->x2_0 + g->n2 * g->dx2 <= 1.0 + 1e-12)) return fail(c, MC_ERR_INVALID_ARG, "x2 range must lie in [0, 1]");
  CU(cudaSetDevice(c->p.device));
  int64_t nz = (int64_t)g->n1 * g->n2 * g->n3;
  size_t esz = (g->dtype == MC_DTYPE_F32) ? 4 : 8;
  // free per-grid buffers
  void *old[] = {c->prim, c->prim_x32, c->zvol, c->zpref, c->zlnuc, c->zgmax, c->znbar, c->counts, c->start, c->bsum,
                 c->partial, c->zbq, c->zbnt, c->zlnw};
  for (void *ptr : old) dev_free(c, ptr);
  c->prim = nullptr;
  c->prim_x32 = nullptr;
  c->zbq = c->zbnt = nullptr;
  c->zlnw = nullptr;
  c->have_grid = false;
  c->have_run = false;
  c->n1 = g->n1; c->n2 = g->n2; c->n3 = g->n3; c->nz = nz;
  c->x1_0 = g->x1_0; c->dx1 = g->dx1; c->x2_0 = g->x2_0; c->dx2 = g->dx2; c->x3_0 = g->x3_0; c->dx3 = g->dx3;
  c->prim_f32 = (g->dtype == MC_DTYPE_F32);
  c->prim = dev_alloc(c, esz * 8 * nz);
  c->zvol = (double *)dev_alloc(c, 8 * nz);
  c->zpref = (double *)dev_alloc(c, 8 * nz);
  c->zlnuc = (double *)dev_alloc(c, 8 * nz);
  c->zgmax = (double *)dev_alloc(c, 8 * nz);
  c->znbar = (double *)dev_alloc(c, 8 * nz);
  c->counts = (int64_t *)dev_alloc(c, 8 * nz);
  c->start = (int64_t *)dev_alloc(c, 8 * nz);
  c->bsum = (int64_t *)dev_alloc(c, 8 * ((nz + 1023) / 1024 + 1));
  c->nchunks = (int)((nz + 2047) / 2048);
  c->partial = (double *)dev_alloc(c, 8 * (size_t)c->nchunks * c->p.n_nu);
  if (!c->prim || !c->zvol || !c->zpref || !c->zlnuc || !c->zgmax || !c->znbar || !c->counts || !c->start || !c->bsum || !c->partial)
    return fail(c, MC_ERR_OOM, "grid allocation failed");
  if (c->p.kappa > 0.0) {
    c->zlnw = (double *)dev_alloc(c, 8 * nz);
    if (!c->zlnw) return fail(c, MC_ERR_OOM, "grid allocation failed");
  }
  if (c->p.brems) {
    c->zbq = (double *)dev_alloc(c, 8 * nz);
    c->zbnt = (double *)dev_alloc(c, 8 * nz);
    if (!c->zbq || !c->zbnt) return fail(c, MC_ERR_OOM, "grid allocation failed");
  }
  const void *src = g->prim;
  void *staging = nullptr;
  if (g->location == MC_LOC_HOST) {
    staging = dev_alloc(c, esz * 8 * nz);
    if (!staging) return fail(c, MC_ERR_OOM, "staging allocation failed");
    CU(cudaMemcpy(staging, g->prim, esz * 8 * nz, cudaMemcpyHostToDevice));
    src = staging;
  }
  CU(cudaMemset(c->bad, 0, sizeof(int)));
  launch_grid_to_aos(src, c->prim_f32, c->prim, c->prim_f32, nz, c->bad, 0);
  if (c->p.precision != MC_PREC_FP64 && !c->prim_f32) {
    // the FP32 coefficient path reads FP32 primitives directly (no per-step conversions)
    c->prim_x32 = (float *)dev_alloc(c, 4 * 8 * nz);
    if (!c->prim_x32) {
      if (staging) dev_free(c, staging);
      return fail(c, MC_ERR_OOM, "grid allocation failed");
    }
    launch_grid_to_aos(src, 0, c->prim_x32, 1, nz, c->bad, 0);
  }
  int bad = 0;
  CU(cudaMemcpy(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (staging) dev_free(c, staging);
  if (bad) return fail(c, MC_ERR_NAN_INPUT, "grid primitives contain non-finite values");
  c->have_grid = true;
  c->grid_epoch++;
  return MC_OK;
}

static void free_childbuf(mc_ctx *c, ChildBuf &q) {
  for (int k = 0; k < 4; ++k) { dev_free(c, q.X[k]); dev_free(c, q.K[k]); }
  dev_free(c, q.w); dev_free(c, q.id); dev_free(c, q.ctr); dev_free(c, q.nsc);
  std::memset(&q, 0, sizeof(q));
}

// Child queues (two generations, ping-pong), the superphoton pool and the two phase lists, all
// sized for `cap` superphotons: 2 x 88 B of queue, 168 B of pool and 8 B of lists per slot.
static const double kQueueSlotBytes = 352.0;
static int ensure_queues(mc_ctx *c, int64_t cap) {
  if (cap <= c->qcap) return MC_OK;
  for (int b = 0; b < 2; ++b) free_childbuf(c, c->q[b]);
  Pool &P = c->pool;
  for (int k = 0; k < 4; ++k) { dev_free(c, P.X[k]); dev_free(c, P.K[k]); dev_free(c, P.A[k]); }
  void *pv[] = {P.w, P.wb, P.ana, P.ans, P.acc, P.x1t, P.id, P.ctr, P.nev, P.nsc, P.nsteps, c->list_grid, c->list_free};
  for (void *ptr : pv) dev_free(c, ptr);
  std::memset(&P, 0, sizeof(P));
  c->list_grid = c->list_free = nullptr;
  c->qcap = 0;
  for (int b = 0; b < 2; ++b) {
    ChildBuf &q = c->q[b];
    for (int k = 0; k < 4; ++k) {
      q.X[k] = (double *)dev_alloc(c, 8 * cap);
      q.K[k] = (double *)dev_alloc(c, 8 * cap);
      if (!q.X[k] || !q.K[k]) return fail(c, MC_ERR_OOM, "queue allocation failed");
    }
    q.w = (double *)dev_alloc(c, 8 * cap);
    q.id = (uint64_t *)dev_alloc(c, 8 * cap);
    q.ctr = (uint32_t *)dev_alloc(c, 4 * cap);
    q.nsc = (int32_t *)dev_alloc(c, 4 * cap);
    if (!q.w || !q.id || !q.ctr || !q.nsc) return fail(c, MC_ERR_OOM, "queue allocation failed");
  }
  for (int k = 0; k < 4; ++k) {
    P.X[k] = (double *)dev_alloc(c, 8 * cap);
    P.K[k] = (double *)dev_alloc(c, 8 * cap);
    P.A[k] = (double *)dev_alloc(c, 8 * cap);
    if (!P.X[k] || !P.K[k] || !P.A[k]) return fail(c, MC_ERR_OOM, "pool allocation failed");
  }
  double **dv[] = {&P.w, &P.wb, &P.ana, &P.ans, &P.acc, &P.x1t};
  for (double **d : dv) {
    *d = (double *)dev_alloc(c, 8 * cap);
    if (!*d) return fail(c, MC_ERR_OOM, "pool allocation failed");
  }
  P.id = (uint64_t *)dev_alloc(c, 8 * cap);
  P.ctr = (uint32_t *)dev_alloc(c, 4 * cap);
  P.nev = (uint32_t *)dev_alloc(c, 4 * cap);
  P.nsc = (int32_t *)dev_alloc(c, 4 * cap);
  P.nsteps = (int32_t *)dev_alloc(c, 4 * cap);
  c->list_grid = (int32_t *)dev_alloc(c, 4 * cap);
  c->list_free = (int32_t *)dev_alloc(c, 4 * cap);
  if (!P.id || !P.ctr || !P.nev || !P.nsc || !P.nsteps || !c->list_grid || !c->list_free)
    return fail(c, MC_ERR_OOM, "pool allocation failed");
  c->qcap = cap;
  return MC_OK;
}

// Enqueues weights, zone counts and scan for (N_s, seed) on st without any host synchronisation
// (usable under stream capture); the job's primary total ends up in c->total_dev.
int generate_async(mc_ctx *c, double n_s, uint64_t seed, cudaStream_t st) {
  DevModel m = make_model(c);
  m.seed = seed;
  cudaError_t e = cudaMemsetAsync(c->bad, 0, sizeof(int), st);
  if (e != cudaSuccess) return (int)e;
  launch_zone_prep(m, c->zvol, c->zpref, c->zlnuc, c->bad, st);
  launch_weights(m, c->zvol, c->zpref, c->zlnuc, c->partial, c->nchunks, n_s, c->p.w_min, c->lnw, c->winv, st);
  launch_counts(m, c->zvol, c->zpref, c->zlnuc, c->zgmax, c->znbar, c->counts, st);
  launch_scan(c->counts, c->start, c->bsum, c->nz, c->total_dev, st);
  c->last_seed = seed;
  c->last_ns = n_s;
  return (int)cudaGetLastError();
}

// Weights, counts and scan for (N_s, seed); leaves the job's primary total in c->last_total.
static int generate(mc_ctx *c, double n_s, uint64_t seed, cudaStream_t st) {
  CU(cudaEventRecord(c->ev[2], st));
  CU((cudaError_t)generate_async(c, n_s, seed, st));
  CU(cudaEventRecord(c->ev[3], st));
  CU(cudaMemcpyAsync(c->cnt_host + CNT_N, c->total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(c->cnt_host + CNT_N + 1, c->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  int bad = (int)(c->cnt_host[CNT_N + 1] & 0xffffffffu);
  if (bad) return fail(c, MC_ERR_NAN_INPUT, "non-finite zone state");
  float ms = 0.0f;
  CU(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
  c->t_generate = ms;
  c->last_total = (int64_t)c->cnt_host[CNT_N];
  c->last_seed = seed;
  c->last_ns = n_s;
  return MC_OK;
}

// Launch helper: records the launch's device time between two events on the stream and reads the
// counters back (the host needs the list lengths to size the next phase).
#define TIMED_LAUNCH(phase, launch_expr)                                                                  \
  do {                                                                                                    \
    CU(cudaEventRecord(c->ev[0], st));                                                                    \
    launch_expr;                                                                                          \
    CU(cudaGetLastError());                                                                               \
    CU(cudaEventRecord(c->ev[1], st));                                                                    \
    CU(cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st)); \
    CU(cudaStreamSynchronize(st));                                                                        \
    float ms_ = 0.0f;                                                                                     \
    CU(cudaEventElapsedTime(&ms_, c->ev[0], c->ev[1]));                                                   \
    c->t_transport += ms_;                                                                                \
    c->t_phase[phase] += ms_;                                                                             \
    c->n_launch++;                                                                                        \
  } while (0)

static int set_counter(mc_ctx *c, int idx, unsigned long long v, cudaStream_t st) {
  unsigned long long *h = c->cnt_host + CNT_N + 2 + idx;   // pinned staging slot per counter
  *h = v;
  CU(cudaMemcpyAsync(c->cnt + idx, h, sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
  return MC_OK;
}

// Transports primaries [u0, u1) (or the uid list) and all their descendants: per batch and per
// scattering generation, k_init fills the pool, then the in-grid and free push phases alternate
// until no superphoton of the generation is left.
// Next generation's bias scale from this generation's children per superphoton (see
// mc_get_bias_scales in mc.h).
static double tune_next_scale(double s, int64_t carried, int64_t children, double target) {
  const double r = carried > 0 ? (double)children / (double)carried : 0.0;
  double f = r > 0.0 ? target / r : 8.0;
  f = std::min(8.0, std::max(0.125, f));
  return std::min(1e12, s * f);
}

static int transport(mc_ctx *c, int64_t u0, int64_t u1, const int64_t *uid_list_dev, int64_t n_list, mc_log_rec *log_dev,
                     int64_t log_cap, uint64_t seed, cudaStream_t st, bool tune) {
  DevModel m = make_model(c);
  m.seed = seed;
  const int n_gen = c->p.n_sc_max + 1;
  if (tune || (int)c->bscale.size() != n_gen) c->bscale.assign(n_gen, 1.0);
  const bool tuning = tune && c->p.bias_target > 0.0;
  const int block = c->p.block ? c->p.block : 128;
  const int prec = c->p.precision;
  int occ[2];
  for (int ph = 0; ph < 2; ++ph) {
    occ[ph] = std::max(1, push_max_blocks_per_sm(prec, ph, block, m.a != 0.0 ? 1 : 0));
    if (c->p.ctas_per_sm > 0) occ[ph] = std::min(occ[ph], (int)c->p.ctas_per_sm);
  }
  const bool use_sur = c->p.surrogate == 1;
  if (use_sur && !c->sur_ready) return fail(c, MC_ERR_STATE, "surrogate requested but no trained weights");
  SurrogateView sv;
  std::memset(&sv, 0, sizeof(sv));
  // four 128-row groups of the network per CTA (tensor-memory kernels run one CTA per SM)
  const int sur_block = 128 * kTcGroupsMax;
  const int sur_smem = tc_smem_bytes(kTcGroupsMax);
  int occ_sur = 1;
  if (use_sur) {
    sv = surrogate_view(c);
    occ_sur = std::max(1, std::min(4, push_sur_max_blocks_per_sm(prec, sur_block, sur_smem)));
    if (c->p.ctas_per_sm > 0) occ_sur = std::min(occ_sur, (int)c->p.ctas_per_sm);
    CU(cudaMemsetAsync(c->sur_err, 0, sizeof(unsigned int), st));
  }
  const int64_t n_prim = uid_list_dev ? n_list : (u1 - u0);
  const int64_t batch_max = 1 << 24;
  int64_t batch = std::min<int64_t>(std::max<int64_t>(n_prim, 1), batch_max);
  int rc = ensure_queues(c, std::max<int64_t>(1 << 20, 2 * batch));
  if (rc) return rc;
  PushIO pio;
  std::memset(&pio, 0, sizeof(pio));
  pio.pool = c->pool;
  pio.spec = c->spec;
  pio.cnt = c->cnt;
  pio.log = log_dev;
  pio.log_cap = log_cap;
  pio.out_cap = c->qcap;
  InitIO iio;
  std::memset(&iio, 0, sizeof(iio));
  iio.pool = c->pool;
  iio.list_grid = c->list_grid;
  iio.list_free = c->list_free;
  iio.cnt = c->cnt;
  for (int64_t b0 = 0; b0 < n_prim; b0 += batch) {
    int64_t nb = std::min(batch, n_prim - b0);
    int gen = 0;
    int64_t n_items = nb;
    while (n_items > 0) {
      if (n_items > c->qcap) return fail(c, MC_ERR_QUEUE_OVERFLOW, "generation larger than the superphoton pool");
      m.bias_scale = c->bscale[std::min(gen, n_gen - 1)];
      m.fbias_scale = (float)m.bias_scale;
      iio.n_items = n_items;
      if (gen == 0) {
        iio.mode = uid_list_dev ? 1 : 0;
        iio.uid0 = u0 + b0;
        iio.uids = uid_list_dev ? uid_list_dev + b0 : nullptr;
      } else {
        iio.mode = 2;
        iio.in = c->q[(gen - 1) & 1];
      }
      pio.out = c->q[gen & 1];
      // cursor, children, phase-list counters start at zero for the generation
      CU(cudaMemsetAsync(c->cnt + CNT_NEXT, 0, 2 * sizeof(unsigned long long), st));
      CU(cudaMemsetAsync(c->cnt + CNT_L0, 0, 2 * sizeof(unsigned long long), st));
      int grid_init = (int)std::min<int64_t>((int64_t)c->sms * 4, (n_items + block - 1) / block);
      TIMED_LAUNCH(0, launch_init(m, iio, prec, grid_init, block, st));
      int64_t n_grid = (int64_t)c->cnt_host[CNT_L0], n_free = (int64_t)c->cnt_host[CNT_L1];
      while (n_grid > 0 || n_free > 0) {
        if (n_grid > 0) {
          rc = set_counter(c, CNT_NEXT, 0, st);
          if (rc) return rc;
          pio.list_in = c->list_grid;
          pio.n_in = n_grid;
          pio.list_out = c->list_free;
          pio.out_counter = CNT_L1;   // continues after the n_free entries already listed
          if (use_sur) {
            int grid = (int)std::min<int64_t>((int64_t)c->sms * occ_sur, (n_grid + sur_block - 1) / sur_block);
            TIMED_LAUNCH(1, launch_push_sur(m, pio, sv, prec, grid, sur_smem, st));
          } else {
            int grid = (int)std::min<int64_t>((int64_t)c->sms * occ[0], (n_grid + block - 1) / block);
            TIMED_LAUNCH(1, launch_push(m, pio, prec, 0, grid, block, st));
          }
          if (c->cnt_host[CNT_ERR] & 1ull) return fail(c, MC_ERR_QUEUE_OVERFLOW, "scattered-superphoton queue overflow");
          n_free = (int64_t)c->cnt_host[CNT_L1];
          n_grid = 0;
          rc = set_counter(c, CNT_L0, 0, st);
          if (rc) return rc;
        }
        if (n_free > 0) {
          rc = set_counter(c, CNT_NEXT, 0, st);
          if (rc) return rc;
          pio.list_in = c->list_free;
          pio.n_in = n_free;
          pio.list_out = c->list_grid;
          pio.out_counter = CNT_L0;
          int grid = (int)std::min<int64_t>((int64_t)c->sms * occ[1], (n_free + block - 1) / block);
          TIMED_LAUNCH(2, launch_push(m, pio, prec, 1, grid, block, st));
          if (c->cnt_host[CNT_ERR] & 1ull) return fail(c, MC_ERR_QUEUE_OVERFLOW, "scattered-superphoton queue overflow");
          n_grid = (int64_t)c->cnt_host[CNT_L0];
          n_free = 0;
          rc = set_counter(c, CNT_L1, 0, st);
          if (rc) return rc;
        }
      }
      const int64_t children = (int64_t)c->cnt_host[CNT_OUT];
      if (tuning && b0 == 0 && gen + 1 < n_gen)
        c->bscale[gen + 1] = tune_next_scale(c->bscale[gen], n_items, children, c->p.bias_target);
      n_items = children;
      ++gen;
    }
  }
  if (use_sur) {
    unsigned int err = 0;
    CU(cudaMemcpy(&err, c->sur_err, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (err) return fail(c, MC_ERR_TIMEOUT, "tensor-core wait timed out in the surrogate push");
  }
  return MC_OK;
}

static void fill_stats(mc_ctx *c, mc_run_stats *s) {
  if (!s) return;
  const unsigned long long *h = c->cnt_host;
  s->n_emit = h[CNT_EMIT]; s->n_child = h[CNT_CHILD]; s->n_rec = h[CNT_REC]; s->n_abs = h[CNT_ABS];
  s->n_capt = h[CNT_CAPT]; s->n_maxst = h[CNT_MAXST]; s->n_steps = h[CNT_STEPS]; s->n_iters = h[CNT_ITERS];
  s->n_nonconv = h[CNT_NONCONV]; s->n_roul_surv = h[CNT_ROUL]; s->n_rej_cap = h[CNT_REJCAP];
  s->n_events = h[CNT_EVENTS]; s->n_total = c->last_total; s->err_flags = (int64_t)h[CNT_ERR];
  s->transport_launches = c->n_launch;
  s->transport_ms = c->t_transport;
  s->generate_ms = c->t_generate;
  s->n_steps_grid = h[CNT_GSTEPS];
  s->n_iters_grid = h[CNT_GITERS];
  s->init_ms = c->t_phase[0];
  s->grid_ms = c->t_phase[1];
  s->free_ms = c->t_phase[2];
}

int mc_run(mc_ctx *c, double n_s, uint64_t seed, int64_t shard, int64_t n_shards, void *stream, mc_run_stats *stats) {
  if (!c) return fail(nullptr, MC_ERR_INVALID_ARG, "null context");
  if (!c->have_grid) return fail(c, MC_ERR_STATE, "mc_set_grid must be called before mc_run");
  if (!(n_s > 0.0) || n_shards < 1 || shard < 0 || shard >= n_shards) return fail(c, MC_ERR_INVALID_ARG, "bad N_s or shard");
  CU(cudaSetDevice(c->p.device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = generate(c, n_s, seed, st);
  if (rc) return rc;
  int64_t T = c->last_total;
  int64_t u0 = (int64_t)((__int128)T * shard / n_shards), u1 = (int64_t)((__int128)T * (shard + 1) / n_shards);
  size_t nspec = (size_t)c->p.n_incl * c->p.n_bins * 3;
  // A scattered generation that outgrows the queues is rerun from the start with larger queues:
  // every superphoton draws from its own counter-based stream, so the rerun gives the same result.
  for (int attempt = 0;; ++attempt) {
    CU(cudaMemsetAsync(c->spec, 0, sizeof(double) * nspec, st));
    CU(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * CNT_N, st));
    c->t_transport = 0.0;
    c->t_phase[0] = c->t_phase[1] = c->t_phase[2] = 0.0;
    c->n_launch = 0;
    rc = transport(c, u0, u1, nullptr, 0, nullptr, 0, seed, st, true);
    if (rc != MC_ERR_QUEUE_OVERFLOW || attempt == 3) break;
    int64_t need = (int64_t)c->cnt_host[CNT_OUT];   // slots the overflowing generation asked for
    int64_t want = std::max<int64_t>(need + need / 2, 2 * c->qcap);
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    if ((double)want * kQueueSlotBytes > 0.9 * ((double)free_b + (double)c->qcap * kQueueSlotBytes)) break;
    rc = ensure_queues(c, want);
    if (rc) return rc;
  }
  if (rc) return rc;
  // final counters (also when the shard had no superphoton and nothing was launched)
  CU(cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  c->have_run = true;
  fill_stats(c, stats);
  return MC_OK;
}

int mc_trace(mc_ctx *c, double n_s, uint64_t seed, const int64_t *uids, size_t n_uids, mc_log_rec *out, size_t cap,
             size_t *n_out, void *stream) {
  if (!c || !uids || !out || !n_out) return fail(c, MC_ERR_INVALID_ARG, "null argument");
  if (!c->have_grid) return fail(c, MC_ERR_STATE, "mc_set_grid must be called before mc_trace");
  CU(cudaSetDevice(c->p.device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = generate(c, n_s, seed, st);
  if (rc) return rc;
  for (size_t i = 0; i < n_uids; ++i)
    if (uids[i] < 0 || uids[i] >= c->last_total) return fail(c, MC_ERR_SIZE, "uid out of range");
  int64_t *ud = (int64_t *)dev_alloc(c, 8 * std::max<size_t>(n_uids, 1));
  mc_log_rec *ld = (mc_log_rec *)dev_alloc(c, sizeof(mc_log_rec) * std::max<size_t>(cap, 1));
  if (!ud || !ld) {
    dev_free(c, ud);
    dev_free(c, ld);
    return fail(c, MC_ERR_OOM, "trace buffers");
  }
  size_t nspec = (size_t)c->p.n_incl * c->p.n_bins * 3;
  cudaError_t e = cudaMemcpyAsync(ud, uids, 8 * n_uids, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->spec, 0, sizeof(double) * nspec, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * CNT_N, st);
  if (e != cudaSuccess) {
    dev_free(c, ud);
    dev_free(c, ld);
    return fail(c, MC_ERR_CUDA, cudaGetErrorString(e));
  }
  rc = (n_uids > 0) ? transport(c, 0, 0, ud, (int64_t)n_uids, ld, (int64_t)cap, seed, st, false) : MC_OK;
  if (rc == MC_OK) {
    size_t n = std::min<size_t>((size_t)c->cnt_host[CNT_LOG], cap);
    e = cudaMemcpyAsync(out, ld, sizeof(mc_log_rec) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(c, MC_ERR_CUDA, cudaGetErrorString(e));
    *n_out = n;
    c->have_run = true;
  }
  dev_free(c, ud);
  dev_free(c, ld);
  return rc;
}

int mc_get_spectrum_sums(mc_ctx *c, double *sums, size_t n_elems) {
  if (!c || !sums) return fail(c, MC_ERR_INVALID_ARG, "null argument");
  size_t nspec = (size_t)c->p.n_incl * c->p.n_bins * 3;
  if (n_elems != nspec) return fail(c, MC_ERR_SIZE, "sums buffer must hold 3*n_incl*n_bins doubles");
  if (!c->have_run) return fail(c, MC_ERR_STATE, "no run yet");
  CU(cudaSetDevice(c->p.device));
  CU(cudaMemcpy(sums, c->spec, sizeof(double) * nspec, cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_get_spectrum(mc_ctx *c, double *nuLnu, double *sigma, double *counts, size_t n_elems) {
  if (!c) return fail(nullptr, MC_ERR_INVALID_ARG, "null context");
  size_t nb = (size_t)c->p.n_incl * c->p.n_bins;
  if (n_elems != nb) return fail(c, MC_ERR_SIZE, "buffers must hold n_incl*n_bins doubles");
  if (!c->have_run) return fail(c, MC_ERR_STATE, "no run yet");
  std::vector<double> s(nb * 3);
  int rc = mc_get_spectrum_sums(c, s.data(), nb * 3);
  if (rc) return rc;
  // nu L_nu = sum(w E) m_e c^2 / (dt dln nu_bin) * 4 pi / dOmega_incl, dt = 1 (section 3, eq. weight_calc)
  double dln = (c->p.lnu_hi - c->p.lnu_lo) / c->p.n_bins * std::log(10.0);
  for (int i = 0; i < c->p.n_incl; ++i) {
    double t0 = 0.5 * kPI * i / c->p.n_incl, t1 = 0.5 * kPI * (i + 1) / c->p.n_incl;
    double dom = 2.0 * 2.0 * kPI * (std::cos(t0) - std::cos(t1));   // both hemispheres
    double f = kME * kCL * kCL / dln * (4.0 * kPI / dom);
    for (int b = 0; b < c->p.n_bins; ++b) {
      size_t k = (size_t)i * c->p.n_bins + b;
      if (nuLnu) nuLnu[k] = s[3 * k] * f;
      if (sigma) sigma[k] = std::sqrt(s[3 * k + 1]) * f;
      if (counts) counts[k] = s[3 * k + 2];
    }
  }
  return MC_OK;
}

int mc_fma_peak(int device, int dtype, double *flops) {
  if (!flops || (dtype != MC_DTYPE_F64 && dtype != MC_DTYPE_F32)) return fail(nullptr, MC_ERR_INVALID_ARG, "bad argument");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, MC_ERR_NO_DEVICE, "no such CUDA device");
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, MC_ERR_CUDA, "cudaSetDevice failed");
  double f = 0.0;
  cudaError_t e = fma_peak(dtype == MC_DTYPE_F64, &f);
  if (e != cudaSuccess) return fail(nullptr, MC_ERR_CUDA, cudaGetErrorString(e));
  *flops = f;
  return MC_OK;
}

int mc_get_bias_scales(mc_ctx *c, double *scales, int n) {
  if (!c || !scales) return fail(c, MC_ERR_INVALID_ARG, "null argument");
  if (!c->have_run || (int)c->bscale.size() != c->p.n_sc_max + 1) return fail(c, MC_ERR_STATE, "no run yet");
  if (n != c->p.n_sc_max + 1) return fail(c, MC_ERR_SIZE, "scales buffer must hold n_sc_max + 1 elements");
  for (int g = 0; g < n; ++g) scales[g] = c->bscale[g];
  return MC_OK;
}

int mc_selftest_math(int which, const double *x, double *y, double *ref, int64_t n) {
  if (which < 0 || which > 10 || n < 0 || (n > 0 && (!x || !y || !ref))) return fail(nullptr, MC_ERR_INVALID_ARG, "bad argument");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(nullptr, MC_ERR_NO_DEVICE, "no CUDA device");
  }
  if (n == 0) return MC_OK;
  double *d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 3 * n) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MC_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = selftest_math(which, d, d + n, d + 2 * n, n);
  if (e == cudaSuccess) e = cudaMemcpy(y, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, d + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, MC_ERR_CUDA, cudaGetErrorString(e));
  return MC_OK;
}

int mc_get_zone_counts(mc_ctx *c, int64_t *counts, size_t n_elems) {
  if (!c || !counts) return fail(c, MC_ERR_INVALID_ARG, "null argument");
  if (!c->have_grid || c->last_ns == 0.0) return fail(c, MC_ERR_STATE, "no run yet");
  if (n_elems != (size_t)c->nz) return fail(c, MC_ERR_SIZE, "counts buffer must hold n1*n2*n3 elements");
  CU(cudaSetDevice(c->p.device));
  CU(cudaMemcpy(counts, c->counts, 8 * c->nz, cudaMemcpyDeviceToHost));
  return MC_OK;
}

}  // extern "C"
