// mc_internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mc.h"
#include "mc_device.cuh"

namespace mcgb {

// Scattered-superphoton queue of one generation (structure of arrays).
struct ChildBuf {
  double *X[4];
  double *K[4];
  double *w;
  uint64_t *id;
  uint32_t *ctr;
  int32_t *nsc;
  int16_t *model;   // model index (batched runs only; NULL otherwise)
};

// Superphoton state between transport phases (structure of arrays, one slot per superphoton
// of the current batch or generation).
struct Pool {
  double *X[4], *K[4], *A[4];
  double *w, *wb, *ana, *ans, *acc, *x1t;
  uint64_t *id;
  uint32_t *ctr, *nev;
  int32_t *nsc, *nsteps;
  int16_t *model;   // model index (batched runs only; NULL otherwise)
};

// Counters written by the transport kernels (unsigned 64-bit for atomics).
enum {
  CNT_NEXT = 0,   // work-item cursor
  CNT_OUT,        // children appended
  CNT_LOG,        // log records appended
  CNT_ERR,        // error bits
  CNT_L0,         // appends to the in-grid list
  CNT_L1,         // appends to the free-streaming list
  CNT_EMIT, CNT_CHILD, CNT_REC, CNT_ABS, CNT_CAPT, CNT_MAXST,
  CNT_STEPS, CNT_ITERS, CNT_NONCONV, CNT_ROUL, CNT_REJCAP, CNT_EVENTS,
  CNT_GSTEPS, CNT_GITERS,   // steps and predictor passes taken by the in-grid phase
  CNT_N
};

// Emission (or loading of scattered children) and transport initialisation into the pool;
// slots are appended to the in-grid list (CNT_L0) or the free list (CNT_L1).
struct InitIO {
  int mode;                 // 0: primaries uid0 .. uid0+n_items; 1: uid list; 2: children
  int64_t uid0, n_items;
  const int64_t *uids;
  ChildBuf in;
  Pool pool;
  int32_t *list_grid, *list_free;
  unsigned long long *cnt;
};

// One phase of transport over the listed pool slots; slots that change phase are appended to
// list_out (counter out_counter).
struct PushIO {
  const int32_t *list_in;
  int64_t n_in;
  int32_t *list_out;
  int out_counter;
  Pool pool;
  ChildBuf out;
  int64_t out_cap;
  double *spec;             // [n_incl][n_bins][3]
  unsigned long long *cnt;  // CNT_N counters
  mc_log_rec *log;
  int64_t log_cap;
};

// tables (mc_tables.cu)
void launch_tables(const DevModel &m, double *lnF, double *lnK2, double *hot, const double *gl_ang,
                   const double *gl_s, const double *gl_mu, cudaStream_t st);
// generation (mc_tables.cu)
void launch_zone_prep(const DevModel &m, double *zvol, double *zpref, double *zlnuc, int *bad, cudaStream_t st);
void launch_weights(const DevModel &m, const double *zvol, const double *zpref, const double *zlnuc, double *partial,
                    int nchunks, double n_s, double w_min, double *lnw, double *winv, cudaStream_t st);
void launch_counts(const DevModel &m, const double *zvol, const double *zpref, const double *zlnuc, double *zgmax,
                   double *znbar, int64_t *counts, cudaStream_t st);
void launch_scan(const int64_t *counts, int64_t *start, int64_t *bsum, int64_t n, int64_t *total_dev, cudaStream_t st);
// grid conversion (mc_tables.cu): caller layout [8][nz] -> zone-major [nz][8]
void launch_grid_to_aos(const void *src, int src_f32, void *dst, int dst_f32, int64_t nz, int *bad, cudaStream_t st);
// FMA-chain throughput of the FP64 or FP32 pipe in FLOP/s (mc_tables.cu)
cudaError_t fma_peak(bool fp64, double *flops);
cudaError_t selftest_math(int which, const double *x_dev, double *y_dev, double *ref_dev, int64_t n);
void df_table_host(df *t);
void launch_to_f32(const double *src, float *dst, int n, cudaStream_t st);
void launch_kappa_tables(double kappa, double *lnF, double *lnJ, double *lnA, double *lnI, double *lnH,
                         const double *gl_mu, cudaStream_t st);
// transport (mc_transport.cu)
// prec: the precision form (MC_PREC_FP64, MC_PREC_MIXED or MC_PREC_SPLIT)
int push_max_blocks_per_sm(int prec, int phase, int block, int kerr);
void launch_init(const DevModel &m, const InitIO &io, int prec, int grid, int block, cudaStream_t st);
// phase 0: superphotons inside the radial extent of the grid; 1: outside it
void launch_push(const DevModel &m, const PushIO &io, int prec, int phase, int grid, int block, cudaStream_t st);
// in-grid push with the coefficient network (mixed or split form; 128-thread row groups)
int push_sur_max_blocks_per_sm(int prec, int block, int smem);
void launch_push_sur(const DevModel &m, const PushIO &io, const SurrogateView &sv, int prec, int grid, int smem,
                     cudaStream_t st);

}  // namespace mcgb

// Context owned by the library (opaque to callers; shared by the library's translation units).
struct mc_ctx {
  // parameters, last error, device properties
  mc_model_params p;
  std::string err;
  int sms = 0;
  // allocations made through the caller's allocator (or cudaMalloc)
  std::vector<void *> allocs;
  // tables
  double *lnF = nullptr, *lnK2 = nullptr, *hot = nullptr, *gl = nullptr;
  int nF = 0, nK2 = 0;
  // grid
  bool have_grid = false;
  std::vector<double> bscale;   // bias scale per scattering generation (last mc_run)
  uint64_t grid_epoch = 0;   // bumped by every mc_set_grid (captured batch graphs hold grid pointers)
  void *prim = nullptr;
  float *prim_x32 = nullptr;   // FP32 copy of an FP64 grid, read by the mixed-precision transport
  double *zbq = nullptr, *zbnt = nullptr;   // per-zone bremsstrahlung normalisation and k T_e / h
  double *zlnw = nullptr;                   // per-zone ln w of the kappa population
  double *kapF = nullptr, *kapJ = nullptr, *kapA = nullptr, *kapI = nullptr;   // kappa tables
  double *kapH = nullptr;                   // kappa hot cross-section [kKapNW][kHotNE]
  mcgb::df *dtab = nullptr;                 // double-float function table (exp2, sin pi)
  double *ftab = nullptr;                   // tables of the FP64 exp_t, log_t, sincospi_t
  float *lnK2f = nullptr, *hotf = nullptr;  // FP32 copies of the K2 and hot cross-section tables
  int prim_f32 = 0;
  int n1 = 0, n2 = 0, n3 = 0;
  int64_t nz = 0;
  double x1_0 = 0, dx1 = 0, x2_0 = 0, dx2 = 0, x3_0 = 0, dx3 = 0;
  // per-run generation data
  double *zvol = nullptr, *zpref = nullptr, *zlnuc = nullptr, *zgmax = nullptr, *znbar = nullptr;
  int64_t *counts = nullptr, *start = nullptr, *bsum = nullptr;
  double *partial = nullptr, *lnw = nullptr, *winv = nullptr;
  int *bad = nullptr;
  int nchunks = 0;
  // transport
  mcgb::ChildBuf q[2];
  int64_t qcap = 0;
  mcgb::Pool pool;
  int32_t *list_grid = nullptr, *list_free = nullptr;
  int64_t pcap = 0;
  unsigned long long *cnt = nullptr;
  int64_t *total_dev = nullptr;
  double *spec = nullptr;
  unsigned long long *cnt_host = nullptr;   // pinned
  bool have_run = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double t_transport = 0.0, t_generate = 0.0, t_phase[3] = {0.0, 0.0, 0.0};
  int64_t n_launch = 0;
  int64_t last_total = 0;
  uint64_t last_seed = 0;
  double last_ns = 0.0;
  // coefficient surrogate network
  float *sur_w = nullptr;              // FP32 master weights
  unsigned char *sur_packed = nullptr; // BF16 tiles for tcgen05 inference
  float *sur_bias = nullptr;
  unsigned int *sur_err = nullptr;     // tensor-core wait timeouts
  bool sur_ready = false;
  // batched runs led by this context (mc_batch.cu)
  void *batch = nullptr;
  double wait_ns = 120e9;   // limit on each device-side grid-barrier wait of a batch led by this context
};

// Tensor-core view of the context's trained network (mc_mlp.cu).
mcgb::SurrogateView surrogate_view(const mc_ctx *c);
// Kernel-side view of a context, device allocation through the context's allocator, and the
// error setter (mc_api.cu).
mcgb::DevModel make_model(const mc_ctx *c);
void *dev_alloc_ext(mc_ctx *c, size_t bytes);
void dev_free_ext(mc_ctx *c, void *ptr);
int set_err(mc_ctx *c, int code, const char *msg);
extern "C" int generate_async(mc_ctx *c, double n_s, uint64_t seed, cudaStream_t st);
void mc_batch_release(mc_ctx *c);

