// mc_batch.cu -- many models of uneven size in one persistent launch (parameter surveys).
//
// The paper motivates GPU Monte Carlo by parameter surveys (section 1: spin x electron heating x
// accretion rate); here a batch of models is transported together.  Per model, the generation
// kernels (weights, counts, scan) run as in mc_run; then ONE cooperative kernel carries every
// superphoton of every model through every phase of every scattering generation:
//   init (emission / child load) -> [in-grid push -> free push]* -> next generation ...
// separated by a grid-wide barrier.  Each superphoton carries its model index; the model
// descriptors sit in shared memory (read through L1 in the 6- and 8-CTA variants).  Phase counters
// are fresh for every phase instance (no resets between barriers).  The whole sequence is captured
// into a CUDA graph and replayed; an autotuner picks the register cap (launch bounds) and the
// resident CTAs per SM.  The kernel itself is in mc_batch.cuh, instantiated per precision form in
// mc_batch_fp64.cu, mc_batch_mixed.cu and mc_batch_split.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mc_batch.cuh"

namespace mcgb {

// prim_off[i + 1] = prim_off[i] + total of model i (totals read from each model's scan).
__global__ void k_batch_offsets(const int64_t *const *totals, int n, int64_t *prim_off) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t acc = 0;
    prim_off[0] = 0;
    for (int i = 0; i < n; ++i) {
      acc += *totals[i];
      prim_off[i + 1] = acc;
    }
  }
}

// Launch-bounds variants per precision form (see each form's translation unit).
static BatchKernel pick_kernel(int prec, bool sur, int minb) {
  if (prec == 1) return batch_kernel_mixed(sur, minb);
  if (prec == 2) return batch_kernel_split(sur, minb);
  return batch_kernel_fp64(sur, minb);
}

}  // namespace mcgb

using namespace mcgb;

// ------------------------------------------------------------------ host side
struct BatchState {
  int n_models = 0;
  int64_t cap = 0;
  DevModel *models = nullptr;
  int64_t **totals = nullptr;
  int64_t *prim_off = nullptr;
  unsigned long long *ph = nullptr;
  unsigned int *bar = nullptr;
  Pool pool;
  ChildBuf q[2];
  int32_t *list_grid = nullptr, *list_free = nullptr;
  std::vector<void *> allocs;
  bool alloc_failed = false;
  // tuned launch configuration
  int tuned = 0, minb = 1, ctas = 0;
  // captured graph and the inputs it was captured for
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> g_ns;
  std::vector<uint64_t> g_seed;
  std::vector<const mc_ctx *> g_ctx;
  std::vector<uint64_t> g_epoch;
  // pinned host staging for the descriptors copied at every launch (a captured copy node reads
  // its host source again at each replay, so the source must outlive the graph)
  DevModel *h_models = nullptr;
  const int64_t **h_totals = nullptr;
  int g_minb = 0, g_ctas = 0;
  double g_wait = 0.0;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static void batch_free(mc_ctx *owner, BatchState *bs) {
  if (!bs) return;
  if (bs->gexec) cudaGraphExecDestroy(bs->gexec);
  if (bs->cap_stream) cudaStreamDestroy(bs->cap_stream);
  if (bs->e0) cudaEventDestroy(bs->e0);
  if (bs->e1) cudaEventDestroy(bs->e1);
  if (bs->h_models) cudaFreeHost(bs->h_models);
  if (bs->h_totals) cudaFreeHost((void *)bs->h_totals);
  for (void *p : bs->allocs) dev_free_ext(owner, p);
  delete bs;
}

void mc_batch_release(mc_ctx *c) {
  if (c && c->batch) {
    batch_free(c, (BatchState *)c->batch);
    c->batch = nullptr;
  }
}

static void *balloc(mc_ctx *owner, BatchState *bs, size_t bytes) {
  void *p = dev_alloc_ext(owner, bytes);
  if (p) bs->allocs.push_back(p);
  else bs->alloc_failed = true;
  return p;
}

// Device bytes per pool slot: superphoton pool 170, two child queues 2 x 90, two phase lists 8.
static const double kBatchSlotBytes = 358.0;

static int batch_alloc(mc_ctx *owner, BatchState *bs, int n, int64_t cap) {
  if (bs->n_models >= n && bs->cap >= cap) return MC_OK;
  for (void *p : bs->allocs) dev_free_ext(owner, p);
  bs->allocs.clear();
  bs->alloc_failed = false;
  bs->n_models = 0;
  bs->cap = 0;
  if (bs->gexec) {
    cudaGraphExecDestroy(bs->gexec);
    bs->gexec = nullptr;
  }
  bs->models = (DevModel *)balloc(owner, bs, sizeof(DevModel) * kMaxBatch);
  bs->totals = (int64_t **)balloc(owner, bs, sizeof(int64_t *) * kMaxBatch);
  bs->prim_off = (int64_t *)balloc(owner, bs, sizeof(int64_t) * (kMaxBatch + 1));
  bs->ph = (unsigned long long *)balloc(owner, bs, sizeof(unsigned long long) * kPhWords);
  bs->bar = (unsigned int *)balloc(owner, bs, 256);
  Pool &P = bs->pool;
  std::memset(&P, 0, sizeof(P));
  for (int k = 0; k < 4; ++k) {
    P.X[k] = (double *)balloc(owner, bs, 8 * cap);
    P.K[k] = (double *)balloc(owner, bs, 8 * cap);
    P.A[k] = (double *)balloc(owner, bs, 8 * cap);
  }
  double **dv[] = {&P.w, &P.wb, &P.ana, &P.ans, &P.acc, &P.x1t};
  for (double **d : dv) *d = (double *)balloc(owner, bs, 8 * cap);
  P.id = (uint64_t *)balloc(owner, bs, 8 * cap);
  P.ctr = (uint32_t *)balloc(owner, bs, 4 * cap);
  P.nev = (uint32_t *)balloc(owner, bs, 4 * cap);
  P.nsc = (int32_t *)balloc(owner, bs, 4 * cap);
  P.nsteps = (int32_t *)balloc(owner, bs, 4 * cap);
  P.model = (int16_t *)balloc(owner, bs, 2 * cap);
  for (int b = 0; b < 2; ++b) {
    ChildBuf &q = bs->q[b];
    std::memset(&q, 0, sizeof(q));
    for (int k = 0; k < 4; ++k) {
      q.X[k] = (double *)balloc(owner, bs, 8 * cap);
      q.K[k] = (double *)balloc(owner, bs, 8 * cap);
    }
    q.w = (double *)balloc(owner, bs, 8 * cap);
    q.id = (uint64_t *)balloc(owner, bs, 8 * cap);
    q.ctr = (uint32_t *)balloc(owner, bs, 4 * cap);
    q.nsc = (int32_t *)balloc(owner, bs, 4 * cap);
    q.model = (int16_t *)balloc(owner, bs, 2 * cap);
  }
  bs->list_grid = (int32_t *)balloc(owner, bs, 4 * cap);
  bs->list_free = (int32_t *)balloc(owner, bs, 4 * cap);
  if (bs->alloc_failed) return set_err(owner, MC_ERR_OOM, "batch allocation failed");
  bs->n_models = kMaxBatch;
  bs->cap = cap;
  return MC_OK;
}

// Fills the pinned staging buffers with the current model descriptors.  The previous launch that
// read them has completed: every mc_run_batch synchronises before returning.
static void stage_descriptors(mc_ctx **ctxs, int n, const uint64_t *seeds, BatchState *bs) {
  for (int i = 0; i < n; ++i) {
    bs->h_models[i] = make_model(ctxs[i]);
    bs->h_models[i].seed = seeds[i];
    bs->h_totals[i] = ctxs[i]->total_dev;
  }
}

// Enqueues one batched run on stream st (no host synchronisation): generation per model, offsets,
// counter resets, the cooperative transport kernel.
static cudaError_t batch_enqueue(mc_ctx **ctxs, int n, const double *n_s, const uint64_t *seeds, BatchState *bs,
                                 int minb, int ctas, cudaStream_t st, bool timed) {
  mc_ctx *c0 = ctxs[0];
  const int prec = c0->p.precision;
  const bool sur = c0->p.surrogate == 1;
  stage_descriptors(ctxs, n, seeds, bs);
  for (int i = 0; i < n; ++i) {
    cudaError_t e = (cudaError_t)generate_async(ctxs[i], n_s[i], seeds[i], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctxs[i]->cnt, 0, sizeof(unsigned long long) * CNT_N, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ctxs[i]->spec, 0, sizeof(double) * ctxs[i]->p.n_incl * ctxs[i]->p.n_bins * 3, st);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(bs->models, bs->h_models, sizeof(DevModel) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bs->totals, bs->h_totals, sizeof(int64_t *) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  k_batch_offsets<<<1, 1, 0, st>>>(bs->totals, n, bs->prim_off);
  e = cudaMemsetAsync(bs->ph, 0, sizeof(unsigned long long) * kPhWords, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bs->bar, 0, 256, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c0->cnt, 0, sizeof(unsigned long long) * CNT_N, st);
  if (e == cudaSuccess && sur) e = cudaMemsetAsync(c0->sur_err, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  BatchIO b;
  std::memset(&b, 0, sizeof(b));
  b.models = bs->models;
  b.n_models = n;
  b.prim_off = bs->prim_off;
  b.pool = bs->pool;
  b.q[0] = bs->q[0];
  b.q[1] = bs->q[1];
  b.list_grid = bs->list_grid;
  b.list_free = bs->list_free;
  b.cap = bs->cap;
  b.cnt = c0->cnt;
  b.ph = bs->ph;
  b.bar = bs->bar;
  if (sur) b.sv = surrogate_view(c0);
  b.timeout_ns = c0->wait_ns;
  BatchKernel kern = pick_kernel(prec, sur, minb);
  const int smem = batch_smem_bytes(sur, minb);
  cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // shared memory over L1: the descriptors take ~48 KB, a CTA with four network row groups ~163 KB more
  cudaFuncSetAttribute((const void *)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  void *args[] = {&b};
  if (timed) cudaEventRecord(bs->e0, st);
  e = cudaLaunchCooperativeKernel((const void *)kern, dim3(ctas), dim3(sur ? 128 * kTcGroupsMax : 128), args, smem, st);
  if (timed) cudaEventRecord(bs->e1, st);
  return e;
}

static int max_ctas(mc_ctx *c0, int minb) {
  const int prec = c0->p.precision;
  const bool sur = c0->p.surrogate == 1;
  BatchKernel kern = pick_kernel(prec, sur, minb);
  const int smem = batch_smem_bytes(sur, minb);
  cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute((const void *)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void *)kern, sur ? 128 * kTcGroupsMax : 128, smem);
  if (sur) n = std::min(n, 512 / kTmemCols);   // TMEM: 512 columns per SM
  return std::max(n, 0);
}

extern "C" int mc_run_batch(mc_ctx **ctxs, int n, const double *n_s, const uint64_t *seeds, int flags, void *stream,
                            mc_run_stats *stats) {
  if (!ctxs || n < 1 || !n_s || !seeds) return set_err(nullptr, MC_ERR_INVALID_ARG, "null argument");
  if (n > kMaxBatch) return set_err(ctxs[0], MC_ERR_SIZE, "at most 64 models per batch");
  mc_ctx *c0 = ctxs[0];
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return set_err(c0, MC_ERR_INVALID_ARG, "null context");
    if (!ctxs[i]->have_grid) return set_err(c0, MC_ERR_STATE, "every model needs a grid");
    if (!(n_s[i] > 0.0)) return set_err(c0, MC_ERR_INVALID_ARG, "N_s must be positive");
    if (ctxs[i]->p.device != c0->p.device || ctxs[i]->p.precision != c0->p.precision ||
        ctxs[i]->p.surrogate != c0->p.surrogate)
      return set_err(c0, MC_ERR_INVALID_ARG, "models of a batch share device, precision and surrogate mode");
    if (ctxs[i]->p.n_sc_max + 2 > kMaxGen) return set_err(c0, MC_ERR_INVALID_ARG, "n_sc_max too large for a batch");
    if (ctxs[i]->p.bias_target > 0.0) return set_err(c0, MC_ERR_INVALID_ARG, "bias tuning runs in mc_run only");
  }
  if (c0->p.surrogate == 1 && !c0->sur_ready) return set_err(c0, MC_ERR_STATE, "surrogate requested but no weights");
  if (cudaSetDevice(c0->p.device) != cudaSuccess) return set_err(c0, MC_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  BatchState *bs = (BatchState *)c0->batch;
  if (!bs) {
    bs = new BatchState();
    c0->batch = bs;
    cudaEventCreate(&bs->e0);
    cudaEventCreate(&bs->e1);
    cudaStreamCreateWithFlags(&bs->cap_stream, cudaStreamNonBlocking);
    if (cudaMallocHost(&bs->h_models, sizeof(DevModel) * kMaxBatch) != cudaSuccess ||
        cudaMallocHost((void **)&bs->h_totals, sizeof(int64_t *) * kMaxBatch) != cudaSuccess) {
      cudaGetLastError();
      batch_free(c0, bs);
      c0->batch = nullptr;
      return set_err(c0, MC_ERR_OOM, "pinned host allocation failed");
    }
  }
  // capacity: every generation of the batch must fit the pool (primaries ~ N_s per model; a larger
  // scattered generation makes the run repeat with a pool twice as large, below)
  double ns_tot = 0.0;
  for (int i = 0; i < n; ++i) ns_tot += n_s[i];
  int64_t cap = std::max<int64_t>((int64_t)(1.5 * ns_tot) + (1 << 20), bs->cap);
  if (cap > (int64_t)2000000000) return set_err(c0, MC_ERR_SIZE, "batch too large for one launch");
  int rc = batch_alloc(c0, bs, n, cap);
  if (rc) return rc;
  // ---- autotuner: register cap x resident CTAs per SM, timed on a calibration run of every model at
  // a fraction of its N_s.  The fraction keeps >= ~5e6 superphotons in the calibration batch: with
  // less, the tails of the phases (a few long paths between grid barriers) hide the throughput.
  if ((flags & 1) && !bs->tuned) {
    std::vector<double> ns_small(n);
    const double frac = std::min(1.0, std::max(0.05, 5e6 / ns_tot));
    for (int i = 0; i < n; ++i) ns_small[i] = std::max(1.0, frac * n_s[i]);
    double best = 1e300;
    const int minbs[5] = {1, 3, 4, 6, 8};   // register caps 255, 168, 128, 80, 64
    for (int mb : minbs) {
      if (mb != 1 && c0->p.surrogate == 1) continue;   // one launch-bounds variant with the network
      if (mb == 4 && c0->p.precision == MC_PREC_SPLIT) continue;   // the split form has the 1 and 3 variants
      if (mb >= 6 && c0->p.precision != MC_PREC_MIXED) continue;   // the double-float form only
      int mx = max_ctas(c0, mb);
      for (int per = (mb >= 6 ? 5 : 1); per <= mx; ++per) {
        int ctas = per * c0->sms;
        cudaError_t e = batch_enqueue(ctxs, n, ns_small.data(), seeds, bs, mb, ctas, st, true);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_err(c0, MC_ERR_CUDA, cudaGetErrorString(e));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, bs->e0, bs->e1);
        if (ms < best) {
          best = ms;
          bs->minb = mb;
          bs->ctas = ctas;
        }
      }
    }
    bs->tuned = 1;
  }
  int minb = bs->tuned ? bs->minb : 1;
  int ctas = bs->tuned ? bs->ctas : std::max(1, max_ctas(c0, 1)) * c0->sms;
  if (c0->p.ctas_per_sm > 0) ctas = std::min(ctas, c0->p.ctas_per_sm * c0->sms);
  unsigned long long h[CNT_N];
  std::vector<int64_t> off(n + 1);
  bool used_graph = false;
  // A batch whose scattered generations outgrow the pool is rerun with a larger one (the result
  // is the same: every superphoton draws from its own counter-based stream).
  for (int attempt = 0;; ++attempt) {
  used_graph = false;
  if (flags & 2) {
    // ---- CUDA graph: capture once per (models, N_s, seeds, launch configuration), then replay
    std::vector<double> vns(n_s, n_s + n);
    std::vector<uint64_t> vseed(seeds, seeds + n);
    std::vector<const mc_ctx *> vctx(ctxs, ctxs + n);
    std::vector<uint64_t> vep(n);
    for (int i = 0; i < n; ++i) vep[i] = ctxs[i]->grid_epoch;
    bool same = bs->gexec && bs->g_ns == vns && bs->g_seed == vseed && bs->g_ctx == vctx && bs->g_epoch == vep &&
                bs->g_minb == minb && bs->g_ctas == ctas && bs->g_wait == c0->wait_ns;
    if (!same) {
      if (bs->gexec) {
        cudaGraphExecDestroy(bs->gexec);
        bs->gexec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(bs->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = batch_enqueue(ctxs, n, n_s, seeds, bs, minb, ctas, bs->cap_stream, false);
        e = cudaStreamEndCapture(bs->cap_stream, &graph);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&bs->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cudaGetLastError();   // capture unsupported: fall back to direct launches
        bs->gexec = nullptr;
      } else {
        bs->g_ns = vns;
        bs->g_seed = vseed;
        bs->g_ctx = vctx;
        bs->g_epoch = vep;
        bs->g_minb = minb;
        bs->g_ctas = ctas;
        bs->g_wait = c0->wait_ns;
      }
    }
    if (bs->gexec) {
      stage_descriptors(ctxs, n, seeds, bs);
      cudaEventRecord(bs->e0, st);
      cudaError_t e = cudaGraphLaunch(bs->gexec, st);
      cudaEventRecord(bs->e1, st);
      if (e != cudaSuccess) return set_err(c0, MC_ERR_CUDA, cudaGetErrorString(e));
      used_graph = true;
    }
  }
  if (!used_graph) {
    cudaError_t e = batch_enqueue(ctxs, n, n_s, seeds, bs, minb, ctas, st, true);
    if (e != cudaSuccess) return set_err(c0, MC_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaMemcpyAsync(h, c0->cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(off.data(), bs->prim_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_err(c0, MC_ERR_CUDA, cudaGetErrorString(e));
  if (h[CNT_ERR] & 4ull) return set_err(c0, MC_ERR_TIMEOUT, "grid barrier timed out");
  if (h[CNT_ERR] & 8ull) return set_err(c0, MC_ERR_SIZE, "more transport phases than one batched launch holds");
  if (!(h[CNT_ERR] & 1ull)) break;
  size_t free_b = 0, total_b = 0;
  int64_t want = 2 * bs->cap;
  if (attempt == 2 || want > (int64_t)2000000000 || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess ||
      (double)want * kBatchSlotBytes > 0.9 * ((double)free_b + (double)bs->cap * kBatchSlotBytes))
    return set_err(c0, MC_ERR_QUEUE_OVERFLOW, "batch queue overflow");
  rc = batch_alloc(c0, bs, n, want);   // also drops the captured graph (it holds the old buffers)
  if (rc) return rc;
  }
  if (c0->p.surrogate == 1) {
    unsigned int err = 0;
    cudaMemcpy(&err, c0->sur_err, sizeof(err), cudaMemcpyDeviceToHost);
    if (err) return set_err(c0, MC_ERR_TIMEOUT, "tensor-core wait timed out");
  }
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, bs->e0, bs->e1);
  for (int i = 0; i < n; ++i) {
    ctxs[i]->have_run = true;
    ctxs[i]->last_total = off[i + 1] - off[i];
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->n_emit = h[CNT_EMIT]; stats->n_child = h[CNT_CHILD]; stats->n_rec = h[CNT_REC]; stats->n_abs = h[CNT_ABS];
    stats->n_capt = h[CNT_CAPT]; stats->n_maxst = h[CNT_MAXST]; stats->n_steps = h[CNT_STEPS];
    stats->n_iters = h[CNT_ITERS]; stats->n_nonconv = h[CNT_NONCONV]; stats->n_roul_surv = h[CNT_ROUL];
    stats->n_rej_cap = h[CNT_REJCAP]; stats->n_events = h[CNT_EVENTS]; stats->n_total = off[n];
    stats->err_flags = (int64_t)h[CNT_ERR];
    stats->n_steps_grid = h[CNT_GSTEPS];
    stats->n_iters_grid = h[CNT_GITERS];
    stats->transport_launches = 1;
    stats->transport_ms = ms;   // with a graph: the whole replay (generation + transport)
    stats->batch_min_blocks = minb;
    stats->batch_ctas = ctas;
    stats->batch_graph = used_graph ? 1 : 0;
  }
  return MC_OK;
}

extern "C" int mc_set_wait_limit(mc_ctx *c, double seconds) {
  if (!c) return set_err(nullptr, MC_ERR_INVALID_ARG, "null context");
  if (!(seconds >= 1e-9 && seconds <= 3600.0)) return set_err(c, MC_ERR_INVALID_ARG, "wait limit must be in [1e-9, 3600] s");
  c->wait_ns = seconds * 1e9;
  return MC_OK;
}
