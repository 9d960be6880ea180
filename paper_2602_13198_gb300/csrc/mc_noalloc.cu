// mc_noalloc.cu -- zone superphoton counts without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the counts: code that
// runs while a CUDA stream is being captured into a graph, code inside a host allocator's own
// callbacks, or applications that hand the GPU to a fixed pool and forbid further cudaMalloc.
// mc_zone_counts_noalloc serves them: it runs the same weight, count and scan kernels as mc_run,
// but every scratch array those kernels need lives in one file-scope __device__ array of fixed
// size (kScratchBytes), which every GPU that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "mc_internal.h"

using namespace mcgb;

namespace {

constexpr int64_t kMaxZones = 131072;   // largest grid accepted: n1*n2*n3 <= 2^17
constexpr int kMaxNu = 512;             // largest weight table accepted
constexpr int64_t kMaxChunks = (kMaxZones + 2047) / 2048;
constexpr int64_t kMaxScanBlocks = (kMaxZones + 1023) / 1024 + 1;
// layout (bytes, each region 256-aligned): 8 per-zone double arrays (volume, emission prefactor,
// ln nu_c, rejection bound, expected count, and the kappa ln w and bremsstrahlung q / nu_T, k T_e / h
// that the zone preparation writes for those models), partial sums, ln w, 1/w, scan block sums, the
// non-finite flag
constexpr int kZoneArrays = 8;
constexpr size_t kZoneBytes = (size_t)kMaxZones * 8;
constexpr size_t kPartialBytes = (size_t)kMaxNu * kMaxChunks * 8;
constexpr size_t kNuBytes = (size_t)kMaxNu * 8;
constexpr size_t kScanBytes = ((size_t)kMaxScanBlocks * 8 + 255) / 256 * 256;
constexpr size_t kScratchBytes = kZoneArrays * kZoneBytes + kPartialBytes + 2 * kNuBytes + kScanBytes + 256;
static_assert(kScratchBytes == 8660480, "scratch size stated in mc.h (8.3 MiB)");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device ordinal, looked up once per device.
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

// A zone state that the preparation flagged non-finite makes the job's total -1 (mc_run fails with
// MC_ERR_NAN_INPUT on the same state), so the caller can tell without a host synchronisation here.
__global__ void k_flag_total(const int *bad, int64_t *total) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *bad) *total = -1;
}

}  // namespace

extern "C" int mc_zone_counts_noalloc(mc_ctx *c, double n_s, uint64_t seed, int64_t *counts, int64_t *start,
                                      int64_t *total, void *stream) {
  if (!c || !counts || !start || !total) {
    if (c) c->err = "null argument";
    return MC_ERR_INVALID_ARG;
  }
  if (!c->have_grid) {
    c->err = "mc_set_grid must be called before mc_zone_counts_noalloc";
    return MC_ERR_STATE;
  }
  if (!(n_s > 0.0)) {
    c->err = "N_s must be positive";
    return MC_ERR_INVALID_ARG;
  }
  if (c->nz > kMaxZones || c->p.n_nu > kMaxNu) {
    c->err = "mc_zone_counts_noalloc supports at most 131072 zones and 512 weight-table nodes";
    return MC_ERR_SIZE;
  }
  int dev = c->p.device;
  if (dev < 0 || dev >= kMaxDevices) {
    c->err = "device ordinal out of range for mc_zone_counts_noalloc";
    return MC_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return MC_ERR_CUDA;
  }
  void *base = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side name g_scratch is not a
    // device address, so the kernels get the address the runtime reports for this device
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        c->err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return MC_ERR_CUDA;
      }
    }
    base = g_addr[dev];
  }
  unsigned char *p = (unsigned char *)base;
  double *zvol = (double *)p;
  double *zpref = (double *)(p + kZoneBytes);
  double *zlnuc = (double *)(p + 2 * kZoneBytes);
  double *zgmax = (double *)(p + 3 * kZoneBytes);
  double *znbar = (double *)(p + 4 * kZoneBytes);
  double *zlnw = (double *)(p + 5 * kZoneBytes);
  double *zbq = (double *)(p + 6 * kZoneBytes);
  double *zbnt = (double *)(p + 7 * kZoneBytes);
  unsigned char *tail = p + kZoneArrays * kZoneBytes;
  double *partial = (double *)tail;
  double *lnw = (double *)(tail + kPartialBytes);
  double *winv = (double *)(tail + kPartialBytes + kNuBytes);
  int64_t *bsum = (int64_t *)(tail + kPartialBytes + 2 * kNuBytes);
  int *bad = (int *)(tail + kPartialBytes + 2 * kNuBytes + kScanBytes);
  cudaStream_t st = (cudaStream_t)stream;
  int nchunks = (int)((c->nz + 2047) / 2048);
  DevModel m = make_model(c);
  m.seed = seed;
  m.zpref = zpref;
  m.zlnuc = zlnuc;
  m.zgmax = zgmax;
  m.lnw = lnw;
  m.winv = winv;
  // the zone preparation writes these per-zone arrays for kappa and bremsstrahlung models: they go
  // to the scratch too, so the context's own arrays (and a run on them) are left alone
  m.zlnw = zlnw;
  m.zbq = zbq;
  m.zbnt = zbnt;
  // the scratch keeps the previous call's contents: every array below is fully rewritten by its
  // kernel; only the non-finite flag must start at zero
  e = cudaMemsetAsync(bad, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    launch_zone_prep(m, zvol, zpref, zlnuc, bad, st);
    launch_weights(m, zvol, zpref, zlnuc, partial, nchunks, n_s, c->p.w_min, lnw, winv, st);
    launch_counts(m, zvol, zpref, zlnuc, zgmax, znbar, counts, st);
    launch_scan(counts, start, bsum, c->nz, total, st);
    k_flag_total<<<1, 32, 0, st>>>(bad, total);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return MC_ERR_CUDA;
  }
  return MC_OK;
}
