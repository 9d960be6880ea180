// mc_batch.cuh -- device side of the batched survey launch (mc_batch.cu): the descriptor of one
// launch, the grid barrier, the phase loop and the cooperative kernel k_batch, templated on the
// precision form.  Each form's instantiations compile in a translation unit of their own
// (mc_batch_fp64.cu, mc_batch_mixed.cu, mc_batch_split.cu), which hand the host code their kernels.
#pragma once
#include "mc_mlp.cuh"
#include "mc_push.cuh"

namespace mcgb {


constexpr int kMaxBatch = 64;
constexpr int kMaxGen = 16;
constexpr int kMaxPhases = 512;
// phase counters: per generation CNT_N, then per phase instance k: grid appends, free appends,
// grid cursor, free cursor
constexpr int kPhBase = kMaxGen * CNT_N;
constexpr int kPhWords = kPhBase + 4 * kMaxPhases;

struct BatchIO {
  const DevModel *models;
  int n_models;
  const int64_t *prim_off;   // [n_models + 1]
  Pool pool;
  ChildBuf q[2];
  int32_t *list_grid, *list_free;
  int64_t cap;
  unsigned long long *cnt;   // CNT_N totals
  unsigned long long *ph;    // kPhWords
  unsigned int *bar;         // grid barrier: arrivals, generation
  SurrogateView sv;
  double timeout_ns;
};

// Grid-wide barrier (all CTAs are co-resident under the cooperative launch).  A CTA waits at most
// timeout_ns; on timeout it raises bit 2 of the error word and every CTA leaves the kernel at its
// next barrier.  Returns false when the kernel must stop.
static __device__ bool grid_sync(const BatchIO &b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *vb = b.bar;
    volatile unsigned long long *verr = b.cnt + CNT_ERR;
    unsigned int gen = vb[1];
    __threadfence();
    unsigned int arrived = atomicAdd(b.bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(b.bar, 0u);
      __threadfence();
      atomicAdd(b.bar + 1, 1u);
    } else {
      unsigned long long t0 = globaltimer();
      while (vb[1] == gen) {
        if ((double)(globaltimer() - t0) > b.timeout_ns || (*verr & 4ull)) {
          ok = 0;
          atomicOr(b.cnt + CNT_ERR, 4ull);
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
    s_ok = ok && !(*verr & 4ull);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
  return *(volatile const unsigned long long *)p;
}

// Persistent loop of one phase over list_in[0, n_in); superphotons that change phase are appended
// to list_out through out_cnt.  With the surrogate, the in-grid phase runs in lockstep per 128-thread
// row group (the network's tile), each group on its own named barrier.
template <int PREC, int PHASE, bool SUR>
__device__ void batch_phase(const DevModel *sm, const BatchIO &b, const PushIO &io, const int32_t *list_in,
                            int64_t n_in, unsigned long long *cursor, int32_t *list_out, unsigned long long *out_cnt,
                            TcMlp &T, LocalStats &ls) {
  const int lane = threadIdx.x & 31;
  PhF<PREC> p;   // the precision form's geodesic and weight scalars
  p.raddr = nullptr;
  int64_t slot = -1;
  bool live = false, exhausted = (n_in == 0);
  SurCarry<typename Form<PREC>::S> sc;
  while (true) {
    if (!exhausted) {
      unsigned idle = __ballot_sync(0xffffffffu, !live);
      if (idle) {
        int cnt = __popc(idle);
        int leader = __ffs(idle) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(cursor, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, leader);
        if (base + cnt >= (unsigned long long)n_in) exhausted = true;
        if (!live) {
          unsigned long long k = base + __popc(idle & ((1u << lane) - 1u));
          if (k < (unsigned long long)n_in) {
            slot = list_in[k];
            load_ph(b.pool, slot, p);
            set_wthr(sm[p.model], p);
            live = true;
          }
        }
      }
    }
    if (SUR && PHASE == 0) {
      // the row group (128 threads) moves in lockstep; the groups of a CTA do not
      const int grp = threadIdx.x >> 7;
      if (!group_or(grp, live)) {
        if (!group_or(grp, !exhausted)) break;
        continue;
      }
      float in[3] = {0.0f, 0.0f, 0.0f}, out[3];
      if (live) {
        step_sur_a(sm[p.model], p, sc, ls);
        in[0] = sc.a.in[0];
        in[1] = sc.a.in[1];
        in[2] = sc.a.in[2];
      }
      tc_mlp_eval(T, in, out);
      if (live) {
        live = step_sur_b<PREC>(sm[p.model], io, p, sc, out, ls);
        if (live && !in_grid(sm[p.model], p.X)) {
          save_ph(b.pool, slot, p);
          list_out[atomicAdd(out_cnt, 1ull)] = (int32_t)slot;
          live = false;
        }
      }
      flush_record(p);
    } else {
      if (!__any_sync(0xffffffffu, live)) break;
      if (live) {
        const DevModel &m = sm[p.model];
        bool handoff;
        if (PHASE == 0) {
          live = step<PREC>(m, io, p, ls);
          handoff = live && !in_grid(m, p.X);
        } else {
          int r = step_free<PREC>(m, io, p, ls);
          live = (r != 1);
          handoff = (r == 2);
        }
        if (handoff) {
          save_ph(b.pool, slot, p);
          list_out[atomicAdd(out_cnt, 1ull)] = (int32_t)slot;
          live = false;
        }
      }
      flush_record(p);
    }
  }
}

// Dynamic shared memory of a batch CTA: the model descriptors, then (surrogate) the network's tiles.
// Variants of 6 or more resident CTAs per SM (the double-float form, latency-bound, gains from resident
// warps) read the descriptors from global memory through L1 instead: ~48 KB per CTA of shared memory
// would cap residency at 4.
constexpr int kModelsSmem = (int)((sizeof(DevModel) * kMaxBatch + 127) / 128 * 128);
__host__ __device__ constexpr bool global_desc(bool sur, int minb) { return !sur && minb >= 6; }
inline int batch_smem_bytes(bool sur, int minb) {
  return (global_desc(sur, minb) ? 0 : kModelsSmem) + (sur ? tc_smem_bytes(kTcGroupsMax) : 0);
}

template <int PREC, bool SUR, int MINB>
__global__ void __launch_bounds__(SUR ? 128 * kTcGroupsMax : 128, MINB) k_batch(BatchIO b) {
  __shared__ int64_t soff[kMaxBatch + 1];
  extern __shared__ __align__(128) unsigned char dyn[];
  const DevModel *sm;
  if constexpr (global_desc(SUR, MINB)) {
    sm = b.models;
  } else {
    DevModel *ds = reinterpret_cast<DevModel *>(dyn);
    const unsigned long long *src = (const unsigned long long *)b.models;
    unsigned long long *dst = (unsigned long long *)ds;
    const int words = (int)(b.n_models * sizeof(DevModel) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    sm = ds;
  }
  for (int i = threadIdx.x; i <= b.n_models; i += blockDim.x) soff[i] = b.prim_off[i];
  __syncthreads();
  TcMlp T;
  if (SUR) tc_setup(T, dyn + (global_desc(SUR, MINB) ? 0 : kModelsSmem), b.sv);
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long *agrid = b.ph + kPhBase, *afree = agrid + kMaxPhases, *cgrid = afree + kMaxPhases,
                     *cfree = cgrid + kMaxPhases;
  int k = 0;
  bool go = true;
  for (int g = 0; g < kMaxGen && go; ++g) {
    unsigned long long *gcnt = b.ph + (int64_t)g * CNT_N;
    const int64_t n_items = (g == 0) ? soff[b.n_models] : (int64_t)vload(b.ph + (int64_t)(g - 1) * CNT_N + CNT_OUT);
    if (n_items == 0) break;
    if (n_items > b.cap) {
      if (threadIdx.x == 0) atomicOr(b.cnt + CNT_ERR, 1ull);
      break;
    }
    const ChildBuf qin = b.q[(g + 1) & 1], qout = b.q[g & 1];
    PushIO io;
    memset(&io, 0, sizeof(io));
    io.pool = b.pool;
    io.out = qout;
    io.out_cap = b.cap;
    io.cnt = gcnt;
    // ---- init: emission or child load, one item per thread (warp-uniform trip count)
    {
      const int64_t stride = (int64_t)gridDim.x * blockDim.x;
      const int64_t n_round = (n_items + stride - 1) / stride * stride;
      for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_round; idx += stride) {
        const bool have = idx < n_items;
        bool gp = false;
        Ph p;
        if (g == 0) {   // emission: every lane of the warp takes part in the frequency rejection
          int lo = 0, hi = b.n_models - 1;
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (soff[mid] <= idx) lo = mid;
            else hi = mid - 1;
          }
          p.model = lo;
          emit_warp<true>(sm[0], sm, have, lo, have ? idx - soff[lo] : 0, p, ls);
          if (have) ls.emit++;
        }
        if (have) {
          if (g != 0) {
            p.model = qin.model[idx];
            load_child<Form<PREC>::K32>(sm[p.model], qin, idx, p, ls);
          }
          init_transport<Form<PREC>::C32>(sm[p.model], p);
          save_ph(b.pool, idx, p);
          gp = in_grid(sm[p.model], p.X);
        }
        const int lane = threadIdx.x & 31;
        unsigned mg = __ballot_sync(0xffffffffu, have && gp), mf = __ballot_sync(0xffffffffu, have && !gp);
        unsigned long long bg = 0, bf = 0;
        if (lane == 0) {
          if (mg) bg = atomicAdd(agrid + k, (unsigned long long)__popc(mg));
          if (mf) bf = atomicAdd(afree + k, (unsigned long long)__popc(mf));
        }
        bg = __shfl_sync(0xffffffffu, bg, 0);
        bf = __shfl_sync(0xffffffffu, bf, 0);
        unsigned below = (1u << lane) - 1u;
        if (have && gp) b.list_grid[bg + __popc(mg & below)] = (int32_t)idx;
        if (have && !gp) b.list_free[bf + __popc(mf & below)] = (int32_t)idx;
      }
    }
    if (!grid_sync(b)) { go = false; break; }
    // ---- alternate in-grid and free-streaming phases until the generation is done
    while (true) {
      int64_t ng = (int64_t)vload(agrid + k);
      batch_phase<PREC, 0, SUR>(sm, b, io, b.list_grid, ng, cgrid + k, b.list_free, afree + k, T, ls);
      if (!grid_sync(b)) { go = false; break; }
      int64_t nf = (int64_t)vload(afree + k);
      batch_phase<PREC, 1, SUR>(sm, b, io, b.list_free, nf, cfree + k, b.list_grid, agrid + k + 1, T, ls);
      if (!grid_sync(b)) { go = false; break; }
      ++k;
      if (k >= kMaxPhases - 1) {
        if (threadIdx.x == 0) atomicOr(b.cnt + CNT_ERR, 8ull);
        go = false;
        break;
      }
      if (vload(agrid + k) == 0) break;
    }
    if (go && vload(gcnt + CNT_ERR) & 1ull) {
      if (threadIdx.x == 0) atomicOr(b.cnt + CNT_ERR, 1ull);
      go = false;
    }
  }
  if (SUR) tc_teardown(T);
  flush_stats(ls, b.cnt);
}

typedef void (*BatchKernel)(BatchIO);

// Kernel of one launch configuration of each precision form (minimum resident CTAs per SM = minb).
BatchKernel batch_kernel_fp64(bool sur, int minb);
BatchKernel batch_kernel_mixed(bool sur, int minb);
BatchKernel batch_kernel_split(bool sur, int minb);

}  // namespace mcgb
