// mc_transport.cu -- superphoton transport kernels (sections 2.3-2.7, 3).
//
// A batch of superphotons (the primaries of a uid range, or the scattered children of the
// previous generation) goes through three kernels:
//   * k_init: emission (zone by binary search in the count scan, frequency and direction by
//     rejection, wavevector in the plasma tetrad) or loading of a child, then the transport
//     initialisation; every lane does the same work, and the state goes to a pool in HBM;
//   * k_push_fp64 / k_push_mixed <phase 0>: superphotons inside the radial extent of the grid:
//     iterated velocity Verlet (FP64, or double-float in the mixed form; metric derivatives
//     evaluated once per step at x_{n+1}, reused by every predictor pass), fluid interpolation and
//     invariant coefficients (FP64, or FP32 in the mixed form),
//     trapezoid optical depths, biased scattering with the event located within the step, Compton
//     kinematics of the child, termination tests; a superphoton that leaves the grid is handed on;
//   * k_push_fp64 / k_push_mixed <phase 1>: superphotons outside the grid, where both trapezoid end points have no plasma
//     and a step reduces to the geodesic and the termination tests (recording at r >= r_record);
//     one that re-enters the grid is handed back.
// Grouping superphotons by phase keeps the lanes of a warp on the same code path; the push kernels
// are persistent and refill a lane from the phase's list as soon as its superphoton leaves.
#include "mc_push.cuh"

namespace mcgb {
// Emission or child loading + transport initialisation, one item per thread (grid-stride; the trip
// count is warp-uniform, so a warp's lanes reach the cooperative frequency rejection together).
template <int PREC, bool KERR>
__global__ void __launch_bounds__(128) k_init(DevModel m, InitIO io) {
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = (io.n_items + stride - 1) / stride * stride;   // warp-uniform trip count
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_round; idx += stride) {
    const bool have = idx < io.n_items;
    bool grid_phase = false;
    Ph p;
    if (io.mode != 2) {   // emission: every lane of the warp takes part in the frequency rejection
      const int64_t uid = !have ? 0 : (io.mode == 1) ? io.uids[idx] : io.uid0 + idx;
      emit_warp(m, nullptr, have, 0, uid, p, ls);
      if (have) ls.emit++;
    }
    if (have) {
      if (io.mode == 2) load_child<Form<PREC>::K32>(m, io.in, idx, p, ls);
      p.model = 0;
      init_transport<Form<PREC>::C32, KERR>(m, p);
      save_ph(io.pool, idx, p);
      grid_phase = in_grid(m, p.X);
    }
    // warp-aggregated appends to the two phase lists
    const int lane = threadIdx.x & 31;
    unsigned mg = __ballot_sync(0xffffffffu, have && grid_phase);
    unsigned mf = __ballot_sync(0xffffffffu, have && !grid_phase);
    unsigned long long bg = 0, bf = 0;
    if (lane == 0) {
      if (mg) bg = atomicAdd(io.cnt + CNT_L0, (unsigned long long)__popc(mg));
      if (mf) bf = atomicAdd(io.cnt + CNT_L1, (unsigned long long)__popc(mf));
    }
    bg = __shfl_sync(0xffffffffu, bg, 0);
    bf = __shfl_sync(0xffffffffu, bf, 0);
    unsigned below = (1u << lane) - 1u;
    if (have && grid_phase) io.list_grid[bg + __popc(mg & below)] = (int32_t)idx;
    if (have && !grid_phase) io.list_free[bf + __popc(mf & below)] = (int32_t)idx;
  }
  flush_stats(ls, io.cnt);
}

// Persistent transport of one phase over io.list_in; PHASE 0 keeps superphotons while they are in
// the grid, PHASE 1 while they are outside it.  A lane whose superphoton ends or changes phase is
// refilled from the list (one atomic per warp).
template <int PREC, int PHASE, bool KERR>
__device__ __forceinline__ void push_body(const DevModel &m, const PushIO &io) {
  const int lane = threadIdx.x & 31;
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  PhF<PREC> p;   // the precision form's geodesic and weight scalars
  p.raddr = nullptr;
  int64_t slot = -1;
  bool live = false;
  bool exhausted = false;
  while (true) {
    if (!exhausted) {
      unsigned idle = __ballot_sync(0xffffffffu, !live);
      if (idle) {
        int cnt = __popc(idle);
        int leader = __ffs(idle) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(io.cnt + CNT_NEXT, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, leader);
        if (base + cnt >= (unsigned long long)io.n_in) exhausted = true;
        if (!live) {
          unsigned long long k = base + __popc(idle & ((1u << lane) - 1u));
          if (k < (unsigned long long)io.n_in) {
            slot = io.list_in[k];
            load_ph(io.pool, slot, p, m);
            live = true;
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, live)) break;
    if (live) {
      bool handoff;
      if (PHASE == 0) {
        live = step<PREC, KERR>(m, io, p, ls);
        handoff = live && !in_grid(m, p.X);
      } else {
        int r = step_free<PREC, KERR>(m, io, p, ls);
        live = (r != 1);
        handoff = (r == 2);
      }
      if (handoff) {
        save_ph(io.pool, slot, p);
        unsigned long long o = atomicAdd(io.cnt + io.out_counter, 1ull);
        io.list_out[o] = (int32_t)slot;
        live = false;
      }
    }
    flush_record(p);
  }
  flush_stats(ls, io.cnt);
}

// Minimum resident CTAs of 128 threads per SM that each form's register cap allows (65536 / (128 x
// CTAs) registers per thread).  FP64 form: the FP64 pipe is the bound.  Mixed form (double-float
// geodesic on the FP32 pipes): latency-bound, it gains from resident warps even with spills at the
// cap; measured on the 3-D snapshot, the 2-D torus and the sphere, 8 CTAs (64 registers) beat 2 to 6
// and 10 to 16.
#ifndef MC_FP64_MINB
#define MC_FP64_MINB 1
#endif
#ifndef MC_MIXED_MINB
#define MC_MIXED_MINB 8
#endif
#ifndef MC_SPLIT_MINB
#define MC_SPLIT_MINB 1
#endif
template <int PHASE, bool KERR>
__global__ void __launch_bounds__(128, MC_FP64_MINB) k_push_fp64(DevModel m, PushIO io) {
  push_body<0, PHASE, KERR>(m, io);
}

template <int PHASE, bool KERR>
__global__ void __launch_bounds__(128, MC_MIXED_MINB) k_push_mixed(DevModel m, PushIO io) {
  push_body<1, PHASE, KERR>(m, io);
}

// Split form (FP64 geodesic, FP32 coefficients and weights).
template <int PHASE, bool KERR>
__global__ void __launch_bounds__(128, MC_SPLIT_MINB) k_push_split(DevModel m, PushIO io) {
  push_body<2, PHASE, KERR>(m, io);
}

// Persistent in-grid push with the network.  Each 128-thread row group reaches its tensor-core
// evaluation once per iteration (idle lanes contribute a zero row) and leaves the loop as a whole;
// the CTA's groups iterate independently and meet again only at the teardown.
template <int PREC>
__global__ void __launch_bounds__(128 * kTcGroupsMax) k_push_sur(DevModel m, PushIO io, SurrogateView sv) {
  extern __shared__ __align__(128) unsigned char smem_sur[];
  TcMlp T;
  tc_setup(T, smem_sur, sv);
  const int lane = threadIdx.x & 31;
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  PhF<PREC> p;
  p.raddr = nullptr;
  int64_t slot = -1;
  bool live = false;
  bool exhausted = false;
  SurCarry<typename Form<PREC>::S> sc;
  while (true) {
    if (!exhausted) {
      unsigned idle = __ballot_sync(0xffffffffu, !live);
      if (idle) {
        int cnt = __popc(idle);
        int leader = __ffs(idle) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(io.cnt + CNT_NEXT, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, leader);
        if (base + cnt >= (unsigned long long)io.n_in) exhausted = true;
        if (!live) {
          unsigned long long k = base + __popc(idle & ((1u << lane) - 1u));
          if (k < (unsigned long long)io.n_in) {
            slot = io.list_in[k];
            load_ph(io.pool, slot, p, m);
            live = true;
          }
        }
      }
    }
    const int grp = threadIdx.x >> 7;   // each 128-thread row group moves in lockstep on its own
    if (!group_or(grp, live)) {
      if (!group_or(grp, !exhausted)) break;
      continue;
    }
    float in[3] = {0.0f, 0.0f, 0.0f}, out[3];
    if (live) {
      step_sur_a(m, p, sc, ls);
      in[0] = sc.a.in[0];
      in[1] = sc.a.in[1];
      in[2] = sc.a.in[2];
    }
    tc_mlp_eval(T, in, out);
    if (live) {
      live = step_sur_b<PREC>(m, io, p, sc, out, ls);
      if (live && !in_grid(m, p.X)) {
        save_ph(io.pool, slot, p);
        unsigned long long o = atomicAdd(io.cnt + io.out_counter, 1ull);
        io.list_out[o] = (int32_t)slot;
        live = false;
      }
    }
    flush_record(p);
  }
  tc_teardown(T);
  flush_stats(ls, io.cnt);
}

static const void *sur_kernel(int prec) {
  return prec == 2 ? (const void *)k_push_sur<2> : (const void *)k_push_sur<1>;
}

int push_sur_max_blocks_per_sm(int prec, int block, int smem) {
  int n = 0;
  const void *k = sur_kernel(prec);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem);
  return n;
}

void launch_push_sur(const DevModel &m, const PushIO &io, const SurrogateView &sv, int prec, int grid, int smem,
                     cudaStream_t st) {
  if (prec == 2) k_push_sur<2><<<grid, 128 * kTcGroupsMax, smem, st>>>(m, io, sv);
  else k_push_sur<1><<<grid, 128 * kTcGroupsMax, smem, st>>>(m, io, sv);
}

// Kernel of one launch configuration: precision form, phase and spin (general Kerr, or a = 0).
template <int PHASE>
static const void *push_kernel(int prec, bool kerr) {
  if (prec == 1) return kerr ? (const void *)k_push_mixed<PHASE, true> : (const void *)k_push_mixed<PHASE, false>;
  if (prec == 2) return kerr ? (const void *)k_push_split<PHASE, true> : (const void *)k_push_split<PHASE, false>;
  return kerr ? (const void *)k_push_fp64<PHASE, true> : (const void *)k_push_fp64<PHASE, false>;
}

int push_max_blocks_per_sm(int prec, int phase, int block, int kerr) {
  int n = 0;
  const void *k = phase == 0 ? push_kernel<0>(prec, kerr != 0) : push_kernel<1>(prec, kerr != 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0);
  return n;
}

template <int PREC>
static void launch_init_t(const DevModel &m, const InitIO &io, int grid, int block, cudaStream_t st) {
  if (m.a != 0.0) k_init<PREC, true><<<grid, block, 0, st>>>(m, io);
  else k_init<PREC, false><<<grid, block, 0, st>>>(m, io);
}

void launch_init(const DevModel &m, const InitIO &io, int prec, int grid, int block, cudaStream_t st) {
  if (prec == 1) launch_init_t<1>(m, io, grid, block, st);
  else if (prec == 2) launch_init_t<2>(m, io, grid, block, st);
  else launch_init_t<0>(m, io, grid, block, st);
}

// a = 0 takes the Schwarzschild form of the metric and of the geodesic acceleration.
void launch_push(const DevModel &m, const PushIO &io, int prec, int phase, int grid, int block, cudaStream_t st) {
  const bool kerr = m.a != 0.0;
  void *args[] = {(void *)&m, (void *)&io};
  const void *k = phase == 0 ? push_kernel<0>(prec, kerr) : push_kernel<1>(prec, kerr);
  cudaLaunchKernel(k, dim3(grid), dim3(block), args, 0, st);
}

}  // namespace mcgb
