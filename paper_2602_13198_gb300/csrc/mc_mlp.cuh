// mc_mlp.cuh -- coefficient surrogate network: layout constants and the tcgen05 inference path.
//
// The network (3 -> 64 -> 64 -> 3, SiLU) maps normalised (ln Theta_e, ln(nu/nu_c), ln eps) to
//   o0 = ln(sigma_h / sigma_T)               (thermal Klein-Nishina hot cross-section, section 2.7)
//   o1 = ln K2(1/Theta_e) - ln(2 Theta_e^2)   (the synchrotron normalisation of section 2.2)
//   o2 = ln F(nu/nu_c) / 10                  (angle-integrated emissivity shape)
// replacing the table lookups of the transport step.  Inference runs on the 5th-generation
// tensor cores: 128 rows (one per thread of a CTA) per MMA, BF16 operands in shared memory in the
// canonical K-major layout without swizzle, FP32 accumulators in tensor memory.  Every product is
// split into BF16 high and low parts, a = a_hi + a_lo, and accumulated as
// a_hi b_hi + a_lo b_hi + a_hi b_lo (three BF16 passes), which keeps the products near FP32
// accuracy: plain BF16 (8-bit mantissa) inputs alone would move ln Theta_e by ~2%.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mcgb {

constexpr int kHid = 64;
// packed FP32 weights: W1[64][3] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 64 * 3, kOffW2 = kOffB1 + 64, kOffB2 = kOffW2 + 64 * 64;
constexpr int kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 3 * 64, kNumW = kOffB3 + 3;   // 4611
// input normalisation: x = (u - centre) / half-width
constexpr double kSurLT0 = -6.907755278982137, kSurLT1 = 6.907755278982137;    // ln Theta in [1e-3, 1e3]
constexpr double kSurLK0 = -9.210340371976184, kSurLK1 = 9.210340371976184;    // ln K in [1e-4, 1e4]
constexpr double kSurLE0 = -27.631021115928547, kSurLE1 = 13.815510557964274; // ln eps in [1e-12, 1e6]
constexpr double kSurThetaK2Min = 0.3;   // o1 trained for Theta_e >= 0.3 only
// BF16 operand tiles (bytes): A1 128x16, A2 128x64 (hi and lo); B1 64x16 holding
// [W1_hi | W1_lo | W1_hi] against A1 = [x_hi | x_hi | x_lo]; B2 64x64 and B3 16x64, hi and lo each
constexpr int kTileA1 = 128 * 16 * 2, kTileA2 = 128 * 64 * 2;
constexpr int kTileB1 = 64 * 16 * 2, kTileB2 = 64 * 64 * 2, kTileB3 = 16 * 64 * 2;
constexpr int kPackedBytes = kTileB1 + 2 * kTileB2 + 2 * kTileB3;   // B1, B2hi, B2lo, B3hi, B3lo
constexpr int kTmemCols = 256;   // 64 columns per row group, up to three groups

// Byte offset of element (row, k) of a rows x K bf16 matrix in the canonical K-major layout without
// swizzle: 8x8 core matrices of 128 contiguous bytes, core (row/8, k/8) at ((row/8)*(K/8) + k/8)*128.
__host__ __device__ __forceinline__ int kmajor_off(int row, int k, int K) {
  return (((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

struct SurrogateView {
  const unsigned char *packed;   // kPackedBytes of BF16 tiles
  const float *bias;             // b1[64] b2[64] b3[3] (FP32)
  unsigned int *err;             // timeout flag
  double wait_ns;                // limit on each tensor-core completion wait (ns)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start >> 4 at [0,14), leading byte offset >> 4 at
// [16,30) (between core matrices along K), stride byte offset >> 4 at [32,46) (between 8-row
// groups), descriptor version 1 at [46,48), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D FP32 (bit 4), A and B BF16 (bits 7 and 10), both K-major,
// N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase (the completion of MMAs this CTA issued).  A wait that lasts
// longer than wait_ns (by the global nanosecond timer, read around each poll) sets bit 0 of the error
// flag and returns false, but only once the MMAs in flight have completed (a second wait of at most
// 2^22 polls; bit 1 if that one runs out too), so that the caller may reuse their operand tiles and
// free the tensor memory.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, unsigned int *err, double wait_ns) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    const bool done = mbar_try_wait(mbar, parity);
    if ((double)(globaltimer() - t0) > wait_ns) {
      if (err) atomicOr(err, 1u);
      if (done) return false;
      break;
    }
    if (done) return true;
  }
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(mbar, parity)) return false;
  if (err) atomicOr(err, 2u);
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Named barrier of one 128-thread row group (ids 1 to 3; id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int grp) {
  if (grp == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
  else if (grp == 1) asm volatile("bar.sync 2, 128;" ::: "memory");
  else if (grp == 2) asm volatile("bar.sync 3, 128;" ::: "memory");
  else asm volatile("bar.sync 4, 128;" ::: "memory");
}

// OR of a predicate over the 128 threads of a row group (every thread gets the result).
__device__ __forceinline__ bool group_or(int grp, bool v) {
  uint32_t r;
  if (grp == 0)
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
  else if (grp == 1)
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
  else if (grp == 2)
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 3, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 4, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
  return r != 0;
}

// z sigmoid(z) with the fast reciprocal division (a few ulp; the BF16 split keeps ~16 bits)
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// Per-CTA state of the tensor-core MLP: shared-memory tiles, TMEM base, one mbarrier and phase per
// row group.  A CTA of 128 x G threads evaluates G groups of 128 rows (G = 1 .. 4); group g has its
// own A tiles, accumulates in TMEM columns [64 g, 64 g + 64), and synchronises on its own named
// barrier: the first thread of the group issues its MMAs and commits them to the group's mbarrier.
// The groups run independently, so one group's transport overlaps another's network wait.  The
// tensor-memory kernels run one CTA per SM, so four groups are how an SM gets sixteen warps (at a
// 128-register cap, which measured faster than eight warps at 255).
constexpr int kTcGroupsMax = 4;
struct TcMlp {
  unsigned char *a1[kTcGroupsMax], *a2[kTcGroupsMax], *a2l[kTcGroupsMax];   // per-group A tiles
  unsigned char *b1, *b2, *b2l, *b3, *b3l;                                  // shared weight tiles
  const float *bias;                        // b1 b2 b3 in shared memory
  uint32_t tmem, mbar[kTcGroupsMax], phase[kTcGroupsMax];
  int groups;
  unsigned int *err;
  double wait_ns;
};

// Shared memory needed by one CTA of `groups` row groups (tiles + biases + mbarrier + TMEM slot).
__host__ __device__ constexpr int tc_smem_bytes(int groups) {
  return groups * (kTileA1 + 2 * kTileA2) + kPackedBytes + 4 * (64 + 64 + 16) + 8 * kTcGroupsMax + 64;
}

// Set-up by all threads of the CTA (blockDim.x = 128 or 256): carve shared memory, copy packed
// weights and biases, initialise the groups' mbarriers, warp 0 allocates kTmemCols TMEM columns.
__device__ __forceinline__ void tc_setup(TcMlp &T, unsigned char *smem, const SurrogateView &sv) {
  const int G = (int)(blockDim.x >> 7);
  T.groups = G;
  unsigned char *q = smem;
  for (int g = 0; g < G; ++g) { T.a1[g] = q; q += kTileA1; }
  for (int g = 0; g < G; ++g) { T.a2[g] = q; q += kTileA2; }
  for (int g = 0; g < G; ++g) { T.a2l[g] = q; q += kTileA2; }
  for (int g = G; g < kTcGroupsMax; ++g) T.a1[g] = T.a2[g] = T.a2l[g] = nullptr;
  T.b1 = q;
  T.b2 = T.b1 + kTileB1;
  T.b2l = T.b2 + kTileB2;
  T.b3 = T.b2l + kTileB2;
  T.b3l = T.b3 + kTileB3;
  float *bias = (float *)(T.b3l + kTileB3);
  uint64_t *mb = (uint64_t *)(bias + 64 + 64 + 16);
  uint32_t *tslot = (uint32_t *)(mb + kTcGroupsMax);
  const int tid = threadIdx.x;
  const uint4 *src = (const uint4 *)sv.packed;
  uint4 *dst = (uint4 *)T.b1;
  for (int i = tid; i < kPackedBytes / 16; i += blockDim.x) dst[i] = src[i];
  for (int i = tid; i < 64 + 64 + 16; i += blockDim.x) bias[i] = (i < 128 + 3) ? sv.bias[i] : 0.0f;
  T.bias = bias;
  T.err = sv.err;
  T.wait_ns = sv.wait_ns;
  for (int g = 0; g < kTcGroupsMax; ++g) {
    T.mbar[g] = smem_addr(mb + g);
    T.phase[g] = 0;
  }
  if (tid == 0)
    for (int g = 0; g < G; ++g) mbar_init(T.mbar[g], 1);
  if ((tid >> 5) == 0) tmem_alloc(smem_addr(tslot), kTmemCols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  T.tmem = *tslot;
}

__device__ __forceinline__ void tc_teardown(TcMlp &T) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(T.tmem, kTmemCols);
}

// One layer of row group g: D_g[128 x N] = sum over the np (A, B) pairs of A_g[128 x K] B[N x K]^T in
// TMEM columns [64 g, 64 g + N), issued by the group's first thread; returns after every thread of
// the group has seen the MMAs complete.
__device__ __forceinline__ bool tc_layer(TcMlp &T, int g, const unsigned char *const *as,
                                         const unsigned char *const *bs, int np, int K, int N) {
  fence_async_smem();
  tc_fence_before();
  group_sync(g);
  tc_fence_after();
  if ((threadIdx.x & 127) == 0) {
    const uint32_t sbo = (K / 8) * 128;
    const uint32_t id = idesc_bf16(128, N);
    for (int p = 0; p < np; ++p) {
      const uint32_t ab = smem_addr(as[p]), bb = smem_addr(bs[p]);
      for (int k = 0; k < K / 16; ++k) {
        // advancing 16 elements along K = two core matrices = 256 bytes
        uint64_t da = umma_desc(ab + k * 256, 128, sbo);
        uint64_t db = umma_desc(bb + k * 256, 128, sbo);
        tc_mma(T.tmem + 64u * g, da, db, id, (p > 0 || k > 0) ? 1u : 0u);
      }
    }
    tc_commit(T.mbar[g]);
  }
  bool ok = mbar_wait_bounded(T.mbar[g], T.phase[g], T.err, T.wait_ns);
  T.phase[g] ^= 1u;
  tc_fence_after();
  return ok;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16(v);
  lo = __float2bfloat16(v - __bfloat162float(hi));
}

// Writes 16 activations (columns c0 .. c0+15) of this thread's row as hi/lo BF16 rows of its group's
// A2 / A2lo (two values per conversion: element 2q in the low half of each packed pair, as in
// memory order).
__device__ __forceinline__ void put_hidden16(TcMlp &T, int grp, int row, int c0, const float *h) {
#pragma unroll
  for (int c = 0; c < 16; c += 8) {
    __nv_bfloat162 hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float a = h[c + 2 * q], b = h[c + 2 * q + 1];
      hi[q] = __floats2bfloat162_rn(a, b);
      const float2 back = __bfloat1622float2(hi[q]);
      lo[q] = __floats2bfloat162_rn(a - back.x, b - back.y);
    }
    *(uint4 *)(T.a2[grp] + kmajor_off(row, c0 + c, 64)) = *(uint4 *)hi;
    *(uint4 *)(T.a2l[grp] + kmajor_off(row, c0 + c, 64)) = *(uint4 *)lo;
  }
}

// Hidden layer epilogue in 16-column chunks (16 live activations instead of 64): TMEM accumulators
// + bias, SiLU, BF16 hi/lo split into the next layer's A tiles.
__device__ __forceinline__ void hidden_epilogue(TcMlp &T, int grp, int row, uint32_t tbase, const float *bias) {
#pragma unroll 1
  for (int c0 = 0; c0 < 64; c0 += 16) {
    float h[16];
    tmem_ld16(tbase + c0, h);
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = silu_f(h[c] + bias[c0 + c]);
    put_hidden16(T, grp, row, c0, h);
  }
}

// Evaluates the network for this thread's row (all 128 threads of the thread's row group must call it).
// in[3]: normalised inputs; out[3]: raw outputs.  Returns false if a wait timed out.
__device__ __forceinline__ bool tc_mlp_eval(TcMlp &T, const float in[3], float out[3]) {
  const int grp = threadIdx.x >> 7, row = threadIdx.x & 127;
  // TMEM lanes of this warp (warp w reads lanes 32 (w mod 4) ...) and this group's columns
  const uint32_t tbase = T.tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + 64u * grp;
  // layer 1 operand: [x_hi(3) | x_hi(3) | x_lo(3) | 0 ...] against [W1_hi | W1_lo | W1_hi]
  {
    __nv_bfloat16 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __float2bfloat16(0.0f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      __nv_bfloat16 hi, lo;
      split_bf16(in[q], hi, lo);
      v[q] = hi;
      v[3 + q] = hi;
      v[6 + q] = lo;
    }
    *(uint4 *)(T.a1[grp] + kmajor_off(row, 0, 16)) = *(uint4 *)v;
    *(uint4 *)(T.a1[grp] + kmajor_off(row, 8, 16)) = *(uint4 *)(v + 8);
  }
  const unsigned char *a_l1[1] = {T.a1[grp]};
  const unsigned char *b_l1[1] = {T.b1};
  bool ok = tc_layer(T, grp, a_l1, b_l1, 1, 16, 64);
  hidden_epilogue(T, grp, row, tbase, T.bias);
  const unsigned char *a_l2[3] = {T.a2[grp], T.a2l[grp], T.a2[grp]};
  const unsigned char *b_l2[3] = {T.b2, T.b2, T.b2l};
  ok = tc_layer(T, grp, a_l2, b_l2, 3, 64, 64) && ok;
  hidden_epilogue(T, grp, row, tbase, T.bias + 64);   // the layer-2 MMAs have completed: A2 may be overwritten
  const unsigned char *b_l3[3] = {T.b3, T.b3, T.b3l};
  ok = tc_layer(T, grp, a_l2, b_l3, 3, 64, 16) && ok;
  float y[16];
  tmem_ld16(tbase, y);
  out[0] = y[0] + T.bias[128];
  out[1] = y[1] + T.bias[129];
  out[2] = y[2] + T.bias[130];
  tc_fence_before();
  group_sync(grp);   // the group's TMEM columns and A tiles free for its next evaluation
  tc_fence_after();
  return ok;
}

}  // namespace mcgb
