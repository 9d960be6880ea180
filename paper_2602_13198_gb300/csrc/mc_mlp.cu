// mc_mlp.cu -- training and standalone inference of the coefficient surrogate network.
//
// Training data come from the library's own FP64 quadratures (the same definitions as its
// lookup tables): sigma_h by the Maxwell-Juettner x Klein-Nishina quadrature, K2 by the trapezoid
// rule on its integral representation, F(K) by 64-node Gauss-Legendre.  Training runs on the GPU
// with this file's FP32 forward/backward kernel (one sample per thread, per-block gradient
// reduction in shared memory) and an Adam update kernel.  The trained weights are packed into
// BF16 tiles for the tensor-core inference in mc_mlp.cuh.
#include <cmath>
#include <cstring>
#include <vector>

#include "mc_internal.h"
#include "mc_mlp.cuh"

using namespace mcgb;

namespace mcgb {

__device__ __forceinline__ float silu32(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu32(float z) {
  float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Training samples: inputs uniform in (ln Theta, ln K, ln eps) over the surrogate's domain, drawn
// from stream 0xD000000000000000 | (tag << 40) | i; targets o0, o1, o2 and their masks.
__global__ void k_sur_data(int64_t n, uint64_t seed, uint64_t tag, const double *glF, const double *glS,
                           const double *glM, float *X, float *T, float *Mk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Rng r;
  rng_init(r, 0xD000000000000000ull | (tag << 40) | (uint64_t)i, 0u);
  double lt = kSurLT0 + (kSurLT1 - kSurLT0) * rng_u(r, seed);
  double lk = kSurLK0 + (kSurLK1 - kSurLK0) * rng_u(r, seed);
  double le = kSurLE0 + (kSurLE1 - kSurLE0) * rng_u(r, seed);
  double th = exp(lt), K = exp(lk), e = exp(le);
  // o0: hot cross-section quadrature (gamma = 1 + Theta s^2, s in [0, 8]; mu in [-1, 1])
  double num = 0.0, den = 0.0;
  for (int a = 0; a < 64; ++a) {
    double s = glS[a];
    double gam = 1.0 + th * s * s;
    double hs = gam * s * s * sqrt(th * (2.0 + th * s * s)) * exp(-s * s);
    double beta = sqrt(1.0 - 1.0 / (gam * gam));
    double q = 0.0;
    for (int b = 0; b < 32; ++b) {
      double om = 1.0 - glM[b] * beta;
      q += glM[32 + b] * om * sigma_kn_ratio(e * gam * om);
    }
    num += glS[64 + a] * hs * 0.5 * q;
    den += glS[64 + a] * hs;
  }
  double o0 = log(num / den);
  // o1: K2(1/Theta) by the trapezoid rule on int_0^inf exp(-x cosh t) cosh 2t dt
  double o1 = 0.0, m1 = 0.0;
  if (th >= kSurThetaK2Min) {
    double x = 1.0 / th, h = 1.0 / 64.0, k2 = 0.5 * exp(-x);
    for (int q = 1; q < 4096; ++q) {
      double t = q * h, ch = cosh(t);
      if (x * ch > 800.0) break;
      k2 += exp(-x * ch) * cosh(2.0 * t);
    }
    o1 = log(k2 * h) - log(2.0 * th * th);
    m1 = 1.0;
  }
  // o2: ln F(K), F = int_0^{pi/2} sin^2 G(K / sin) (64-node Gauss-Legendre)
  double F = 0.0;
  for (int q = 0; q < 64; ++q) {
    double st = sin(glF[q]);
    F += glF[64 + q] * st * st * Gsyn(K / st);
  }
  double o2 = log(F);
  X[3 * i + 0] = (float)((lt - 0.5 * (kSurLT0 + kSurLT1)) / (0.5 * (kSurLT1 - kSurLT0)));
  X[3 * i + 1] = (float)((lk - 0.5 * (kSurLK0 + kSurLK1)) / (0.5 * (kSurLK1 - kSurLK0)));
  X[3 * i + 2] = (float)((le - 0.5 * (kSurLE0 + kSurLE1)) / (0.5 * (kSurLE1 - kSurLE0)));
  T[3 * i + 0] = (float)o0;
  T[3 * i + 1] = (float)o1;
  T[3 * i + 2] = (float)(o2 / 10.0);
  Mk[3 * i + 0] = 1.0f;
  Mk[3 * i + 1] = (float)m1;
  Mk[3 * i + 2] = 1.0f;
}

constexpr int kGB = 64;          // samples per block in the gradient kernel
constexpr int kLd = 65;          // padded row length of the activation tiles
constexpr int kWPad = 4616;      // kNumW rounded up to a multiple of 4

// Masked mean-squared-error gradient over samples [first, first + n) (FP32).  One sample per
// thread; the block's contributions to every weight gradient are reduced in shared memory and
// added to G with one atomic per weight.  loss_acc (if not NULL) accumulates sum m (y - t)^2.
__global__ void __launch_bounds__(kGB) k_sur_grad(const float *W, const float *X, const float *T, const float *Mk,
                                                  int64_t first, int64_t n, float inv_norm, float *G, double *loss_acc) {
  extern __shared__ float sh[];
  float *w = sh;
  float *h1 = w + kWPad, *s1 = h1 + kGB * kLd, *h2 = s1 + kGB * kLd, *dz2 = h2 + kGB * kLd, *dz1 = dz2 + kGB * kLd;
  float *xs = dz1 + kGB * kLd, *dys = xs + kGB * 4;
  const int t = threadIdx.x;
  for (int i = t; i < kNumW; i += kGB) w[i] = W[i];
  const int64_t sidx = (int64_t)blockIdx.x * kGB + t;
  const bool valid = sidx < n;
  const int64_t gi = first + sidx;
  float x[3] = {0.f, 0.f, 0.f}, tg[3] = {0.f, 0.f, 0.f}, mk[3] = {0.f, 0.f, 0.f};
  if (valid) {
    for (int c = 0; c < 3; ++c) {
      x[c] = X[3 * gi + c];
      tg[c] = T[3 * gi + c];
      mk[c] = Mk[3 * gi + c];
    }
  }
  __syncthreads();
  const float *W1 = w + kOffW1, *B1 = w + kOffB1, *W2 = w + kOffW2, *B2 = w + kOffB2, *W3 = w + kOffW3, *B3 = w + kOffB3;
  for (int j = 0; j < 64; ++j) {
    float z = B1[j] + W1[3 * j] * x[0] + W1[3 * j + 1] * x[1] + W1[3 * j + 2] * x[2];
    h1[t * kLd + j] = silu32(z);
    s1[t * kLd + j] = dsilu32(z);
  }
  float y[3] = {B3[0], B3[1], B3[2]};
  for (int i = 0; i < 64; ++i) {
    float z = B2[i];
    for (int j = 0; j < 64; ++j) z += W2[64 * i + j] * h1[t * kLd + j];
    float hv = silu32(z);
    h2[t * kLd + i] = hv;
    dz2[t * kLd + i] = dsilu32(z);   // holds silu'(z2) until overwritten below
    y[0] += W3[i] * hv;
    y[1] += W3[64 + i] * hv;
    y[2] += W3[128 + i] * hv;
  }
  float dy[3];
  double lsum = 0.0;
  for (int k = 0; k < 3; ++k) {
    float d = y[k] - tg[k];
    dy[k] = valid ? 2.0f * mk[k] * d * inv_norm : 0.0f;
    if (valid) lsum += (double)mk[k] * d * d;
  }
  for (int c = 0; c < 3; ++c) {
    xs[t * 4 + c] = x[c];
    dys[t * 4 + c] = dy[c];
  }
  for (int j = 0; j < 64; ++j) {
    float dh2 = W3[j] * dy[0] + W3[64 + j] * dy[1] + W3[128 + j] * dy[2];
    dz2[t * kLd + j] = dh2 * dz2[t * kLd + j];
  }
  for (int j = 0; j < 64; ++j) {
    float dh1 = 0.0f;
    for (int i = 0; i < 64; ++i) dh1 += W2[64 * i + j] * dz2[t * kLd + i];
    dz1[t * kLd + j] = dh1 * s1[t * kLd + j];
  }
  __syncthreads();
  // thread t owns column j = t of W2 (and row j of W1, b1, b2, column j of W3)
  const int j = t;
  float acc[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) acc[i] = 0.0f;
  float g1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f, g3[3] = {0.f, 0.f, 0.f};
  for (int s = 0; s < kGB; ++s) {
    float hj = h1[s * kLd + j];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] += dz2[s * kLd + i] * hj;
    float d1 = dz1[s * kLd + j];
    g1[0] += d1 * xs[s * 4];
    g1[1] += d1 * xs[s * 4 + 1];
    g1[2] += d1 * xs[s * 4 + 2];
    gb1 += d1;
    gb2 += dz2[s * kLd + j];
    float h2j = h2[s * kLd + j];
    g3[0] += dys[s * 4] * h2j;
    g3[1] += dys[s * 4 + 1] * h2j;
    g3[2] += dys[s * 4 + 2] * h2j;
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) atomicAdd(G + kOffW2 + 64 * i + j, acc[i]);
  for (int c = 0; c < 3; ++c) atomicAdd(G + kOffW1 + 3 * j + c, g1[c]);
  atomicAdd(G + kOffB1 + j, gb1);
  atomicAdd(G + kOffB2 + j, gb2);
  for (int k = 0; k < 3; ++k) atomicAdd(G + kOffW3 + 64 * k + j, g3[k]);
  if (t < 3) {
    float gb = 0.f;
    for (int s = 0; s < kGB; ++s) gb += dys[s * 4 + t];
    atomicAdd(G + kOffB3 + t, gb);
  }
  if (loss_acc) {
    // block sum of the loss through warp shuffles
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) atomicAdd(loss_acc, lsum);
  }
}

__global__ void k_adam(float *W, float *G, float *Mo, float *Vo, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = G[i];
  float m = b1 * Mo[i] + (1.0f - b1) * g;
  float v = b2 * Vo[i] + (1.0f - b2) * g * g;
  Mo[i] = m;
  Vo[i] = v;
  W[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  G[i] = 0.0f;
}

// Standalone tensor-core inference: rows of X (n x 3) -> Y (n x 3), 128 rows per CTA.
__global__ void __launch_bounds__(128) k_sur_infer_tc(SurrogateView sv, const float *X, float *Y, int64_t n) {
  extern __shared__ __align__(128) unsigned char smem_tc[];
  TcMlp T;
  tc_setup(T, smem_tc, sv);
  int64_t row = (int64_t)blockIdx.x * 128 + threadIdx.x;
  float in[3] = {0.f, 0.f, 0.f}, out[3];
  if (row < n) {
    in[0] = X[3 * row];
    in[1] = X[3 * row + 1];
    in[2] = X[3 * row + 2];
  }
  tc_mlp_eval(T, in, out);
  if (row < n) {
    Y[3 * row] = out[0];
    Y[3 * row + 1] = out[1];
    Y[3 * row + 2] = out[2];
  }
  tc_teardown(T);
}

// FP32 reference inference on CUDA cores (one row per thread).
__global__ void k_sur_infer_fp32(const float *W, const float *X, float *Y, int64_t n) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  float x[3] = {X[3 * row], X[3 * row + 1], X[3 * row + 2]};
  float h1[64];
  for (int j = 0; j < 64; ++j)
    h1[j] = silu32(W[kOffB1 + j] + W[kOffW1 + 3 * j] * x[0] + W[kOffW1 + 3 * j + 1] * x[1] + W[kOffW1 + 3 * j + 2] * x[2]);
  float y[3] = {W[kOffB3], W[kOffB3 + 1], W[kOffB3 + 2]};
  for (int i = 0; i < 64; ++i) {
    float z = W[kOffB2 + i];
    for (int j = 0; j < 64; ++j) z += W[kOffW2 + 64 * i + j] * h1[j];
    float hv = silu32(z);
    for (int k = 0; k < 3; ++k) y[k] += W[kOffW3 + 64 * k + i] * hv;
  }
  for (int k = 0; k < 3; ++k) Y[3 * row + k] = y[k];
}

}  // namespace mcgb

// ------------------------------------------------------------------ host side
static void pack_bf16(const float *W, std::vector<unsigned char> &out, std::vector<float> &bias) {
  out.assign(kPackedBytes, 0);
  auto put = [&](unsigned char *tile, int row, int k, int K, __nv_bfloat16 b) {
    std::memcpy(tile + kmajor_off(row, k, K), &b, 2);
  };
  auto hi = [](float v) { return __float2bfloat16(v); };
  auto lo = [](float v) { return __float2bfloat16(v - __bfloat162float(__float2bfloat16(v))); };
  unsigned char *B1 = out.data(), *B2 = B1 + kTileB1, *B2l = B2 + kTileB2, *B3 = B2l + kTileB2, *B3l = B3 + kTileB3;
  const __nv_bfloat16 z = __float2bfloat16(0.0f);
  for (int n = 0; n < 64; ++n)
    for (int k = 0; k < 16; ++k) {
      // [W1_hi | W1_lo | W1_hi | 0]
      __nv_bfloat16 v = z;
      if (k < 3) v = hi(W[kOffW1 + 3 * n + k]);
      else if (k < 6) v = lo(W[kOffW1 + 3 * n + k - 3]);
      else if (k < 9) v = hi(W[kOffW1 + 3 * n + k - 6]);
      put(B1, n, k, 16, v);
    }
  for (int n = 0; n < 64; ++n)
    for (int k = 0; k < 64; ++k) {
      put(B2, n, k, 64, hi(W[kOffW2 + 64 * n + k]));
      put(B2l, n, k, 64, lo(W[kOffW2 + 64 * n + k]));
    }
  for (int n = 0; n < 16; ++n)
    for (int k = 0; k < 64; ++k) {
      put(B3, n, k, 64, n < 3 ? hi(W[kOffW3 + 64 * n + k]) : z);
      put(B3l, n, k, 64, n < 3 ? lo(W[kOffW3 + 64 * n + k]) : z);
    }
  bias.assign(131, 0.0f);
  for (int i = 0; i < 64; ++i) {
    bias[i] = W[kOffB1 + i];
    bias[64 + i] = W[kOffB2 + i];
  }
  for (int k = 0; k < 3; ++k) bias[128 + k] = W[kOffB3 + k];
}

static int ensure_sur(mc_ctx *c) {
  if (c->sur_w) return MC_OK;
  c->sur_w = (float *)dev_alloc_ext(c, sizeof(float) * kWPad);
  c->sur_packed = (unsigned char *)dev_alloc_ext(c, kPackedBytes);
  c->sur_bias = (float *)dev_alloc_ext(c, sizeof(float) * 144);
  c->sur_err = (unsigned int *)dev_alloc_ext(c, sizeof(unsigned int) * 4);
  if (!c->sur_w || !c->sur_packed || !c->sur_bias || !c->sur_err) return set_err(c, MC_ERR_OOM, "surrogate allocation");
  cudaMemset(c->sur_err, 0, sizeof(unsigned int) * 4);
  return MC_OK;
}

// Uploads FP32 weights, packs the BF16 tiles and biases for inference.
static int load_weights(mc_ctx *c, const float *w_host) {
  int rc = ensure_sur(c);
  if (rc) return rc;
  std::vector<unsigned char> packed;
  std::vector<float> bias;
  pack_bf16(w_host, packed, bias);
  if (cudaMemcpy(c->sur_w, w_host, sizeof(float) * kNumW, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->sur_packed, packed.data(), kPackedBytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->sur_bias, bias.data(), sizeof(float) * 131, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(c, MC_ERR_CUDA, "weight upload failed");
  c->sur_ready = true;
  return MC_OK;
}

mcgb::SurrogateView surrogate_view(const mc_ctx *c) {
  SurrogateView v;
  v.packed = c->sur_packed;
  v.bias = c->sur_bias;
  v.err = c->sur_err;
  v.wait_ns = std::min(c->wait_ns, 1e9);   // a completion takes microseconds: at most 1 s
  return v;
}

extern "C" {

int mc_surrogate_set_weights(mc_ctx *c, const float *w) {
  if (!c || !w) return set_err(c, MC_ERR_INVALID_ARG, "null argument");
  if (cudaSetDevice(c->p.device) != cudaSuccess) return set_err(c, MC_ERR_CUDA, "cudaSetDevice failed");
  return load_weights(c, w);
}

int mc_surrogate_get_weights(mc_ctx *c, float *w) {
  if (!c || !w) return set_err(c, MC_ERR_INVALID_ARG, "null argument");
  if (!c->sur_ready) return set_err(c, MC_ERR_STATE, "no surrogate weights");
  if (cudaMemcpy(w, c->sur_w, sizeof(float) * kNumW, cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_err(c, MC_ERR_CUDA, "weight download failed");
  return MC_OK;
}

int mc_surrogate_grad(mc_ctx *c, const float *w, const float *x, const float *t, const float *mask, int64_t n,
                      float *grad, double *loss) {
  if (!c || !w || !x || !t || !mask || !grad || n < 1) return set_err(c, MC_ERR_INVALID_ARG, "bad argument");
  if (cudaSetDevice(c->p.device) != cudaSuccess) return set_err(c, MC_ERR_CUDA, "cudaSetDevice failed");
  double msum = 0.0;
  for (int64_t i = 0; i < 3 * n; ++i) msum += mask[i];
  if (!(msum > 0.0)) return set_err(c, MC_ERR_INVALID_ARG, "empty mask");
  float *dw = (float *)dev_alloc_ext(c, sizeof(float) * kWPad), *dg = (float *)dev_alloc_ext(c, sizeof(float) * kWPad);
  float *dx = (float *)dev_alloc_ext(c, sizeof(float) * 3 * n), *dt = (float *)dev_alloc_ext(c, sizeof(float) * 3 * n);
  float *dm = (float *)dev_alloc_ext(c, sizeof(float) * 3 * n);
  double *dl = (double *)dev_alloc_ext(c, sizeof(double));
  int rc = MC_OK;
  if (!dw || !dg || !dx || !dt || !dm || !dl) rc = set_err(c, MC_ERR_OOM, "gradient buffers");
  if (rc == MC_OK) {
    cudaMemcpy(dw, w, sizeof(float) * kNumW, cudaMemcpyHostToDevice);
    cudaMemset(dg, 0, sizeof(float) * kWPad);
    cudaMemcpy(dx, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dt, t, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dm, mask, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
    cudaMemset(dl, 0, sizeof(double));
    size_t sm = sizeof(float) * (kWPad + 5 * kGB * kLd + 8 * kGB);
    cudaFuncSetAttribute(k_sur_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_sur_grad<<<(unsigned)((n + kGB - 1) / kGB), kGB, sm>>>(dw, dx, dt, dm, 0, n, (float)(1.0 / msum), dg, dl);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = set_err(c, MC_ERR_CUDA, cudaGetErrorString(e));
    cudaMemcpy(grad, dg, sizeof(float) * kNumW, cudaMemcpyDeviceToHost);
    double l = 0.0;
    cudaMemcpy(&l, dl, sizeof(double), cudaMemcpyDeviceToHost);
    if (loss) *loss = l / msum;
  }
  void *bufs[] = {dw, dg, dx, dt, dm, dl};
  for (void *b : bufs) dev_free_ext(c, b);
  return rc;
}

int mc_surrogate_infer(mc_ctx *c, const float *x, float *y, int64_t n, int tensor_cores) {
  if (!c || !x || !y || n < 1) return set_err(c, MC_ERR_INVALID_ARG, "bad argument");
  if (!c->sur_ready) return set_err(c, MC_ERR_STATE, "no surrogate weights");
  if (cudaSetDevice(c->p.device) != cudaSuccess) return set_err(c, MC_ERR_CUDA, "cudaSetDevice failed");
  float *dx = (float *)dev_alloc_ext(c, sizeof(float) * 3 * n), *dy = (float *)dev_alloc_ext(c, sizeof(float) * 3 * n);
  int rc = MC_OK;
  if (!dx || !dy) rc = set_err(c, MC_ERR_OOM, "inference buffers");
  if (rc == MC_OK) {
    cudaMemcpy(dx, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
    cudaMemset(c->sur_err, 0, sizeof(unsigned int));
    if (tensor_cores) {
      // >= 56 KB of shared memory per CTA keeps at most four CTAs (4 x 128 TMEM columns) on an SM
      int sm = tc_smem_bytes(1);
      cudaFuncSetAttribute(k_sur_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
      k_sur_infer_tc<<<(unsigned)((n + 127) / 128), 128, sm>>>(surrogate_view(c), dx, dy, n);
    } else {
      k_sur_infer_fp32<<<(unsigned)((n + 127) / 128), 128>>>(c->sur_w, dx, dy, n);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = set_err(c, MC_ERR_CUDA, cudaGetErrorString(e));
    unsigned int err = 0;
    cudaMemcpy(&err, c->sur_err, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    if (rc == MC_OK && err) rc = set_err(c, MC_ERR_TIMEOUT, "tensor-core wait timed out");
    cudaMemcpy(y, dy, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost);
  }
  dev_free_ext(c, dx);
  dev_free_ext(c, dy);
  return rc;
}

int mc_surrogate_train(mc_ctx *c, int64_t n_train, int64_t steps, int64_t batch, double lr, uint64_t seed,
                       double *val_loss) {
  if (!c || n_train < 1024 || steps < 1 || batch < kGB || !(lr > 0.0))
    return set_err(c, MC_ERR_INVALID_ARG, "bad training argument");
  if (cudaSetDevice(c->p.device) != cudaSuccess) return set_err(c, MC_ERR_CUDA, "cudaSetDevice failed");
  int rc = ensure_sur(c);
  if (rc) return rc;
  const int64_t n_val = 16384;
  float *X = (float *)dev_alloc_ext(c, sizeof(float) * 3 * (n_train + n_val));
  float *T = (float *)dev_alloc_ext(c, sizeof(float) * 3 * (n_train + n_val));
  float *M = (float *)dev_alloc_ext(c, sizeof(float) * 3 * (n_train + n_val));
  float *G = (float *)dev_alloc_ext(c, sizeof(float) * kWPad), *Mo = (float *)dev_alloc_ext(c, sizeof(float) * kWPad);
  float *Vo = (float *)dev_alloc_ext(c, sizeof(float) * kWPad);
  double *L = (double *)dev_alloc_ext(c, sizeof(double));
  if (!X || !T || !M || !G || !Mo || !Vo || !L) rc = set_err(c, MC_ERR_OOM, "training buffers");
  if (rc == MC_OK) {
    const double *gl = c->gl;   // [0,128): angle rule, [128,256): s rule, [256,320): mu rule
    k_sur_data<<<(unsigned)((n_train + 127) / 128), 128>>>(n_train, seed, 1, gl, gl + 128, gl + 256, X, T, M);
    k_sur_data<<<(unsigned)((n_val + 127) / 128), 128>>>(n_val, seed, 2, gl, gl + 128, gl + 256, X + 3 * n_train,
                                                         T + 3 * n_train, M + 3 * n_train);
    // deterministic initial weights: N(0, 1/fan_in) from the run seed
    std::vector<float> w(kNumW, 0.0f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 12345;
    auto nrm = [&]() {
      // Box-Muller on a 64-bit linear congruential stream (host-side initialisation only)
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      double u1 = ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      double u2 = ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < 64 * 3; ++i) w[kOffW1 + i] = (float)(nrm() / std::sqrt(3.0));
    for (int i = 0; i < 64 * 64; ++i) w[kOffW2 + i] = (float)(nrm() / 8.0);
    for (int i = 0; i < 3 * 64; ++i) w[kOffW3 + i] = (float)(nrm() / 8.0);
    cudaMemcpy(c->sur_w, w.data(), sizeof(float) * kNumW, cudaMemcpyHostToDevice);
    cudaMemset(G, 0, sizeof(float) * kWPad);
    cudaMemset(Mo, 0, sizeof(float) * kWPad);
    cudaMemset(Vo, 0, sizeof(float) * kWPad);
    size_t sm = sizeof(float) * (kWPad + 5 * kGB * kLd + 8 * kGB);
    cudaFuncSetAttribute(k_sur_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const float b1 = 0.9f, b2 = 0.999f;
    double p1 = 1.0, p2 = 1.0;
    const int64_t nb = n_train / batch;
    // each batch carries ~3 masked targets per sample; normalising by 3 * batch keeps the loss
    // a mean over targets
    const float inv_norm = (float)(1.0 / (3.0 * batch));
    for (int64_t it = 0; it < steps; ++it) {
      int64_t first = (it % nb) * batch;
      k_sur_grad<<<(unsigned)((batch + kGB - 1) / kGB), kGB, sm>>>(c->sur_w, X, T, M, first, batch, inv_norm, G, nullptr);
      p1 *= b1;
      p2 *= b2;
      double lr_t = lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(3.141592653589793 * (double)it / steps)));
      k_adam<<<(kNumW + 255) / 256, 256>>>(c->sur_w, G, Mo, Vo, kNumW, (float)lr_t, b1, b2, 1e-8f, (float)(1.0 - p1),
                                          (float)(1.0 - p2));
    }
    cudaMemset(L, 0, sizeof(double));
    cudaMemset(G, 0, sizeof(float) * kWPad);
    k_sur_grad<<<(unsigned)((n_val + kGB - 1) / kGB), kGB, sm>>>(c->sur_w, X, T, M, n_train, n_val,
                                                                  (float)(1.0 / (3.0 * n_val)), G, L);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = set_err(c, MC_ERR_CUDA, cudaGetErrorString(e));
    double l = 0.0;
    cudaMemcpy(&l, L, sizeof(double), cudaMemcpyDeviceToHost);
    if (val_loss) *val_loss = l / (3.0 * n_val);
    if (rc == MC_OK) {
      cudaMemcpy(w.data(), c->sur_w, sizeof(float) * kNumW, cudaMemcpyDeviceToHost);
      rc = load_weights(c, w.data());
    }
  }
  void *bufs[] = {X, T, M, G, Mo, Vo, L};
  for (void *b : bufs) dev_free_ext(c, b);
  return rc;
}

}  // extern "C"
