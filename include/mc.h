/* mc.h -- C ABI of the GB300 (sm_103a) Monte Carlo radiative-transfer hot path.
 *
 * The library computes the emergent spectrum nu L_nu of a relativistic plasma by the
 * superphoton Monte Carlo method of GPUmonty (arXiv 2602.13198): superphoton generation
 * per grid zone from the thermal synchrotron emissivity (sections 2.1-2.3), transport
 * along Kerr-Schild null geodesics by iterated velocity Verlet (section 2.4) with
 * synchrotron absorption (sections 2.5-2.6), biased Compton scattering off thermal
 * electrons (section 2.7), and binning of escaping superphotons (section 3).
 *
 * Conventions (all entry points):
 *   - return MC_OK (0) on success, a negative MC_ERR_* code on failure; no exception
 *     or longjmp crosses the boundary; mc_last_error() gives a message;
 *   - pointers are plain host or device pointers as stated per argument; sizes are in
 *     elements unless stated; nothing is retained beyond the call unless stated;
 *   - a context is not thread-safe; use one context per host thread;
 *   - device memory is obtained through the caller's allocator callbacks when given
 *     (PyTorch's caching allocator from Python), else cudaMalloc.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_ERR_INVALID_ARG (-1)
#define MC_ERR_NO_DEVICE (-2)
#define MC_ERR_OOM (-3)
#define MC_ERR_TIMEOUT (-4)
#define MC_ERR_QUEUE_OVERFLOW (-5)
#define MC_ERR_NAN_INPUT (-6)
#define MC_ERR_SIZE (-7)
#define MC_ERR_STATE (-8)
#define MC_ERR_CUDA (-9)

enum { MC_PREC_FP64 = 0, MC_PREC_MIXED = 1, MC_PREC_SPLIT = 2 };
enum { MC_DTYPE_F64 = 0, MC_DTYPE_F32 = 1 };
enum { MC_LOC_HOST = 0, MC_LOC_DEVICE = 1 };
enum { MC_BIAS_CONST = 0, MC_BIAS_GENERATION = 1, MC_BIAS_THETAE2 = 2 };

typedef struct mc_ctx mc_ctx;

/* Device allocator callbacks: alloc returns a device pointer aligned to 256 bytes, or NULL. */
typedef void *(*mc_alloc_fn)(size_t bytes, void *user);
typedef void (*mc_free_fn)(void *ptr, void *user);

/* Model parameters: the problem statement of the paper (metric and units, section 4.3;
 * emission band and weight floor, sections 2.1-2.3 and 4.3; Verlet tolerance, section
 * 2.4; bias b >= 1, section 2.7; record radius and spectrum bins, sections 4.1-4.3). */
typedef struct mc_model_params {
  double a;            /* black-hole spin a/M */
  double mass;         /* 1: Kerr-Schild with M = 1 (code units); 0: flat spacetime */
  double hslope;       /* modified Kerr-Schild theta(x2) = pi x2 + (1-hslope)/2 sin(2 pi x2) */
  double L_unit;       /* code length [cm] (GM/c^2 for mass 1) */
  double M_unit;       /* mass unit [g]: rho_unit = M_unit / L_unit^3 */
  double R_high, R_low;/* electron temperature model T_i/T_e = (R_high beta^2 + R_low)/(1 + beta^2) */
  double gam;          /* adiabatic index used by the temperature model */
  double thetae_min;   /* no synchrotron emission below this Theta_e */
  double thetae_max;   /* Theta_e ceiling */
  double nu_min, nu_max;   /* emission band [Hz] */
  double w_min;        /* superphoton weight floor */
  double n_s;          /* unused by mc_run (pass N_s there); kept for layout symmetry */
  double eps_geo;      /* step control: each internal coordinate moves at most eps_geo of its scale */
  double verlet_tol;   /* relative error bound of the Verlet predictor loop (paper: 1e-3) */
  double r_record;     /* record superphotons at r >= r_record [code lengths] */
  double dh;           /* capture at r <= r_h (1 + dh) */
  double bias_p0;      /* bias parameter; see bias_mode */
  double lnu_lo, lnu_hi;   /* spectrum range, log10(nu/Hz) */
  double roulette_w, roulette_p;  /* Russian roulette when w < roulette_w * w_birth, survival roulette_p */
  double bias_max;     /* upper bound on the bias b (any b >= 1 leaves the estimate unbiased) */
  double kappa;        /* 0: thermal (Maxwell-Juettner) electrons; in (3, 1e8]: kappa-distributed electrons of
                          width w = Theta_e (kappa - 3) / kappa for synchrotron emission, absorption and
                          Compton scattering (non-thermal electrons of section 6; not with the surrogate) */
  double bias_target;  /* > 0: tune the bias per scattering generation on the fly so that each
                          generation produces about bias_target scattered superphotons per
                          superphoton it carries (mc_run only); 0: the bias as configured */
  int64_t max_steps;   /* drop a superphoton after this many steps */
  int32_t n_nu;        /* weight-table nodes in ln nu (>= 2) */
  int32_t verlet_maxit;/* cap on Verlet predictor iterations */
  int32_t bias_mode;   /* MC_BIAS_CONST: b = max(1,p0); _GENERATION: max(1, p0 (n_sc+1)^2); _THETAE2: max(1, p0 Theta_e^2) */
  int32_t n_sc_max;    /* largest scattering generation that is produced */
  int32_t n_bins, n_incl;  /* spectrum bins in log nu, inclination bins over [0, pi/2] (hemispheres folded) */
  int32_t k2_mode;     /* 0: exact K2(1/Theta_e); 1: K2 ~ 2 Theta_e^2 (section 2.2) */
  int32_t scatter;     /* 0: Compton scattering off */
  /* --- execution (not part of the physics) --- */
  int32_t precision;   /* MC_PREC_FP64: everything FP64; MC_PREC_MIXED: geodesics at FP64-level accuracy in
                          double-float (FP32 pairs, 48-bit significand); plasma coefficients, optical
                          depths, weights (carried relative to each superphoton's FP64 birth weight)
                          and the scattering decision in FP32; emission and Compton kinematics FP64;
                          MC_PREC_SPLIT: geodesic and step size in FP64; plasma coefficients, optical
                          depths, weights (carried relative to each superphoton's FP64 birth weight),
                          the scattering decision and the Compton kinematics in FP32; emission
                          sampling FP64 */
  int32_t surrogate;   /* 0: closed forms and tables; 1: MLP surrogate for the coefficients (needs weights;
                          MC_PREC_MIXED or MC_PREC_SPLIT) */
  int32_t block;       /* threads per CTA of the transport kernel (0: default 128) */
  int32_t ctas_per_sm; /* resident CTAs per SM for the persistent launch (0: occupancy maximum) */
  int32_t device;      /* CUDA device ordinal */
  int32_t brems;       /* 1: add thermal bremsstrahlung emission and absorption (not with the surrogate) */
  mc_alloc_fn alloc;   /* optional device allocator (NULL: cudaMalloc) */
  mc_free_fn free;
  void *alloc_user;
} mc_model_params;

/* Fluid grid: primitives rho, u, B^1..3, U^1..3 (U^i: 4-velocity relative to the normal
 * observer; B^i: field 3-vector; modified Kerr-Schild internal coordinates x1 = ln r,
 * x2 in [0,1], x3 = phi), laid out [8][n1*n2*n3] with zone index (i*n2 + j)*n3 + k. */
typedef struct mc_grid_desc {
  int32_t n1, n2, n3;
  int32_t dtype;       /* MC_DTYPE_F64 or MC_DTYPE_F32 */
  double x1_0, dx1, x2_0, dx2, x3_0, dx3;
  int32_t location;    /* MC_LOC_HOST: copied into the context; MC_LOC_DEVICE: copied device-to-device */
  int32_t pad0;
  const void *prim;    /* 8 * n1*n2*n3 elements of dtype */
} mc_grid_desc;

/* Counters of one run (sums over all generations). */
typedef struct mc_run_stats {
  int64_t n_emit;      /* primaries emitted */
  int64_t n_child;     /* scattered superphotons created */
  int64_t n_rec, n_abs, n_capt, n_maxst;   /* recorded / absorbed / captured / dropped at max_steps */
  int64_t n_steps;     /* geodesic steps */
  int64_t n_iters;     /* Verlet predictor iterations */
  int64_t n_nonconv;   /* steps whose predictor loop hit verlet_maxit */
  int64_t n_roul_surv; /* roulette survivals */
  int64_t n_rej_cap;   /* rejection loops that hit their cap */
  int64_t n_events;    /* scattering events */
  int64_t n_total;     /* primaries of the whole job (all shards) */
  int64_t err_flags;   /* bit 0: child queue overflow; bit 1: log overflow */
  int64_t transport_launches;  /* transport kernel launches (one per generation and batch) */
  double transport_ms; /* summed device time of those launches (CUDA events on the launching stream) */
  double generate_ms;  /* device time of weights, counts and scan */
  int64_t n_steps_grid;  /* steps taken inside the radial extent of the grid (the rest free-stream) */
  int64_t n_iters_grid;  /* Verlet predictor passes of those steps */
  double init_ms, grid_ms, free_ms;   /* transport device time by phase: emission/initialisation,
                                         in-grid push, free-streaming push */
  int32_t batch_min_blocks;  /* mc_run_batch: register-cap variant (minimum resident CTAs per SM) */
  int32_t batch_ctas;        /* mc_run_batch: persistent grid size in CTAs */
  int32_t batch_graph;       /* mc_run_batch: 1 if the run replayed a captured CUDA graph */
  int32_t pad0;
} mc_run_stats;

/* One finished superphoton, for per-photon parity checks (layout matches the test oracle's). */
typedef struct mc_log_rec {
  uint64_t id;         /* random-stream id: the primary's uid, or the child's derived id */
  int32_t gen, status; /* scattering generation; 1 recorded, 2 absorbed, 3 captured, 4 max steps */
  double X[4], K[4];   /* end position (internal coordinates) and wavevector */
  double w;            /* end weight */
  int64_t nsteps;
  int32_t nev, pad;    /* scattering events of this superphoton */
} mc_log_rec;

/* Creates a context on p->device, builds the device tables (synchrotron angle integral,
 * K2, hot cross-section; sections 2.2 and 2.7).  *out owned by the library until mc_free.
 * Errors: INVALID_ARG (bad parameters), NO_DEVICE, OOM, CUDA. */
int mc_init_model(mc_ctx **out, const mc_model_params *p);

/* Sets the fluid grid (section 3: "reading data from external files"); the library keeps
 * its own copy in a zone-major layout.  Errors: INVALID_ARG, NAN_INPUT (non-finite
 * primitive), OOM, CUDA. */
int mc_set_grid(mc_ctx *c, const mc_grid_desc *g);

/* Runs the whole hot path for N_s target superphotons and Philox seed `seed`: weights
 * (eq. weight_calc), zone counts (section 2.3), then transport of the primaries of shard
 * `shard` of `n_shards` (contiguous uid ranges) and of all their scattered descendants,
 * generation by generation (section 3).  The spectrum sums are reset at the start of the
 * call.  `stream` is a cudaStream_t (NULL: default stream); the call returns after the
 * work on `stream` is complete (it reads the counters back).  stats may be NULL.
 * A scattered generation that exceeds the queues makes the call grow them and start again
 * (same result: every superphoton has its own counter-based stream), up to three times while
 * device memory allows.  Errors: STATE (no grid, or the surrogate on without trained weights),
 * INVALID_ARG, QUEUE_OVERFLOW (the queues could not grow enough; results invalid), TIMEOUT (a
 * tensor-core wait of the surrogate ran out, see mc_set_wait_limit), NAN_INPUT, OOM, CUDA. */
int mc_run(mc_ctx *c, double n_s, uint64_t seed, int64_t shard, int64_t n_shards, void *stream,
           mc_run_stats *stats);

/* Bias scales s_g (g = 0 .. n_sc_max) of the last mc_run: generation g scatters with
 * b = clamp(s_g b_0, 1, bias_max), b_0 the configured bias.  s_0 = 1; with bias_target > 0, after
 * generation g of the first batch of primaries, s_{g+1} = s_g clamp(bias_target / r_g, 1/8, 8) with
 * r_g = (children produced) / (superphotons carried) (8 when r_g = 0); later batches and
 * mc_trace reuse the sequence.  Without tuning every s_g = 1.  Errors: STATE (no run),
 * SIZE (n != n_sc_max + 1). */
int mc_get_bias_scales(mc_ctx *c, double *scales, int n);

/* Spectrum of the last mc_run: nu L_nu [erg/s] per (inclination, frequency) bin, its Monte
 * Carlo standard error, and the superphoton count, each n_incl*n_bins host doubles
 * (inclination-major).  Any pointer may be NULL.  Errors: SIZE if n_elems != n_incl*n_bins. */
int mc_get_spectrum(mc_ctx *c, double *nuLnu, double *sigma, double *counts, size_t n_elems);

/* Raw spectrum sums (sum w E, sum (w E)^2, count) [n_incl][n_bins][3] into host memory, for
 * reductions across shards.  Errors: SIZE if n_elems != 3*n_incl*n_bins. */
int mc_get_spectrum_sums(mc_ctx *c, double *sums, size_t n_elems);

/* Zone superphoton counts of the last mc_run (int64, n1*n2*n3 host elements).
 * Errors: STATE before any run, SIZE. */
int mc_get_zone_counts(mc_ctx *c, int64_t *counts, size_t n_elems);

/* Transports only the listed primaries (host array of uids of the job defined by N_s and
 * seed) and their descendants, writing one mc_log_rec per finished superphoton to the host
 * buffer `out` (capacity `cap`, number written in *n_out).  The spectrum sums of these
 * superphotons replace the context's.  With bias tuning the generations scatter with the bias
 * scales of the context's last mc_run (see mc_get_bias_scales), so a trace after a run of the same
 * job follows the run's histories.  Errors: SIZE (uid out of range), STATE, CUDA. */
int mc_trace(mc_ctx *c, double n_s, uint64_t seed, const int64_t *uids, size_t n_uids, mc_log_rec *out,
             size_t cap, size_t *n_out, void *stream);

/* Measures the arithmetic pipe throughput of the current device with a chain of independent
 * fused multiply-adds (no memory traffic): dtype MC_DTYPE_F64 or MC_DTYPE_F32; writes the achieved
 * FLOP/s (2 per FMA) to *flops.  Used as the roofline peak of the FP64 and FP32 pipes, which the
 * paper's compute-bound transport kernels are measured against (section 5).  Errors: INVALID_ARG,
 * NO_DEVICE, CUDA. */
int mc_fma_peak(int device, int dtype, double *flops);

/* Test hook: evaluates, on the current device, one of the library's own implementations of a
 * special function next to CUDA's for the same inputs.  which = 0: sine of |x| < 1/2 by the Taylor
 * series used in the metric (ref: CUDA sin); 1: its cosine (ref: CUDA cos); 2: x^(1/6) by the
 * FP32-seeded Newton iteration used in the synchrotron function (ref: cbrt(sqrt(x))); 3: e^x in
 * double-float arithmetic, as the mixed-precision geodesic evaluates r = e^x1 (ref: CUDA exp,
 * |x| < 80); 4, 5: sin(pi x), cos(pi x) in double-float (ref: CUDA sincospi).  Inputs 3-5 are split
 * to double-float first and results joined back to double.  6: e^x and 7: ln x by the table-driven
 * FP64 functions of the FP64 transport (ref: CUDA exp, log); 8, 9: their sin(pi x), cos(pi x) (ref:
 * CUDA sincospi); 10: their e^x - 1 (ref: CUDA expm1).  x, y, ref are n host doubles (caller-owned).  Errors: INVALID_ARG, NO_DEVICE, CUDA. */
int mc_selftest_math(int which, const double *x, double *y, double *ref, int64_t n);

/* Zone superphoton counts for (N_s, seed) -- the same numbers mc_run computes and
 * mc_get_zone_counts returns -- without allocating any device memory, for callers that cannot
 * allocate at this point (a stream being captured into a graph, a custom allocator's callback,
 * an application that has given all device memory to its own pool).  The paper has no
 * counterpart; it is an execution variant of the weight/count/scan kernels of mc_run.
 *   counts: device int64[n1*n2*n3], written; start: device int64[n1*n2*n3], the exclusive scan
 *   (first uid of each zone), written; total: device int64[1], the job's primary count, written.
 *   All three are caller-owned device pointers; the call is asynchronous on `stream`.
 *   A zone state that turns non-finite (mc_run fails with MC_ERR_NAN_INPUT on it) makes *total
 *   -1; counts and start are then meaningless.  The call itself cannot see this without waiting
 *   for the GPU, so it still returns MC_OK: read *total after the stream's work is done.
 * Scratch lives in one static device array of fixed size (8.3 MiB: eight per-zone arrays, the
 * weight-table partial sums and the scan's block sums) that every GPU loading the library keeps
 * until the process exits; grids above 131072 zones or weight tables above 512 nodes are rejected
 * with MC_ERR_SIZE.  The first call on a device looks up that array's device address (once per
 * device, with the device current) and keeps it for the life of the process (a cudaDeviceReset
 * in between is not supported); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls whose work overlaps on
 * the GPU (different streams, or different contexts on the same device) race and must be ordered
 * by the caller.  The context's tables, grid and per-zone arrays are read, not modified (the
 * kappa and bremsstrahlung zone arrays are rebuilt in the scratch).
 * Errors: INVALID_ARG, STATE (no grid), SIZE, CUDA. */
int mc_zone_counts_noalloc(mc_ctx *c, double n_s, uint64_t seed, int64_t *counts, int64_t *start, int64_t *total,
                           void *stream);

/* ---- coefficient surrogate (not in the paper: an addition of this library) ----
 * A 3 -> 64 -> 64 -> 3 SiLU network maps normalised inputs
 *   x0 = ln(Theta_e)/ln(1e3), x1 = ln(nu/nu_c)/ln(1e4), x2 = (ln(eps) - ln(1e-3))/ln(1e9)
 * to o0 = ln(sigma_h/sigma_T) (hot cross-section, section 2.7), o1 = ln K2(1/Theta_e) -
 * ln(2 Theta_e^2) (section 2.2) and o2 = ln F(nu/nu_c)/10 (angle-integrated synchrotron
 * shape).  Weights are 4611 floats: W1[64][3] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]. */

/* Trains the context's network on the device: n_train samples uniform in the input domain with
 * targets from the library's own FP64 quadratures, `steps` Adam steps of `batch` samples, cosine
 * learning-rate decay from lr; then packs BF16 tiles for tensor-core inference.  *val_loss gets the
 * mean squared error on 16384 held-out samples.  Errors: INVALID_ARG, OOM, CUDA. */
int mc_surrogate_train(mc_ctx *c, int64_t n_train, int64_t steps, int64_t batch, double lr, uint64_t seed,
                       double *val_loss);

/* Sets / gets the FP32 weights (host arrays of 4611 floats).  Errors: INVALID_ARG, STATE (get
 * before any weights), CUDA. */
int mc_surrogate_set_weights(mc_ctx *c, const float *w);
int mc_surrogate_get_weights(mc_ctx *c, float *w);

/* Gradient of the masked mean squared error sum m (y - t)^2 / sum m with respect to the 4611
 * weights w, over n samples (host arrays x, t, mask of n*3 floats), computed by the library's
 * training kernel; *loss gets the loss.  Errors: INVALID_ARG, OOM, CUDA. */
int mc_surrogate_grad(mc_ctx *c, const float *w, const float *x, const float *t, const float *mask, int64_t n,
                      float *grad, double *loss);

/* Evaluates the network on n input rows (host x, y: n*3 floats) with the BF16 tensor-core kernel
 * (tensor_cores = 1) or the FP32 reference kernel (0).  Errors: STATE (no weights), TIMEOUT (a
 * tensor-core wait ran out), CUDA. */
int mc_surrogate_infer(mc_ctx *c, const float *x, float *y, int64_t n, int tensor_cores);

/* Batched survey (section 1's parameter surveys): runs n <= 64 models (contexts with grids, same
 * device, precision and surrogate mode) together, each with its own N_s (n_s[i]) and seed.  Per
 * model the weights/counts/scan run as in mc_run; then ONE cooperative persistent kernel
 * transports every superphoton of every model through all scattering generations.  flags: bit 0
 * (MC_BATCH_AUTOTUNE): before the first batched run of this leading context, time calibration runs
 * (every model at the same fraction of its N_s, >= 5% and >= ~5e6 superphotons in all, at most the
 * whole batch) over the register-cap variants and resident CTAs per SM and keep the fastest;
 * bit 1 (MC_BATCH_GRAPH): capture the whole sequence into a CUDA graph (re-captured when models,
 * N_s, seeds or the launch configuration change) and replay it.  Each model's spectrum is read
 * with mc_get_spectrum on its own context; `stats` (may be NULL) gets the totals and the launch
 * configuration.  State (queues, graph, tuning) is kept by ctxs[0].  A scattered generation larger
 * than the pool makes the batch run again with a pool twice as large (same result; up to two times).
 * Errors: INVALID_ARG, SIZE (more than 64 models, or more transport phases than one launch holds),
 * STATE, QUEUE_OVERFLOW (the pool cannot grow further), TIMEOUT (grid barrier or tensor-core wait), OOM,
 * CUDA. */
#define MC_BATCH_AUTOTUNE 1
#define MC_BATCH_GRAPH 2
int mc_run_batch(mc_ctx **ctxs, int n, const double *n_s, const uint64_t *seeds, int flags, void *stream,
                 mc_run_stats *stats);

/* Limit, in seconds, on each device-side wait of the grid barrier between the phases of a batched
 * run led by c (ctxs[0] of mc_run_batch); default 120.  A wait that runs out raises an error bit on
 * the device; every CTA then leaves the kernel at its next barrier, and mc_run_batch returns
 * MC_ERR_TIMEOUT with the context still usable (the next call starts from reset counters).  The
 * limit is part of a captured batch graph's key, so changing it re-captures.  The same limit, capped
 * at 1 s, bounds each wait of the surrogate network for its tensor-core products (mc_run,
 * mc_run_batch and mc_surrogate_infer with the surrogate on): a wait that runs out still lets the
 * products in flight complete before the kernel goes on, and the call returns MC_ERR_TIMEOUT.  Not
 * in the paper: a guard of this library's persistent and tensor-core launches (section 3 launches
 * one kernel per stage).  Errors: INVALID_ARG (c NULL, or seconds outside [1e-9, 3600]). */
int mc_set_wait_limit(mc_ctx *c, double seconds);

/* Releases the context and all its device memory.  NULL is a no-op. */
void mc_free(mc_ctx *c);

/* Message of the last failing call on c (or of the last mc_init_model failure when c is NULL). */
const char *mc_last_error(const mc_ctx *c);

/* Library version string. */
const char *mc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
