/*
 * xrdvi — variational sparse Bayesian crystalline-phase search on one GPU.
 *
 * C ABI of the Monte-Carlo ELBO step of Murakami et al., "Rapid, Comprehensive
 * Search of Crystalline Phases from X-ray Diffraction in Seconds via
 * GPU-Accelerated Bayesian Variational Inference" (arXiv 2501.09308):
 *
 *   problem   (Appendix A.1)  pattern D = {(x_i, y_i)}, i = 1..N, 2-theta in
 *             degrees and integer counts; K candidate phases, phase k a list
 *             of M_k (position p_m, relative intensity I_m) pairs;
 *   model     (Appendix A.2)  f(x) = B(x) + sum_k h_k sum_m I_m V(x; p_m + mu_k,
 *             w_k, r_k, alpha_k), V the split pseudo-Voigt (1-r) G + r L;
 *   likelihood(Appendix A.2)  y_i ~ Poisson(f(x_i));
 *   priors    (Sec. 2.2, Appendix B.2)  h ~ Exp(1/max(Y-B)), mu ~ N(0,0.03),
 *             alpha ~ N(1,0.2), r ~ U(0,1), w ~ Gam(3, rate 100);
 *   inference (Sec. 3.2)  mean-field normal q over the unconstrained
 *             parameters u = (ln h, mu, ln w, logit r, alpha), fitted by
 *             maximising the reparameterised Monte-Carlo ELBO with Adam.
 *
 * Every compute step runs in CUDA kernels built for sm_103a; there is no CPU
 * fallback.  A context owns all of its device memory.  Unless stated, pointers
 * are HOST pointers owned by the caller, copied during the call; "_dev"
 * entry points take DEVICE pointers (caller-owned, must stay valid until the
 * call returns on the context's stream).  No call keeps a caller pointer.
 *
 * Errors: every call returns an xrdvi_status; xrdvi_last_error() gives a
 * thread-local message for the last failing call on the calling thread.
 * A context is not thread-safe: use one context per host thread.
 *
 * Parameter layout (all entry points): per phase k, j = 0 intensity h,
 * 1 shift mu, 2 width w (FWHM, degrees), 3 Gauss-Lorentz ratio r,
 * 4 asymmetry alpha.  loc/raw are float [K*5] (index k*5+j) with
 * sigma = softplus(raw).  Gradients are float [K*10]: grad[k*10+j] =
 * dELBO/dloc[k][j], grad[k*10+5+j] = dELBO/draw[k][j].  Monte-Carlo noise is
 * float [S*K*5] (index (s*K+k)*5+j).
 */
#ifndef XRDVI_H
#define XRDVI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XRDVI_OK = 0,
    XRDVI_EINVAL = 1,      /* invalid argument or input data                    */
    XRDVI_ENOMEM = 2,      /* device allocation failed / over the memory budget */
    XRDVI_ECUDA = 3,       /* CUDA runtime error (no device, launch failure)    */
    XRDVI_ETIMEOUT = 4,    /* bounded wait ran out                               */
    XRDVI_ENONFINITE = 5,  /* ELBO or gradient became NaN/Inf                    */
    XRDVI_EBUSY = 6,       /* resource temporarily unavailable                   */
    XRDVI_ECANCELED = 7    /* served request cancelled before it ran             */
} xrdvi_status;

typedef struct xrdvi_ctx xrdvi_ctx;

/* Candidate phase set F (Appendix A.1) in CSR form.  offsets[0] = 0,
 * offsets[k+1] - offsets[k] = M_k >= 1.  Positions in (0, 180) degrees,
 * relative intensities in [0, 1].  Peaks need not be sorted. */
typedef struct {
    int32_t K;
    const int32_t *offsets;   /* [K+1]            */
    const float *pos_deg;     /* [offsets[K]]     */
    const float *rel_int;     /* [offsets[K]]     */
} xrdvi_peaks;

/* Measured pattern D (Appendix A.1) and the fixed background B (Appendix A.2,
 * estimated before fitting).  x strictly increasing in (0, 180); y >= 0 and
 * integer-valued; bg >= 0. */
typedef struct {
    int32_t N;
    const float *x_deg;       /* [N] */
    const float *y_counts;    /* [N] */
    const float *bg;          /* [N] */
} xrdvi_pattern;

/* Flags */
#define XRDVI_FLAG_BF16_INT   (1u << 0)  /* keep relative intensities as bfloat16 */
#define XRDVI_FLAG_NAIVE_SUM  (1u << 1)  /* plain instead of compensated f32 sum over phases */
/* Estimator variants (the paper's model is the Poisson likelihood and the ELBO):
 * GAUSS_LIK replaces the Poisson likelihood by a Gaussian with variance
 * max(y_i, 1), ln p(Y|Phi) = sum_i [-(y_i - f_i)^2 / (2 v_i) - ln(2 pi v_i)/2]
 * (a weighted residual sum of squares); IW_ELBO makes the fit maximise the
 * importance-weighted bound ln (1/S) sum_s w_s over the S draws of a step
 * (Burda, Grosse & Salakhutdinov, ICLR 2016), whose gradient weights each
 * draw by w_s / sum w instead of 1/S; the ELBO values reported (trace,
 * xrdvi_elbo_grad, forward_dev) are then that bound. */
#define XRDVI_FLAG_GAUSS_LIK  (1u << 2)
#define XRDVI_FLAG_IW_ELBO    (1u << 3)
/* Shared-shape estimator: the shapes (mu, w, r, alpha) of all S samples of a
 * step take sample 0's noise, the intensities h each sample's own (an
 * unbiased estimator of the same ELBO; with injected noise, eps[s][k][1..4]
 * is replaced by eps[0][k][1..4]).  The profile then factors into phase
 * profiles evaluated once per step, and both the forward contraction over
 * phases and the backward's per-(sample, phase) sums run as GEMMs on the
 * tensor cores (xrdvi_gemm_nt_tf32x3).  Not with sub-model batches or the
 * static entry. */
#define XRDVI_FLAG_SHARED_SHAPES (1u << 4)
/* Angle-dependent width (model variant; the paper names a sec term in App.
 * A.2 without a formula): every side width at point x is multiplied by
 * sec(theta) with theta = x/2 (x the 2-theta of the point in degrees), so the
 * peaks broaden towards high angles.  Needs every x below 174 degrees. */
#define XRDVI_FLAG_SEC_WIDTH  (1u << 5)
/* Background fitted in-model (model variant; the paper fixes B beforehand,
 * App. A.2): B_i(beta) = B_i exp(sum_{j<3} beta_j T_j(z_i)) with Chebyshev T_j
 * and z_i the grid mapped onto [-1, 1]; each beta_j has the prior
 * N(0, bg_prior_sd^2) and is point-estimated (ln p(beta) joins every draw's
 * log joint, beta takes the Adam step rule).  xrdvi_get_background reads it. */
#define XRDVI_FLAG_FIT_BACKGROUND (1u << 6)
/* Shape parameters held fixed (model options): the Gauss-Lorentz ratio r at
 * fix_r_value and / or the asymmetry alpha at fix_alpha_value, for every
 * phase.  A fixed parameter is a constant of the model, not part of q: it has
 * no prior, Jacobian, entropy or ln q term, its gradient is zero and its
 * variational parameters are not updated. */
#define XRDVI_FLAG_FIX_R      (1u << 7)
#define XRDVI_FLAG_FIX_ALPHA  (1u << 8)
/* xrdvi_create: the peak and pattern arrays (offsets, pos_deg, rel_int,
 * x_deg, y_counts, bg) are DEVICE pointers; they are read back once for
 * validation and preparation (sorting, the data constants), then handled as
 * host input.  K and N stay host values. */
#define XRDVI_FLAG_DEVICE_PTRS (1u << 9)
/* Area-normalised profiles (the alternative to the height normalisation the
 * paper's lambda = 1 / max(Y - B) suggests): each phase's profile is divided
 * by the area of its unit-height shape, a(w, alpha, r) = ((1 + alpha) w / 2)
 * [(1 - r) sqrt(pi / ln 2) / 2 + r pi / 2], so h is an integrated intensity
 * (per unit relative intensity), the posterior's area of phase k is
 * h_k sum_m I_m, and the initial h is scaled by the initial shape's area. */
#define XRDVI_FLAG_AREA_NORM  (1u << 10)
/* Explicit phase gates (model variant, not in the paper, whose sparsity
 * comes from the exponential prior on h): each phase's profile is scaled by a
 * binary-Concrete gate z = sigmoid((a_k + L)/tau) (Maddison, Mnih & Teh,
 * ICLR 2017) with logistic noise L and a learned logit a_k (starting at 0);
 * the prior is the same family with logit ln(gate_prior / (1 - gate_prior)),
 * and each draw's log joint gains ln p(y) - ln q(y) of the logit y.  The
 * logits take the Adam step rule; xrdvi_get_gates reads them.  With injected
 * noise (xrdvi_elbo_grad) eps holds [S*K*5] normals followed by [S*K]
 * logistic gate noise values.  The posterior's areas use z h. */
#define XRDVI_FLAG_GATES      (1u << 11)
/* Every peak evaluated directly at every point.  By default the Lorentzian
 * tails of peaks more than half a tile width (of 256 points) beyond a tile,
 * and beyond their Gaussian reach, are summed at 32 Chebyshev nodes of the
 * tile and interpolated (error below 1e-8 of those tails, under FP32
 * rounding); the shared-shape variant always runs dense. */
#define XRDVI_FLAG_DENSE      (1u << 12)

typedef struct {
    uint32_t size;            /* sizeof(xrdvi_config): set by xrdvi_config_default */
    int32_t S;                /* Monte-Carlo samples per ELBO step (>= 1)          */
    float lr, beta1, beta2, adam_eps;   /* Adam on -ELBO                          */
    uint64_t seed;            /* Philox4x32-10 key for the fit's noise stream      */
    float prior_mu_sd;        /* mu ~ N(0, prior_mu_sd)                 (B.2)      */
    float prior_alpha_mean;   /* alpha ~ N(mean, sd)                    (B.2)      */
    float prior_alpha_sd;
    float prior_w_shape;      /* w ~ Gam(shape, rate)                   (B.2)      */
    float prior_w_rate;
    float alpha_min;          /* profile clamp: alpha_eff = max(alpha, alpha_min)  */
    float init_h_frac;        /* initial h = init_h_frac * max(Y - B)              */
    float init_sigma;         /* initial sigma of every q factor                   */
    uint32_t flags;           /* XRDVI_FLAG_*                                      */
    float bg_prior_sd;        /* prior sd of the fitted-background coefficients    */
    float fix_r_value;        /* r with XRDVI_FLAG_FIX_R (in [0, 1])              */
    float fix_alpha_value;    /* alpha with XRDVI_FLAG_FIX_ALPHA                  */
    float gate_tau;           /* gate temperature (XRDVI_FLAG_GATES)              */
    float gate_prior;         /* prior inclusion probability of a gate, (0, 1)     */
} xrdvi_config;

/* Fills the defaults: S 256, Adam lr 0.01 betas (0.9, 0.999) eps 1e-8, seed 0,
 * priors of Appendix B.2, alpha_min 1e-3, init_h_frac 0.1, init_sigma 0.1,
 * bg_prior_sd 0.1, fix_r_value 0.5, fix_alpha_value 1, gate_tau 2/3,
 * gate_prior 0.5. */
void xrdvi_config_default(xrdvi_config *cfg);

/* Validates and uploads the problem (one host-to-device copy), computes
 * lambda = 1 / max(Y - B) (Sec. 2.2) and the data constant of the Poisson
 * log-likelihood, allocates the device state and initialises q.
 * EINVAL on malformed input (K < 1, an empty phase, x not increasing,
 * y negative / non-integer / non-finite, bg < 0, max(Y - B) <= 0, S < 1, sizes
 * above the documented limits: K <= 1024, total peaks <= 24000, N <= 2^24,
 * S <= 65536).  On success *out owns all device memory. */
xrdvi_status xrdvi_create(const xrdvi_peaks *peaks, const xrdvi_pattern *pattern,
                          const xrdvi_config *cfg, xrdvi_ctx **out);

/* Frees the context and all of its device memory (NULL is a no-op). */
void xrdvi_destroy(xrdvi_ctx *ctx);

/* Runs subsequent work on `cuda_stream`, a cudaStream_t (cudaStreamLegacy
 * and cudaStreamPerThread are accepted); NULL selects the context's own
 * non-blocking stream (the default).  Waits for the previous stream first. */
xrdvi_status xrdvi_set_stream(xrdvi_ctx *ctx, void *cuda_stream);

/* Stochastic variational inference (Sec. 3.2): `iters` steps of
 * sample -> profile/likelihood -> backward -> Adam, replayed as a CUDA graph
 * with no host synchronisation inside.  elbo_trace (NULL or [iters]) receives
 * the ELBO estimate of each step before its update.  Returns ENONFINITE if
 * the last ELBO is not finite.  Blocks until the work is done. */
xrdvi_status xrdvi_fit(xrdvi_ctx *ctx, int32_t iters, double *elbo_trace);

/* Batched SVI (continuous batching without the server): advances the n
 * contexts ctxs[0..n) (1 <= n <= 64, distinct, one device) by `iters` steps
 * each, the steps of all n fits sharing their kernel launches: sampling,
 * window ranges, the likelihood and the gradient are one launch each whose
 * work lists span every fit, whatever its K, N and peak counts; the profile
 * passes of fits too small to fill the GPU alone share launches per group of
 * equal occupancy, while a fit with enough work for the whole GPU runs its
 * own profile and likelihood kernels back to back.  A context whose
 * configuration the batched step does not cover (shared shapes,
 * angle-dependent width, fitted background, naive sums, importance weights)
 * takes its own kernels between those launches.  Every context ends exactly
 * as xrdvi_fit(ctx, iters) would leave it (same kernels per work item, fixed
 * reduction orders).  The step graphs captured for the array are kept with
 * ctxs[0] and reused by the next call with the same contexts in the same
 * order (unless one of them was restored by xrdvi_set_state since); they are
 * freed with ctxs[0].  Do not call it on a context that another thread is
 * using.  Runs on ctxs[0]'s stream after waiting for every context's stream;
 * blocks until done.  last_elbo (NULL or host [n]) receives each fit's last
 * ELBO estimate.  ENONFINITE if any fit's last ELBO or gradient is not
 * finite.  No counterpart in the paper, which fits one pattern at a time. */
xrdvi_status xrdvi_fit_batch(xrdvi_ctx *const *ctxs, int32_t n, int32_t iters, double *last_elbo);

/* One ELBO + gradient evaluation at the current q, without an update.
 * eps: NULL (noise from the fit stream at the current step) or injected
 * standard normals [S*K*5] (with XRDVI_FLAG_GATES [S*K*6]: the normals, then
 * [S*K] logistic gate noise).  Outputs (each may be NULL): elbo [1],
 * grad [K*10], f_out profile [S*N], ll_out [S] log-likelihood per sample,
 * lpj_out [S] log prior + log Jacobian per sample. */
xrdvi_status xrdvi_elbo_grad(xrdvi_ctx *ctx, const float *eps, double *elbo, float *grad,
                             float *f_out, double *ll_out, double *lpj_out);

/* Posterior over phase combinations from the fitted q: how probable each
 * subset of the candidate phases is given the data (Abstract, Sec. 1), with a
 * phase counted as present when its share of the total peak area is at least
 * 1 % (Sec. 4).  Draws S_post samples (Philox key `seed`),
 * computes per-sample inclusion bits, marginal inclusion probabilities
 * pi_k = (count_k + 1/2) / (S_post + 1), the top_m most probable combinations
 * of the mean-field product (exact best-first order), their FP64 log-sum-exp
 * coverage, and the importance-sampled log evidence with its effective
 * sample size.  Outputs (host, may be NULL): pi [K]; combos [top_m * W] bit
 * masks with W = ceil(K/64) words per combination, bit k%64 of word k/64 =
 * phase k; combo_logp [top_m]; log_evidence [1]; ess [1]; coverage_log [1].
 * 1 <= S_post <= 65536, 1 <= top_m <= 4096. */
xrdvi_status xrdvi_posterior(xrdvi_ctx *ctx, int32_t S_post, uint64_t seed, int32_t top_m,
                             double *pi, uint64_t *combos, double *combo_logp,
                             double *log_evidence, double *ess, double *coverage_log);

/* Variational parameters (host float [K*5] each). */
xrdvi_status xrdvi_get_params(xrdvi_ctx *ctx, float *loc, float *raw);
xrdvi_status xrdvi_set_params(xrdvi_ctx *ctx, const float *loc, const float *raw);

/* Checkpoint / resume.  The state is loc, raw, the Adam moments, the step
 * counter and the seed; a resumed fit replays the same noise (Philox counters
 * are keyed by step) and is bit-identical to an uninterrupted one.
 * xrdvi_get_state with buf == NULL stores the required size in *len. */
xrdvi_status xrdvi_get_state(xrdvi_ctx *ctx, void *buf, size_t *len);
xrdvi_status xrdvi_set_state(xrdvi_ctx *ctx, const void *buf, size_t len);

typedef struct {
    int32_t K, N, S, M_total;
    int64_t step;             /* optimisation steps taken                   */
    double eta;               /* max(Y - B)                                  */
    double lambda_;           /* 1 / eta                                     */
    double data_const;        /* sum_i [y ln y - y - ln y!] (Gaussian variant:
                                 -sum_i ln(2 pi max(y_i, 1)) / 2)            */
    size_t device_bytes;      /* device memory held by the context           */
    int32_t point_tiles;      /* 2-theta tiles of the profile kernels        */
} xrdvi_info;

xrdvi_status xrdvi_get_info(xrdvi_ctx *ctx, xrdvi_info *info);

/* Device-pointer entry points used by the torch.autograd.Function wrapper.
 * d_loc, d_raw: float [K*5]; d_eps: float [S*K*5] standard normals (with
 * XRDVI_FLAG_GATES [S*K*6]: the normals, then [S*K] logistic gate noise).
 * xrdvi_forward_dev writes the ELBO estimate (double) to d_elbo.
 * xrdvi_backward_dev recomputes the profiles (nothing of size S*K*N is kept)
 * and writes dELBO/d(loc, raw) to d_grad (float [K*10]).
 * Both are asynchronous on the context's stream. */
xrdvi_status xrdvi_forward_dev(xrdvi_ctx *ctx, const float *d_loc, const float *d_raw,
                               const float *d_eps, double *d_elbo);
xrdvi_status xrdvi_backward_dev(xrdvi_ctx *ctx, const float *d_loc, const float *d_raw,
                                const float *d_eps, float *d_grad);

/* Runs `steps` ordinary fit steps (identical to xrdvi_fit's, advancing the
 * fit) but launches each kernel individually between CUDA events on the
 * context's stream, and returns in kernel_ms[5] the mean duration per launch
 * of: sampling, profile+likelihood, backward, gradient reduction + Adam, ELBO
 * finalisation.  Blocks until done.  For measurement only; xrdvi_fit is the
 * fast path. */
xrdvi_status xrdvi_profile_steps(xrdvi_ctx *ctx, int32_t steps, float *kernel_ms);

/* Per-kernel form of xrdvi_profile_steps (the same fit steps): kernel_ms
 * [XRDVI_PROFILE_KERNELS] receives the mean duration per step (ms) of
 *   0 sampling, 1 peak ranges, 2 profile (with the far-field node sums),
 *   3 reserved (~0), 4 likelihood (with the far-field interpolation),
 *   5 backward sums (with the far field at the nodes; the side-uniform
 *   ranges only with XRDVI_FLAG_DENSE), 6 backward near sums
 *   (XRDVI_FLAG_DENSE; else ~0), 7 reserved (~0), 8 gradient reduction +
 *   Adam, 9 ELBO
 * (a kernel the configuration does not launch reads ~0; the shared-shape
 * variant's contractions count as 2 and 5).  work (NULL or
 * [XRDVI_PROFILE_WORK], HOST) receives the last step's evaluation counts,
 * (peak, point) pairs over all samples: 0 direct on side-uniform ranges, 1 on
 * mixed ranges, 2 Gaussian terms beyond the mixed range, 3 far-field (peak,
 * node) pairs; and the Gaussian terms the backward evaluates, which skips a
 * block of 64 points (a warp's pair of point rows) that lies wholly beyond a
 * peak's Gaussian reach: 4 on mixed ranges, 5 beyond them (zeros for the
 * shared-shape variant).  Blocks until done.  For measurement only. */
#define XRDVI_PROFILE_KERNELS 10
#define XRDVI_PROFILE_WORK 6
xrdvi_status xrdvi_profile_kernels(xrdvi_ctx *ctx, int32_t steps, float *kernel_ms, int64_t *work);

/* Allocation-free variant of xrdvi_elbo_grad, for callers that may not
 * allocate device memory themselves: code whose device memory is owned by
 * something else (a framework's caching allocator, a host application that
 * enforces a fixed memory budget) and that therefore cannot create a context.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  The paper
 * has no counterpart; this is an interface convenience.
 *
 * Inputs (DEVICE pointers, caller-owned): the peak table in CSR form
 * (d_offsets [K+1], d_pos / d_inten [M_total], peaks in any order within a
 * phase: the call sorts each phase by position into its scratch, a stable
 * sort like xrdvi_create's), the pattern (d_x, d_y, d_bg [N]), d_loc / d_raw
 * [K*5], d_eps [S*K*5] standard normals; cfg (HOST) gives S, the priors,
 * alpha_min and flags.  Accepted flags: XRDVI_FLAG_BF16_INT (intensities
 * rounded to bfloat16 on the device, as xrdvi_create rounds them on the host),
 * XRDVI_FLAG_NAIVE_SUM, XRDVI_FLAG_GAUSS_LIK, XRDVI_FLAG_DENSE (the profile
 * is always evaluated with every peak at every point here); IW_ELBO,
 * SHARED_SHAPES, SEC_WIDTH, FIT_BACKGROUND, FIX_R, FIX_ALPHA, AREA_NORM, GATES
 * and DEVICE_PTRS give EINVAL.  data_const = sum_i [y ln y - y - ln y!] (with
 * XRDVI_FLAG_GAUSS_LIK: -sum_i ln(2 pi max(y_i, 1)) / 2) and lambda_ =
 * 1 / max(Y - B) are the values xrdvi_create derives from the pattern
 * (xrdvi_get_info reports both).  Outputs (DEVICE): d_elbo [1] (double),
 * d_grad [K*10] (float), written asynchronously on cuda_stream (a
 * cudaStream_t; NULL is the legacy default stream).
 *
 * Validation: sizes, pointers, flags and the scratch size are checked on the
 * host (EINVAL before any work).  The device arrays are checked on the device,
 * before any kernel indexes with them, against the rules of xrdvi_create
 * (offsets[0] = 0, offsets[K] = M_total, every phase non-empty; positions in
 * (0, 180); intensities in [0, 1]; x strictly increasing in (0, 180); y
 * non-negative integers; bg finite and >= 0).  Since the call does not wait
 * for the GPU, a violation cannot change the returned status: it makes
 * *d_elbo and every d_grad entry NaN instead (lambda_ and data_const are the
 * caller's and are not re-derived).
 *
 * Scratch: one file-scope device array of XRDVI_STATIC_SCRATCH_BYTES
 * (32 MiB), which every GPU that loads the library holds until the process
 * exits.  A problem needing more (48*S*K*T + 2056*S*T + 104*S*K + 16*S +
 * 1416*K + 8*M_total + 32 bytes with T = ceil(N/256), plus up to 255 bytes of
 * alignment for each of its 18 arrays) is rejected with EINVAL before any
 * work.  The first call on a device looks up the array's device address (a
 * one-time set-up per device); make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (every element is rewritten before use, nothing needs clearing):
 * calls that overlap on the GPU — on different streams, or from different
 * threads — race, so serialise them. */
#define XRDVI_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
xrdvi_status xrdvi_elbo_grad_static(int32_t K, int32_t M_total, const int32_t *d_offsets,
                                    const float *d_pos, const float *d_inten, int32_t N,
                                    const float *d_x, const float *d_y, const float *d_bg,
                                    double data_const, double lambda_, const xrdvi_config *cfg,
                                    const float *d_loc, const float *d_raw, const float *d_eps,
                                    double *d_elbo, float *d_grad, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of fits (a runtime around the fit kernels; the
 * paper runs one fit at a time).
 *
 * A server owns a FIFO request queue, max_slots worker threads with one CUDA
 * stream each, and a stream-ordered device memory pool.  A worker takes the
 * head request as soon as its device footprint (xrdvi_footprint_bytes) fits
 * into hbm_budget next to the fits already running, so requests arriving
 * while others run are admitted as slots and memory free up, and fits in
 * different slots overlap on the GPU.  Each fit keeps its whole state on the
 * device from creation to posterior and runs the same deterministic kernels
 * as a standalone context, so its result is the same alone and in the mix.
 * All server calls are thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct xrdvi_server xrdvi_server;

typedef struct {
    int32_t iters;        /* SVI steps of the fit (>= 0)                       */
    int32_t S_post;       /* posterior draws (0: no posterior)                 */
    uint64_t post_seed;   /* Philox key of the posterior draws                 */
    int32_t top_m;        /* combinations reported (1..4096 when S_post > 0)   */
} xrdvi_request_opts;

/* Result of a served fit.  The pointer fields are CALLER buffers (NULL to
 * skip): pi [K], combos [top_m * ceil(K/64)] (layout of xrdvi_posterior),
 * combo_logp [top_m], loc / raw [K*5] (fitted q). */
typedef struct {
    int32_t status;            /* xrdvi_status of the fit itself              */
    int32_t K;
    double t_submit, t_admit, t_done;  /* seconds since xrdvi_server_create    */
    double final_elbo, log_evidence, ess, coverage_log;
    double elbo_tail_mean;     /* mean ELBO estimate over the last max(1, iters/4)
                                  steps, at most 65536 (the sub-model score of
                                  xrdvi_enumerate) */
    size_t footprint_bytes;
    double *pi;
    uint64_t *combos;
    double *combo_logp;
    float *loc, *raw;
} xrdvi_result;

typedef struct {
    int64_t queued, running, completed;
    size_t bytes_in_use, peak_bytes, budget;
    int32_t slots;
} xrdvi_server_stats;

/* Upper bound of the device bytes one fit of this size holds (problem,
 * sample workspaces, state, posterior buffers).  Host arithmetic only; 0 on
 * invalid sizes. */
size_t xrdvi_footprint_bytes(int32_t K, int32_t N, int32_t M_total, int32_t S, int32_t S_post,
                             int32_t top_m);

/* Creates a server on the current device.  hbm_budget: device bytes the
 * admitted fits may hold together; max_slots in [1, 64]. */
xrdvi_status xrdvi_server_create(size_t hbm_budget, int32_t max_slots, xrdvi_server **out);

/* Queues a fit; inputs are copied and validated when the fit runs (a bad
 * problem completes with status EINVAL).  ENOMEM if the request alone exceeds
 * the budget.  *req_id identifies it for poll / cancel. */
xrdvi_status xrdvi_server_submit(xrdvi_server *srv, const xrdvi_peaks *peaks, const xrdvi_pattern *pattern,
                                 const xrdvi_config *cfg, const xrdvi_request_opts *opts, uint64_t *req_id);

/* Waits up to timeout_ms for the request; on completion copies the result
 * into *res (res->status is the fit's own status), forgets the request and
 * returns OK.  ETIMEOUT if it is still queued or running; EINVAL for an
 * unknown or already collected id. */
xrdvi_status xrdvi_server_poll(xrdvi_server *srv, uint64_t req_id, int32_t timeout_ms, xrdvi_result *res);

/* Cancels a request that has not started (its poll reports ECANCELED);
 * EBUSY if it is running or done. */
xrdvi_status xrdvi_server_cancel(xrdvi_server *srv, uint64_t req_id);

xrdvi_status xrdvi_server_get_stats(xrdvi_server *srv, xrdvi_server_stats *stats);

/* Cancels queued requests, waits for running fits, frees everything. */
void xrdvi_server_destroy(xrdvi_server *srv);

/* Exact posterior over phase combinations for small K, by enumeration (the
 * small-K check of the method: every combination c of the K candidates is a
 * sub-model with the phases outside c removed; the paper states the problem
 * as a search over such combinations, Sec. 1 and App. A.1).
 *
 * Every non-empty combination c = 1 .. 2^K - 1 (bit k set = phase k kept,
 * in input order) is fitted by the same SVI as xrdvi_fit: cfg (S, seed,
 * priors, ...) for each, iters steps from the standard initialisation, the
 * pattern and its rate lambda = 1/max(y - B) unchanged, the Monte-Carlo noise
 * of a fit of the sub-model alone (Philox counters with the sample and phase
 * indices local to the sub-model).  Its score is the mean ELBO estimate of
 * the last max(1, iters/4) steps; under a uniform prior over combinations,
 * log p(c | Y) = ELBO_c - logsumexp_c' ELBO_c' (FP64 log-sum-exp on the GPU).
 *
 * The sub-models are fitted in batches: one batch is one problem of
 * B*S samples in which each block of S samples carries its sub-model's phase
 * mask and variational state, so one SVI step advances the whole batch in the
 * same eight kernels.  B is as large as 65536 samples and hbm_budget device
 * bytes allow (xrdvi_enumerate_footprint_bytes).  Outputs are CALLER host
 * buffers of 2^K - 1 doubles, entry c - 1 for combination c: elbo_c (may be
 * NULL) and logp_c.  Blocks until done.  EINVAL for K outside [1, 16],
 * iters < 1 or a bad problem (validated as by xrdvi_create); ENOMEM if one
 * sub-model alone exceeds hbm_budget; ENONFINITE if a score is not finite.
 * The paper has no GPU enumeration of its own. */
xrdvi_status xrdvi_enumerate(const xrdvi_peaks *peaks, const xrdvi_pattern *pattern, const xrdvi_config *cfg,
                             int32_t iters, size_t hbm_budget, double *elbo_c, double *logp_c);

/* Device bytes of one enumeration batch of nsub sub-models (host arithmetic;
 * 0 on invalid sizes). */
size_t xrdvi_enumerate_footprint_bytes(int32_t K, int32_t N, int32_t M_total, int32_t S, int32_t nsub);

/* Gate variant: the logits a [K] and the objective's gradient in them from
 * the last xrdvi_elbo_grad [K] (each may be NULL), HOST buffers.  EINVAL
 * without the flag. */
xrdvi_status xrdvi_get_gates(xrdvi_ctx *ctx, float *logits, float *grad);

/* Fitted-background variant: beta [3], the background curve B(beta) [N] and
 * the objective's gradient in beta from the last xrdvi_elbo_grad [3] (each
 * may be NULL), HOST buffers.  EINVAL without the flag. */
xrdvi_status xrdvi_get_background(xrdvi_ctx *ctx, float *beta, float *bg_curve, float *grad_beta);

/* Tensor-core GEMM used by the shared-shape variant (XRDVI_FLAG_SHARED_SHAPES),
 * exported for testing: C[M x N] = A[M x K] . B[N x K]^T with A, B, C DEVICE
 * row-major FP32 matrices (K contiguous in A and B; leading dimensions lda,
 * ldb, ldc in elements), computed on the 5th-generation tensor cores
 * (tcgen05.mma kind::tf32, accumulators in tensor memory) with the 3xTF32
 * split a = a_hi + a_lo (a_hi = a truncated to TF32): a b ~ a_hi b_hi +
 * a_hi b_lo + a_lo b_hi, FP32 accumulation, split-K partials added in a
 * fixed order (deterministic).  K, lda and ldb must be multiples of 4 with
 * lda, ldb >= K, ldc >= N, and A, B 16-byte aligned (EINVAL otherwise).
 * Allocates its scratch on cuda_stream (stream-ordered) and synchronises it;
 * ETIMEOUT if a pipeline wait gave up.  No counterpart in the paper. */
xrdvi_status xrdvi_gemm_nt_tf32x3(int32_t M, int32_t N, int32_t K, const float *d_A, int32_t lda,
                                  const float *d_B, int32_t ldb, float *d_C, int32_t ldc, void *cuda_stream);

/* The Monte-Carlo noise generator, exported for known-answer tests: Philox4x32
 * with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11), run on the GPU by the
 * same device function that draws every sample's normals (Box-Muller of the
 * top 24 bits of each word; the reparameterised draw of Sec. 3.2).  Block i
 * takes counter ctr[4i..4i+3] and key key[2i..2i+1] and writes out[4i..4i+3]
 * (HOST arrays, caller-owned).  0 <= n <= 2^20 (EINVAL otherwise).  Allocates
 * and frees a small device buffer on a private stream; blocks until done.
 * No counterpart in the paper, which does not name its generator. */
xrdvi_status xrdvi_philox4x32_10(int32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* Bounds-check build.  The library compiled with XRDVI_DEBUG defined (the
 * Python binding loads it when the environment has XRDVI_DEBUG=1) clamps every
 * peak-table index and every decoded peak range of the profile kernels into
 * bounds and records the number of the first check that failed in a device
 * word (1-3 table lookups, 4-9 the range bounds), without a trap or an early
 * exit, so a fault becomes a status: xrdvi_fit, xrdvi_elbo_grad and
 * xrdvi_fit_batch return ECUDA naming the check.  xrdvi_debug_word copies the
 * word to *word (0: no violation) and clears it if reset is non-zero.
 * xrdvi_debug_selftest runs one lookup past the end of a one-entry table
 * through the same check (the access itself is clamped to the table) so that a
 * test can see the word set.  In a regular build both return EINVAL.  No
 * counterpart in the paper. */
xrdvi_status xrdvi_debug_word(int32_t *word, int32_t reset);
xrdvi_status xrdvi_debug_selftest(void);

/* Thread-local message of the last failing call ("" if none). */
const char *xrdvi_last_error(void);

/* Library version string. */
const char *xrdvi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XRDVI_H */
