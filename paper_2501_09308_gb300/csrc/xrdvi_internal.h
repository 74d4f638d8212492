// Internal declarations shared by the kernel and host translation units of
// the xrdvi library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/xrdvi.h"

namespace xrdvi {

// NVTX range over a host scope (a profiler timeline shows create, fit,
// posterior and the server's admission, slices and posteriors).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Profile kernels: 8 warps per block; each warp owns one (sample, 2-theta
// tile) work item of 32 * kPts consecutive points, lane l holding points
// l, l+32, ..., l+32*(kPts-1) of the tile.
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kPts = 8;
constexpr int kTile = 32 * kPts;
// Gradient partial sums per (sample, phase, tile) written by the backward.
constexpr int kGradSums = 10;
// Phases are split into up to kMaxChunks chunks of similar peak count so that
// the profile kernels have enough equal-sized work items to fill the GPU.
constexpr int kMaxChunks = 8;
constexpr int kItemsPerWarp = 8;
constexpr int kGredVals = 11;      // per-(phase, sample block) gradient partials: loc 5, raw 5, gate 1   // profile work items per resident warp the phase chunking aims for
// Far field: the Lorentzian tails of peaks more than kFarGap tile half-widths
// beyond a 2-theta tile (and beyond their Gaussian reach) are summed at
// kFarNodes Chebyshev nodes of the tile's span and interpolated at its points.
constexpr int kFarNodes = 32;
constexpr float kFarGap = 0.5f;
// Second far-field level: super-tiles of kSuperTiles tiles with their own
// kFarNodes nodes take the peaks far beyond the super-tile; their node sums
// are translated to (forward) and from (backward) the tiles' nodes.
constexpr int kSuperTiles = 4;
// Largest interpolation table (kFarNodes weights per point) the far field uses.
constexpr size_t kFarMaxLamBytes = static_cast<size_t>(64) << 20;
// Work counters of the profile kernels of one sample set.
constexpr int kCounters = 4;
// Sample blocks per phase in the gradient reduction.
constexpr int kGradBlocks = 16;

// Fits one multi-fit launch can hold (continuous batching), and the block
// ranges of the fits in one such launch: fit f owns blocks [start[f], start[f+1]).
constexpr int kMaxBatch = 64;
struct FitMap {
    int n = 0;
    int start[kMaxBatch + 1] = {0};
};

// The Gaussian component 2^-u of a peak is evaluated only for warps with a
// point inside the peak's reach u < kGaussU; beyond it 2^-u < 2^-128, which
// flushes to zero in single precision anyway.
constexpr float kGaussU = 128.0f;

// Limits checked at create time.
constexpr int kMaxK = 1024;
constexpr int kMaxPeaks = 24000;
constexpr int kMaxS = 65536;
constexpr int kMaxN = 1 << 24;
constexpr int kTraceCap = 1 << 16;   // ring buffer of ELBO values (power of two)

// Per (sample, phase) constants of the profile kernels (64 bytes).  With
// d = x - p - mu and side width w_side = w (d < 0) or alpha*w (d >= 0):
//   s(d) = 2 / w_side,  t = s(d) d,  u = t^2 = (2 d / w_side)^2,
//   G = 2^-u = exp(-4 ln2 (d/w_side)^2),  L = 1 / (1 + u).
// On ranges where every point lies on one side of the peak,
// t = s_side (x - p) + (-s_side mu) with the side's sl / sr and nslmu / nsrmu.
struct __align__(16) PhaseConst {
    float mu;            // peak shift
    float hl, hg;        // h * r, h * (1 - r)
    float rl, rr;        // Gaussian reach left / right of the peak (degrees)
    float sl, sr;        // 2 / w (d < 0), 2 / (alpha w) (d >= 0)
    float nslmu, nsrmu;  // -sl * mu, -sr * mu
    float absent;        // 1: phase removed from this sample's sub-model (no peaks evaluated)
    float pad[6];
};

struct PriorConst {
    double lambda;        // rate of the exponential prior on h
    double mu_sd;
    double alpha_mean, alpha_sd;
    double w_shape, w_rate, lgamma_w_shape;
    double alpha_min;
    double lp_const;      // parameter-free part of ln p(theta) per phase
};

// A tensor-core GEMM out[M x N] = A[M x K] . B[N x K]^T with its TMA
// descriptors (A, B as TF32 hi / lo parts), built once for fixed buffers.
struct GemmPlan {
    CUtensorMap tAh, tAl, tBh, tBl;
    int M = 0, N = 0, K = 0, ldo = 0, tn = 64, nkb = 0, kb_per_split = 1, splits = 1;
    float *out = nullptr, *work = nullptr;
    int *err = nullptr;
};

// Buffers of one sample set (the fit's S, or the posterior's S_post).
struct Workspace {
    int S = 0;
    float *eps = nullptr;        // [S*K*5] standard normals used
    float *theta = nullptr;      // [S*K*5] physical parameters
    PhaseConst *cst = nullptr;   // [S*K]
    double *lpj = nullptr;       // [S] log prior + log Jacobian
    double *lq = nullptr;        // [S] log q(u)
    double *ll = nullptr;        // [S] log-likelihood
    float *g = nullptr;          // [S*Npad] y/f - 1 (0 on padding)
    double *llpart = nullptr;    // [S*T] deviance partial sums per tile
    float *gpart = nullptr;      // [S*K*T*kGradSums] gradient partial sums (fit only)
    float *fpart = nullptr;      // [C*S*Npad] partial profiles per phase chunk
    ushort4 *ranges = nullptr;   // [S*K*T] peak index ranges per (sample, phase, tile)
    ushort2 *franges = nullptr;  // [S*K*T] end of the far peaks below / start of those above (far field)
    ushort2 *sranges = nullptr;  // [S*K*Tg] the same for the super-tiles' far peaks
    float *fnode = nullptr;      // [kMaxChunks*S*T*kFarNodes] far-field node sums of each phase chunk
    float *fnode2 = nullptr;     // [kMaxChunks*S*Tg*kFarNodes] the same at the super-tiles' nodes
    float *wfar = nullptr;       // [S*T*kFarNodes] sum_i g_i lam_p(x_i) per tile (fit only)
    float *wfar2 = nullptr;      // [S*T*kFarNodes] the tile's part of the super-tile's node weights (fit only)
    int *counters = nullptr;     // [kCounters] work counters of the profile kernels
    double *gred = nullptr;      // [K*kGradBlocks*10] gradient partials per sample block (fit only)
    int *tickets = nullptr;      // [K] arrival tickets of the gradient reduction (fit only)
    size_t fpart_cap = 0;        // elements allocated for fpart
    // Sub-model batch: the S samples form B blocks of S_sub, block b fits the
    // sub-model keeping the phases set in mask[b] (bit k = phase k, K <= 32),
    // with its own variational parameters and Adam state [B*K*...].  B = 1 and
    // mask = null: one model over all phases.
    int B = 1, S_sub = 0;
    const uint32_t *mask = nullptr;   // [B] device
    double *tail_sum = nullptr;       // [B] sum of the ELBO estimates from step tail_start on
    float *bgpart = nullptr;          // [S*T*3] per-(sample, tile) sums g B(beta) T_j (fitted background)
    float *gzy = nullptr;             // [S*K*2] gate z and y of every draw and phase (gates)
    double *iw = nullptr;             // [S] normalised importance weights (importance-weighted
                                      //     objective; null: the ELBO, weights 1/S)
    // Shared-shape variant (one shape draw per step for all samples): the
    // profile and the backward's sums become GEMMs over phase profiles.
    bool shared = false;
    // GEMM operands are kept split for the 3xTF32 products: each array holds
    // the TF32 hi parts followed by the lo parts (2x the size given)
    int Kpad = 0;                     // phases padded to a multiple of 32
    float *H = nullptr;               // [S*Kpad] intensities h_sk (GEMM A of the forward)
    float *Ct = nullptr;              // [Npad*Kpad] phase profiles C_k(x_i), point-major
    float *D = nullptr;               // [K*10*Npad] derivative profiles D_jk(x_i) (GEMM B of the backward)
    float *ghl = nullptr;             // [S*Npad] y/f - 1 (GEMM A of the backward)
    float *gemm_work = nullptr;       // split-K partials of the backward GEMM
    int gemm_splits = 1;
    int *gemm_err = nullptr;          // set if a tensor-core pipeline wait gives up
    GemmPlan plan_fwd, plan_bwd;      // the forward and backward contractions
    int tail_start = 0;
    int C = 1;                   // phase chunks
    int chunk[kMaxChunks + 1] = {0};
    size_t bytes = 0;
};

struct Problem {
    int K = 0, N = 0, Npad = 0, T = 0, Mtot = 0;
    float *pos = nullptr;        // [Mtot] sorted by position within each phase
    float *inten = nullptr;      // [Mtot] (f32 copy; bf16-rounded with the flag)
    int *off = nullptr;          // [K+1]
    float *x = nullptr, *y = nullptr, *bg = nullptr;   // [N]
    double *isum = nullptr;      // [K] sum_m I_m per phase
    double csum = 0.0;           // sum_i [y ln y - y - ln y!]
    PriorConst prior{};
    size_t smem = 0;             // dynamic shared memory of the backward profile kernels
    size_t smem_fwd = 0;         // ... of the forward kernel (compact table)
    bool wide = false;           // backward peak table stored as (-p, -p, I, I) float4
    // Far field (off: every peak evaluated at every point)
    bool far = false;
    float *node_x = nullptr;     // [T*kFarNodes] Chebyshev nodes of each tile's span
    float *node_c = nullptr;     // [T*kFarNodes] cos(x/2) at the nodes (angle-dependent width)
    float *lam = nullptr;        // [T*kFarNodes*kTile] Lagrange weights lam_p(x_i) of the tile's points
    int *far_order = nullptr;    // [K] phases by decreasing peak count (work balance)
    int Tg = 0;                  // super-tiles (second far-field level; 0: one level)
    float *node_x2 = nullptr;    // [Tg*kFarNodes] nodes of each super-tile's span
    float *node_c2 = nullptr;    // [Tg*kFarNodes] cos(x/2) there (angle-dependent width)
    float *sgap = nullptr;       // [Tg] distance beyond a super-tile from which a peak is super-far
    float *Mf = nullptr;         // [T*kFarNodes*kFarNodes] Mf[(t, P, p)] = super-level weight of node P at tile node p
    float *Mb = nullptr;         // [T*kFarNodes*kFarNodes] the same as Mb[(t, p, P)]
    bool gauss = false;          // Gaussian likelihood variant (variance max(y, 1))
    bool fix_r = false, fix_alpha = false;   // r / alpha held at r_value / alpha_value
    bool area_norm = false;      // area-normalised profiles (h = integrated intensity)
    // binary-Concrete phase gates: logits a[K], temperature, prior logit
    bool gates = false;
    float gate_tau = 2.f / 3.f, gate_a0 = 0.f;
    float *gate_a = nullptr, *m_gate = nullptr, *v_gate = nullptr, *grad_gate = nullptr;   // [K]
    float r_value = 0.5f, alpha_value = 1.f;
    bool sec = false;            // angle-dependent width variant (side widths times sec(x/2))
    float *csec = nullptr;       // [N] cos(x_i / 2) for that variant
    float sec_max = 1.f;         // max_i sec(x_i / 2)
    // fitted-background variant: B(beta) = B exp(sum_j beta_j T_j(z))
    bool bgfit = false;
    float bg_sd = 0.1f;
    float *beta = nullptr, *m_beta = nullptr, *v_beta = nullptr;   // [3] coefficients, Adam moments
    float *Tb = nullptr;         // [3*N] Chebyshev terms T_j(z_i)
    float *Bb = nullptr;         // [N] B(beta) of the current step
    int grid_fwd = 0, grid_bwd = 0, grid_bwd_direct = 0, grid_fwd_direct = 0;
    int *nonfinite = nullptr;    // [1] set by the gradient reduction on a NaN / infinite gradient (may be null)
};

// --- kernel launchers (xrdvi_kernels.cu) ------------------------------------
// Sampling: eps_in (device, may be null) or Philox(seed, tag, step).
// d_step: device step counter (null: use `step`); d_iter: receives the step
// used (may be null); ent: receives the entropy of q (may be null).
void launch_sample(const Problem &P, Workspace &W, const float *loc, const float *raw,
                   const float *eps_in, uint64_t seed, uint32_t tag, const int *d_step,
                   uint32_t step, int *d_iter, double *ent, cudaStream_t st);
// marks (may be null): events recorded between the kernels, for per-kernel
// timing: forward after k_ranges, the direct profile and the far field [3];
// backward after the side-uniform and the near sums [2].
void launch_forward(const Problem &P, Workspace &W, float *f_out, bool naive, cudaStream_t st,
                    cudaEvent_t *marks = nullptr);
void launch_backward(const Problem &P, Workspace &W, cudaStream_t st, cudaEvent_t *marks = nullptr);
// Reduces gradient partials per phase and optionally applies Adam (when
// grad_out or adam), then finalises the ELBO (when elbo_out or trace: writes
// ll[S], *elbo_out, trace[step] and advances *d_step).
struct AdamConst { float lr, b1, b2, eps; };
void launch_grad(const Problem &P, Workspace &W, const float *loc_in, const float *raw_in,
                 float *loc_out, float *raw_out, float *grad_out, bool adam, AdamConst ac,
                 float *m, float *v, const int *d_iter, int *d_step, const double *ent,
                 double *elbo_out, double *trace, cudaStream_t st);
// Posterior: per-sample log weights and inclusion bits, marginals, IS
// evidence, and the best-first top-M combinations.
struct PostBuffers {
    double *logw = nullptr;      // [S]
    uint8_t *bits = nullptr;     // [S*K]
    double *pi = nullptr;        // [K]
    double *scalars = nullptr;   // [4]: log_evidence, ess, coverage_log, (spare)
    uint64_t *combos = nullptr;  // [top_m * W]
    double *combo_logp = nullptr;// [top_m]
    int *order = nullptr;        // [K]
    double *cost = nullptr;      // [K]
    double *heap_cost = nullptr; // [2*top_m + 2]
    int *heap_node = nullptr;    // [2*top_m + 2]
    uint64_t *node_mask = nullptr; // [(2*top_m + 2) * ceil(K/64)] flip sets
    int *node_last = nullptr;    // [2*top_m + 2]
    int cap_S = 0, cap_M = 0;
};
void launch_posterior(const Problem &P, Workspace &W, PostBuffers &B, int top_m, cudaStream_t st);

// Error reporting shared by the host translation units (sets the thread-local
// message returned by xrdvi_last_error).
xrdvi_status report_error(xrdvi_status st, const std::string &msg);

// Context creation; with a pool, every device buffer comes from the pool by
// stream-ordered allocation on `stream` (which the context then uses and does
// not own), so creating and destroying contexts never synchronises the device.
xrdvi_status create_context(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                            cudaMemPool_t pool, cudaStream_t stream, xrdvi_ctx **out);
// A context fitting nsub sub-models of the problem at once: sub-model b keeps
// the phases set in masks[b] (K <= 32) and gets its own variational
// parameters, Adam state and cfg->S samples; one SVI step advances all of them
// in the same kernels.  The ELBO estimates of every step from tail_start on
// are summed per sub-model (tail sums, read by batch_tail_sums).  Only fit is
// meaningful on such a context.
xrdvi_status create_batch_context(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                                  int nsub, const uint32_t *masks, cudaMemPool_t pool, cudaStream_t stream,
                                  xrdvi_ctx **out);
xrdvi_status batch_set_tail(xrdvi_ctx *c, int tail_start);
// Copies the nsub tail sums (FP64) to host memory.
xrdvi_status batch_tail_sums(xrdvi_ctx *c, double *host);

// Continuous batching: one SVI step of several fits in shared launches
// (sampling, ranges and the gradient one launch each for the whole batch; the
// profile and likelihood launches per group of small fits of equal occupancy,
// a fit's own kernels for a fit that fills the GPU alone).  FitStep names a
// fit's device state;
// only fits that run the plain far-field step qualify (multi_fit_eligible):
// no shared shapes, angle-dependent width, fitted background, naive sums,
// importance weights or sub-model batches.
struct FitStep {
    const Problem *P = nullptr;
    Workspace *W = nullptr;
    float *loc = nullptr, *raw = nullptr, *m = nullptr, *v = nullptr;
    int *iter = nullptr, *step = nullptr;
    double *ent = nullptr, *elbo = nullptr, *trace = nullptr;
    uint64_t seed = 0;
    AdamConst ac{};
};
struct MultiStepPlan;
MultiStepPlan *multi_plan_create(int cap);   // launch plan for up to cap <= kMaxBatch fits (host memory)
void multi_plan_destroy(MultiStepPlan *p);
bool multi_fit_eligible(const Problem &P, const Workspace &W, bool naive, bool iw);
// Builds the batch's kernel arguments and block maps (host only: the
// arguments are passed by value with every launch; st is unused).
bool multi_plan_set(MultiStepPlan *p, const FitStep *fits, int n, int sm_count, cudaStream_t st);
// Enqueues one SVI step (sample, ranges, profile, likelihood, backward,
// gradient + Adam + ELBO) of every fit of the plan.
void multi_plan_launch_step(const MultiStepPlan *p, cudaStream_t st);

// Context access for the continuous-batching server (xrdvi_capi.cu).
void ctx_fit_step(xrdvi_ctx *c, FitStep *out);
bool ctx_multi_eligible(const xrdvi_ctx *c);
void ctx_enqueue_steps(xrdvi_ctx *c, int n, cudaStream_t st);   // n fit steps, kernel by kernel
void ctx_advance(xrdvi_ctx *c, int n);                          // host step counter += n
// `steps` SVI steps of a batch (multi-fit launches of the plan, if any, then
// the solo contexts' own kernels) captured on stream cap as one graph.
xrdvi_status capture_batch_steps(const MultiStepPlan *plan, xrdvi_ctx *const *solo, int nsolo, int steps,
                                 cudaStream_t cap, cudaGraphExec_t *out);
cudaStream_t ctx_stream(const xrdvi_ctx *c);
xrdvi_status ctx_read_trace(xrdvi_ctx *c, int n, double *host);  // last n ELBO estimates

// Host validation of a problem and config (the checks of xrdvi_create).
xrdvi_status validate_problem(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg);

// logp[c] = elbo[c] - logsumexp(elbo[0..n)) in FP64 with a fixed reduction
// order (one block).
void launch_enum_lse(const double *elbo, int n, double *logp, cudaStream_t st);

// Bounds-check build (XRDVI_DEBUG): whether it is one, the device word of the
// first violated check (0: none; cleared when reset), and a one-lookup
// self-test of the check (d_out: one device float).
bool debug_build();
int debug_word(bool reset);
cudaError_t debug_selftest(float *d_out);

// Philox4x32-10 blocks of n (counter [4], key [2]) pairs, device arrays.
void launch_philox_words(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st);

// Fitted-background variant: B(beta) for the step (before the likelihood),
// and after the gradient sums the beta gradient (weights 1/S or the
// importance weights) with Adam on beta (adam) or written to grad_out [3].
void launch_bg_curve(const Problem &P, cudaStream_t st);
void launch_bg_grad(const Problem &P, Workspace &W, bool adam, AdamConst ac, const int *d_iter, float *grad_out,
                    cudaStream_t st);

// k_lik alone (f = B + chunk partials, deviance, g), over the first C chunks.
void launch_lik(const Problem &P, Workspace &W, float *f_out, int C, cudaStream_t st);
// Shared-shape variant (xrdvi_tc.cu): phase and derivative profiles of sample
// 0's shapes, the forward GEMM into fpart and k_lik; the backward GEMM into
// gpart (one tile per (sample, phase)).
void launch_shared_forward(const Problem &P, Workspace &W, float *f_out, cudaStream_t st);
void launch_shared_backward(const Problem &P, Workspace &W, cudaStream_t st);

// Tensor-core GEMM (xrdvi_tc.cu): out[M x N] = A[M x K] . B[N x K]^T, A and B
// given as TF32 hi / lo parts (launch_tf32_split), row-major with K contiguous
// (K, lda, ldb multiples of 4, 16-byte aligned), loaded by TMA and multiplied
// 3xTF32 on tcgen05 with FP32 accumulation; split-K partials (work,
// gemm_workspace_floats) are added in a fixed order.  gemm_plan encodes the
// TMA descriptors (false if that fails); err (device int) is set if an
// mbarrier wait gives up.
size_t gemm_smem_bytes();
cudaError_t gemm_configure();   // shared-memory attribute of the GEMM kernel (call before capture)
int gemm_splits(int M, int N, int K, int sm_count);
size_t gemm_workspace_floats(int M, int N, int splits);
bool gemm_plan(GemmPlan &p, int M, int N, int K, const float *Ahi, const float *Alo, int lda, const float *Bhi,
               const float *Blo, int ldb, float *out, int ldo, int splits, float *work, int *err);
void launch_gemm(const GemmPlan &p, cudaStream_t st);
void launch_tf32_split(const float *a, size_t n, float *hi, float *lo, cudaStream_t st);

// TF32 high part of a float (low 13 mantissa bits cleared); a - hi is exact.
__device__ __forceinline__ float tf32_hi(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u); }

// Occupancy-based persistent grid sizes.
void configure_grids(Problem &P, int sm_count);
// Phase chunks for a sample set of S samples: enough work items for about
// four per resident warp, chunk boundaries balancing the peak counts
// (offsets: host copy of the CSR offsets, K+1 entries).
void choose_chunks(const Problem &P, const int *offsets, int S, Workspace &W, int max_chunks = kMaxChunks);

}  // namespace xrdvi
