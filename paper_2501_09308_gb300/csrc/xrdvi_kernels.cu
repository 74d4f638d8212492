// CUDA kernels of the Monte-Carlo ELBO step (arXiv 2501.09308), sm_103a.
//
//   k_sample    reparameterised draw u = loc + softplus(raw) eps (Sec. 3.2),
//               transforms to (h, mu, w, r, alpha), per-(s,k) profile
//               constants, log prior + log Jacobian (Sec. 2.2, Appendix B.2)
//   k_forward   f = B + sum_k h_k sum_m I_m V over all phases, peaks and
//               points (the triple loop of Sec. 2.3), then the Poisson
//               log-likelihood (Appendix A.2) in deviance form and y/f - 1
//   k_backward  profile recomputation with the likelihood gradient sums
//   k_grad      deterministic reduction to dELBO/d(loc, raw), Adam, ELBO
//   k_post_*    posterior over phase combinations (area ratio >= 1 %)
//
// The profile kernels are bound by the FP32 and MUFU pipes: per evaluation one
// reciprocal (Lorentzian) and, only near a peak, one exp2 (Gaussian).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math_constants.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "xrdvi_internal.h"

namespace xrdvi {
namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2Pi = 1.8378770664093454836;  // ln(2 pi)

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the two-multiplier
// bijection with Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0];
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ float u01(uint32_t v) {
    return (static_cast<float>(v >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float softplusf(float x) {
    return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x));
}

__device__ __forceinline__ float sigmoidf(float x) {
    if (x >= 0.f) return 1.f / (1.f + expf(-x));
    const float e = expf(x);
    return e / (1.f + e);
}

// Area of the unit-height split pseudo-Voigt of FWHM w (left) and alpha w
// (right): ((1 + alpha) w / 2) [(1 - r) sqrt(pi / ln 2) / 2 + r pi / 2].
__device__ __forceinline__ float area_factorf(float w, float alpha_c, float r) {
    constexpr float kAG = 1.0644670194312262f;   // sqrt(pi / ln 2) / 2
    constexpr float kAL = 1.5707963267948966f;   // pi / 2
    return 0.5f * (1.f + alpha_c) * w * fmaf(r, kAL - kAG, kAG);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum with a fixed reduction tree (deterministic).  `sh`
// holds blockDim.x/32 doubles.  Result valid in every thread.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double t = (l < nw) ? sh[l] : 0.0;
    t = warp_sum(t);
    return t;
}

__device__ double block_max(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double t = (l < nw) ? sh[l] : -CUDART_INF;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

// ---------------------------------------------------------------------------
// Sampling
// ---------------------------------------------------------------------------
struct SampleArgs {
    int S, K;
    const float *loc, *raw, *eps_in;
    uint32_t key0, key1, tag, step;
    const int *d_step;
    int *d_iter;
    double *ent;
    PriorConst pr;
    float *eps, *theta;
    PhaseConst *cst;
    double *lpj, *lq;
    int *counters;
    int *tickets;   // [B*K] arrival tickets of k_grad, zeroed here
    int B, S_sub;
    const uint32_t *mask;  // [B] phases kept by each sub-model (null: all)
    float reach_scale;     // Gaussian reach factor: max sec(x/2) of the pattern (angle-dependent width), else 1
    const float *beta;     // [3] fitted-background coefficients (null: fixed background)
    float bg_sd;
    int fix_r, fix_a;      // r / alpha held fixed (model constants, not in q)
    float r_value, a_value;
    int area_norm;         // area-normalised profiles: h / a(w, alpha, r) scales the profile
    const float *gate_a;   // [K] gate logits (null: no gates)
    float gate_tau, gate_a0;   // temperature, prior logit
    float *gzy;            // [S*K*2] gate z and y per draw and phase
    int shared;            // shape noise of every sample = sample 0's (shared-shape variant)
    float *H;              // [S*Kpad] h_sk for the forward GEMM (shared-shape variant)
    int Kpad;
    // FP32 copies of the prior constants used per (s, k)
    float pr_lambda, pr_mu_isd, pr_alpha_mean, pr_alpha_isd, pr_wsm1, pr_wrate;
};

// Block indices of a kernel body: the launch's own (re-read from the special
// register wherever used, which keeps register pressure as in a plain kernel)
// or a fixed value (a block of a multi-fit launch, relative to its fit).
struct GridBlock {
    __device__ __forceinline__ int x() const { return static_cast<int>(blockIdx.x); }
    __device__ __forceinline__ int y() const { return static_cast<int>(blockIdx.y); }
};
struct FixedBlock {
    int bx, by;
    __device__ __forceinline__ int x() const { return bx; }
    __device__ __forceinline__ int y() const { return by; }
};

// Draw s of one sample set (one block of 128 threads per draw).
__device__ __forceinline__ void sample_body(const SampleArgs &a, int s) {
    __shared__ double sh[4];
    const uint32_t step = a.d_step ? static_cast<uint32_t>(*a.d_step) : a.step;
    if (s == 0 && threadIdx.x == 0) {
        if (a.d_iter) *a.d_iter = static_cast<int>(step);
        for (int i = 0; i < kCounters; ++i) a.counters[i] = 0;  // work counters of the profile kernels
    }
    const float sq = sqrtf(kGaussU);
    // sub-model of this sample; the noise counters use the sample and phase
    // indices local to the sub-model, as a fit of the sub-model alone would
    const int b = s / a.S_sub, s_loc = s - b * a.S_sub;
    const uint32_t mk = a.mask ? a.mask[b] : 0u;
    const float *loc = a.loc + static_cast<size_t>(b) * a.K * 5;
    const float *raw = a.raw + static_cast<size_t>(b) * a.K * 5;
    double acc = 0.0, accq = 0.0;
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const size_t base = (static_cast<size_t>(s) * a.K + k) * 5;
        if (a.mask && !((mk >> k) & 1u)) {
            PhaseConst pc = {};
            pc.absent = 1.f;
            a.cst[static_cast<size_t>(s) * a.K + k] = pc;
#pragma unroll
            for (int j = 0; j < 5; ++j) a.theta[base + j] = 0.f;
            continue;
        }
        const uint32_t kl = a.mask ? static_cast<uint32_t>(__popc(mk & ((1u << k) - 1u))) : static_cast<uint32_t>(k);
        float e[8];
        // shared-shape variant: h takes this sample's noise, the shapes sample 0's
        const size_t sh_base = a.shared ? (static_cast<size_t>(b) * a.S_sub * a.K + k) * 5 : base;
        if (a.eps_in) {
            e[0] = a.eps_in[base];
#pragma unroll
            for (int j = 1; j < 5; ++j) e[j] = a.eps_in[sh_base + j];
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t c[4] = {static_cast<uint32_t>(s_loc), kl, step,
                                 a.tag * 256u + static_cast<uint32_t>(j)};
                philox4x32_10(c, a.key0, a.key1);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float r1 = u01(c[2 * q]), r2 = u01(c[2 * q + 1]);
                    const float rad = sqrtf(-2.0f * logf(r1));
                    float sn, cs;
                    sincospif(2.0f * r2, &sn, &cs);
                    e[4 * j + 2 * q] = rad * cs;
                    e[4 * j + 2 * q + 1] = rad * sn;
                }
            }
            if (a.shared && s_loc != 0) {
                const float e0 = e[0];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint32_t c[4] = {0u, kl, step, a.tag * 256u + static_cast<uint32_t>(j)};
                    philox4x32_10(c, a.key0, a.key1);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float r1 = u01(c[2 * q]), r2 = u01(c[2 * q + 1]);
                        const float rad = sqrtf(-2.0f * logf(r1));
                        float sn, cs;
                        sincospif(2.0f * r2, &sn, &cs);
                        e[4 * j + 2 * q] = rad * cs;
                        e[4 * j + 2 * q + 1] = rad * sn;
                    }
                }
                e[0] = e0;
            }
        }
        float u[5], sig[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            sig[j] = softplusf(raw[k * 5 + j]);
            u[j] = fmaf(sig[j], e[j], loc[k * 5 + j]);
            a.eps[base + j] = e[j];
        }
        if (a.fix_r) u[3] = 0.f;   // fixed parameters: not drawn (their noise is unused)
        if (a.fix_a) u[4] = a.a_value;
        const float h = expf(u[0]);
        const float mu = u[1];
        const float w = expf(u[2]);
        const float r = a.fix_r ? a.r_value : sigmoidf(u[3]);
        const float al = u[4];
        a.theta[base + 0] = h;
        a.theta[base + 1] = mu;
        a.theta[base + 2] = w;
        a.theta[base + 3] = r;
        a.theta[base + 4] = al;
        const float ac = al > static_cast<float>(a.pr.alpha_min) ? al : static_cast<float>(a.pr.alpha_min);
        const float wl = w, wr = ac * w;
        const float sl = 2.0f / wl, sr = 2.0f / wr;
        // area-normalised profiles divide by the area of the unit-height shape
        // a(w, alpha, r) = ((1 + alpha) w / 2) [(1 - r) sqrt(pi/ln2)/2 + r pi/2]
        float he = a.area_norm ? __fdiv_rn(h, area_factorf(w, ac, r)) : h;
        float glp = 0.f;
        if (a.gate_a) {
            // binary-Concrete gate: y = (a + L)/tau with logistic noise L, z = sigmoid(y)
            // scales the profile; the draw's log joint gains ln p(y) - ln q(y)
            float L;
            if (a.eps_in) {
                L = a.eps_in[static_cast<size_t>(5) * a.S * a.K + static_cast<size_t>(s) * a.K + k];
            } else {
                uint32_t c[4] = {static_cast<uint32_t>(s_loc), kl, step, a.tag * 256u + 2u};
                philox4x32_10(c, a.key0, a.key1);
                // ln u - ln(1 - u) with 1 - u taken from the complemented counter
                // word (exactly 1 - u in real arithmetic), so that the rounding
                // of u to 1.0f near the top never gives an infinite L
                L = logf(u01(c[0])) - logf(u01(~c[0]));
            }
            const float ga = a.gate_a[k], tau = a.gate_tau;
            const float y = __fdiv_rn(ga + L, tau);
            const float z = sigmoidf(y);
            const float lq = logf(tau) + ga - tau * y - 2.f * softplusf(ga - tau * y);
            const float lp = logf(tau) + a.gate_a0 - tau * y - 2.f * softplusf(a.gate_a0 - tau * y);
            glp = lp - lq;
            he *= z;
            a.gzy[(static_cast<size_t>(s) * a.K + k) * 2] = z;
            a.gzy[(static_cast<size_t>(s) * a.K + k) * 2 + 1] = y;
        }
        if (a.H) {   // TF32 hi / lo parts of the profile scale for the forward GEMM
            const float hh = tf32_hi(he);
            a.H[static_cast<size_t>(s) * a.Kpad + k] = hh;
            a.H[static_cast<size_t>(a.S) * a.Kpad + static_cast<size_t>(s) * a.Kpad + k] = he - hh;
        }
        PhaseConst pc;
        pc.mu = mu;
        pc.hl = he * r;
        pc.hg = he * (1.0f - r);
        pc.rl = 0.5f * sq * wl * a.reach_scale;
        pc.rr = 0.5f * sq * wr * a.reach_scale;
        pc.sl = sl;
        pc.sr = sr;
        pc.nslmu = -sl * mu;
        pc.nsrmu = -sr * mu;
        pc.absent = 0.f;
        pc.pad[0] = pc.pad[1] = pc.pad[2] = pc.pad[3] = pc.pad[4] = pc.pad[5] = 0.f;
        a.cst[static_cast<size_t>(s) * a.K + k] = pc;
        // log prior (Sec. 2.2, Appendix B.2) + log Jacobian of the transform:
        // the parameter-free part is the host constant lp_const; the rest is
        // O(1) per phase and evaluated in FP32 (ln w = u_w exactly), summed in FP64.
        const float zm = mu * a.pr_mu_isd;
        const float za = a.fix_a ? 0.f : (al - a.pr_alpha_mean) * a.pr_alpha_isd;   // fixed: no prior
        const float lpf = -a.pr_lambda * h - 0.5f * zm * zm - 0.5f * za * za + a.pr_wsm1 * u[2] - a.pr_wrate * w;
        const float ljf = u[0] + u[2] - (a.fix_r ? 0.f : softplusf(-u[3]) + softplusf(u[3]));
        acc += a.pr.lp_const + static_cast<double>(lpf) + static_cast<double>(ljf) + static_cast<double>(glp);
        if (a.lq) {
            float q = 0.f;
            int nfree = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                if ((j == 3 && a.fix_r) || (j == 4 && a.fix_a)) continue;   // not part of q
                q += -0.5f * e[j] * e[j] - logf(sig[j]);
                ++nfree;
            }
            accq += static_cast<double>(q) - 0.5 * nfree * kLog2Pi;
        }
    }
    if (s == 0 && a.tickets)
        for (int k = threadIdx.x; k < a.B * a.K; k += blockDim.x) a.tickets[k] = 0;
    if (a.beta && threadIdx.x == 0) {   // ln p(beta) of the fitted background joins every draw's log joint
        for (int j = 0; j < 3; ++j) {
            const double z = static_cast<double>(a.beta[j]) / a.bg_sd;
            acc += -0.5 * z * z - log(static_cast<double>(a.bg_sd)) - 0.5 * kLog2Pi;
        }
    }
    const double tot = block_sum(acc, sh);
    const double totq = a.lq ? block_sum(accq, sh) : 0.0;
    if (threadIdx.x == 0) {
        a.lpj[s] = tot;
        if (a.lq) a.lq[s] = totq;
    }
    if (s_loc == 0 && a.ent) {
        // Gaussian entropy sum_j (ln sigma_j + (1 + ln 2 pi)/2): the terms in FP32
        // (FP64 transcendentals are slow on this part), their sum in FP64
        double H = 0.0;
        for (int i = threadIdx.x; i < 5 * a.K; i += blockDim.x)
            if ((!a.mask || ((mk >> (i / 5)) & 1u)) && !((i % 5 == 3 && a.fix_r) || (i % 5 == 4 && a.fix_a)))
                H += static_cast<double>(logf(softplusf(raw[i]))) + 0.5 * (1.0 + kLog2Pi);
        H = block_sum(H, sh);
        if (threadIdx.x == 0) a.ent[b] = H;
    }
}

__global__ void __launch_bounds__(128) k_sample(SampleArgs a) { sample_body(a, blockIdx.x); }

// ---------------------------------------------------------------------------
// Profile kernels
// ---------------------------------------------------------------------------
//
// With d = x - p - mu and s(d) = 2 / w_side, t = s(d) d, u = t^2,
// L = 1 / (1 + u), G = 2^-u.  Peaks are sorted by position within a phase,
// so for one tile of points [xlo, xhi] the peaks of a phase fall into three
// contiguous index ranges: peaks left of every point (all d > 0, the
// right-hand width applies), peaks among the points, peaks right of every
// point (all d < 0).  k_ranges finds them once per step for every (sample,
// phase, tile), together with the range of peaks whose Gaussian reaches the
// tile (beyond it 2^-u < 2^-128 is zero in FP32).
//
// The Lorentzian over the two side-uniform ranges is almost all of the work
// (the mixed range holds the few peaks inside the tile); there s is a
// constant and
//   t = fma(s, x - p, -s mu)
// (x - p is exact near the peak, so t keeps full precision there).  The
// mixed range (side chosen per point, both components) and the Gaussian on
// the uniform ranges form the near part.  The forward does both in one
// kernel; the backward's heavier near part runs in its own kernel
// (k_bwd_near), which keeps the hot kernel's code small.
//
// Work item: one warp owns (sample s, tile of kTile consecutive points, chunk
// c of the phases); lane l holds points i0 + l + 32 j, j < kPts, as kPts/2
// packed pairs (points 2q and 2q+1 of the lane in one 64-bit register;
// arithmetic without an |x| operand runs as packed f32x2 instructions).
// Items are taken from an atomic work counter (zeroed by k_sample).
struct ProfArgs {
    int S, K, N, Npad, T, Mtot, C;
    int chunk[kMaxChunks + 1];  // phase boundaries of the C chunks
    const float *pos, *inten;
    const int *off;
    const float *x, *y, *bg;
    const PhaseConst *cst;
    ushort4 *ranges;   // [S*K*T] (m1, m2, nb, ne) relative to the phase's first peak
    float *g;          // [S*Npad]
    float *f_out;      // [S*N] or null
    double *llpart;    // [S*T]
    float *gpart;      // [S*K*T*kGradSums]
    float *fpart;      // [C*S*Npad] partial profiles per phase chunk
    int *counter;      // work counter of this kernel (zeroed by k_sample)
    int gauss;         // Gaussian likelihood variant
    const float *csec; // [N] cos(x/2) of the angle-dependent width variant (null: constant width)
    float *ghl;        // [2*S*Npad] TF32 hi / lo parts of g (shared-shape variant; null otherwise)
    const float *Tb;   // [3*N] Chebyshev terms (fitted background; null: fixed background)
    float *bgpart;     // [S*T*3] per-(sample, tile) sums of g B(beta) T_j
    // far field (null: every peak evaluated at every point)
    ushort2 *franges;  // [S*K*T] (fb, fe) relative to the phase's first peak
    float *fnode;      // [C*S*T*kFarNodes] far-field profile at the tile nodes per phase chunk
    float *wfar;       // [S*T*kFarNodes] node weights of g (null: not needed)
    float *wfar2;      // [S*T*kFarNodes] per tile: sum_p Mb[t][p][P] W_t,p (null: no second level)
    const float *node_x, *node_c, *lam;
    const int *far_order;   // [K] phases by decreasing peak count
    // second far-field level (Tg = 0: none)
    int Tg;
    ushort2 *sranges;  // [S*K*Tg] super-far ends relative to the phase's first peak
    float *fnode2;     // [C*S*Tg*kFarNodes] super-level node sums per phase chunk
    const float *node_x2, *node_c2, *sgap, *Mf, *Mb;
};

typedef unsigned long long f2_t;   // two packed floats

__device__ __forceinline__ f2_t pk2(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2_t bc2(float v) { return pk2(v, v); }
__device__ __forceinline__ float sum2(f2_t v) {
    float a, b;
    up2(v, a, b);
    return a + b;
}

__device__ __forceinline__ f2_t rcp2(f2_t v) {
    float a, b;
    up2(v, a, b);
    return pk2(rcp_approx(a), rcp_approx(b));
}

__device__ __forceinline__ f2_t ex2neg2(f2_t u) {
    float a, b;
    up2(u, a, b);
    return pk2(ex2_approx(-a), ex2_approx(-b));
}

// Does any point of the warp's pair block lie inside the Gaussian's reach
// (u < kGaussU)?  Beyond it ex2.approx.ftz returns exactly 0, so skipping the
// Gaussian terms there leaves every sum bit-identical.  Warp-uniform.
__device__ __forceinline__ bool any_gauss(f2_t u) {
    float a, b;
    up2(u, a, b);
    return __any_sync(0xffffffffu, fminf(a, b) < kGaussU);
}

constexpr int kPairs = kPts / 2;

// Range marker of a phase removed from a sample's sub-model (peak offsets
// stay below kMaxPeaks < 0xffff).
constexpr unsigned short kAbsentRange = 0xffffu;

// Margin (degrees) keeping the side-uniform ranges clear of d = 0.
constexpr float kSideMargin = 1e-4f;

// First m in [lo, hi) with pos[m] > bound (strict) or >= bound (kInclusive).
template <bool kInclusive>
__device__ __forceinline__ int first_beyond(const float *pos, int lo, int hi, float bound) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float p = pos[mid];
        const bool beyond = kInclusive ? (p >= bound) : (p > bound);
        if (beyond) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Peak index ranges of every (sample, phase, tile):
//   [mb, m1) all d > 0,  [m1, m2) mixed,  [m2, me) all d < 0,  [nb, ne) Gaussian reach.
__device__ __forceinline__ void ranges_body(const ProfArgs &a, int vb, int vgrid) {
    const int total = a.S * a.K * a.T;
    for (int idx = vb * blockDim.x + threadIdx.x; idx < total; idx += vgrid * blockDim.x) {
        const int tile = idx % a.T;
        const int sk = idx / a.T;
        const int k = sk % a.K;
        const PhaseConst c = a.cst[sk];
        if (c.absent != 0.f) {
            a.ranges[idx] = make_ushort4(kAbsentRange, 0, 0, 0);
            if (a.franges) a.franges[idx] = make_ushort2(0, 0);
            if (a.sranges && tile % kSuperTiles == 0)
                a.sranges[(idx / a.T) * a.Tg + tile / kSuperTiles] = make_ushort2(0, 0);
            continue;
        }
        const float xlo = a.x[tile * kTile];
        const float xhi = a.x[min(tile * kTile + kTile - 1, a.N - 1)];
        const int mb = a.off[k], me = a.off[k + 1];
        const int m1 = first_beyond<true>(a.pos, mb, me, xlo - c.mu - kSideMargin);
        const int m2 = first_beyond<false>(a.pos, m1, me, xhi - c.mu + kSideMargin);
        const int nb = first_beyond<false>(a.pos, mb, me, xlo - c.mu - c.rr);
        const int ne = first_beyond<true>(a.pos, nb, me, xhi - c.mu + c.rl);
        a.ranges[idx] = make_ushort4(static_cast<unsigned short>(m1 - mb), static_cast<unsigned short>(m2 - mb),
                                     static_cast<unsigned short>(nb - mb), static_cast<unsigned short>(ne - mb));
        if (a.franges) {
            // far peaks: more than kFarGap half-widths of the tile beyond it and
            // beyond their Gaussian reach, so only their Lorentzian reaches it
            const float gap = fmaxf(kFarGap * 0.5f * (xhi - xlo), kSideMargin);
            const int fb = min(min(first_beyond<true>(a.pos, mb, m1, xlo - c.mu - gap), nb), m1);
            const int fe = max(max(first_beyond<false>(a.pos, m2, me, xhi - c.mu + gap), ne), m2);
            a.franges[idx] = make_ushort2(static_cast<unsigned short>(fb - mb), static_cast<unsigned short>(fe - mb));
            if (a.sranges && tile % kSuperTiles == 0) {
                // super-far peaks: beyond the super-tile by sgap (which exceeds
                // every member tile's far gap) and beyond the Gaussian reach, so
                // they are far for every tile of it
                const int g = tile / kSuperTiles;
                const float slo = a.x[g * kSuperTiles * kTile];
                const float shi = a.x[min((g + 1) * kSuperTiles * kTile - 1, a.N - 1)];
                const float sg = a.sgap[g];
                const int sfb = first_beyond<true>(a.pos, mb, fb, slo - c.mu - fmaxf(sg, c.rr));
                const int sfe = first_beyond<false>(a.pos, fe, me, shi - c.mu + fmaxf(sg, c.rl));
                a.sranges[(idx / a.T) * a.Tg + g] =
                    make_ushort2(static_cast<unsigned short>(sfb - mb), static_cast<unsigned short>(sfe - mb));
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_ranges(ProfArgs a) { ranges_body(a, blockIdx.x, gridDim.x); }

// Bounds-check build (XRDVI_DEBUG): every peak-table index and every decoded
// peak range is clamped into bounds, and the first violation's check number is
// recorded in a device word that the host reads after the call.  Control flow
// is unchanged (no early return, no trap), so no warp or barrier is left
// waiting; a regular build compiles the checks away.
#ifdef XRDVI_DEBUG
__device__ int g_debug_word = 0;
__device__ __forceinline__ int dbg_index(int i, int n, int code) {
    if (i < 0 || i >= n) {
        atomicCAS(&g_debug_word, 0, code);
        return i < 0 ? 0 : (n > 0 ? n - 1 : 0);
    }
    return i;
}
__device__ __forceinline__ int dbg_range(int v, int lo, int hi, int code) {
    if (v < lo || v > hi) {
        atomicCAS(&g_debug_word, 0, code);
        return v < lo ? lo : hi;
    }
    return v;
}
#else
__device__ __forceinline__ int dbg_index(int i, int, int) { return i; }
__device__ __forceinline__ int dbg_range(int v, int, int, int) { return v; }
#endif

// Shared-memory peak table.  Entries hold -p (so that x + (-p) is one packed
// add) and I.  The wide layout's entry m also holds peak m + 1's values,
// (-p_m, -p_m+1, I_m, I_m+1), so that a single 16-byte load yields the packed
// pairs of two consecutive peaks (the far-field loops run two peaks per
// packed instruction); it is used when the table is small enough not to
// limit occupancy.
template <bool kWide>
struct PeakTable;
template <>
struct PeakTable<false> {
    const float2 *p;
    int n;   // entries (for the bounds-check build)
    __device__ __forceinline__ void get(int m, f2_t &np, f2_t &I) const {
        const float2 v = p[dbg_index(m, n, 1)];
        np = bc2(v.x);
        I = bc2(v.y);
    }
    // peaks m and m + 1 as packed pairs
    __device__ __forceinline__ void pair(int m, f2_t &np, f2_t &I) const {
        const float2 v0 = p[dbg_index(m, n - 1, 2)], v1 = p[dbg_index(m + 1, n, 2)];
        np = pk2(v0.x, v1.x);
        I = pk2(v0.y, v1.y);
    }
    __device__ __forceinline__ void scalar(int m, float &np, float &I) const {
        const float2 v = p[dbg_index(m, n, 3)];
        np = v.x;
        I = v.y;
    }
};
template <>
struct PeakTable<true> {
    const float4 *p;
    int n;   // entries (for the bounds-check build)
    __device__ __forceinline__ void get(int m, f2_t &np, f2_t &I) const {
        const float4 v = p[dbg_index(m, n, 1)];
        np = bc2(v.x);
        I = bc2(v.z);
    }
    __device__ __forceinline__ void pair(int m, f2_t &np, f2_t &I) const {
        const float4 v = p[dbg_index(m, n - 1, 2)];   // entry m also holds peak m + 1
        np = pk2(v.x, v.y);
        I = pk2(v.z, v.w);
    }
    __device__ __forceinline__ void scalar(int m, float &np, float &I) const {
        const float4 v = p[dbg_index(m, n, 3)];
        np = v.x;
        I = v.z;
    }
};

template <bool kWide>
__device__ __forceinline__ PeakTable<kWide> load_table(const ProfArgs &a, float4 *s_raw, int *&s_off) {
    PeakTable<kWide> t;
    if constexpr (kWide) {
        float4 *q = s_raw;
        for (int i = threadIdx.x; i < a.Mtot; i += blockDim.x) {
            const int j = i + 1 < a.Mtot ? i + 1 : i;
            q[i] = make_float4(-a.pos[i], -a.pos[j], a.inten[i], a.inten[j]);
        }
        t.p = q;
        t.n = a.Mtot;
        s_off = reinterpret_cast<int *>(q + a.Mtot);
    } else {
        float2 *q = reinterpret_cast<float2 *>(s_raw);
        for (int i = threadIdx.x; i < a.Mtot; i += blockDim.x) q[i] = make_float2(-a.pos[i], a.inten[i]);
        t.p = q;
        t.n = a.Mtot;
        s_off = reinterpret_cast<int *>(q + a.Mtot);
    }
    for (int i = threadIdx.x; i <= a.K; i += blockDim.x) s_off[i] = a.off[i];
    __syncthreads();
    return t;
}

// Peak ranges of one (sample, phase, tile): [mb, fb) far below, [fb, m1)
// near below, [m1, m2) mixed, [m2, fe) near above, [fe, me) far above, and
// the Gaussian reach [nb, ne) (inside [fb, fe)); of the far peaks, [mb, sfb)
// and [sfe, me) are super-far (beyond the tile's super-tile).  Without the
// far field fb = sfb = mb and fe = sfe = me; without the second level
// sfb = mb and sfe = me.
struct Ranges {
    int mb, m1, m2, me, nb, ne, fb, fe, sfb, sfe;
};

__device__ __forceinline__ Ranges load_ranges(const ProfArgs &a, const int *s_off, int s, int k, int tile) {
    const size_t sk = static_cast<size_t>(s) * a.K + k;
    const size_t id = sk * a.T + tile;
    // every load is issued before any of them is used: one round trip per phase
    const ushort4 r = a.ranges[id];
    const ushort2 f = a.franges ? a.franges[id] : make_ushort2(0, 0);
    const ushort2 g = a.sranges ? a.sranges[sk * a.Tg + tile / kSuperTiles] : make_ushort2(0, 0);
    Ranges o;
    o.mb = s_off[k];
    if (r.x == kAbsentRange) {  // phase not in this sample's sub-model: every range empty
        o.me = o.m1 = o.m2 = o.nb = o.ne = o.fb = o.fe = o.sfb = o.sfe = o.mb;
        return o;
    }
    o.me = s_off[k + 1];
    o.m1 = o.mb + r.x;
    o.m2 = o.mb + r.y;
    o.nb = o.mb + r.z;
    o.ne = o.mb + r.w;
    o.fb = a.franges ? o.mb + f.x : o.mb;
    o.fe = a.franges ? o.mb + f.y : o.me;
    o.sfb = a.sranges ? o.mb + g.x : o.mb;
    o.sfe = a.sranges ? o.mb + g.y : o.me;
#ifdef XRDVI_DEBUG
    // every range within the phase's peaks (check numbers 4-9)
    o.m1 = dbg_range(o.m1, o.mb, o.me, 4);
    o.m2 = dbg_range(o.m2, o.m1, o.me, 5);
    o.nb = dbg_range(o.nb, o.mb, o.me, 6);
    o.ne = dbg_range(o.ne, o.nb, o.me, 6);
    o.fb = dbg_range(o.fb, o.mb, o.m1, 7);
    o.fe = dbg_range(o.fe, o.m2, o.me, 7);
    o.sfb = dbg_range(o.sfb, o.mb, o.fb, 8);
    o.sfe = dbg_range(o.sfe, o.fe, o.me, 9);
#endif
    return o;
}

// Is there any work for the near kernels (mixed range, or Gaussian reach
// beyond it)?  Warp-uniform.
__device__ __forceinline__ bool near_work(const Ranges &r) {
    return r.m1 < r.m2 || r.nb < r.m1 || r.m2 < r.ne;
}

// t = s(d) d for a packed pair on the mixed range: the side's scale is
// selected per point (exact for any asymmetry).
// The side's scale s_l + m (s_r - s_l) with the mask m = sat(d 2^100): 1 for
// d >= 2^-100, 0 for d <= 0 (the saturating multiply runs on the FMA pipe;
// a comparison and a select per point would take the busier ALU pipe).  For
// 0 < d < 2^-100, where m is fractional, |t| < 1e-27: L = G = 1 and every
// t-weighted term vanishes in FP32 whichever scale is used.
__device__ __forceinline__ float mul_sat(float a, float b) {
    float r;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2_t t_mixed(f2_t x2, f2_t np, f2_t nmu2, f2_t sl2, f2_t ds2) {
    const f2_t d2 = add2(add2(x2, np), nmu2);
    float d0, d1;
    up2(d2, d0, d1);
    const f2_t m2 = pk2(mul_sat(d0, 0x1p100f), mul_sat(d1, 0x1p100f));
    return mul2(d2, fma2(m2, ds2, sl2));
}

__device__ __forceinline__ void item_points(const ProfArgs &a, int i0, int lane, f2_t (&x2)[kPairs]) {
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        const int i_a = min(i0 + (2 * q) * 32 + lane, a.N - 1);
        const int i_b = min(i0 + (2 * q + 1) * 32 + lane, a.N - 1);
        x2[q] = pk2(a.x[i_a], a.x[i_b]);
    }
}

// Per-point width factor of the angle-dependent variant: the side width at
// point x is w_side sec(x/2), so t = s d cos(x/2); the mu-gradient sums carry
// one more factor cos(x/2) (dt/dmu = -s cos(x/2)), the other sums none.
// PtScale<false> is the constant-width model and costs nothing.
template <bool kSec>
struct PtScale {
    __device__ __forceinline__ void load(const ProfArgs &, int, int) {}
    __device__ __forceinline__ f2_t operator()(f2_t t, int) const { return t; }
};
template <>
struct PtScale<true> {
    f2_t c[kPairs];
    __device__ __forceinline__ void load(const ProfArgs &a, int i0, int lane) {
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            const int i_a = min(i0 + (2 * q) * 32 + lane, a.N - 1);
            const int i_b = min(i0 + (2 * q + 1) * 32 + lane, a.N - 1);
            c[q] = pk2(a.csec[i_a], a.csec[i_b]);
        }
    }
    __device__ __forceinline__ f2_t operator()(f2_t t, int q) const { return mul2(t, c[q]); }
};

__device__ __forceinline__ int next_item(int *counter, int lane) {
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, it, 0);
}

// Neumaier-compensated accumulation of packed per-point values.
template <bool kNaive>
__device__ __forceinline__ void acc_points(float (&fs)[kPts], float (&fc)[kPts], const f2_t (&v2)[kPairs]) {
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        float v[2];
        up2(v2[q], v[0], v[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * q + h;
            if (kNaive) {
                fs[j] += v[h];
            } else {
                const float t = fs[j] + v[h];
                fc[j] += (fabsf(fs[j]) >= fabsf(v[h])) ? ((fs[j] - t) + v[h]) : ((v[h] - t) + fs[j]);
                fs[j] = t;
            }
        }
    }
}

// --- forward ------------------------------------------------------------------
// Side-uniform ranges take the points relative to the tile's edge on the
// range's side, x0 (the first point for peaks below the tile, the last for
// peaks above it): t = s (x - x0) + b with b = s (x0 - p) - s mu.  Over such a
// range both terms have the sign of t, so t keeps full relative accuracy and
// costs one FMA per evaluation.  The b of up to 32 peaks are formed at once,
// one per lane, into the warp's buffer as (b, b, I, I).
template <class Tab>
__device__ __forceinline__ void fill_offsets(const Tab &tab, float4 *wb, int lane, int mb, int n, float sc,
                                             float cmu, float x0) {
    __syncwarp();   // the previous batch's reads are done
    if (lane < n) {
        float np, I;
        tab.scalar(mb + lane, np, I);
        const float b = fmaf(sc, x0 + np, cmu);
        wb[lane] = make_float4(b, b, I, I);
    }
    __syncwarp();
}

// The lane's points relative to x0, x - x0 (exact for points of one tile away
// from x = 0), loaded again for each range so that no point coordinates stay
// in registers across the phase loop.
__device__ __forceinline__ void rel_points(const ProfArgs &a, int i0, int lane, float x0, f2_t (&dx2)[kPairs]) {
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        const int i_a = min(i0 + (2 * q) * 32 + lane, a.N - 1);
        const int i_b = min(i0 + (2 * q + 1) * 32 + lane, a.N - 1);
        dx2[q] = pk2(a.x[i_a] - x0, a.x[i_b] - x0);
    }
}

// Lorentzian sums on a side-uniform range, one reciprocal per two peaks:
// I0/d0 + I1/d1 = (I0 d1 + I1 d0) / (d0 d1)  (d = 1 + t^2; d0 d1 stays finite
// while s |d| < 1e9).
template <class Tab, class Sc>
__device__ __forceinline__ void fwdL_uniform(const ProfArgs &a, const Tab &tab, float4 *wb, int i0, int lane, int m0,
                                             int m1, float sc, float cmu, float x0, const Sc &ps, f2_t (&sl)[kPairs]) {
    if (m0 >= m1) return;
    const f2_t s2 = bc2(sc), one2 = bc2(1.f);
    f2_t dx2[kPairs];
    rel_points(a, i0, lane, x0, dx2);
    for (int mb = m0; mb < m1; mb += 32) {
        const int n = min(32, m1 - mb);
        fill_offsets(tab, wb, lane, mb, n, sc, cmu, x0);
        int j = 0;
        for (; j + 1 < n; j += 2) {
            const float4 v0 = wb[j], v1 = wb[j + 1];
            const f2_t b0 = pk2(v0.x, v0.y), I0 = pk2(v0.z, v0.w);
            const f2_t b1 = pk2(v1.x, v1.y), I1 = pk2(v1.z, v1.w);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t t0 = ps(fma2(s2, dx2[q], b0), q);
                const f2_t t1 = ps(fma2(s2, dx2[q], b1), q);
                const f2_t d0 = fma2(t0, t0, one2), d1 = fma2(t1, t1, one2);
                const f2_t num = fma2(I0, d1, mul2(I1, d0));
                sl[q] = fma2(num, rcp2(mul2(d0, d1)), sl[q]);
            }
        }
        if (j < n) {
            const float4 v = wb[j];
            const f2_t b = pk2(v.x, v.y), I = pk2(v.z, v.w);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t t = ps(fma2(s2, dx2[q], b), q);
                sl[q] = fma2(I, rcp2(fma2(t, t, one2)), sl[q]);
            }
        }
    }
}

// Near part of one phase's profile on the tile: the mixed range (both
// components, side chosen per point) and the Gaussian on the side-uniform
// ranges within its reach.
template <class Tab, class Sc, class PC>
__device__ __forceinline__ void fwd_near(const ProfArgs &a, const Tab &tab, const Ranges &r, const PC &cp,
                                         int i0, int lane, const Sc &ps, f2_t (&sl)[kPairs], f2_t (&sg)[kPairs]) {
    f2_t x2[kPairs];
    item_points(a, i0, lane, x2);
    const f2_t nmu2 = bc2(-cp.mu), one2 = bc2(1.f), sl2 = bc2(cp.sl), ds2 = bc2(cp.sr - cp.sl);
    // two peaks per pass, their Lorentzians over one reciprocal as in
    // fwdL_uniform (d = 1 + t^2 stays small on the mixed range)
    int m = r.m1;
    for (; m + 1 < r.m2; m += 2) {
        f2_t np0, I0, np1, I1;
        tab.get(m, np0, I0);
        tab.get(m + 1, np1, I1);
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            const f2_t t0 = ps(t_mixed(x2[q], np0, nmu2, sl2, ds2), q);
            const f2_t t1 = ps(t_mixed(x2[q], np1, nmu2, sl2, ds2), q);
            const f2_t u0 = mul2(t0, t0), u1 = mul2(t1, t1);
            const f2_t d0 = add2(u0, one2), d1 = add2(u1, one2);
            sl[q] = fma2(fma2(I0, d1, mul2(I1, d0)), rcp2(mul2(d0, d1)), sl[q]);
            sg[q] = fma2(I1, ex2neg2(u1), fma2(I0, ex2neg2(u0), sg[q]));
        }
    }
    if (m < r.m2) {
        f2_t np, I;
        tab.get(m, np, I);
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            const f2_t t = ps(t_mixed(x2[q], np, nmu2, sl2, ds2), q);
            const f2_t u = mul2(t, t);
            sl[q] = fma2(I, rcp2(add2(u, one2)), sl[q]);
            sg[q] = fma2(I, ex2neg2(u), sg[q]);
        }
    }
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int m0 = side ? r.m2 : min(r.nb, r.m1), m1 = side ? max(r.ne, r.m2) : r.m1;
        const f2_t s2 = bc2(side ? cp.sl : cp.sr), c2 = bc2(side ? cp.nslmu : cp.nsrmu);
        for (int m = m0; m < m1; ++m) {
            f2_t np, I;
            tab.get(m, np, I);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t t = ps(fma2(s2, add2(x2[q], np), c2), q);
                sg[q] = fma2(I, ex2neg2(mul2(t, t)), sg[q]);
            }
        }
    }
}

// Partial profile of one phase chunk: fpart[c][s][i] = sum over the chunk's
// phases of h sum_m I_m [(1 - r) G + r L] (Neumaier-compensated over phases).
template <bool kNaive, bool kWide, bool kSec = false>
__global__ void __launch_bounds__(kThreads, 3) k_forward(ProfArgs a) {
    extern __shared__ float4 s_raw[];
    __shared__ float4 s_wb[kWarps][32];
    int *s_off;
    const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
    const int lane = threadIdx.x & 31;
    float4 *wb = s_wb[threadIdx.x >> 5];
    const int items = a.S * a.T * a.C;
    for (int item = next_item(a.counter, lane); item < items; item = next_item(a.counter, lane)) {
        const int c = item % a.C;
        const int st = item / a.C;
        const int s = st / a.T, tile = st - s * a.T;
        const int i0 = tile * kTile;
        const float xlo = a.x[i0], xhi = a.x[min(i0 + kTile - 1, a.N - 1)];
        PtScale<kSec> ps;
        ps.load(a, i0, lane);
        float fs[kPts], fc[kPts];
#pragma unroll
        for (int j = 0; j < kPts; ++j) fs[j] = fc[j] = 0.f;
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = a.chunk[c]; k < a.chunk[c + 1]; ++k) {
            const PhaseConst cp = cs[k];
            const Ranges r = load_ranges(a, s_off, s, k, tile);
            f2_t sl[kPairs], sg[kPairs];
#pragma unroll
            for (int q = 0; q < kPairs; ++q) sl[q] = sg[q] = 0ull;
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                fwdL_uniform(a, tab, wb, i0, lane, side ? r.m2 : r.fb, side ? r.fe : r.m1, side ? cp.sl : cp.sr,
                             side ? cp.nslmu : cp.nsrmu, side ? xhi : xlo, ps, sl);
            }
            if (near_work(r)) fwd_near(a, tab, r, cp, i0, lane, ps, sl, sg);  // warp-uniform
            const f2_t hl2 = bc2(cp.hl), hg2 = bc2(cp.hg);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) sl[q] = fma2(hl2, sl[q], mul2(hg2, sg[q]));
            acc_points<kNaive>(fs, fc, sl);
        }
        float *dst = a.fpart + (static_cast<size_t>(c) * a.S + s) * a.Npad + i0 + lane;
#pragma unroll
        for (int j = 0; j < kPts; ++j) dst[j * 32] = fs[j] + fc[j];
    }
}

// --- far field -------------------------------------------------------------------
// The Lorentzian tails that reach a tile from peaks beyond kFarGap half-widths
// of it are analytic on the tile's span, with poles x = rho +- i/s at least
// 1.5 half-widths from its centre.  Their sums are therefore evaluated at
// kFarNodes Chebyshev nodes of the first kind of the span (Trefethen,
// "Approximation Theory and Approximation Practice", ch. 8 bounds the
// interpolation error by a power of the Bernstein-ellipse parameter; for
// these poles it is below 1e-8 of the tail, under FP32 rounding) and
// interpolated at the tile's points with Lagrange weights lam_p(x_i):
//   forward   f_far(x_i) = sum_p lam_p(x_i) F_p          (in k_lik)
//   backward  sum_i g_i phi(x_i) = sum_p W_p phi(x_p),  W_p = sum_i g_i lam_p(x_i).
// A second level does the same on super-tiles of kSuperTiles tiles for the
// peaks far beyond the super-tile.  The node evaluations run inside the
// direct kernels, lane p taking node p, in the same loop over phases.

// One phase's far Lorentzian sum at this lane's node x: sum_m I_m L(t_m(x))
// over [lo0, hi0) (peaks below, scale sr) and [lo1, hi1) (peaks above, sl).
template <class Tab, class PC, bool kSec>
__device__ __forceinline__ float far_node_sum(const Tab &tab, const PC &cp, float x, float cx, int lo0, int hi0,
                                              int lo1, int hi1) {
    const f2_t x2 = bc2(x), one2 = bc2(1.f);
    float acc = 0.f;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int m0 = side ? lo1 : lo0, m1 = side ? hi1 : hi0;
        const float sc = side ? cp.sl : cp.sr, cm = side ? cp.nslmu : cp.nsrmu;
        const f2_t sc2 = bc2(sc), cm2 = bc2(cm);
        int m = m0;
        for (; m + 1 < m1; m += 2) {
            f2_t np2, I2;
            tab.pair(m, np2, I2);
            f2_t t2 = fma2(sc2, add2(x2, np2), cm2);
            if (kSec) t2 = mul2(t2, bc2(cx));
            // I0/d0 + I1/d1 = (I0 d1 + I1 d0) / (d0 d1): one reciprocal per two
            // peaks (finite while s |x - p| < 1e9, as in fwdL_uniform)
            float d0, d1, i0, i1;
            up2(fma2(t2, t2, one2), d0, d1);
            up2(I2, i0, i1);
            acc = fmaf(fmaf(i0, d1, i1 * d0), rcp_approx(d0 * d1), acc);
        }
        if (m < m1) {
            float np, I;
            tab.scalar(m, np, I);
            float t = fmaf(sc, x + np, cm);
            if (kSec) t *= cx;
            acc = fmaf(I, rcp_approx(fmaf(t, t, 1.f)), acc);
        }
    }
    return acc;
}

// One phase's far gradient sums at this lane's node (weight w, w cos(x/2) for
// the mu sums): adds w sum I L to S1 and, per side, w c sum I L^2 t to A and
// w (sum I L - sum I L^2) to B.
template <class Tab, class PC, bool kSec>
__device__ __forceinline__ void far_node_grad(const Tab &tab, const PC &cp, float x, float cx, float w, float wa,
                                              int lo0, int hi0, int lo1, int hi1, float &S1, float (&A)[2],
                                              float (&B)[2]) {
    const f2_t x2 = bc2(x), one2 = bc2(1.f);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int m0 = side ? lo1 : lo0, m1 = side ? hi1 : hi0;
        if (m0 >= m1) continue;
        const float sc = side ? cp.sl : cp.sr, cm = side ? cp.nslmu : cp.nsrmu;
        const f2_t sc2 = bc2(sc), cm2 = bc2(cm);
        f2_t s1p = 0ull, anp = 0ull, c2p = 0ull;   // two peaks per packed instruction
        int m = m0;
        for (; m + 1 < m1; m += 2) {
            f2_t np2, I2;
            tab.pair(m, np2, I2);
            f2_t t2 = fma2(sc2, add2(x2, np2), cm2);
            if (kSec) t2 = mul2(t2, bc2(cx));
            const f2_t L2 = rcp2(fma2(t2, t2, one2));
            const f2_t q1 = mul2(I2, L2);
            s1p = add2(s1p, q1);
            const f2_t q2 = mul2(q1, L2);
            anp = fma2(q2, t2, anp);
            c2p = add2(c2p, q2);
        }
        float s1 = sum2(s1p), an = sum2(anp), c2 = sum2(c2p);
        if (m < m1) {   // the odd peak
            float np, I;
            tab.scalar(m, np, I);
            float t = fmaf(sc, x + np, cm);
            if (kSec) t *= cx;
            const float L = rcp_approx(fmaf(t, t, 1.f));
            const float q1 = I * L;
            s1 += q1;
            const float q2 = q1 * L;
            an = fmaf(q2, t, an);
            c2 += q2;
        }
        S1 = fmaf(w, s1, S1);
        if (side) {
            A[1] = fmaf(wa, an, A[1]);
            B[1] = fmaf(w, s1 - c2, B[1]);
        } else {
            A[0] = fmaf(wa, an, A[0]);
            B[0] = fmaf(w, s1 - c2, B[0]);
        }
    }
}

// Far peaks of one (sample, phase, tile): level 1 (the tile's nodes) [lo0,
// hi0) below and [lo1, hi1) above the tile without the super-far ones; level
// 2 (the super-tile's nodes) the super-far ones.
struct FarRanges {
    int l1[4], l2[4];
};
__device__ __forceinline__ FarRanges far_ranges(const Ranges &r) {
    FarRanges f;
    f.l1[0] = r.sfb; f.l1[1] = r.fb; f.l1[2] = r.fe; f.l1[3] = r.sfe;
    f.l2[0] = r.mb; f.l2[1] = r.sfb; f.l2[2] = r.sfe; f.l2[3] = r.me;
    return f;
}

// Profile with the far field on: per (sample, tile, phase chunk), each
// phase's near band [fb, m1), [m2, fe) (a few peaks: t = s (x - p) - s mu per
// evaluation), its mixed range and its Gaussian reach at the tile's points
// (the Gaussian at every point of them: beyond its reach 2^-u is exactly 0,
// and a branch-free loop beats a warp vote per pair block here).  Phase
// contributions are summed with packed Kahan compensation (all terms are
// non-negative).  Lane p also sums the phase's far peaks at node p
// of the tile (and, for a super-tile's first tile, its super-far peaks at node
// p of the super-tile), Kahan-compensated over the phases, into the chunk's
// node partials fnode (fnode2), which k_lik combines and interpolates.
template <bool kNaive, bool kWide, bool kSec>
__device__ __forceinline__ void fwd_direct_items(const ProfArgs &a, const PeakTable<kWide> &tab, const int *s_off) {
    const int lane = threadIdx.x & 31;
    const f2_t one2 = bc2(1.f);
    const int items = a.S * a.T * a.C;
    for (int item = next_item(a.counter, lane); item < items; item = next_item(a.counter, lane)) {
        const int c = item % a.C;
        const int st = item / a.C;
        const int s = st / a.T, tile = st - s * a.T;
        const int i0 = tile * kTile;
        f2_t x2[kPairs];
        item_points(a, i0, lane, x2);
        PtScale<kSec> ps;
        ps.load(a, i0, lane);
        f2_t fs[kPairs], fc[kPairs];
#pragma unroll
        for (int q = 0; q < kPairs; ++q) fs[q] = fc[q] = 0ull;
        // far field: this lane's node of the tile (and of the super-tile)
        const bool lvl2 = a.Tg && tile % kSuperTiles == 0;
        const int g = tile / kSuperTiles;
        const float xn = a.node_x[tile * kFarNodes + lane];
        const float xn2 = lvl2 ? a.node_x2[g * kFarNodes + lane] : 0.f;
        const float cn = kSec ? a.node_c[tile * kFarNodes + lane] : 1.f;
        const float cn2 = kSec && lvl2 ? a.node_c2[g * kFarNodes + lane] : 1.f;
        float F = 0.f, Fc = 0.f, F2 = 0.f, F2c = 0.f;
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = a.chunk[c]; k < a.chunk[c + 1]; ++k) {
            const PhaseConst cp = cs[k];
            const Ranges r = load_ranges(a, s_off, s, k, tile);
            {   // far peaks at the nodes
                const FarRanges fr = far_ranges(r);
                const float v = cp.hl * far_node_sum<PeakTable<kWide>, PhaseConst, kSec>(
                                            tab, cp, xn, cn, fr.l1[0], fr.l1[1], fr.l1[2], fr.l1[3]);
                const float y = v - Fc, t = F + y;   // Kahan (non-negative terms)
                Fc = (t - F) - y;
                F = t;
                if (lvl2) {
                    const float v2 = cp.hl * far_node_sum<PeakTable<kWide>, PhaseConst, kSec>(
                                                 tab, cp, xn2, cn2, fr.l2[0], fr.l2[1], fr.l2[2], fr.l2[3]);
                    const float y2 = v2 - F2c, t2 = F2 + y2;
                    F2c = (t2 - F2) - y2;
                    F2 = t2;
                }
            }
            f2_t sl[kPairs], sg[kPairs];
#pragma unroll
            for (int q = 0; q < kPairs; ++q) sl[q] = sg[q] = 0ull;
            // near band, Lorentzian (its Gaussian part is in the reach loops below)
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                const int m0 = side ? r.m2 : r.fb, m1 = side ? r.fe : r.m1;
                const f2_t s2 = bc2(side ? cp.sl : cp.sr), c2 = bc2(side ? cp.nslmu : cp.nsrmu);
                for (int m = m0; m < m1; ++m) {
                    f2_t np, I;
                    tab.get(m, np, I);
#pragma unroll
                    for (int q = 0; q < kPairs; ++q) {
                        const f2_t t = ps(fma2(s2, add2(x2[q], np), c2), q);
                        sl[q] = fma2(I, rcp2(fma2(t, t, one2)), sl[q]);
                    }
                }
            }
            if (near_work(r)) {   // warp-uniform
                const f2_t nmu2 = bc2(-cp.mu), sl2 = bc2(cp.sl), ds2 = bc2(cp.sr - cp.sl);
                for (int m = r.m1; m < r.m2; ++m) {
                    f2_t np, I;
                    tab.get(m, np, I);
#pragma unroll
                    for (int q = 0; q < kPairs; ++q) {
                        const f2_t t = ps(t_mixed(x2[q], np, nmu2, sl2, ds2), q);
                        const f2_t u = mul2(t, t);
                        sl[q] = fma2(I, rcp2(add2(u, one2)), sl[q]);
                        sg[q] = fma2(I, ex2neg2(u), sg[q]);
                    }
                }
#pragma unroll 1
                for (int side = 0; side < 2; ++side) {
                    const int m0 = side ? r.m2 : min(r.nb, r.m1), m1 = side ? max(r.ne, r.m2) : r.m1;
                    const f2_t s2 = bc2(side ? cp.sl : cp.sr), c2 = bc2(side ? cp.nslmu : cp.nsrmu);
                    for (int m = m0; m < m1; ++m) {
                        f2_t np, I;
                        tab.get(m, np, I);
#pragma unroll
                        for (int q = 0; q < kPairs; ++q) {
                            const f2_t t = ps(fma2(s2, add2(x2[q], np), c2), q);
                            const f2_t u = mul2(t, t);
                            sg[q] = fma2(I, ex2neg2(u), sg[q]);
                        }
                    }
                }
            }
            const f2_t hl2 = bc2(cp.hl), hg2 = bc2(cp.hg);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t v = fma2(hl2, sl[q], mul2(hg2, sg[q]));
                if (kNaive) {
                    fs[q] = add2(fs[q], v);
                } else {   // Kahan: fc holds the rounding error of fs (subtracted at the end)
                    const f2_t y = sub2(v, fc[q]);
                    const f2_t t = add2(fs[q], y);
                    fc[q] = sub2(sub2(t, fs[q]), y);
                    fs[q] = t;
                }
            }
        }
        float *dst = a.fpart + (static_cast<size_t>(c) * a.S + s) * a.Npad + i0 + lane;
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            float lo, hi;
            up2(kNaive ? fs[q] : sub2(fs[q], fc[q]), lo, hi);
            dst[(2 * q) * 32] = lo;
            dst[(2 * q + 1) * 32] = hi;
        }
        a.fnode[((static_cast<size_t>(c) * a.S + s) * a.T + tile) * kFarNodes + lane] = F - Fc;
        if (lvl2) a.fnode2[((static_cast<size_t>(c) * a.S + s) * a.Tg + g) * kFarNodes + lane] = F2 - F2c;
    }
}

template <bool kNaive, bool kWide, bool kSec>
__global__ void __launch_bounds__(kThreads, 3) k_fwd_direct(ProfArgs a) {
    extern __shared__ float4 s_raw[];
    int *s_off;
    const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
    fwd_direct_items<kNaive, kWide, kSec>(a, tab, s_off);
}

// Poisson log-likelihood term minus its data constant, D(y, f) =
// y ln(f / y) - (f - y) (= -f for y = 0).  Near f = y it is evaluated by the
// series of Loader (2000, "Fast and accurate computation of binomial
// probabilities") in v = (y - f)/(y + f):
//   y ln(y/f) + f - y = (y - f) v + 2 y sum_{j>=1} v^(2j+1) / (2j+1),
// which avoids the cancellation of the direct form.
__device__ __forceinline__ float deviance_term(float y, float f) {
    if (y == 0.f) return -f;
    const float dif = y - f;
    const float v = __fdiv_rn(dif, y + f);
    if (fabsf(v) < 0.1f) {
        const float v2 = v * v;
        const float ser = fmaf(v2, fmaf(v2, fmaf(v2, fmaf(v2, 1.f / 11.f, 1.f / 9.f), 1.f / 7.f), 1.f / 5.f), 1.f / 3.f);
        const float bd0 = fmaf(dif, v, 2.f * y * v * v2 * ser);
        return -bd0;
    }
    return -(y * logf(__fdiv_rn(y, f)) - dif);
}

// f = B + sum of the C chunk partials (fixed order; all terms are positive,
// so the FP32 sum errs by at most C ulps), then the deviance term, g = y/f - 1
// and the per-tile deviance sum (all terms <= 0: an FP32 tree sum without
// cancellation, stored in FP64).  One block per (sample, tile);
// kTile == blockDim.x.
template <class Blk>
__device__ __forceinline__ void lik_body(const ProfArgs &a, Blk blk) {
    __shared__ float shf[kTile / 32];
    __shared__ float sFn[kFarNodes], sF2[kFarNodes];
    // unsigned division (the indices are non-negative; cheaper than the signed form)
    const int s = static_cast<int>(static_cast<unsigned>(blk.x()) / static_cast<unsigned>(a.T)), tile = blk.x() - s * a.T;
    const int i = tile * kTile + threadIdx.x;
    float dev = 0.f;
    float gv = 0.f;
    const float *lam = a.fnode ? a.lam + static_cast<size_t>(tile) * kFarNodes * kTile + threadIdx.x : nullptr;
    __shared__ __align__(16) float sMb[kFarNodes * kFarNodes];
    __shared__ float sW2[kTile / 32][kFarNodes];
    if (a.wfar2) {
        // the tile's backward translation matrix (4 KB, 16 bytes a thread), copied
        // asynchronously so that no warp waits for it before the node weights
        static_assert(kFarNodes * kFarNodes * 4 == kTile * 16, "one 16-byte copy per thread");
        const float *M = a.Mb + static_cast<size_t>(tile) * kFarNodes * kFarNodes + threadIdx.x * 4;
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(sMb + threadIdx.x * 4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(M) : "memory");
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (lam) {
        // far-field node values: the chunks' partial node sums, plus the
        // super-tile's (summed over chunks) translated to this tile's nodes.
        // The translation is split over the eight warps (warp w takes super
        // nodes [4w, 4w + 4)), whose matrix entries are loaded while warp 0
        // sums the super-level chunks and warp 1 the tile's, so the node values
        // cost about one round trip instead of a warp's 32-term chain.
        constexpr int kPer = kFarNodes / (kTile / 32);
        static_assert(kPer * (kTile / 32) == kFarNodes, "super nodes split evenly over the warps");
        __shared__ float sFc[kFarNodes], sPart[kTile / 32][kFarNodes];
        const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int g = tile / kSuperTiles;
        float mf[kPer];
        if (a.Tg) {
            const float *M = a.Mf + (static_cast<size_t>(tile) * kFarNodes + w * kPer) * kFarNodes + l;
#pragma unroll
            for (int j = 0; j < kPer; ++j) mf[j] = M[j * kFarNodes];
        }
        if (w == 0 && a.Tg) {
            float F2 = 0.f;
            for (int c = 0; c < a.C; ++c) F2 += a.fnode2[((static_cast<size_t>(c) * a.S + s) * a.Tg + g) * kFarNodes + l];
            sF2[l] = F2;
        }
        if (w == 1) {
            float F = 0.f;
            for (int c = 0; c < a.C; ++c) F += a.fnode[((static_cast<size_t>(c) * a.S + s) * a.T + tile) * kFarNodes + l];
            sFc[l] = F;
        }
        __syncthreads();
        if (a.Tg) {
            float part = 0.f;
#pragma unroll
            for (int j = 0; j < kPer; ++j) part = fmaf(mf[j], sF2[w * kPer + j], part);
            sPart[w][l] = part;
            __syncthreads();
        }
        if (w == 0) {
            float F = sFc[l];
            if (a.Tg) {
#pragma unroll
                for (int ww = 0; ww < kTile / 32; ++ww) F += sPart[ww][l];
            }
            sFn[l] = F;
        }
        __syncthreads();
    }
    if (i < a.N) {
        float f = a.bg[i];
        for (int c = 0; c < a.C; ++c) f += a.fpart[(static_cast<size_t>(c) * a.S + s) * a.Npad + i];
        if (lam) {   // far field: interpolated from the tile's nodes
            float ff = 0.f;
#pragma unroll 8
            for (int p = 0; p < kFarNodes; ++p) ff = fmaf(lam[p * kTile], sFn[p], ff);
            f += ff;
        }
        const float yv = a.y[i];
        if (a.gauss) {
            // Gaussian variant: -(y - f)^2 / (2 v), d/df = (y - f) / v, v = max(y, 1)
            const float v = fmaxf(yv, 1.f), r = yv - f;
            gv = __fdiv_rn(r, v);
            dev = -0.5f * r * gv;
        } else {
            dev = deviance_term(yv, f);
            gv = (yv > 0.f) ? __fdiv_rn(yv, f) - 1.0f : -1.0f;
        }
        if (a.f_out) a.f_out[static_cast<size_t>(s) * a.N + i] = f;
    }
    a.g[static_cast<size_t>(s) * a.Npad + i] = gv;
    if (a.ghl) {   // shared-shape variant: TF32 hi / lo parts for the backward GEMM
        const float gh = tf32_hi(gv);
        a.ghl[static_cast<size_t>(s) * a.Npad + i] = gh;
        a.ghl[static_cast<size_t>(a.S) * a.Npad + static_cast<size_t>(s) * a.Npad + i] = gv - gh;
    }
    dev = warp_sumf(dev);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) shf[w] = dev;
    if (a.wfar) {
        // node weights of g: W_p = sum_i g_i lam_p(x_i).  A reduce-scatter
        // leaves lane p of each warp with its warp's sum for node p.
        __shared__ float shw[kTile / 32][kFarNodes];
        float v[kFarNodes];
#pragma unroll
        for (int p = 0; p < kFarNodes; ++p) v[p] = gv * lam[p * kTile];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const bool up = (l & o) != 0;
#pragma unroll
            for (int j = 0; j < o; ++j) {
                const float send = up ? v[j] : v[j + o];
                const float keep = up ? v[j + o] : v[j];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        shw[w][l] = v[0];
        if (a.wfar2) asm volatile("cp.async.wait_all;\n" ::: "memory");   // sMb complete before the sync
        __syncthreads();
        // every warp forms W_p at lane p (the same sum in each)
        float t = 0.f;
#pragma unroll
        for (int ww = 0; ww < kTile / 32; ++ww) t += shw[ww][l];
        if (w == 0) a.wfar[static_cast<size_t>(blk.x()) * kFarNodes + l] = t;
        if (a.wfar2) {
            // this tile's part of the super-tile's node weights, sum_p Mb[t][p][P] W_t,p
            // at lane P: warp w takes nodes p of [w n, (w + 1) n), the sum of the parts
            // follows the last sync (k_bwd_direct adds the member tiles' sums in tile order)
            constexpr int n = kFarNodes / (kTile / 32);
            static_assert(n * (kTile / 32) == kFarNodes, "nodes split evenly over the warps");
            float w2 = 0.f;
#pragma unroll
            for (int j = 0; j < n; ++j)
                w2 = fmaf(sMb[(w * n + j) * kFarNodes + l], __shfl_sync(0xffffffffu, t, w * n + j), w2);
            sW2[w][l] = w2;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < kTile / 32 ? shf[threadIdx.x] : 0.f;
        t = warp_sumf(t);
        if (threadIdx.x == 0) a.llpart[static_cast<size_t>(s) * a.T + tile] = static_cast<double>(t);
        if (a.wfar2) {
            float w2 = 0.f;
#pragma unroll
            for (int ww = 0; ww < kTile / 32; ++ww) w2 += sW2[ww][threadIdx.x];
            a.wfar2[static_cast<size_t>(blk.x()) * kFarNodes + threadIdx.x] = w2;
        }
    }
    if (a.Tb) {   // fitted background: d LL / d beta_j = sum_i g_i B_i(beta) T_j(z_i), per tile
        __shared__ float shb[3][kTile / 32];
        float v[3] = {0.f, 0.f, 0.f};
        if (i < a.N) {
            const float gb = gv * a.bg[i];
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = gb * a.Tb[static_cast<size_t>(j) * a.N + i];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            v[j] = warp_sumf(v[j]);
            if (l == 0) shb[j][w] = v[j];
        }
        __syncthreads();
        if (threadIdx.x < 32) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float t = threadIdx.x < kTile / 32 ? shb[j][threadIdx.x] : 0.f;
                t = warp_sumf(t);
                if (threadIdx.x == 0) a.bgpart[(static_cast<size_t>(s) * a.T + tile) * 3 + j] = t;
            }
        }
    }
}

__global__ void __launch_bounds__(kTile) k_lik(ProfArgs a) { lik_body(a, GridBlock()); }

// --- backward -----------------------------------------------------------------
// Gradient sums per (sample, phase, tile), with q = (y/f - 1) I:
//   0 S1G = sum q G          1 S1L = sum q L
//   2 AG  = sum q G t        3 AL  = sum q L^2 t
//   4 AGs = sum q G |t|      5 ALs = sum q L^2 |t|
//   6 BG  = sum q G t^2      7 BL  = sum q L^2 t^2
//   8 BGs = sum q G t|t|     9 BLs = sum q L^2 t|t|
// (t carries the sign of d, so the |t| sums separate the two sides; on a
// side-uniform range |t| = +-t and those sums follow from the plain ones).

// Lorentzian part on one side-uniform range: S1 += sum q L, A += sum q L^2 t,
// C2 += sum q L^2.  Since L (1 + t^2) = 1, q L^2 t^2 = q L - q L^2, so the
// range's sum q L^2 t^2 is S1 - C2 and needs no product of its own.  The
// sums over the range's peaks are taken per point without the point's factor
// g = y/f - 1, which multiplies them once at the end (q = g I).
template <class Tab, class Sc>
__device__ __forceinline__ void bwdL_uniform(const ProfArgs &a, const Tab &tab, float4 *wb, int i0, int lane,
                                             const float *gs, int m0, int m1, float sc, float cmu, float x0,
                                             const Sc &ps, f2_t &S1, f2_t &A, f2_t &C2) {
    if (m0 >= m1) return;
    const f2_t s2 = bc2(sc), one2 = bc2(1.f);
    f2_t dx2[kPairs];
    rel_points(a, i0, lane, x0, dx2);
    f2_t S1p[kPairs], Ap[kPairs], C2p[kPairs];
#pragma unroll
    for (int q = 0; q < kPairs; ++q) S1p[q] = Ap[q] = C2p[q] = 0ull;
    for (int mb = m0; mb < m1; mb += 32) {
        const int n = min(32, m1 - mb);
        fill_offsets(tab, wb, lane, mb, n, sc, cmu, x0);
        for (int j = 0; j < n; ++j) {
            const float4 v = wb[j];
            const f2_t b = pk2(v.x, v.y), I = pk2(v.z, v.w);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t t = ps(fma2(s2, dx2[q], b), q);
                const f2_t L = rcp2(fma2(t, t, one2));
                const f2_t q1 = mul2(I, L);
                S1p[q] = add2(S1p[q], q1);
                const f2_t q2 = mul2(q1, L);
                Ap[q] = fma2(q2, t, Ap[q]);
                C2p[q] = add2(C2p[q], q2);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        const f2_t g2 = pk2(gs[(2 * q) * 32], gs[(2 * q + 1) * 32]);   // g = y/f - 1 (0 on padding)
        S1 = fma2(g2, S1p[q], S1);
        A = fma2(ps(g2, q), Ap[q], A);   // mu sums: g cos(x/2) in the angle-dependent variant
        C2 = fma2(g2, C2p[q], C2);
    }
}

template <bool kWide, bool kSec = false>
__global__ void __launch_bounds__(kThreads, 4) k_bwd_uniform(ProfArgs a) {
    extern __shared__ float4 s_raw[];
    __shared__ float4 s_wb[kWarps][32];
    int *s_off;
    const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
    const int lane = threadIdx.x & 31;
    float4 *wb = s_wb[threadIdx.x >> 5];
    const int items = a.S * a.T * a.C;
    for (int item = next_item(a.counter, lane); item < items; item = next_item(a.counter, lane)) {
        const int c = item % a.C;
        const int st = item / a.C;
        const int s = st / a.T, tile = st - s * a.T;
        const int i0 = tile * kTile;
        const float xlo = a.x[i0], xhi = a.x[min(i0 + kTile - 1, a.N - 1)];
        PtScale<kSec> ps;
        ps.load(a, i0, lane);
        const float *gs = a.g + static_cast<size_t>(s) * a.Npad + i0 + lane;
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = a.chunk[c]; k < a.chunk[c + 1]; ++k) {
            const PhaseConst cp = cs[k];
            const Ranges r = load_ranges(a, s_off, s, k, tile);
            // the lane's sums over its points, per side
            float S1 = 0.f, A[2] = {0.f, 0.f}, B[2] = {0.f, 0.f};
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                f2_t S1s = 0ull, As = 0ull, C2s = 0ull;
                bwdL_uniform(a, tab, wb, i0, lane, gs, side ? r.m2 : r.fb, side ? r.fe : r.m1, side ? cp.sl : cp.sr,
                             side ? cp.nslmu : cp.nsrmu, side ? xhi : xlo, ps, S1s, As, C2s);
                S1 += sum2(S1s);
                const float as = sum2(As), bs = sum2(sub2(S1s, C2s));
                if (side) { A[1] = as; B[1] = bs; } else { A[0] = as; B[0] = bs; }
            }
            // side 0: all d > 0 (|t| = t); side 1: all d < 0 (|t| = -t)
            float v[5] = {S1, A[0] + A[1], A[0] - A[1], B[0] + B[1], B[0] - B[1]};
#pragma unroll
            for (int j = 0; j < 5; ++j) v[j] = warp_sumf(v[j]);
            if (lane == 0) {
                float2 *dst = reinterpret_cast<float2 *>(
                    a.gpart + ((static_cast<size_t>(s) * a.K + k) * a.T + tile) * kGradSums);
#pragma unroll
                for (int j = 0; j < 5; ++j) dst[j] = make_float2(0.f, v[j]);
            }
        }
    }
}

// Accumulate v * |t| into a packed pair of sums (scalar FMAs: |t| is a free
// operand modifier of the scalar instruction).
__device__ __forceinline__ f2_t fma_abs2(f2_t v, f2_t t, f2_t acc) {
    float t0, t1, v0, v1, a0, a1;
    up2(t, t0, t1);
    up2(v, v0, v1);
    up2(acc, a0, a1);
    return pk2(fmaf(v0, fabsf(t0), a0), fmaf(v1, fabsf(t1), a1));
}

// Near part of one phase's gradient sums on a tile (mixed range: both
// components with the side chosen per point; Gaussian terms on the
// side-uniform ranges within its reach), accumulated into acc[kGradSums]
// (even entries Gaussian, odd Lorentzian: S1, A, A|t|, B, B|t|).
template <class Tab, class Sc, class PC>
__device__ __forceinline__ void bwd_near_sums(const Tab &tab, const Ranges &r, const PC &cp,
                                              const f2_t (&x2)[kPairs], const f2_t (&g2)[kPairs], const Sc &ps,
                                              f2_t (&acc)[kGradSums]) {
    const f2_t nmu2 = bc2(-cp.mu), one2 = bc2(1.f), sl2 = bc2(cp.sl), ds2 = bc2(cp.sr - cp.sl);
    for (int m = r.m1; m < r.m2; ++m) {
        f2_t np, I;
        tab.get(m, np, I);
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            const f2_t t = ps(t_mixed(x2[q], np, nmu2, sl2, ds2), q);
            const f2_t tA = ps(t, q);   // t for the mu sums (times cos(x/2) once more)
            const f2_t u = mul2(t, t);
            const f2_t L = rcp2(add2(u, one2));
            const f2_t gI = mul2(g2[q], I);
            const f2_t q1 = mul2(gI, L);
            acc[1] = add2(acc[1], q1);
            const f2_t q2 = mul2(q1, L);
            acc[3] = fma2(q2, tA, acc[3]);
            acc[5] = fma_abs2(q2, tA, acc[5]);
            const f2_t q3 = mul2(q2, t);
            acc[7] = fma2(q3, t, acc[7]);
            acc[9] = fma_abs2(q3, t, acc[9]);
            if (any_gauss(u)) {
                const f2_t qg = mul2(gI, ex2neg2(u));
                acc[0] = add2(acc[0], qg);
                acc[2] = fma2(qg, tA, acc[2]);
                acc[4] = fma_abs2(qg, tA, acc[4]);
                const f2_t q3g = mul2(qg, t);
                acc[6] = fma2(q3g, t, acc[6]);
                acc[8] = fma_abs2(q3g, t, acc[8]);
            }
        }
    }
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int m0 = side ? r.m2 : min(r.nb, r.m1), m1 = side ? max(r.ne, r.m2) : r.m1;
        const f2_t s2 = bc2(side ? cp.sl : cp.sr), c2 = bc2(side ? cp.nslmu : cp.nsrmu);
        f2_t S1 = 0ull, A = 0ull, B = 0ull;
        for (int m = m0; m < m1; ++m) {
            f2_t np, I;
            tab.get(m, np, I);
#pragma unroll
            for (int q = 0; q < kPairs; ++q) {
                const f2_t t = ps(fma2(s2, add2(x2[q], np), c2), q);
                const f2_t u = mul2(t, t);
                if (any_gauss(u)) {
                    const f2_t qg = mul2(mul2(g2[q], I), ex2neg2(u));
                    S1 = add2(S1, qg);
                    A = fma2(qg, ps(t, q), A);
                    B = fma2(mul2(qg, t), t, B);
                }
            }
        }
        acc[0] = add2(acc[0], S1);
        acc[2] = add2(acc[2], A);
        acc[6] = add2(acc[6], B);
        acc[4] = side ? sub2(acc[4], A) : add2(acc[4], A);
        acc[8] = side ? sub2(acc[8], B) : add2(acc[8], B);
    }
}

// Near part of the gradient sums (mixed range: both components; Gaussian on
// the side-uniform ranges), added to the sums k_bwd_uniform wrote.  The
// ranges of 32 phases are loaded at once, one per lane, and only the phases
// with near work on this tile (a warp ballot) are visited.
template <bool kWide, bool kSec = false>
__global__ void __launch_bounds__(kThreads, 3) k_bwd_near(ProfArgs a) {
    extern __shared__ float4 s_raw[];
    int *s_off;
    const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
    const int lane = threadIdx.x & 31;
    const int items = a.S * a.T * a.C;
    for (int item = next_item(a.counter, lane); item < items; item = next_item(a.counter, lane)) {
        const int c = item % a.C;
        const int st = item / a.C;
        const int s = st / a.T, tile = st - s * a.T;
        const int i0 = tile * kTile;
        f2_t x2[kPairs], g2[kPairs];
        PtScale<kSec> ps;
        bool loaded = false;
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        const int kend = a.chunk[c + 1];
        for (int kb = a.chunk[c]; kb < kend; kb += 32) {
            const int kl = kb + lane;
            Ranges rl;
            bool work = false;
            if (kl < kend) {
                rl = load_ranges(a, s_off, s, kl, tile);
                work = near_work(rl);
            }
            unsigned mask = __ballot_sync(0xffffffffu, work);
            if (mask && !loaded) {
                item_points(a, i0, lane, x2);
                ps.load(a, i0, lane);
                const float *gs = a.g + static_cast<size_t>(s) * a.Npad + i0 + lane;
#pragma unroll
                for (int q = 0; q < kPairs; ++q) g2[q] = pk2(gs[(2 * q) * 32], gs[(2 * q + 1) * 32]);
                loaded = true;
            }
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int k = kb + src;
                Ranges r;
                r.mb = __shfl_sync(0xffffffffu, rl.mb, src);
                r.m1 = __shfl_sync(0xffffffffu, rl.m1, src);
                r.m2 = __shfl_sync(0xffffffffu, rl.m2, src);
                r.me = __shfl_sync(0xffffffffu, rl.me, src);
                r.nb = __shfl_sync(0xffffffffu, rl.nb, src);
                r.ne = __shfl_sync(0xffffffffu, rl.ne, src);
                const PhaseConst cp = cs[k];
                f2_t acc[kGradSums];
#pragma unroll
                for (int j = 0; j < kGradSums; ++j) acc[j] = 0ull;
                bwd_near_sums(tab, r, cp, x2, g2, ps, acc);
                float v[kGradSums];
#pragma unroll
                for (int j = 0; j < kGradSums; ++j) v[j] = warp_sumf(sum2(acc[j]));
                if (lane == 0) {
                    float2 *dst = reinterpret_cast<float2 *>(
                        a.gpart + ((static_cast<size_t>(s) * a.K + k) * a.T + tile) * kGradSums);
#pragma unroll
                    for (int j = 0; j < kGradSums; j += 2) {
                        const float2 o = dst[j / 2];
                        dst[j / 2] = make_float2(o.x + v[j], o.y + v[j + 1]);
                    }
                }
            }
        }
    }
}

// Direct backward sums with the far field on: per (sample, tile, phase chunk)
// and phase, the Lorentzian sums of the side-uniform band [fb, m1), [m2, fe)
// and the near part (bwd_near_sums), reduced once and written to gpart (the
// far-field kernel adds its part afterwards).  The band holds a few peaks per
// phase, so one kernel with the point coordinates and g in registers replaces
// the dense path's side-uniform + near pair.
// Warp sum of 16 values by recursive halving (8 + 4 + 2 + 1 + 1 shuffles):
// lane l ends with the total of value (l >> 1) & 15 in v[0].
template <class V>
__device__ __forceinline__ void warp_reduce_scatter16(V (&v)[16], int lane) {
#pragma unroll
    for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const V send = up ? v[j] : v[j + n];
            const V keep = up ? v[j + n] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Gradient sums with the far field on: per (sample, tile, phase chunk) and
// phase, the direct sums at the tile's points (near band, mixed range,
// Gaussian reach) plus, at lane p, the far sums at node p weighted by W_p
// (and, for a super-tile's first tile, the super-far sums at super node p
// weighted by W2_p, which k_grad attributes to the phase like any tile's),
// reduced once and written to gpart.
template <bool kWide, bool kSec>
__device__ __forceinline__ void bwd_direct_items(const ProfArgs &a, const PeakTable<kWide> &tab, const int *s_off) {
    const int lane = threadIdx.x & 31;
    const f2_t one2 = bc2(1.f);
    const int items = a.S * a.T * a.C;
    for (int item = next_item(a.counter, lane); item < items; item = next_item(a.counter, lane)) {
        const int c = item % a.C;
        const int st = item / a.C;
        const int s = st / a.T, tile = st - s * a.T;
        const int i0 = tile * kTile;
        f2_t x2[kPairs], g2[kPairs];
        item_points(a, i0, lane, x2);
        PtScale<kSec> ps;
        ps.load(a, i0, lane);
        const float *gs = a.g + static_cast<size_t>(s) * a.Npad + i0 + lane;
#pragma unroll
        for (int q = 0; q < kPairs; ++q) g2[q] = pk2(gs[(2 * q) * 32], gs[(2 * q + 1) * 32]);
        // far field: this lane's node, its weight W_p = sum_i g_i lam_p(x_i), and
        // for a super-tile's first tile the super node and W2_P = sum_t sum_p Mb[t][p][P] W_t,p
        // (k_lik leaves each tile's sum over p in wfar2)
        const bool lvl2 = a.Tg && tile % kSuperTiles == 0;
        const int g = tile / kSuperTiles;
        const float xn = a.node_x[tile * kFarNodes + lane];
        const float cn = kSec ? a.node_c[tile * kFarNodes + lane] : 1.f;
        const float wn = a.wfar[(static_cast<size_t>(s) * a.T + tile) * kFarNodes + lane];
        float xn2 = 0.f, cn2 = 1.f, wn2 = 0.f;
        if (lvl2) {
            xn2 = a.node_x2[g * kFarNodes + lane];
            if (kSec) cn2 = a.node_c2[g * kFarNodes + lane];
            const int t1 = min(tile + kSuperTiles, a.T);
            for (int t = tile; t < t1; ++t) wn2 += a.wfar2[(static_cast<size_t>(s) * a.T + t) * kFarNodes + lane];
        }
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = a.chunk[c]; k < a.chunk[c + 1]; ++k) {
            const PhaseConst cp = cs[k];
            const Ranges r = load_ranges(a, s_off, s, k, tile);
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
            // near band: lane-local Lorentzian sums per side (a few peaks; g applied per point at the end)
            float A[2] = {0.f, 0.f}, B[2] = {0.f, 0.f};
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                const int m0 = side ? r.m2 : r.fb, m1 = side ? r.fe : r.m1;
                if (m0 >= m1) continue;
                const f2_t s2 = bc2(side ? cp.sl : cp.sr), c2 = bc2(side ? cp.nslmu : cp.nsrmu);
                f2_t S1p[kPairs], Ap[kPairs], C2p[kPairs];
#pragma unroll
                for (int q = 0; q < kPairs; ++q) S1p[q] = Ap[q] = C2p[q] = 0ull;
                for (int m = m0; m < m1; ++m) {
                    f2_t np, I;
                    tab.get(m, np, I);
#pragma unroll
                    for (int q = 0; q < kPairs; ++q) {
                        const f2_t t = ps(fma2(s2, add2(x2[q], np), c2), q);
                        const f2_t L = rcp2(fma2(t, t, one2));
                        const f2_t q1 = mul2(I, L);
                        S1p[q] = add2(S1p[q], q1);
                        const f2_t q2 = mul2(q1, L);
                        Ap[q] = fma2(q2, t, Ap[q]);
                        C2p[q] = add2(C2p[q], q2);
                    }
                }
                f2_t S1s = 0ull, As = 0ull, C2s = 0ull;
#pragma unroll
                for (int q = 0; q < kPairs; ++q) {
                    S1s = fma2(g2[q], S1p[q], S1s);
                    As = fma2(ps(g2[q], q), Ap[q], As);
                    C2s = fma2(g2[q], C2p[q], C2s);
                }
                v[1] += sum2(S1s);
                A[side] = sum2(As);
                B[side] = sum2(sub2(S1s, C2s));
            }
            {   // far peaks at the nodes (lane-local, folded into the same sums)
                const FarRanges fr = far_ranges(r);
                far_node_grad<PeakTable<kWide>, PhaseConst, kSec>(tab, cp, xn, cn, wn, wn * cn, fr.l1[0], fr.l1[1],
                                                                  fr.l1[2], fr.l1[3], v[1], A, B);
                if (lvl2)
                    far_node_grad<PeakTable<kWide>, PhaseConst, kSec>(tab, cp, xn2, cn2, wn2, wn2 * cn2, fr.l2[0],
                                                                      fr.l2[1], fr.l2[2], fr.l2[3], v[1], A, B);
            }
            // side 0: all d > 0 (|t| = t); side 1: all d < 0 (|t| = -t)
            v[3] = A[0] + A[1];
            v[5] = A[0] - A[1];
            v[7] = B[0] + B[1];
            v[9] = B[0] - B[1];
            if (near_work(r)) {   // warp-uniform
                f2_t acc[kGradSums];
#pragma unroll
                for (int j = 0; j < kGradSums; ++j) acc[j] = 0ull;
                bwd_near_sums(tab, r, cp, x2, g2, ps, acc);
#pragma unroll
                for (int j = 0; j < kGradSums; ++j) v[j] += sum2(acc[j]);
            }
            warp_reduce_scatter16(v, lane);
            const int j = (lane >> 1) & 15;
            if ((lane & 1) == 0 && j < kGradSums)
                a.gpart[((static_cast<size_t>(s) * a.K + k) * a.T + tile) * kGradSums + j] = v[0];
        }
    }
}

template <bool kWide, bool kSec>
__global__ void __launch_bounds__(kThreads, 3) k_bwd_direct(ProfArgs a) {
    extern __shared__ float4 s_raw[];
    int *s_off;
    const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
    bwd_direct_items<kWide, kSec>(a, tab, s_off);
}

// ---------------------------------------------------------------------------
// Gradient reduction + Adam + ELBO
// ---------------------------------------------------------------------------
struct GradArgs {
    int S, K, T;
    PriorConst pr;
    double csum;
    const float *gpart, *theta, *eps;
    const float *loc_in, *raw_in;
    float *loc_out, *raw_out, *grad_out;
    int adam;
    AdamConst ac;
    float *m, *v;
    const int *d_iter;
    int *d_step;
    const double *llpart, *lpj, *ent;
    double *ll, *elbo_out, *trace;
    double *gred;   // [B*K*kGradBlocks*10] per-sample-block partial sums
    int *tickets;   // [B*K] arrival tickets (zeroed by k_sample, reset by the last block)
    int NB;         // sample blocks per phase
    int B, S_sub;   // sub-model batch (B = 1, S_sub = S: one model)
    const uint32_t *mask;
    double *tail_sum;   // [B] (may be null): ELBO estimates summed from step tail_start on
    int tail_start;
    int elbo_blocks;    // k_grad's grid carries this many extra blocks that do k_elbo's work (0: none)
    const double *lq;   // [S] ln q(u_s) (importance-weighted objective)
    double *iw;         // [S] normalised importance weights (null: the ELBO)
    int Tg;             // tiles per (sample, phase) record of gpart (T, or 1 for the shared-shape variant)
    // FP32 prior constants of the per-sample gradient
    float pr_lambda, pr_mu_isd2, pr_w_shape, pr_w_rate, pr_alpha_mean, pr_alpha_isd2;
    int fix_r, fix_a;   // r / alpha held fixed: zero gradient, no update
    int area_norm;      // area-normalised profiles
    const float *gzy;   // [S*K*2] gate z, y (null: no gates)
    float gate_tau, gate_a0;
    float *gate_a, *m_gate, *v_gate;   // [K] gate logits and their Adam moments
    float *grad_gate;   // [K] gate gradient out (may be null)
    int *nonfinite;     // set to 1 when a gradient entry is NaN or infinite (may be null)
};

// ELBO = mean_s [LL_s + log prior + log Jacobian] + entropy, in FP64 with a
// fixed summation order; also advances the step counter of the fit loop.
__device__ void elbo_block(const GradArgs &a, int b) {   // b: sub-model
    __shared__ double sh[8];
    double acc = 0.0;
    for (int s = b * a.S_sub + threadIdx.x; s < (b + 1) * a.S_sub; s += blockDim.x) {
        double ll = a.csum;
        const double *lp = a.llpart + static_cast<size_t>(s) * a.T;
        for (int t = 0; t < a.T; ++t) ll += lp[t];
        a.ll[s] = ll;
        acc += ll + a.lpj[s];
    }
    double iw_bound = 0.0;
    if (a.iw) {
        // importance-weighted bound (Burda et al. 2016): ln w_s = LL + ln p + ln|J| - ln q,
        // L = logsumexp(ln w) - ln S; the normalised weights drive k_grad
        __syncthreads();   // a.ll of this block written
        double mx = -CUDART_INF;
        for (int s = b * a.S_sub + threadIdx.x; s < (b + 1) * a.S_sub; s += blockDim.x)
            mx = fmax(mx, a.ll[s] + a.lpj[s] - a.lq[s]);
        mx = block_max(mx, sh);
        double se = 0.0;
        for (int s = b * a.S_sub + threadIdx.x; s < (b + 1) * a.S_sub; s += blockDim.x)
            se += exp(a.ll[s] + a.lpj[s] - a.lq[s] - mx);
        se = block_sum(se, sh);
        for (int s = b * a.S_sub + threadIdx.x; s < (b + 1) * a.S_sub; s += blockDim.x)
            a.iw[s] = exp(a.ll[s] + a.lpj[s] - a.lq[s] - mx) / se;
        iw_bound = mx + log(se) - log(static_cast<double>(a.S_sub));
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        const double elbo = a.iw ? iw_bound : acc / a.S_sub + a.ent[b];
        if (a.elbo_out) a.elbo_out[b] = elbo;
        if (a.d_iter) {
            const int it = *a.d_iter;
            if (a.trace && b == 0) a.trace[it & (kTraceCap - 1)] = elbo;
            if (a.tail_sum && it >= a.tail_start) a.tail_sum[b] += elbo;
            if (a.d_step && b == 0) *a.d_step = it + 1;
        }
    }
}

__global__ void __launch_bounds__(256) k_elbo(GradArgs a) { elbo_block(a, blockIdx.x); }

// Gradient of the ELBO for phase k = blockIdx.x over sample block
// blockIdx.y, 32 samples at a time.  Stage 1: one warp per (sample, phase)
// record, the lanes read the record's tiles (coalesced) and tree-sum the ten
// partial sums in FP32 into shared memory.  Stage 2: warp 0, one sample per
// lane, forms the per-sample gradient in FP64 and accumulates it; the lanes
// are combined by a fixed shuffle tree.  The last block of the phase to
// arrive adds the block totals in a fixed order (deterministic) and applies
// Adam.
template <class Blk>
__device__ __forceinline__ void grad_body(const GradArgs &a, Blk blk) {
    __shared__ float qs[32][kGradSums + 1];
    __shared__ double red[kGredVals];
    __shared__ int is_last;
    const int bk = blk.x(), b = blk.y();   // (sub-model, phase), sample block
    if (a.elbo_blocks && bk >= a.B * a.K) {   // extra blocks: the ELBO of sub-model bk - B K, beside the gradient
        if (b == 0) elbo_block(a, bk - a.B * a.K);
        return;
    }
    const int sm = bk / a.K, k = bk - sm * a.K;
    if (a.mask && !((a.mask[sm] >> k) & 1u)) return;   // phase not in this sub-model (whole block)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = sm * a.S_sub + static_cast<int>((static_cast<long long>(a.S_sub) * b) / a.NB);
    const int s1 = sm * a.S_sub + static_cast<int>((static_cast<long long>(a.S_sub) * (b + 1)) / a.NB);
    double accl[5] = {0, 0, 0, 0, 0}, acce[5] = {0, 0, 0, 0, 0}, accg = 0.0;
    for (int c0 = s0; c0 < s1; c0 += 32) {
        const int nc = s1 - c0 < 32 ? s1 - c0 : 32;
        for (int i = warp; i < nc; i += kWarps) {
            const size_t sk = static_cast<size_t>(c0 + i) * a.K + k;
            const float2 *gp = reinterpret_cast<const float2 *>(a.gpart + sk * a.Tg * kGradSums);
            float qf[16];   // the ten sums, padded for one reduce-scatter (16 shuffles for all ten)
#pragma unroll
            for (int j = 0; j < 16; ++j) qf[j] = 0.f;
            for (int t = lane; t < a.Tg; t += 32) {
#pragma unroll
                for (int j = 0; j < kGradSums / 2; ++j) {
                    const float2 v = gp[t * (kGradSums / 2) + j];
                    qf[2 * j] += v.x;
                    qf[2 * j + 1] += v.y;
                }
            }
            warp_reduce_scatter16(qf, lane);   // lane 2j holds the warp's total of sum j
            if ((lane & 1) == 0 && (lane >> 1) < kGradSums) qs[i][lane >> 1] = qf[0];
        }
        __syncthreads();
        if (warp == 0 && lane < nc) {
            // per-sample gradient in FP32 (its inputs are FP32 sums; FP64 keeps
            // the accumulation over samples, where the terms cancel)
            float q[kGradSums];
#pragma unroll
            for (int j = 0; j < kGradSums; ++j) q[j] = qs[lane][j];
            const size_t sk = static_cast<size_t>(c0 + lane) * a.K + k;
            const float *th = a.theta + sk * 5;
            const float *ep = a.eps + sk * 5;
            const float h = th[0], mu = th[1], w = th[2], r = th[3], al = th[4];
            const float amin = static_cast<float>(a.pr.alpha_min);
            const bool clamped = !(al > amin);
            const float acl = clamped ? amin : al;
            const float sl = __fdiv_rn(2.f, w), sr = __fdiv_rn(2.f, acl * w);
            const float ln2f = static_cast<float>(kLn2);
            // side splits: X+ = (X + Xs)/2 (d >= 0), X- = (X - Xs)/2 (d < 0)
            const float AGp = 0.5f * (q[2] + q[4]), AGm = 0.5f * (q[2] - q[4]);
            const float ALp = 0.5f * (q[3] + q[5]), ALm = 0.5f * (q[3] - q[5]);
            const float BGp = 0.5f * (q[6] + q[8]), BLp = 0.5f * (q[7] + q[9]);
            float G[5];
            // the profile scale he: h, or h / a(w, alpha, r) for area-normalised
            // profiles, whose derivatives add -he * dLL/dhe * d ln a / d(u_w, r, alpha)
            const float aw = a.area_norm ? area_factorf(w, acl, r) : 1.f;
            const float zg = a.gzy ? a.gzy[sk * 2] : 1.f;   // gate of this draw and phase
            const float he = (a.area_norm ? __fdiv_rn(h, aw) : h) * zg;
            const float LLh = (1.f - r) * q[0] + r * q[1];   // d LL / d he
            constexpr float kAG = 1.0644670194312262f, kAL = 1.5707963267948966f;
            const float dlna_dr = a.area_norm ? __fdiv_rn(kAL - kAG, fmaf(r, kAL - kAG, kAG)) : 0.f;
            // likelihood part (chained to u) + prior/Jacobian part
            G[0] = he * LLh + (1.f - a.pr_lambda * h);
            G[1] = 2.f * he * ((1.f - r) * ln2f * (sl * AGm + sr * AGp) + r * (sl * ALm + sr * ALp)) -
                   mu * a.pr_mu_isd2;
            G[2] = 2.f * he * ((1.f - r) * ln2f * q[6] + r * q[7]) - (a.area_norm ? he * LLh : 0.f) +
                   (a.pr_w_shape - a.pr_w_rate * w);
            G[3] = a.fix_r ? 0.f : r * (1.f - r) * he * (q[1] - q[0] - dlna_dr * LLh) + (1.f - 2.f * r);
            const float gal = clamped ? 0.f
                                      : __fdiv_rn(2.f * he, acl) * ((1.f - r) * ln2f * BGp + r * BLp) -
                                            (a.area_norm ? __fdiv_rn(he * LLh, 1.f + acl) : 0.f);
            G[4] = a.fix_a ? 0.f : gal - (al - a.pr_alpha_mean) * a.pr_alpha_isd2;
            const double wt = a.iw ? __ldcg(&a.iw[c0 + lane]) : 1.0;   // importance weight w_s / sum w
            if (a.gzy) {   // gate logit: (1/tau) [dLL/dy + d ln p/dy], dLL/dy = he dLL/dhe (1 - z)
                const float yg = a.gzy[sk * 2 + 1];
                const float dlnp = a.gate_tau * (2.f * sigmoidf(a.gate_a0 - a.gate_tau * yg) - 1.f);
                const float gg = __fdiv_rn(he * LLh * (1.f - zg) + dlnp, a.gate_tau);
                accg += a.iw ? wt * static_cast<double>(gg) : static_cast<double>(gg);
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const double gj = a.iw ? wt * static_cast<double>(G[j]) : static_cast<double>(G[j]);
                accl[j] += gj;
                acce[j] += gj * static_cast<double>(ep[j]);
            }
        }
        __syncthreads();
    }
    if (warp == 0) {
        // the block's 11 sums over its samples by one FP64 reduce-scatter
        // (16 additions instead of 55 for 11 butterfly sums)
        static_assert(kGredVals <= 16, "block sums fit one reduce-scatter");
        double v[16];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            v[j] = accl[j];
            v[5 + j] = acce[j];
        }
        v[10] = accg;
#pragma unroll
        for (int j = 11; j < 16; ++j) v[j] = 0.0;
        warp_reduce_scatter16(v, lane);
        const int j = (lane >> 1) & 15;
        if ((lane & 1) == 0 && j < kGredVals) a.gred[(static_cast<size_t>(bk) * a.NB + b) * kGredVals + j] = v[0];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&a.tickets[bk], 1) == a.NB - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x < kGredVals) {
        double tot = 0.0;
        for (int bb = 0; bb < a.NB; ++bb)
            tot += __ldcg(&a.gred[(static_cast<size_t>(bk) * a.NB + bb) * kGredVals + threadIdx.x]);
        red[threadIdx.x] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.tickets[bk] = 0;
    if (threadIdx.x == 10 && a.gzy) {   // gate logit of phase bk (one model: bk = k)
        const double grad = a.iw ? red[10] : red[10] / a.S_sub;
        if (a.grad_gate) a.grad_gate[bk] = static_cast<float>(grad);
        if (a.adam) {
            const int t = *a.d_iter + 1;
            const double gm = -grad;
            const double mm = a.ac.b1 * static_cast<double>(a.m_gate[bk]) + (1.0 - a.ac.b1) * gm;
            const double vv = a.ac.b2 * static_cast<double>(a.v_gate[bk]) + (1.0 - a.ac.b2) * gm * gm;
            a.m_gate[bk] = static_cast<float>(mm);
            a.v_gate[bk] = static_cast<float>(vv);
            const double c1 = 1.0 - static_cast<double>(powf(a.ac.b1, static_cast<float>(t)));
            const double c2 = 1.0 - static_cast<double>(powf(a.ac.b2, static_cast<float>(t)));
            a.gate_a[bk] = static_cast<float>(a.gate_a[bk] - a.ac.lr * (mm / c1) / (sqrt(vv / c2) + a.ac.eps));
        }
    }
    if (threadIdx.x < 10) {
        const int j = threadIdx.x % 5;
        const bool is_raw = threadIdx.x >= 5;
        const double rw = a.raw_in[bk * 5 + j];
        double grad;
        // importance weights are already normalised; the ELBO takes the sample mean
        if (!is_raw) {
            grad = a.iw ? red[j] : red[j] / a.S_sub;
        } else {
            // d/d raw of sigma = softplus(raw): sigmoid(raw); entropy gradient 1 / sigma
            // (both in FP32: FP64 transcendentals are slow on this part)
            const float rwf = static_cast<float>(rw);
            grad = ((a.iw ? red[5 + j] : red[5 + j] / a.S_sub) + static_cast<double>(1.f / softplusf(rwf))) *
                   static_cast<double>(sigmoidf(rwf));
        }
        const bool fixed = (j == 3 && a.fix_r) || (j == 4 && a.fix_a);   // not part of q: no gradient
        if (fixed) grad = 0.0;
        if (a.grad_out) a.grad_out[bk * 10 + threadIdx.x] = static_cast<float>(grad);
        if (a.nonfinite && !isfinite(grad)) atomicOr(a.nonfinite, 1);
        if (a.adam && !fixed) {
            const int t = *a.d_iter + 1;
            const int idx = bk * 10 + threadIdx.x;
            // the Adam rule in FP32 (its state is FP32; FP64 division and square
            // root are slow on this part)
            const float gm = -static_cast<float>(grad);  // minimise -ELBO
            const float b1 = a.ac.b1, b2 = a.ac.b2;
            const float mm = fmaf(b1, a.m[idx], (1.f - b1) * gm);
            const float vv = fmaf(b2, a.v[idx], (1.f - b2) * gm * gm);
            a.m[idx] = mm;
            a.v[idx] = vv;
            const float c1 = 1.f - powf(b1, static_cast<float>(t));
            const float c2 = 1.f - powf(b2, static_cast<float>(t));
            const double step = a.ac.lr * __fdiv_rn(mm, c1) / (sqrtf(__fdiv_rn(vv, c2)) + a.ac.eps);
            if (!is_raw) {
                a.loc_out[bk * 5 + j] = static_cast<float>(a.loc_in[bk * 5 + j] - step);
            } else {
                a.raw_out[bk * 5 + j] = static_cast<float>(rw - step);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_grad(GradArgs a) { grad_body(a, GridBlock()); }

// ---------------------------------------------------------------------------
// Multi-fit step kernels (continuous batching of fits of different K and N):
// one launch runs one SVI-step kernel for every fit of a batch.  Fit f owns
// the blocks [start[f], start[f+1]) of the per-fit grid (sampling, ranges,
// likelihood, gradient); every fit's arguments travel in the launch's
// parameters, and the per-fit body runs on block indices relative to the fit.  The two profile
// kernels are persistent over all fits: a block starts on the fit its index
// falls in and then helps the others, re-staging the peak table for each fit
// it visits; each fit's items come from that fit's own work counter.  Every
// fit's work items and reductions are those of its standalone kernels, so a
// fit's result does not depend on the batch it runs in.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fit_of_block(const FitMap &m, int b) {
    int lo = 0, hi = m.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (m.start[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// The arguments of every fit of a batch, passed by value: they live in the
// kernel's parameter space like a plain kernel's, which the compiler reloads
// instead of holding in registers (a copy in shared memory made the backward
// spill).  Under the 32 KB parameter limit for kMaxBatch fits.
template <class T>
struct MultiArgs {
    T fit[kMaxBatch];
};
static_assert(sizeof(MultiArgs<ProfArgs>) + sizeof(FitMap) < 32000, "kernel parameter space");
static_assert(sizeof(MultiArgs<SampleArgs>) + sizeof(FitMap) < 32000, "kernel parameter space");
static_assert(sizeof(MultiArgs<GradArgs>) + sizeof(FitMap) < 32000, "kernel parameter space");

__global__ void __launch_bounds__(128) k_sample_multi(const __grid_constant__ MultiArgs<SampleArgs> ma, FitMap m) {
    const int f = fit_of_block(m, blockIdx.x);
    sample_body(ma.fit[f], static_cast<int>(blockIdx.x) - m.start[f]);
}

__global__ void __launch_bounds__(256) k_ranges_multi(const __grid_constant__ MultiArgs<ProfArgs> ma, FitMap m) {
    const int f = fit_of_block(m, blockIdx.x);
    ranges_body(ma.fit[f], static_cast<int>(blockIdx.x) - m.start[f], m.start[f + 1] - m.start[f]);
}

__global__ void __launch_bounds__(kTile) k_lik_multi(const __grid_constant__ MultiArgs<ProfArgs> ma, FitMap m) {
    const int f = fit_of_block(m, blockIdx.x);
    lik_body(ma.fit[f], FixedBlock{static_cast<int>(blockIdx.x) - m.start[f], 0});
}

__global__ void __launch_bounds__(256) k_grad_multi(const __grid_constant__ MultiArgs<GradArgs> ma, FitMap m) {
    const int f = fit_of_block(m, blockIdx.x);
    const GradArgs &a = ma.fit[f];
    const int lb = static_cast<int>(blockIdx.x) - m.start[f];
    const int X = a.B * a.K + a.elbo_blocks;   // blocks per sample block (phases, then ELBO blocks)
    grad_body(a, FixedBlock{lb % X, lb / X});
}

// Persistent profile kernels over all fits (forward: kFwd, else backward).
template <bool kFwd, bool kWide>
__global__ void __launch_bounds__(kThreads, 3) k_direct_multi(const __grid_constant__ MultiArgs<ProfArgs> ma,
                                                              FitMap m) {
    extern __shared__ float4 s_raw[];
    __shared__ int s_done;
    const int f0 = fit_of_block(m, blockIdx.x);
    for (int v = 0; v < m.n; ++v) {
        const int f = f0 + v < m.n ? f0 + v : f0 + v - m.n;
        const ProfArgs &a = ma.fit[f];
        __syncthreads();   // every warp is done with the previous fit's table
        if (threadIdx.x == 0) s_done = atomicAdd(a.counter, 0) >= a.S * a.T * a.C;   // nothing left: skip the table
        __syncthreads();
        if (s_done) continue;
        int *s_off;
        const PeakTable<kWide> tab = load_table<kWide>(a, s_raw, s_off);
        if constexpr (kFwd)
            fwd_direct_items<false, kWide, false>(a, tab, s_off);
        else
            bwd_direct_items<kWide, false>(a, tab, s_off);
    }
}

// ---------------------------------------------------------------------------
// Posterior over phase combinations
// ---------------------------------------------------------------------------
struct PostArgs {
    int S, K, T, W, top_m;
    double csum, alpha_min;
    int area_norm;   // area-normalised profiles: the area of phase k is h_k sum_m I_m
    const float *gzy;   // [S*K*2] gate z of each draw (null: no gates)
    const double *llpart, *lpj, *lq, *isum;
    const float *theta;
    double *logw, *pi, *scalars, *combo_logp, *cost;
    uint8_t *bits;
    uint64_t *combos;
    int *order;
    double *heap_cost;
    int *heap_node;
    uint64_t *node_mask;  // [(2*top_m+2) * WK]
    int *node_last;
};

// One block per sample: log importance weight and area-ratio inclusion bits.
__global__ void __launch_bounds__(128) k_post_sample(PostArgs a) {
    __shared__ double sh[4];
    const int s = blockIdx.x;
    const double AG = 0.5 * sqrt(CUDART_PI / kLn2), AL = 0.5 * CUDART_PI;
    double tot = 0.0;
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const float *th = a.theta + (static_cast<size_t>(s) * a.K + k) * 5;
        const double ac = th[4] > static_cast<float>(a.alpha_min) ? static_cast<double>(th[4]) : a.alpha_min;
        // area-normalised profiles: h is already the area per unit intensity
        const double hz = static_cast<double>(th[0]) * (a.gzy ? a.gzy[(static_cast<size_t>(s) * a.K + k) * 2] : 1.f);
        const double area = a.area_norm ? hz * a.isum[k]
                                        : hz * a.isum[k] * ((1.0 + ac) * th[2] * 0.5) *
                                              ((1.0 - th[3]) * AG + static_cast<double>(th[3]) * AL);
        tot += area;
    }
    tot = block_sum(tot, sh);
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const float *th = a.theta + (static_cast<size_t>(s) * a.K + k) * 5;
        const double ac = th[4] > static_cast<float>(a.alpha_min) ? static_cast<double>(th[4]) : a.alpha_min;
        // area-normalised profiles: h is already the area per unit intensity
        const double hz = static_cast<double>(th[0]) * (a.gzy ? a.gzy[(static_cast<size_t>(s) * a.K + k) * 2] : 1.f);
        const double area = a.area_norm ? hz * a.isum[k]
                                        : hz * a.isum[k] * ((1.0 + ac) * th[2] * 0.5) *
                                              ((1.0 - th[3]) * AG + static_cast<double>(th[3]) * AL);
        a.bits[static_cast<size_t>(s) * a.K + k] = (area / tot >= 0.01) ? 1 : 0;
    }
    if (threadIdx.x == 0) {
        double ll = a.csum;
        const double *lp = a.llpart + static_cast<size_t>(s) * a.T;
        for (int t = 0; t < a.T; ++t) ll += lp[t];
        a.logw[s] = ll + a.lpj[s] - a.lq[s];
    }
}

// Block k < K: marginal pi_k and its flip cost.  Block K: IS evidence and ESS.
__global__ void __launch_bounds__(256) k_post_reduce(PostArgs a) {
    __shared__ double sh[8];
    const int k = blockIdx.x;
    if (k < a.K) {
        double cnt = 0.0;
        for (int s = threadIdx.x; s < a.S; s += blockDim.x) cnt += a.bits[static_cast<size_t>(s) * a.K + k];
        cnt = block_sum(cnt, sh);
        if (threadIdx.x == 0) {
            const double p = (cnt + 0.5) / (a.S + 1.0);
            a.pi[k] = p;
            a.cost[k] = fabs(log(p) - log1p(-p));
        }
        return;
    }
    double mx = -CUDART_INF;
    for (int s = threadIdx.x; s < a.S; s += blockDim.x) mx = fmax(mx, a.logw[s]);
    mx = block_max(mx, sh);
    double e1 = 0.0, e2 = 0.0;
    for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
        e1 += exp(a.logw[s] - mx);
        e2 += exp(2.0 * (a.logw[s] - mx));
    }
    e1 = block_sum(e1, sh);
    e2 = block_sum(e2, sh);
    if (threadIdx.x == 0) {
        const double lse1 = mx + log(e1), lse2 = 2.0 * mx + log(e2);
        a.scalars[0] = lse1 - log(static_cast<double>(a.S));
        a.scalars[1] = exp(2.0 * lse1 - lse2);
    }
}

// Stable rank sort of the flip costs (one block).
__global__ void __launch_bounds__(1024) k_post_sort(PostArgs a) {
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const double ck = a.cost[k];
        int rank = 0;
        for (int j = 0; j < a.K; ++j) {
            const double cj = a.cost[j];
            rank += (cj < ck) || (cj == ck && j < k);
        }
        a.order[rank] = k;
    }
}

__device__ __forceinline__ bool heap_less(double c1, int n1, double c2, int n2) {
    return c1 < c2 || (c1 == c2 && n1 < n2);
}

// Best-first enumeration of the top_m most probable combinations (one
// thread).  A flip set is a set of sorted positions; from a set whose largest
// position is `last`, the children are "append last+1" and "replace last by
// last+1".  Costs are sums of non-negative sorted costs, so sets leave the heap
// in non-decreasing cost order and each set is generated exactly once.
__global__ void k_post_topm(PostArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int K = a.K;
    const int WK = (K + 63) / 64;
    double lmode = 0.0;
    for (int k = 0; k < K; ++k) {
        const double p = a.pi[k];
        lmode += (p > 0.5) ? log(p) : log1p(-p);
    }
    int nnodes = 0, hsize = 0;
    // root
    for (int w = 0; w < WK; ++w) a.node_mask[w] = 0ull;
    a.node_last[0] = -1;
    a.heap_cost[0] = 0.0;
    a.heap_node[0] = 0;
    nnodes = 1;
    hsize = 1;
    double lse_m = -CUDART_INF, lse_s = 0.0;
    int out = 0;
    while (hsize > 0 && out < a.top_m) {
        // pop
        const double cst = a.heap_cost[0];
        const int n = a.heap_node[0];
        --hsize;
        if (hsize > 0) {
            const double lc = a.heap_cost[hsize];
            const int ln = a.heap_node[hsize];
            int i = 0;
            for (;;) {
                int l = 2 * i + 1, r = l + 1, b = i;
                double bc = lc;
                int bn = ln;
                if (l < hsize && heap_less(a.heap_cost[l], a.heap_node[l], bc, bn)) { b = l; bc = a.heap_cost[l]; bn = a.heap_node[l]; }
                if (r < hsize && heap_less(a.heap_cost[r], a.heap_node[r], bc, bn)) { b = r; }
                if (b == i) break;
                a.heap_cost[i] = a.heap_cost[b];
                a.heap_node[i] = a.heap_node[b];
                i = b;
            }
            a.heap_cost[i] = lc;
            a.heap_node[i] = ln;
        }
        // emit combination = mode xor flips
        const uint64_t *msk = a.node_mask + static_cast<size_t>(n) * WK;
        uint64_t *dst = a.combos + static_cast<size_t>(out) * a.W;
        for (int w = 0; w < a.W; ++w) dst[w] = 0ull;
        for (int k = 0; k < K; ++k)
            if (a.pi[k] > 0.5) dst[k >> 6] |= 1ull << (k & 63);
        for (int j = 0; j < K; ++j)
            if ((msk[j >> 6] >> (j & 63)) & 1ull) {
                const int k = a.order[j];
                dst[k >> 6] ^= 1ull << (k & 63);
            }
        const double lp = lmode - cst;
        a.combo_logp[out] = lp;
        if (lp > lse_m) {
            lse_s = lse_s * exp(lse_m - lp) + 1.0;
            lse_m = lp;
        } else {
            lse_s += exp(lp - lse_m);
        }
        ++out;
        // children
        const int last = a.node_last[n];
        const int j = last + 1;
        if (j < K) {
            for (int c = 0; c < (last >= 0 ? 2 : 1); ++c) {
                const int nn = nnodes++;
                uint64_t *nm = a.node_mask + static_cast<size_t>(nn) * WK;
                for (int w = 0; w < WK; ++w) nm[w] = msk[w];
                double cc;
                if (c == 0) {
                    nm[j >> 6] |= 1ull << (j & 63);
                    cc = cst + a.cost[a.order[j]];
                } else {
                    nm[last >> 6] &= ~(1ull << (last & 63));
                    nm[j >> 6] |= 1ull << (j & 63);
                    cc = cst - a.cost[a.order[last]] + a.cost[a.order[j]];
                }
                a.node_last[nn] = j;
                // push
                int i = hsize++;
                while (i > 0) {
                    const int p = (i - 1) / 2;
                    if (!heap_less(cc, nn, a.heap_cost[p], a.heap_node[p])) break;
                    a.heap_cost[i] = a.heap_cost[p];
                    a.heap_node[i] = a.heap_node[p];
                    i = p;
                }
                a.heap_cost[i] = cc;
                a.heap_node[i] = nn;
            }
        }
    }
    a.scalars[2] = lse_m + log(lse_s);
    a.scalars[3] = static_cast<double>(out);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Largest table for which the wide layout is used (keeps four blocks per SM).
constexpr size_t kWideTableBytes = 56 * 1024;

template <class F>
static void set_smem_attr(F f, int bytes) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void configure_grids(Problem &P, int sm_count) {
    const size_t offs = static_cast<size_t>(P.K + 1) * sizeof(int);
    P.wide = static_cast<size_t>(P.Mtot) * sizeof(float4) + offs <= kWideTableBytes;
    P.smem = static_cast<size_t>(P.Mtot) * (P.wide ? sizeof(float4) : sizeof(float2)) + offs;
    P.smem_fwd = static_cast<size_t>(P.Mtot) * sizeof(float2) + offs;
    // The attribute is per function, shared by every context: always allow the
    // largest table any context may have, never the current problem's size.
    const int smax = static_cast<int>(static_cast<size_t>(kMaxPeaks) * sizeof(float2) +
                                      static_cast<size_t>(kMaxK + 1) * sizeof(int));
    set_smem_attr(k_forward<false, false>, smax);
    set_smem_attr(k_forward<true, false>, smax);

    set_smem_attr(k_bwd_uniform<false>, smax);
    set_smem_attr(k_bwd_uniform<true>, smax);
    set_smem_attr(k_bwd_near<false>, smax);
    set_smem_attr(k_bwd_near<true>, smax);
    set_smem_attr(k_forward<false, false, true>, smax);
    set_smem_attr(k_bwd_uniform<false, true>, smax);
    set_smem_attr(k_bwd_uniform<true, true>, smax);
    set_smem_attr(k_bwd_near<false, true>, smax);
    set_smem_attr(k_bwd_near<true, true>, smax);
    set_smem_attr(k_fwd_direct<false, false, false>, smax);
    set_smem_attr(k_fwd_direct<false, true, false>, smax);
    set_smem_attr(k_fwd_direct<true, false, false>, smax);
    set_smem_attr(k_fwd_direct<true, true, false>, smax);
    set_smem_attr(k_fwd_direct<false, false, true>, smax);
    set_smem_attr(k_fwd_direct<false, true, true>, smax);
    set_smem_attr(k_bwd_direct<false, false>, smax);
    set_smem_attr(k_bwd_direct<true, false>, smax);
    set_smem_attr(k_bwd_direct<false, true>, smax);
    set_smem_attr(k_bwd_direct<true, true>, smax);
    int bf = 1, bb = 1;
    int bd = 1;
    if (P.wide)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_bwd_direct<true, false>, kThreads, P.smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_bwd_direct<false, false>, kThreads, P.smem);
    if (bd < 1) bd = 1;
    P.grid_bwd_direct = bd * sm_count;
    int bfd = 1;
    if (P.wide)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bfd, k_fwd_direct<false, true, false>, kThreads, P.smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bfd, k_fwd_direct<false, false, false>, kThreads, P.smem);
    if (bfd < 1) bfd = 1;
    P.grid_fwd_direct = bfd * sm_count;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_forward<false, false>, kThreads, P.smem_fwd);
    if (P.wide)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_bwd_uniform<true>, kThreads, P.smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_bwd_uniform<false>, kThreads, P.smem);
    if (bf < 1) bf = 1;
    if (bb < 1) bb = 1;
    P.grid_fwd = bf * sm_count;
    P.grid_bwd = bb * sm_count;
}

static ProfArgs prof_args(const Problem &P, Workspace &W, float *f_out) {
    ProfArgs a;
    a.S = W.S; a.K = P.K; a.N = P.N; a.Npad = P.Npad; a.T = P.T; a.Mtot = P.Mtot; a.C = W.C;
    for (int c = 0; c <= kMaxChunks; ++c) a.chunk[c] = c <= W.C ? W.chunk[c] : P.K;
    a.pos = P.pos; a.inten = P.inten; a.off = P.off;
    a.x = P.x; a.y = P.y; a.bg = P.bg;
    a.cst = W.cst; a.ranges = W.ranges; a.g = W.g; a.f_out = f_out; a.llpart = W.llpart; a.gpart = W.gpart;
    a.fpart = W.fpart; a.counter = W.counters;
    a.gauss = P.gauss ? 1 : 0;
    a.csec = P.csec;
    a.ghl = W.ghl;
    if (P.bgfit) a.bg = P.Bb;   // fitted background: the current curve B(beta)
    a.bgpart = P.bgfit ? W.bgpart : nullptr;
    a.Tb = a.bgpart ? P.Tb : nullptr;   // beta sums only where the sample set keeps them
    const bool far = P.far && W.franges;
    a.franges = far ? W.franges : nullptr;
    a.fnode = far ? W.fnode : nullptr;
    a.wfar = far ? W.wfar : nullptr;
    a.node_x = P.node_x; a.node_c = P.node_c; a.lam = P.lam; a.far_order = P.far_order;
    a.Tg = far && W.sranges ? P.Tg : 0;
    a.sranges = a.Tg ? W.sranges : nullptr;
    a.fnode2 = a.Tg ? W.fnode2 : nullptr;
    a.wfar2 = a.Tg && a.wfar ? W.wfar2 : nullptr;
    a.node_x2 = P.node_x2; a.node_c2 = P.node_c2; a.sgap = P.sgap; a.Mf = P.Mf; a.Mb = P.Mb;
    return a;
}

static int grid_for(int grid_max, int items) {
    const int need = (items + kWarps - 1) / kWarps;
    return need < grid_max ? need : grid_max;
}

void choose_chunks(const Problem &P, const int *offsets, int S, Workspace &W, int max_chunks) {
    const long long base = static_cast<long long>(S) * P.T;
    const long long resident = static_cast<long long>(P.far ? P.grid_fwd_direct : P.grid_fwd) * kWarps;
    const int per_warp = kItemsPerWarp;
    int C = static_cast<int>((per_warp * resident + base - 1) / base);
    C = C < 1 ? 1 : C;
    C = C > kMaxChunks ? kMaxChunks : C;
    C = C > max_chunks ? max_chunks : C;
    C = C < 1 ? 1 : C;
    C = C > P.K ? P.K : C;
    // cut at the first phase boundary reaching c * Mtot / C peaks, leaving at
    // least one phase for every later chunk
    W.chunk[0] = 0;
    int k = 0;
    for (int c = 1; c < C; ++c) {
        const long long target = static_cast<long long>(P.Mtot) * c / C;
        const int kmax = P.K - (C - c);
        int kk = k + 1;
        while (kk < kmax && offsets[kk] < target) ++kk;
        W.chunk[c] = kk;
        k = kk;
    }
    W.chunk[C] = P.K;
    W.C = C;
}

static SampleArgs sample_args(const Problem &P, Workspace &W, const float *loc, const float *raw,
                              const float *eps_in, uint64_t seed, uint32_t tag, const int *d_step, uint32_t step,
                              int *d_iter, double *ent) {
    SampleArgs a;
    a.S = W.S; a.K = P.K; a.loc = loc; a.raw = raw; a.eps_in = eps_in;
    a.key0 = static_cast<uint32_t>(seed & 0xffffffffu);
    a.key1 = static_cast<uint32_t>(seed >> 32);
    a.tag = tag; a.step = step; a.d_step = d_step; a.d_iter = d_iter; a.ent = ent;
    a.pr = P.prior; a.eps = W.eps; a.theta = W.theta; a.cst = W.cst; a.lpj = W.lpj; a.lq = W.lq;
    a.counters = W.counters;
    a.tickets = W.tickets;
    a.B = W.B; a.S_sub = W.B > 1 || W.mask ? W.S_sub : W.S; a.mask = W.mask;
    a.shared = W.shared ? 1 : 0; a.H = W.H; a.Kpad = W.Kpad;
    a.reach_scale = P.sec ? P.sec_max : 1.0f;
    a.beta = P.bgfit ? P.beta : nullptr; a.bg_sd = P.bg_sd;
    a.fix_r = P.fix_r ? 1 : 0; a.fix_a = P.fix_alpha ? 1 : 0; a.r_value = P.r_value; a.a_value = P.alpha_value;
    a.area_norm = P.area_norm ? 1 : 0;
    a.gate_a = P.gates ? P.gate_a : nullptr; a.gate_tau = P.gate_tau; a.gate_a0 = P.gate_a0; a.gzy = W.gzy;
    a.pr_lambda = static_cast<float>(P.prior.lambda);
    a.pr_mu_isd = static_cast<float>(1.0 / P.prior.mu_sd);
    a.pr_alpha_mean = static_cast<float>(P.prior.alpha_mean);
    a.pr_alpha_isd = static_cast<float>(1.0 / P.prior.alpha_sd);
    a.pr_wsm1 = static_cast<float>(P.prior.w_shape - 1.0);
    a.pr_wrate = static_cast<float>(P.prior.w_rate);
    return a;
}

void launch_sample(const Problem &P, Workspace &W, const float *loc, const float *raw,
                   const float *eps_in, uint64_t seed, uint32_t tag, const int *d_step,
                   uint32_t step, int *d_iter, double *ent, cudaStream_t st) {
    k_sample<<<W.S, 128, 0, st>>>(sample_args(P, W, loc, raw, eps_in, seed, tag, d_step, step, d_iter, ent));
}

void launch_lik(const Problem &P, Workspace &W, float *f_out, int C, cudaStream_t st) {
    ProfArgs a = prof_args(P, W, f_out);
    a.C = C;
    k_lik<<<W.S * P.T, kTile, 0, st>>>(a);
}

void launch_forward(const Problem &P, Workspace &W, float *f_out, bool naive, cudaStream_t st, cudaEvent_t *marks) {
    ProfArgs a = prof_args(P, W, f_out);
    const int nr = W.S * P.K * P.T;
    k_ranges<<<(nr + 255) / 256 < 4096 ? (nr + 255) / 256 : 4096, 256, 0, st>>>(a);
    if (marks) cudaEventRecord(marks[0], st);
    // the forward reads the compact table (measured faster than the wide one)
    const int grid = grid_for(P.grid_fwd, W.S * P.T * W.C);
    if (a.fnode) {   // far field on: the direct part only (peak table as the backward's)
        const int gd = grid_for(P.grid_fwd_direct, W.S * P.T * W.C);
        if (P.sec) {
            if (P.wide) k_fwd_direct<false, true, true><<<gd, kThreads, P.smem, st>>>(a);
            else k_fwd_direct<false, false, true><<<gd, kThreads, P.smem, st>>>(a);
        } else if (naive) {
            if (P.wide) k_fwd_direct<true, true, false><<<gd, kThreads, P.smem, st>>>(a);
            else k_fwd_direct<true, false, false><<<gd, kThreads, P.smem, st>>>(a);
        } else {
            if (P.wide) k_fwd_direct<false, true, false><<<gd, kThreads, P.smem, st>>>(a);
            else k_fwd_direct<false, false, false><<<gd, kThreads, P.smem, st>>>(a);
        }
    } else if (P.sec) {   // angle-dependent width (compensated sums)
        k_forward<false, false, true><<<grid, kThreads, P.smem_fwd, st>>>(a);
    } else if (naive) {
        k_forward<true, false><<<grid, kThreads, P.smem_fwd, st>>>(a);
    } else {
        k_forward<false, false><<<grid, kThreads, P.smem_fwd, st>>>(a);
    }
    if (marks) cudaEventRecord(marks[1], st);
    if (marks) cudaEventRecord(marks[2], st);
    k_lik<<<W.S * P.T, kTile, 0, st>>>(a);
}

void launch_backward(const Problem &P, Workspace &W, cudaStream_t st, cudaEvent_t *marks) {
    ProfArgs a = prof_args(P, W, nullptr);
    const int grid = grid_for(P.grid_bwd, W.S * P.T * W.C);
    a.counter = W.counters + 2;
    if (a.wfar) {   // far field on: one direct kernel, then the far-field sums
        const int grid = grid_for(P.grid_bwd_direct, W.S * P.T * W.C);
        if (P.sec) {
            if (P.wide) k_bwd_direct<true, true><<<grid, kThreads, P.smem, st>>>(a);
            else k_bwd_direct<false, true><<<grid, kThreads, P.smem, st>>>(a);
        } else {
            if (P.wide) k_bwd_direct<true, false><<<grid, kThreads, P.smem, st>>>(a);
            else k_bwd_direct<false, false><<<grid, kThreads, P.smem, st>>>(a);
        }
        if (marks) cudaEventRecord(marks[0], st);
    } else if (P.sec) {   // angle-dependent width
        if (P.wide)
            k_bwd_uniform<true, true><<<grid, kThreads, P.smem, st>>>(a);
        else
            k_bwd_uniform<false, true><<<grid, kThreads, P.smem, st>>>(a);
        if (marks) cudaEventRecord(marks[0], st);
        a.counter = W.counters + 3;
        if (P.wide)
            k_bwd_near<true, true><<<grid, kThreads, P.smem, st>>>(a);
        else
            k_bwd_near<false, true><<<grid, kThreads, P.smem, st>>>(a);
    } else {
        if (P.wide)
            k_bwd_uniform<true><<<grid, kThreads, P.smem, st>>>(a);
        else
            k_bwd_uniform<false><<<grid, kThreads, P.smem, st>>>(a);
        if (marks) cudaEventRecord(marks[0], st);
        a.counter = W.counters + 3;
        if (P.wide)
            k_bwd_near<true><<<grid, kThreads, P.smem, st>>>(a);
        else
            k_bwd_near<false><<<grid, kThreads, P.smem, st>>>(a);
    }
    if (marks) cudaEventRecord(marks[1], st);
}

static GradArgs grad_args(const Problem &P, Workspace &W, const float *loc_in, const float *raw_in,
                          float *loc_out, float *raw_out, float *grad_out, bool adam, AdamConst ac, float *m,
                          float *v, const int *d_iter, int *d_step, const double *ent, double *elbo_out,
                          double *trace) {
    GradArgs a;
    a.S = W.S; a.K = P.K; a.T = P.T; a.pr = P.prior; a.csum = P.csum;
    a.gpart = W.gpart; a.theta = W.theta; a.eps = W.eps;
    a.loc_in = loc_in; a.raw_in = raw_in; a.loc_out = loc_out; a.raw_out = raw_out;
    a.grad_out = grad_out; a.adam = adam ? 1 : 0; a.ac = ac; a.m = m; a.v = v;
    a.d_iter = d_iter; a.d_step = d_step; a.llpart = W.llpart; a.lpj = W.lpj; a.ent = ent;
    a.ll = W.ll; a.elbo_out = elbo_out; a.trace = trace;
    a.gred = W.gred; a.tickets = W.tickets;
    a.B = W.B; a.S_sub = W.B > 1 || W.mask ? W.S_sub : W.S; a.mask = W.mask;
    a.tail_sum = W.tail_sum; a.tail_start = W.tail_start;
    a.lq = W.lq; a.iw = W.iw;
    a.Tg = W.shared ? 1 : P.T;
    a.pr_lambda = static_cast<float>(P.prior.lambda);
    a.pr_mu_isd2 = static_cast<float>(1.0 / (P.prior.mu_sd * P.prior.mu_sd));
    a.pr_w_shape = static_cast<float>(P.prior.w_shape);
    a.pr_w_rate = static_cast<float>(P.prior.w_rate);
    a.pr_alpha_mean = static_cast<float>(P.prior.alpha_mean);
    a.pr_alpha_isd2 = static_cast<float>(1.0 / (P.prior.alpha_sd * P.prior.alpha_sd));
    a.fix_r = P.fix_r ? 1 : 0; a.fix_a = P.fix_alpha ? 1 : 0;
    a.area_norm = P.area_norm ? 1 : 0;
    a.nonfinite = P.nonfinite;
    a.gzy = P.gates ? W.gzy : nullptr; a.gate_tau = P.gate_tau; a.gate_a0 = P.gate_a0;
    a.gate_a = P.gate_a; a.m_gate = P.m_gate; a.v_gate = P.v_gate; a.grad_gate = grad_out ? P.grad_gate : nullptr;
    a.NB = (a.S_sub + 31) / 32;   // 32 samples (4 per warp) per block
    a.NB = a.NB < kGradBlocks ? a.NB : kGradBlocks;
    a.elbo_blocks = 0;
    return a;
}

void launch_grad(const Problem &P, Workspace &W, const float *loc_in, const float *raw_in,
                 float *loc_out, float *raw_out, float *grad_out, bool adam, AdamConst ac,
                 float *m, float *v, const int *d_iter, int *d_step, const double *ent,
                 double *elbo_out, double *trace, cudaStream_t st) {
    GradArgs a = grad_args(P, W, loc_in, raw_in, loc_out, raw_out, grad_out, adam, ac, m, v, d_iter, d_step, ent,
                           elbo_out, trace);
    const bool want_grad = grad_out || adam, want_elbo = elbo_out || trace || W.tail_sum;
    a.elbo_blocks = 0;
    if (W.iw) {
        // the importance weights (k_elbo) come before the weighted gradient
        k_elbo<<<W.B, 256, 0, st>>>(a);
        if (want_grad) k_grad<<<dim3(W.B * P.K, a.NB), 256, 0, st>>>(a);
    } else if (want_grad && want_elbo) {
        // the ELBO (which the gradient does not need) in extra blocks of k_grad
        a.elbo_blocks = W.B;
        k_grad<<<dim3(W.B * P.K + W.B, a.NB), 256, 0, st>>>(a);
    } else {
        if (want_grad) k_grad<<<dim3(W.B * P.K, a.NB), 256, 0, st>>>(a);
        if (want_elbo) k_elbo<<<W.B, 256, 0, st>>>(a);
    }
}

// --- multi-fit step (continuous batching) ---------------------------------------
// Fits whose peak tables take the same layout and allow the same number of
// resident profile blocks per SM share one persistent launch; a fit with a
// larger table (fewer blocks per SM) does not lower the others' occupancy.
struct MultiClass {
    bool wide = true;
    int n = 0;
    size_t smem = 0;
    int grid1_fwd = 0, grid1_bwd = 0;   // a class of one fit runs the fit's own kernels on these grids
    int grid1_lik = 0;                  // ... and, if it fills the GPU by itself, its own likelihood kernel
    bool own = false;                   // a fit that fills the GPU by itself: never shared
    MultiArgs<ProfArgs> pf, pb;   // forward (work counter 0) and backward (counter 2) arguments
    FitMap m_fwd, m_bwd;
};

struct MultiStepPlan {
    int cap = 0, n = 0;
    MultiArgs<SampleArgs> sa;
    MultiArgs<ProfArgs> pf;       // every fit: ranges
    MultiArgs<ProfArgs> pl;       // the fits that share profile launches: likelihood
    MultiArgs<GradArgs> ga;
    FitMap m_sample, m_ranges, m_lik, m_grad;
    std::vector<MultiClass> classes;
};

void multi_plan_destroy(MultiStepPlan *p) { delete p; }

MultiStepPlan *multi_plan_create(int cap) {
    if (cap < 1 || cap > kMaxBatch) return nullptr;
    MultiStepPlan *p = new MultiStepPlan();
    p->cap = cap;
    // the shared-memory attribute of the persistent kernels (largest table any fit may have)
    const int smax = static_cast<int>(static_cast<size_t>(kMaxPeaks) * sizeof(float2) +
                                      static_cast<size_t>(kMaxK + 1) * sizeof(int));
    set_smem_attr(k_direct_multi<true, true>, smax);
    set_smem_attr(k_direct_multi<true, false>, smax);
    set_smem_attr(k_direct_multi<false, true>, smax);
    set_smem_attr(k_direct_multi<false, false>, smax);
    return p;
}

bool multi_fit_eligible(const Problem &P, const Workspace &W, bool naive, bool iw) {
    return P.far && W.franges && W.wfar && !W.shared && !P.sec && !P.bgfit && !naive && !iw && W.B == 1 &&
           !W.mask;
}

// Splits `grid` persistent blocks over the fits in proportion to their work
// (at least one block each); blocks that finish their fit help the others.
static void persistent_map(FitMap &m, const std::vector<long long> &items, int grid) {
    const int n = static_cast<int>(items.size());
    long long tot = 0;
    for (long long v : items) tot += v;
    if (grid < n) grid = n;
    m.n = n;
    m.start[0] = 0;
    long long acc = 0;
    for (int f = 0; f < n; ++f) {
        acc += items[f];
        int e = static_cast<int>((acc * grid + tot - 1) / tot);
        e = e < m.start[f] + 1 ? m.start[f] + 1 : e;
        e = e > grid - (n - 1 - f) ? grid - (n - 1 - f) : e;
        m.start[f + 1] = e;
    }
    m.start[n] = grid;
}

static int direct_occupancy(bool fwd, bool wide, size_t smem) {
    int occ = 1;
    if (fwd) {
        if (wide) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direct_multi<true, true>, kThreads, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direct_multi<true, false>, kThreads, smem);
    } else {
        if (wide) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direct_multi<false, true>, kThreads, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direct_multi<false, false>, kThreads, smem);
    }
    return occ < 1 ? 1 : occ;
}

bool multi_plan_set(MultiStepPlan *p, const FitStep *fits, int n, int sm_count, cudaStream_t st) {
    (void)st;
    if (!p || n < 1 || n > p->cap) return false;
    p->n = n;
    p->classes.clear();
    int bs = 0, br = 0, bl = 0, bg = 0;
    p->m_sample.n = p->m_ranges.n = p->m_grad.n = n;
    p->m_lik.n = 0;
    std::vector<long long> work(n), items(n);
    std::vector<int> cls(n);
    for (int f = 0; f < n; ++f) {
        const FitStep &F = fits[f];
        const Problem &P = *F.P;
        Workspace &W = *F.W;
        SampleArgs sa = sample_args(P, W, F.loc, F.raw, nullptr, F.seed, 0u, F.step, 0u, F.iter, F.ent);
        ProfArgs pf = prof_args(P, W, nullptr);
        GradArgs ga = grad_args(P, W, F.loc, F.raw, F.loc, F.raw, nullptr, true, F.ac, F.m, F.v, F.iter, F.step,
                                F.ent, F.elbo, F.trace);
        ga.elbo_blocks = W.B;   // the ELBO in extra blocks of the gradient kernel, as in a fit step
        p->sa.fit[f] = sa;
        p->pf.fit[f] = pf;
        p->ga.fit[f] = ga;
        p->m_sample.start[f] = bs;
        bs += W.S;
        p->m_ranges.start[f] = br;
        const int nr = W.S * P.K * P.T;
        br += (nr + 255) / 256 < 4096 ? (nr + 255) / 256 : 4096;
        p->m_grad.start[f] = bg;
        bg += (W.B * P.K + ga.elbo_blocks) * ga.NB;
        // the fit's own table layout and residency, as in its standalone kernels
        const size_t tb = P.smem;
        const int occ = std::min(direct_occupancy(true, P.wide, tb), direct_occupancy(false, P.wide, tb));
        // a fit with at least four work items per resident warp fills the GPU
        // by itself: it keeps its own persistent kernels (per-fit arguments in
        // the constant bank), and only the smaller fits share multi-fit launches
        const long long fit_items = static_cast<long long>(W.S) * P.T * W.C;
        const bool own = fit_items >= 4LL * occ * sm_count * kWarps;
        int c = own ? static_cast<int>(p->classes.size()) : 0;
        for (; c < static_cast<int>(p->classes.size()); ++c) {
            if (!p->classes[c].own && p->classes[c].wide == P.wide &&
                std::min(direct_occupancy(true, P.wide, p->classes[c].smem),
                         direct_occupancy(false, P.wide, p->classes[c].smem)) == occ)
                break;
        }
        if (c == static_cast<int>(p->classes.size())) {
            p->classes.emplace_back();
            p->classes[c].wide = P.wide;
            p->classes[c].own = own;
        }
        MultiClass &C = p->classes[c];
        if (!own) {   // likelihood in the shared launch
            p->pl.fit[p->m_lik.n] = pf;
            p->m_lik.start[p->m_lik.n++] = bl;
            bl += W.S * P.T;
        }
        C.grid1_lik = W.S * P.T;
        C.smem = std::max(C.smem, tb);
        C.grid1_fwd = grid_for(P.grid_fwd_direct, W.S * P.T * W.C);
        C.grid1_bwd = grid_for(P.grid_bwd_direct, W.S * P.T * W.C);
        ProfArgs pb = pf;
        pb.counter = W.counters + 2;
        C.pf.fit[C.n] = pf;
        C.pb.fit[C.n] = pb;
        cls[f] = c;
        work[f] = static_cast<long long>(W.S) * P.T * P.Mtot;   // (sample, tile, peak) triples
        items[f] = static_cast<long long>(W.S) * P.T * W.C;
        ++C.n;
    }
    p->m_sample.start[n] = bs;
    p->m_ranges.start[n] = br;
    p->m_lik.start[p->m_lik.n] = bl;
    p->m_grad.start[n] = bg;
    for (int c = 0; c < static_cast<int>(p->classes.size()); ++c) {
        MultiClass &C = p->classes[c];
        std::vector<long long> w;
        long long nitems = 0;
        for (int f = 0; f < n; ++f)
            if (cls[f] == c) {
                w.push_back(work[f]);
                nitems += items[f];
            }
        const auto grid = [&](int occ) {
            const long long need = (nitems + kWarps - 1) / kWarps;
            const long long g = static_cast<long long>(occ) * sm_count;
            return static_cast<int>(need < g ? need : g);
        };
        persistent_map(C.m_fwd, w, grid(direct_occupancy(true, C.wide, C.smem)));
        persistent_map(C.m_bwd, w, grid(direct_occupancy(false, C.wide, C.smem)));
    }
    return true;
}

void multi_plan_launch_step(const MultiStepPlan *p, cudaStream_t st) {
    // the arguments travel with each launch (kernel parameters)
    k_sample_multi<<<p->m_sample.start[p->n], 128, 0, st>>>(p->sa, p->m_sample);
    k_ranges_multi<<<p->m_ranges.start[p->n], 256, 0, st>>>(p->pf, p->m_ranges);
    // fits that fill the GPU by themselves: their own profile, likelihood and
    // backward kernels back to back (their intermediates stay in L2)
    for (const MultiClass &C : p->classes) {
        if (!C.own) continue;
        const ProfArgs &a = C.pf.fit[0];
        if (C.wide) k_fwd_direct<false, true, false><<<C.grid1_fwd, kThreads, C.smem, st>>>(a);
        else k_fwd_direct<false, false, false><<<C.grid1_fwd, kThreads, C.smem, st>>>(a);
        k_lik<<<C.grid1_lik, kTile, 0, st>>>(a);
        if (C.wide) k_bwd_direct<true, false><<<C.grid1_bwd, kThreads, C.smem, st>>>(C.pb.fit[0]);
        else k_bwd_direct<false, false><<<C.grid1_bwd, kThreads, C.smem, st>>>(C.pb.fit[0]);
    }
    for (const MultiClass &C : p->classes) {
        if (C.own) continue;
        if (C.n == 1) {   // alone in its class: the fit's own kernel (arguments in the constant bank)
            if (C.wide) k_fwd_direct<false, true, false><<<C.grid1_fwd, kThreads, C.smem, st>>>(C.pf.fit[0]);
            else k_fwd_direct<false, false, false><<<C.grid1_fwd, kThreads, C.smem, st>>>(C.pf.fit[0]);
        } else if (C.wide) {
            k_direct_multi<true, true><<<C.m_fwd.start[C.n], kThreads, C.smem, st>>>(C.pf, C.m_fwd);
        } else {
            k_direct_multi<true, false><<<C.m_fwd.start[C.n], kThreads, C.smem, st>>>(C.pf, C.m_fwd);
        }
    }
    if (p->m_lik.n > 0) k_lik_multi<<<p->m_lik.start[p->m_lik.n], kTile, 0, st>>>(p->pl, p->m_lik);
    for (const MultiClass &C : p->classes) {
        if (C.own) continue;
        if (C.n == 1) {
            if (C.wide) k_bwd_direct<true, false><<<C.grid1_bwd, kThreads, C.smem, st>>>(C.pb.fit[0]);
            else k_bwd_direct<false, false><<<C.grid1_bwd, kThreads, C.smem, st>>>(C.pb.fit[0]);
        } else if (C.wide) {
            k_direct_multi<false, true><<<C.m_bwd.start[C.n], kThreads, C.smem, st>>>(C.pb, C.m_bwd);
        } else {
            k_direct_multi<false, false><<<C.m_bwd.start[C.n], kThreads, C.smem, st>>>(C.pb, C.m_bwd);
        }
    }
    k_grad_multi<<<p->m_grad.start[p->n], 256, 0, st>>>(p->ga, p->m_grad);
}

void launch_posterior(const Problem &P, Workspace &W, PostBuffers &B, int top_m, cudaStream_t st) {
    PostArgs a;
    a.S = W.S; a.K = P.K; a.T = P.T; a.W = (P.K + 63) / 64; a.top_m = top_m;
    a.csum = P.csum; a.alpha_min = static_cast<double>(static_cast<float>(P.prior.alpha_min));
    a.area_norm = P.area_norm ? 1 : 0;
    a.gzy = P.gates ? W.gzy : nullptr;
    a.llpart = W.llpart; a.lpj = W.lpj; a.lq = W.lq; a.isum = P.isum; a.theta = W.theta;
    a.logw = B.logw; a.pi = B.pi; a.scalars = B.scalars; a.combo_logp = B.combo_logp;
    a.cost = B.cost; a.bits = B.bits; a.combos = B.combos; a.order = B.order;
    a.heap_cost = B.heap_cost; a.heap_node = B.heap_node;
    a.node_mask = B.node_mask;
    a.node_last = B.node_last;
    k_post_sample<<<W.S, 128, 0, st>>>(a);
    k_post_reduce<<<P.K + 1, 256, 0, st>>>(a);
    k_post_sort<<<1, 1024, 0, st>>>(a);
    k_post_topm<<<1, 32, 0, st>>>(a);
}


namespace {
// Raw Philox4x32-10 blocks through the same device function the sampling
// kernel draws its noise with (exported for known-answer tests).
__global__ void k_philox_words(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox4x32_10(c, key[2 * i], key[2 * i + 1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) out[4 * i + j] = c[j];
}
}  // namespace

#ifdef XRDVI_DEBUG
namespace {
// One lookup through the table check with an index past a one-entry table:
// the check records its number and reads entry 0 instead.
__global__ void k_debug_selftest(float *out) {
    __shared__ float2 one[1];
    if (threadIdx.x == 0) one[0] = make_float2(1.f, 2.f);
    __syncthreads();
    PeakTable<false> t;
    t.p = one;
    t.n = 1;
    float np, I;
    t.scalar(1 + static_cast<int>(threadIdx.x), np, I);
    if (threadIdx.x == 0) *out = np + I;
}
}  // namespace

bool debug_build() { return true; }
int debug_word(bool reset) {
    int w = 0;
    cudaMemcpyFromSymbol(&w, g_debug_word, sizeof(int));
    if (reset) {
        const int z = 0;
        cudaMemcpyToSymbol(g_debug_word, &z, sizeof(int));
    }
    return w;
}
cudaError_t debug_selftest(float *d_out) {
    k_debug_selftest<<<1, 32>>>(d_out);
    return cudaDeviceSynchronize();
}
#else
bool debug_build() { return false; }
int debug_word(bool) { return 0; }
cudaError_t debug_selftest(float *) { return cudaErrorNotSupported; }
#endif

void launch_philox_words(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st) {
    if (n > 0) k_philox_words<<<(n + 127) / 128, 128, 0, st>>>(n, ctr, key, out);
}

namespace {
// Normalised log-probabilities of enumerated combinations: logp = elbo -
// logsumexp(elbo), FP64, strided per-thread partials combined by a fixed
// tree (one block, deterministic).
__global__ void __launch_bounds__(256) k_enum_lse(const double *elbo, int n, double *logp) {
    __shared__ double sh[8];
    double m = -CUDART_INF;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, elbo[i]);
    m = block_max(m, sh);
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += exp(elbo[i] - m);
    acc = block_sum(acc, sh);
    const double lse = m + log(acc);
    for (int i = threadIdx.x; i < n; i += blockDim.x) logp[i] = elbo[i] - lse;
}
}  // namespace

void launch_enum_lse(const double *elbo, int n, double *logp, cudaStream_t st) {
    k_enum_lse<<<1, 256, 0, st>>>(elbo, n, logp);
}


namespace {
// Fitted background curve B_i(beta) = B_i exp(sum_j beta_j T_j(z_i)).
__global__ void k_bg_curve(int N, const float *bg, const float *Tb, const float *beta, float *Bb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float e = beta[0] * Tb[i] + beta[1] * Tb[N + i] + beta[2] * Tb[2 * N + i];
    Bb[i] = bg[i] * expf(e);
}

// beta gradient: sum over draws (weight 1/S, or the importance weights) of
// the tile sums, in a fixed order, minus beta / sd^2; then Adam on beta (the
// step rule of k_grad) or the gradient written out.  One block of 3 warps.
__global__ void k_bg_grad(int S, int T, const float *bgpart, const double *iw, float *beta, float *m, float *v,
                          float bg_sd, int adam, AdamConst ac, const int *d_iter, float *grad_out) {
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= 3) return;
    double acc = 0.0;
    for (int s = lane; s < S; s += 32) {
        double t = 0.0;
        for (int tile = 0; tile < T; ++tile) t += bgpart[(static_cast<size_t>(s) * T + tile) * 3 + j];
        acc += iw ? iw[s] * t : t;
    }
    acc = warp_sumd(acc);
    if (lane != 0) return;
    const double b = beta[j];
    const double grad = (iw ? acc : acc / S) - b / (static_cast<double>(bg_sd) * bg_sd);
    if (grad_out) grad_out[j] = static_cast<float>(grad);
    if (adam) {
        const int t = *d_iter + 1;
        const double gm = -grad;
        const double mm = ac.b1 * static_cast<double>(m[j]) + (1.0 - ac.b1) * gm;
        const double vv = ac.b2 * static_cast<double>(v[j]) + (1.0 - ac.b2) * gm * gm;
        m[j] = static_cast<float>(mm);
        v[j] = static_cast<float>(vv);
        const double c1 = 1.0 - pow(static_cast<double>(ac.b1), t), c2 = 1.0 - pow(static_cast<double>(ac.b2), t);
        beta[j] = static_cast<float>(b - ac.lr * (mm / c1) / (sqrt(vv / c2) + ac.eps));
    }
}
}  // namespace

void launch_bg_curve(const Problem &P, cudaStream_t st) {
    k_bg_curve<<<(P.N + 255) / 256, 256, 0, st>>>(P.N, P.bg, P.Tb, P.beta, P.Bb);
}

void launch_bg_grad(const Problem &P, Workspace &W, bool adam, AdamConst ac, const int *d_iter, float *grad_out,
                    cudaStream_t st) {
    k_bg_grad<<<1, 96, 0, st>>>(W.S, P.T, W.bgpart, W.iw, P.beta, P.m_beta, P.v_beta, P.bg_sd, adam ? 1 : 0, ac,
                                d_iter, grad_out);
}

}  // namespace xrdvi
