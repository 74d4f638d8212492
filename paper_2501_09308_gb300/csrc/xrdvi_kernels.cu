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

#include <cstdint>

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

__device__ __forceinline__ double softplusd(double x) {
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

__device__ __forceinline__ float sigmoidf(float x) {
    if (x >= 0.f) return 1.f / (1.f + expf(-x));
    const float e = expf(x);
    return e / (1.f + e);
}

__device__ __forceinline__ double sigmoidd(double x) {
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x));
    const double e = exp(x);
    return e / (1.0 + e);
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
};

__global__ void __launch_bounds__(128) k_sample(SampleArgs a) {
    __shared__ double sh[4];
    const int s = blockIdx.x;
    const uint32_t step = a.d_step ? static_cast<uint32_t>(*a.d_step) : a.step;
    if (s == 0 && threadIdx.x == 0 && a.d_iter) *a.d_iter = static_cast<int>(step);
    const float sq = sqrtf(kGaussU);
    double acc = 0.0, accq = 0.0;
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const size_t base = (static_cast<size_t>(s) * a.K + k) * 5;
        float e[8];
        if (a.eps_in) {
#pragma unroll
            for (int j = 0; j < 5; ++j) e[j] = a.eps_in[base + j];
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t c[4] = {static_cast<uint32_t>(s), static_cast<uint32_t>(k), step,
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
        }
        float u[5], sig[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            sig[j] = softplusf(a.raw[k * 5 + j]);
            u[j] = fmaf(sig[j], e[j], a.loc[k * 5 + j]);
            a.eps[base + j] = e[j];
        }
        const float h = expf(u[0]);
        const float mu = u[1];
        const float w = expf(u[2]);
        const float r = sigmoidf(u[3]);
        const float al = u[4];
        a.theta[base + 0] = h;
        a.theta[base + 1] = mu;
        a.theta[base + 2] = w;
        a.theta[base + 3] = r;
        a.theta[base + 4] = al;
        const float ac = al > static_cast<float>(a.pr.alpha_min) ? al : static_cast<float>(a.pr.alpha_min);
        const float wl = w, wr = ac * w;
        const float cl = 4.0f / (wl * wl), cr = 4.0f / (wr * wr);
        PhaseConst pc;
        pc.mu = mu;
        pc.split = (ac >= 0.5f && ac <= 2.0f) ? 0 : 1;
        pc.a = pc.split ? cl : 0.5f * (cr + cl);
        pc.b = pc.split ? cr : 0.5f * (cr - cl);
        pc.hl = h * r;
        pc.hg = h * (1.0f - r);
        pc.rl = 0.5f * sq * wl;
        pc.rr = 0.5f * sq * wr;
        a.cst[static_cast<size_t>(s) * a.K + k] = pc;
        // log prior (Sec. 2.2, Appendix B.2) + log Jacobian of the transform
        const double hd = h, mud = mu, wd = w, ald = al;
        double lp = log(a.pr.lambda) - a.pr.lambda * hd;
        const double zm = mud / a.pr.mu_sd;
        lp += -0.5 * zm * zm - log(a.pr.mu_sd) - 0.5 * kLog2Pi;
        const double za = (ald - a.pr.alpha_mean) / a.pr.alpha_sd;
        lp += -0.5 * za * za - log(a.pr.alpha_sd) - 0.5 * kLog2Pi;
        lp += a.pr.w_shape * log(a.pr.w_rate) - a.pr.lgamma_w_shape +
              (a.pr.w_shape - 1.0) * log(wd) - a.pr.w_rate * wd;
        const double lj = static_cast<double>(u[0]) + static_cast<double>(u[2]) -
                          softplusd(-static_cast<double>(u[3])) - softplusd(static_cast<double>(u[3]));
        acc += lp + lj;
        if (a.lq) {
#pragma unroll
            for (int j = 0; j < 5; ++j)
                accq += -0.5 * static_cast<double>(e[j]) * e[j] - log(static_cast<double>(sig[j])) - 0.5 * kLog2Pi;
        }
    }
    const double tot = block_sum(acc, sh);
    const double totq = a.lq ? block_sum(accq, sh) : 0.0;
    if (threadIdx.x == 0) {
        a.lpj[s] = tot;
        if (a.lq) a.lq[s] = totq;
    }
    if (s == 0 && a.ent) {
        double H = 0.0;
        for (int i = threadIdx.x; i < 5 * a.K; i += blockDim.x)
            H += log(softplusd(static_cast<double>(a.raw[i]))) + 0.5 * (1.0 + kLog2Pi);
        H = block_sum(H, sh);
        if (threadIdx.x == 0) *a.ent = H;
    }
}

// ---------------------------------------------------------------------------
// Profile kernels
// ---------------------------------------------------------------------------
struct ProfArgs {
    int S, K, N, Npad, T, Mtot;
    const float *pos, *inten;
    const int *off;
    const float *x, *y, *bg;
    const PhaseConst *cst;
    float *g;          // [S*Npad]
    float *f_out;      // [S*N] or null
    double *llpart;    // [S*T]
    float *gpart;      // [S*K*T*8]
};

__device__ __forceinline__ void load_table(const ProfArgs &a, float2 *s_pk, int *s_off) {
    for (int i = threadIdx.x; i < a.Mtot; i += blockDim.x) s_pk[i] = make_float2(a.pos[i], a.inten[i]);
    for (int i = threadIdx.x; i <= a.K; i += blockDim.x) s_off[i] = a.off[i];
    __syncthreads();
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

// c(d) * d for one side-width form (see PhaseConst).
template <bool kSplit>
__device__ __forceinline__ float cd_of(const PhaseConst &c, float d) {
    if (kSplit) return (d >= 0.f ? c.b : c.a) * d;
    return fmaf(c.b, fabsf(d), c.a * d);
}

// Forward sums over the peaks [mb, me) of one phase: sl += I L, sg += I G.
template <bool kSplit>
__device__ __forceinline__ void fwd_phase(const float2 *s_pk, int mb, int me, const PhaseConst &c,
                                          float plo, float phi, const float (&xj)[kPts],
                                          float (&sl)[kPts], float (&sg)[kPts]) {
    for (int m = mb; m < me; ++m) {
        const float2 pk = s_pk[m];
        float u[kPts];
#pragma unroll
        for (int j = 0; j < kPts; ++j) {
            const float d = (xj[j] - pk.x) - c.mu;
            u[j] = d * cd_of<kSplit>(c, d);
            sl[j] = fmaf(pk.y, rcp_approx(u[j] + 1.0f), sl[j]);
        }
        if (pk.x > plo && pk.x < phi) {  // warp-uniform
#pragma unroll
            for (int j = 0; j < kPts; ++j) sg[j] = fmaf(pk.y, ex2_approx(-u[j]), sg[j]);
        }
    }
}

// Backward sums over the peaks of one phase (layout of k_backward's acc).
template <bool kSplit>
__device__ __forceinline__ bool bwd_phase(const float2 *s_pk, int mb, int me, const PhaseConst &c,
                                          float plo, float phi, const float (&xj)[kPts],
                                          const float (&gj)[kPts], float (&acc)[8]) {
    bool anyg = false;
    for (int m = mb; m < me; ++m) {
        const float2 pk = s_pk[m];
        float u[kPts], cd[kPts], ud[kPts], q[kPts];
#pragma unroll
        for (int j = 0; j < kPts; ++j) {
            const float d = (xj[j] - pk.x) - c.mu;
            cd[j] = cd_of<kSplit>(c, d);
            u[j] = d * cd[j];
            ud[j] = fabsf(d) * cd[j];
            q[j] = gj[j] * pk.y;
            const float L = rcp_approx(u[j] + 1.0f);
            const float q1 = q[j] * L;
            acc[1] += q1;
            const float q2 = q1 * L;
            acc[3] = fmaf(q2, cd[j], acc[3]);
            acc[5] = fmaf(q2, u[j], acc[5]);
            acc[7] = fmaf(q2, ud[j], acc[7]);
        }
        if (pk.x > plo && pk.x < phi) {  // warp-uniform
            anyg = true;
#pragma unroll
            for (int j = 0; j < kPts; ++j) {
                const float qg = q[j] * ex2_approx(-u[j]);
                acc[0] += qg;
                acc[2] = fmaf(qg, cd[j], acc[2]);
                acc[4] = fmaf(qg, u[j], acc[4]);
                acc[6] = fmaf(qg, ud[j], acc[6]);
            }
        }
    }
    return anyg;
}

template <bool kNaive>
__global__ void __launch_bounds__(kThreads) k_forward(ProfArgs a) {
    extern __shared__ float2 s_pk[];
    int *s_off = reinterpret_cast<int *>(s_pk + a.Mtot);
    load_table(a, s_pk, s_off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int items = a.S * a.T;
    for (int item = blockIdx.x * kWarps + warp; item < items; item += gridDim.x * kWarps) {
        const int s = item / a.T, tile = item - s * a.T;
        const int i0 = tile * kTile;
        float xj[kPts], fs[kPts], fc[kPts];
#pragma unroll
        for (int j = 0; j < kPts; ++j) {
            const int ic = min(i0 + j * 32 + lane, a.N - 1);
            xj[j] = a.x[ic];
            fs[j] = a.bg[ic];
            fc[j] = 0.f;
        }
        const float xlo = a.x[i0];
        const float xhi = a.x[min(i0 + kTile - 1, a.N - 1)];
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = 0; k < a.K; ++k) {
            const PhaseConst c = cs[k];
            const float plo = xlo - c.mu - c.rr;   // peak p is "near" iff plo < p < phi
            const float phi = xhi - c.mu + c.rl;
            float sl[kPts], sg[kPts];
#pragma unroll
            for (int j = 0; j < kPts; ++j) sl[j] = sg[j] = 0.f;
            if (c.split)
                fwd_phase<true>(s_pk, s_off[k], s_off[k + 1], c, plo, phi, xj, sl, sg);
            else
                fwd_phase<false>(s_pk, s_off[k], s_off[k + 1], c, plo, phi, xj, sl, sg);
#pragma unroll
            for (int j = 0; j < kPts; ++j) {
                const float v = fmaf(c.hl, sl[j], c.hg * sg[j]);
                if (kNaive) {
                    fs[j] += v;
                } else {
                    // Neumaier compensated summation over phases
                    const float t = fs[j] + v;
                    fc[j] += (fabsf(fs[j]) >= fabsf(v)) ? ((fs[j] - t) + v) : ((v - t) + fs[j]);
                    fs[j] = t;
                }
            }
        }
        double dev = 0.0;
#pragma unroll
        for (int j = 0; j < kPts; ++j) {
            const int i = i0 + j * 32 + lane;
            float gv = 0.f;
            if (i < a.N) {
                const float f = fs[j] + fc[j];
                const float yv = a.y[i];
                dev += static_cast<double>(deviance_term(yv, f));
                gv = (yv > 0.f) ? __fdiv_rn(yv, f) - 1.0f : -1.0f;
                if (a.f_out) a.f_out[static_cast<size_t>(s) * a.N + i] = f;
            }
            a.g[static_cast<size_t>(s) * a.Npad + i] = gv;
        }
        dev = warp_sum(dev);
        if (lane == 0) a.llpart[static_cast<size_t>(s) * a.T + tile] = dev;
    }
}

// Gradient sums per (s, k, tile), with q = (y/f - 1) I_m, t = c(d) d, u = t d:
//   0 S1G = sum q G        1 S1L = sum q L
//   2 S2G = sum q G t      3 S2L = sum q L^2 t
//   4 S3G = sum q G u      5 S3L = sum q L^2 u
//   6 S4G = sum q G u sgn  7 S4L = sum q L^2 u sgn      (sgn = sign(d))
__global__ void __launch_bounds__(kThreads) k_backward(ProfArgs a) {
    extern __shared__ float2 s_pk[];
    int *s_off = reinterpret_cast<int *>(s_pk + a.Mtot);
    load_table(a, s_pk, s_off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int items = a.S * a.T;
    for (int item = blockIdx.x * kWarps + warp; item < items; item += gridDim.x * kWarps) {
        const int s = item / a.T, tile = item - s * a.T;
        const int i0 = tile * kTile;
        float xj[kPts], gj[kPts];
#pragma unroll
        for (int j = 0; j < kPts; ++j) {
            const int i = i0 + j * 32 + lane;
            xj[j] = a.x[min(i, a.N - 1)];
            gj[j] = a.g[static_cast<size_t>(s) * a.Npad + i];
        }
        const float xlo = a.x[i0];
        const float xhi = a.x[min(i0 + kTile - 1, a.N - 1)];
        const PhaseConst *cs = a.cst + static_cast<size_t>(s) * a.K;
        for (int k = 0; k < a.K; ++k) {
            const PhaseConst c = cs[k];
            const float plo = xlo - c.mu - c.rr;
            const float phi = xhi - c.mu + c.rl;
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool anyg;
            if (c.split)
                anyg = bwd_phase<true>(s_pk, s_off[k], s_off[k + 1], c, plo, phi, xj, gj, acc);
            else
                anyg = bwd_phase<false>(s_pk, s_off[k], s_off[k + 1], c, plo, phi, xj, gj, acc);
            float s1l = acc[1], s2l = acc[3], s3l = acc[5], s4l = acc[7];
            float s1g = acc[0], s2g = acc[2], s3g = acc[4], s4g = acc[6];
            s1l = warp_sumf(s1l);
            s2l = warp_sumf(s2l);
            s3l = warp_sumf(s3l);
            s4l = warp_sumf(s4l);
            if (anyg) {  // warp-uniform
                s1g = warp_sumf(s1g);
                s2g = warp_sumf(s2g);
                s3g = warp_sumf(s3g);
                s4g = warp_sumf(s4g);
            }
            if (lane == 0) {
                float4 *dst = reinterpret_cast<float4 *>(
                    a.gpart + ((static_cast<size_t>(s) * a.K + k) * a.T + tile) * 8);
                dst[0] = make_float4(s1g, s1l, s2g, s2l);
                dst[1] = make_float4(s3g, s3l, s4g, s4l);
            }
        }
    }
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
};

// ELBO = mean_s [LL_s + log prior + log Jacobian] + entropy, in FP64 with a
// fixed summation order; also advances the step counter of the fit loop.
__global__ void __launch_bounds__(256) k_elbo(GradArgs a) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
        double ll = a.csum;
        const double *lp = a.llpart + static_cast<size_t>(s) * a.T;
        for (int t = 0; t < a.T; ++t) ll += lp[t];
        a.ll[s] = ll;
        acc += ll + a.lpj[s];
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        const double elbo = acc / a.S + *a.ent;
        if (a.elbo_out) *a.elbo_out = elbo;
        if (a.d_iter) {
            const int it = *a.d_iter;
            if (a.trace) a.trace[it & (kTraceCap - 1)] = elbo;
            if (a.d_step) *a.d_step = it + 1;
        }
    }
}

__global__ void __launch_bounds__(256) k_grad(GradArgs a) {
    __shared__ double sh[8];
    __shared__ double red[10];
    const int k = blockIdx.x;
    double accl[5] = {0, 0, 0, 0, 0}, acce[5] = {0, 0, 0, 0, 0};
    const double ln2 = kLn2;
    for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
        const size_t sk = static_cast<size_t>(s) * a.K + k;
        const float *gp = a.gpart + sk * a.T * 8;
        double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < a.T; ++t) {
            const float4 v0 = reinterpret_cast<const float4 *>(gp + t * 8)[0];
            const float4 v1 = reinterpret_cast<const float4 *>(gp + t * 8)[1];
            q[0] += v0.x; q[1] += v0.y; q[2] += v0.z; q[3] += v0.w;
            q[4] += v1.x; q[5] += v1.y; q[6] += v1.z; q[7] += v1.w;
        }
        const float *th = a.theta + sk * 5;
        const float *ep = a.eps + sk * 5;
        const double h = th[0], mu = th[1], w = th[2], r = th[3], al = th[4];
        const bool clamped = !(th[4] > static_cast<float>(a.pr.alpha_min));
        const double acl = clamped ? static_cast<double>(static_cast<float>(a.pr.alpha_min)) : al;
        double G[5];
        // likelihood part (chain to u) + prior/Jacobian part
        G[0] = h * ((1.0 - r) * q[0] + r * q[1]) + (1.0 - a.pr.lambda * h);
        G[1] = 2.0 * h * ((1.0 - r) * ln2 * q[2] + r * q[3]) - mu / (a.pr.mu_sd * a.pr.mu_sd);
        G[2] = 2.0 * h * ((1.0 - r) * ln2 * q[4] + r * q[5]) + (a.pr.w_shape - a.pr.w_rate * w);
        G[3] = r * (1.0 - r) * h * (q[1] - q[0]) + (1.0 - 2.0 * r);
        const double gal = clamped ? 0.0
                                   : (h / acl) * ((1.0 - r) * ln2 * (q[4] + q[6]) + r * (q[5] + q[7]));
        G[4] = gal - (al - a.pr.alpha_mean) / (a.pr.alpha_sd * a.pr.alpha_sd);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            accl[j] += G[j];
            acce[j] += G[j] * static_cast<double>(ep[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const double v1 = block_sum(accl[j], sh);
        const double v2 = block_sum(acce[j], sh);
        if (threadIdx.x == 0) {
            red[j] = v1;
            red[5 + j] = v2;
        }
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        const int j = threadIdx.x % 5;
        const bool is_raw = threadIdx.x >= 5;
        const double rw = a.raw_in[k * 5 + j];
        double grad;
        if (!is_raw) {
            grad = red[j] / a.S;
        } else {
            grad = (red[5 + j] / a.S + 1.0 / softplusd(rw)) * sigmoidd(rw);
        }
        if (a.grad_out) a.grad_out[k * 10 + threadIdx.x] = static_cast<float>(grad);
        if (a.adam) {
            const int t = *a.d_iter + 1;
            const int idx = k * 10 + threadIdx.x;
            const double gm = -grad;  // minimise -ELBO
            const double mm = a.ac.b1 * static_cast<double>(a.m[idx]) + (1.0 - a.ac.b1) * gm;
            const double vv = a.ac.b2 * static_cast<double>(a.v[idx]) + (1.0 - a.ac.b2) * gm * gm;
            a.m[idx] = static_cast<float>(mm);
            a.v[idx] = static_cast<float>(vv);
            const double c1 = 1.0 - pow(static_cast<double>(a.ac.b1), t);
            const double c2 = 1.0 - pow(static_cast<double>(a.ac.b2), t);
            const double step = a.ac.lr * (mm / c1) / (sqrt(vv / c2) + a.ac.eps);
            if (!is_raw) {
                a.loc_out[k * 5 + j] = static_cast<float>(a.loc_in[k * 5 + j] - step);
            } else {
                a.raw_out[k * 5 + j] = static_cast<float>(rw - step);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Posterior over phase combinations
// ---------------------------------------------------------------------------
struct PostArgs {
    int S, K, T, W, top_m;
    double csum, alpha_min;
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
        const double area = static_cast<double>(th[0]) * a.isum[k] * ((1.0 + ac) * th[2] * 0.5) *
                            ((1.0 - th[3]) * AG + static_cast<double>(th[3]) * AL);
        tot += area;
    }
    tot = block_sum(tot, sh);
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const float *th = a.theta + (static_cast<size_t>(s) * a.K + k) * 5;
        const double ac = th[4] > static_cast<float>(a.alpha_min) ? static_cast<double>(th[4]) : a.alpha_min;
        const double area = static_cast<double>(th[0]) * a.isum[k] * ((1.0 + ac) * th[2] * 0.5) *
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
void configure_grids(Problem &P, int sm_count) {
    P.smem = static_cast<size_t>(P.Mtot) * sizeof(float2) + static_cast<size_t>(P.K + 1) * sizeof(int);
    // The attribute is per function, shared by every context: always allow the
    // largest table any context may have, never the current problem's size.
    const int smax = static_cast<int>(static_cast<size_t>(kMaxPeaks) * sizeof(float2) +
                                      static_cast<size_t>(kMaxK + 1) * sizeof(int));
    cudaFuncSetAttribute(k_forward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_forward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    int bf = 1, bb = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_forward<false>, kThreads, P.smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_backward, kThreads, P.smem);
    if (bf < 1) bf = 1;
    if (bb < 1) bb = 1;
    P.grid_fwd = bf * sm_count;
    P.grid_bwd = bb * sm_count;
}

static ProfArgs prof_args(const Problem &P, Workspace &W, float *f_out) {
    ProfArgs a;
    a.S = W.S; a.K = P.K; a.N = P.N; a.Npad = P.Npad; a.T = P.T; a.Mtot = P.Mtot;
    a.pos = P.pos; a.inten = P.inten; a.off = P.off;
    a.x = P.x; a.y = P.y; a.bg = P.bg;
    a.cst = W.cst; a.g = W.g; a.f_out = f_out; a.llpart = W.llpart; a.gpart = W.gpart;
    return a;
}

static int grid_for(int grid_max, int items) {
    const int need = (items + kWarps - 1) / kWarps;
    return need < grid_max ? need : grid_max;
}

void launch_sample(const Problem &P, Workspace &W, const float *loc, const float *raw,
                   const float *eps_in, uint64_t seed, uint32_t tag, const int *d_step,
                   uint32_t step, int *d_iter, double *ent, cudaStream_t st) {
    SampleArgs a;
    a.S = W.S; a.K = P.K; a.loc = loc; a.raw = raw; a.eps_in = eps_in;
    a.key0 = static_cast<uint32_t>(seed & 0xffffffffu);
    a.key1 = static_cast<uint32_t>(seed >> 32);
    a.tag = tag; a.step = step; a.d_step = d_step; a.d_iter = d_iter; a.ent = ent;
    a.pr = P.prior; a.eps = W.eps; a.theta = W.theta; a.cst = W.cst; a.lpj = W.lpj; a.lq = W.lq;
    k_sample<<<W.S, 128, 0, st>>>(a);
}

void launch_forward(const Problem &P, Workspace &W, float *f_out, bool naive, cudaStream_t st) {
    ProfArgs a = prof_args(P, W, f_out);
    const int grid = grid_for(P.grid_fwd, W.S * P.T);
    if (naive)
        k_forward<true><<<grid, kThreads, P.smem, st>>>(a);
    else
        k_forward<false><<<grid, kThreads, P.smem, st>>>(a);
}

void launch_backward(const Problem &P, Workspace &W, cudaStream_t st) {
    ProfArgs a = prof_args(P, W, nullptr);
    const int grid = grid_for(P.grid_bwd, W.S * P.T);
    k_backward<<<grid, kThreads, P.smem, st>>>(a);
}

void launch_grad(const Problem &P, Workspace &W, const float *loc_in, const float *raw_in,
                 float *loc_out, float *raw_out, float *grad_out, bool adam, AdamConst ac,
                 float *m, float *v, const int *d_iter, int *d_step, const double *ent,
                 double *elbo_out, double *trace, cudaStream_t st) {
    GradArgs a;
    a.S = W.S; a.K = P.K; a.T = P.T; a.pr = P.prior; a.csum = P.csum;
    a.gpart = W.gpart; a.theta = W.theta; a.eps = W.eps;
    a.loc_in = loc_in; a.raw_in = raw_in; a.loc_out = loc_out; a.raw_out = raw_out;
    a.grad_out = grad_out; a.adam = adam ? 1 : 0; a.ac = ac; a.m = m; a.v = v;
    a.d_iter = d_iter; a.d_step = d_step; a.llpart = W.llpart; a.lpj = W.lpj; a.ent = ent;
    a.ll = W.ll; a.elbo_out = elbo_out; a.trace = trace;
    if (grad_out || adam) k_grad<<<P.K, 256, 0, st>>>(a);
    if (elbo_out || trace) k_elbo<<<1, 256, 0, st>>>(a);
}

void launch_posterior(const Problem &P, Workspace &W, PostBuffers &B, int top_m, cudaStream_t st) {
    PostArgs a;
    a.S = W.S; a.K = P.K; a.T = P.T; a.W = (P.K + 63) / 64; a.top_m = top_m;
    a.csum = P.csum; a.alpha_min = static_cast<double>(static_cast<float>(P.prior.alpha_min));
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

}  // namespace xrdvi
