// Allocation-free ELBO + gradient evaluation (xrdvi_elbo_grad_static).
//
// For callers that may not allocate device memory themselves: everything the
// evaluation needs beyond the caller's inputs and outputs comes from one
// file-scope device array, so the entry point calls no cudaMalloc, cudaFree or
// allocating library routine.  Before the kernels of xrdvi_elbo_grad
// (sampling from injected noise, profile + likelihood, backward, gradient
// reduction, ELBO) it checks the caller's arrays on the device and sorts each
// phase's peaks by position into the scratch array, which xrdvi_create does on
// the host; invalid input turns the ELBO and gradient into NaN.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/xrdvi.h"
#include "xrdvi_internal.h"

namespace {

// The scratch array: one per GPU that loads this library, held until exit.
// In host code this name is only a host-side stand-in; the device address is
// looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[XRDVI_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

size_t align256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }

// Checks the CSR offsets (offsets[0] = 0, offsets[K] = M, every phase
// non-empty) and copies them to soff; invalid offsets are replaced by an even
// split of the M peaks (valid indices for every later kernel) and flagged.
// One block; it also clears the error word of the call.
__global__ void k_static_offsets(int K, int M, const int *off, int *soff, int *err) {
    int bad = 0;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) {
        const int o = off[k];
        if (o < 0 || o > M) bad = 1;
        if (k == 0 && o != 0) bad = 1;
        if (k == K && o != M) bad = 1;
        if (k < K && !(off[k + 1] > o)) bad = 1;
    }
    bad = __syncthreads_or(bad);
    for (int k = threadIdx.x; k <= K; k += blockDim.x)
        soff[k] = bad ? static_cast<int>((static_cast<long long>(k) * M) / K) : off[k];
    if (threadIdx.x == 0) *err = bad;
}

// Stable sort of every phase's peaks by position (the order xrdvi_create's
// host sort gives): peak i of phase k goes to slot soff[k] + rank, rank = the
// number of the phase's peaks with a smaller position, or an equal one and a
// smaller index.  O(M_k) comparisons per peak.  Intensities are rounded to
// bfloat16 (nearest even) with the BF16 flag, as on the host.  Also checks
// the values xrdvi_create validates (positions in (0, 180), intensities in
// [0, 1], x strictly increasing in (0, 180), integer counts >= 0, finite
// background >= 0) and sets *err on any violation.
__global__ void k_static_prep(int K, int M, int N, const int *soff, const float *pos, const float *inten,
                              const float *x, const float *y, const float *bg, int bf16, float *spos,
                              float *sint, int *err) {
    const int stride = gridDim.x * blockDim.x;
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        int lo = 0, hi = K;   // phase k with soff[k] <= i < soff[k + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (soff[mid] <= i) lo = mid; else hi = mid;
        }
        const int mb = soff[lo], me = soff[lo + 1];
        const float p = pos[i], I = inten[i];
        if (!(p > 0.f && p < 180.f) || !(I >= 0.f && I <= 1.f)) bad = 1;   // also rejects NaN
        int rank = 0;
        for (int j = mb; j < me; ++j) {
            const float q = pos[j];
            rank += (q < p || (q == p && j < i)) ? 1 : 0;
        }
        spos[mb + rank] = p;
        sint[mb + rank] = bf16 ? __bfloat162float(__float2bfloat16_rn(I)) : I;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const float xv = x[i], yv = y[i], b = bg[i];
        if (!(xv > 0.f && xv < 180.f) || (i > 0 && !(xv > x[i - 1]))) bad = 1;
        if (!(yv >= 0.f && yv < 3.0e38f && floorf(yv) == yv)) bad = 1;
        if (!(b >= 0.f && b < 3.0e38f)) bad = 1;
    }
    if (bad) atomicExch(err, 1);
}

// Invalid input: the outputs become NaN.
__global__ void k_static_poison(const int *err, double *elbo, float *grad, int n) {
    if (*err == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *elbo = __longlong_as_double(0x7ff8000000000000ll);
    if (i < n) grad[i] = __int_as_float(0x7fc00000);
}

}  // namespace


extern "C" xrdvi_status xrdvi_elbo_grad_static(int32_t K, int32_t M_total, const int32_t *d_offsets,
                                               const float *d_pos, const float *d_inten, int32_t N,
                                               const float *d_x, const float *d_y, const float *d_bg,
                                               double data_const, double lambda_, const xrdvi_config *cfg,
                                               const float *d_loc, const float *d_raw, const float *d_eps,
                                               double *d_elbo, float *d_grad, void *cuda_stream) {
    using namespace xrdvi;
    if (!cfg || !d_offsets || !d_pos || !d_inten || !d_x || !d_y || !d_bg || !d_loc || !d_raw || !d_eps ||
        !d_elbo || !d_grad)
        return report_error(XRDVI_EINVAL, "elbo_grad_static: null argument");
    if (cfg->size != sizeof(xrdvi_config)) return report_error(XRDVI_EINVAL, "elbo_grad_static: config.size mismatch");
    if (K < 1 || K > kMaxK) return report_error(XRDVI_EINVAL, "elbo_grad_static: K must be in [1, 1024]");
    if (M_total < K || M_total > kMaxPeaks)
        return report_error(XRDVI_EINVAL, "elbo_grad_static: M_total must be in [K, 24000]");
    if (N < 1 || N > kMaxN) return report_error(XRDVI_EINVAL, "elbo_grad_static: N must be in [1, 2^24]");
    const int S = cfg->S;
    if (S < 1 || S > kMaxS) return report_error(XRDVI_EINVAL, "elbo_grad_static: S must be in [1, 65536]");
    if (!(std::isfinite(lambda_) && lambda_ > 0.0) || !std::isfinite(data_const))
        return report_error(XRDVI_EINVAL, "elbo_grad_static: lambda_ must be positive, data_const finite");
    if (cfg->flags &
        (XRDVI_FLAG_IW_ELBO | XRDVI_FLAG_SHARED_SHAPES | XRDVI_FLAG_SEC_WIDTH | XRDVI_FLAG_FIT_BACKGROUND |
         XRDVI_FLAG_FIX_R | XRDVI_FLAG_FIX_ALPHA | XRDVI_FLAG_AREA_NORM | XRDVI_FLAG_GATES | XRDVI_FLAG_DEVICE_PTRS))
        return report_error(XRDVI_EINVAL, "elbo_grad_static: the importance-weighted, shared-shape, angle-dependent "
                                          "width, fitted-background, fixed-shape, area-normalised and gated variants "
                                          "and XRDVI_FLAG_DEVICE_PTRS are not accepted");

    // Layout of the scratch array for this call.
    const size_t T = (static_cast<size_t>(N) + kTile - 1) / kTile;
    const size_t Npad = T * kTile;
    const size_t SK = static_cast<size_t>(S) * K;
    size_t off = 0;
    const size_t o_eps = off;    off += align256(SK * 5 * sizeof(float));
    const size_t o_theta = off;  off += align256(SK * 5 * sizeof(float));
    const size_t o_cst = off;    off += align256(SK * sizeof(PhaseConst));
    const size_t o_lpj = off;    off += align256(static_cast<size_t>(S) * sizeof(double));
    const size_t o_ll = off;     off += align256(static_cast<size_t>(S) * sizeof(double));
    const size_t o_ent = off;    off += align256(sizeof(double));
    const size_t o_g = off;      off += align256(static_cast<size_t>(S) * Npad * sizeof(float));
    const size_t o_llp = off;    off += align256(static_cast<size_t>(S) * T * sizeof(double));
    const size_t o_gp = off;     off += align256(SK * T * kGradSums * sizeof(float));
    const size_t o_fp = off;     off += align256(static_cast<size_t>(S) * Npad * sizeof(float));
    const size_t o_rg = off;     off += align256(SK * T * sizeof(ushort4));
    const size_t o_cnt = off;    off += align256(kCounters * sizeof(int));
    const size_t o_gred = off;   off += align256(static_cast<size_t>(K) * kGradBlocks * kGredVals * sizeof(double));
    const size_t o_tk = off;     off += align256(static_cast<size_t>(K) * sizeof(int));
    const size_t o_off = off;    off += align256(static_cast<size_t>(K + 1) * sizeof(int));
    const size_t o_pos = off;    off += align256(static_cast<size_t>(M_total) * sizeof(float));
    const size_t o_int = off;    off += align256(static_cast<size_t>(M_total) * sizeof(float));
    const size_t o_err = off;    off += align256(sizeof(int));
    if (off > XRDVI_STATIC_SCRATCH_BYTES)
        return report_error(XRDVI_EINVAL, "elbo_grad_static: this problem needs " + std::to_string(off) +
                                              " bytes of scratch, more than the " +
                                              std::to_string(XRDVI_STATIC_SCRATCH_BYTES) +
                                              " bytes of the static array");

    // Set-up, once per device, with that device current.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report_error(XRDVI_EINVAL, "elbo_grad_static: device ordinal above 63");
    unsigned char *base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return report_error(XRDVI_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
            g_sm_count[dev] = n;
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_scratch_addr[dev]);
        sms = g_sm_count[dev];
    }

    Problem P;
    P.K = K;
    P.N = N;
    P.Mtot = M_total;
    P.T = static_cast<int>(T);
    P.Npad = static_cast<int>(Npad);
    // the kernels read the checked offsets and the sorted table in the scratch array
    int *soff = reinterpret_cast<int *>(base + o_off);
    float *spos = reinterpret_cast<float *>(base + o_pos);
    float *sint = reinterpret_cast<float *>(base + o_int);
    int *err = reinterpret_cast<int *>(base + o_err);
    P.pos = spos;
    P.inten = sint;
    P.off = soff;
    P.x = const_cast<float *>(d_x);
    P.y = const_cast<float *>(d_y);
    P.bg = const_cast<float *>(d_bg);
    P.csum = data_const;
    P.gauss = (cfg->flags & XRDVI_FLAG_GAUSS_LIK) != 0;
    P.prior.lambda = lambda_;
    P.prior.mu_sd = cfg->prior_mu_sd;
    P.prior.alpha_mean = cfg->prior_alpha_mean;
    P.prior.alpha_sd = cfg->prior_alpha_sd;
    P.prior.w_shape = cfg->prior_w_shape;
    P.prior.w_rate = cfg->prior_w_rate;
    P.prior.lgamma_w_shape = std::lgamma(static_cast<double>(cfg->prior_w_shape));
    P.prior.alpha_min = cfg->alpha_min;
    P.prior.lp_const = std::log(lambda_) - std::log(static_cast<double>(cfg->prior_mu_sd)) -
                       std::log(static_cast<double>(cfg->prior_alpha_sd)) - std::log(2.0 * M_PI) +
                       cfg->prior_w_shape * std::log(static_cast<double>(cfg->prior_w_rate)) -
                       P.prior.lgamma_w_shape;
    configure_grids(P, sms);

    // Every scratch element is written before it is read in one call (the
    // partial sums of every sample, phase and tile, the padded tail of g, the
    // work counters, which the sampling kernel zeroes, the error word, which
    // the offsets check clears), so nothing has to be cleared here; the array
    // keeps the last call's contents.
    Workspace W;
    W.S = S;
    W.eps = reinterpret_cast<float *>(base + o_eps);
    W.theta = reinterpret_cast<float *>(base + o_theta);
    W.cst = reinterpret_cast<PhaseConst *>(base + o_cst);
    W.lpj = reinterpret_cast<double *>(base + o_lpj);
    W.lq = nullptr;
    W.ll = reinterpret_cast<double *>(base + o_ll);
    W.g = reinterpret_cast<float *>(base + o_g);
    W.llpart = reinterpret_cast<double *>(base + o_llp);
    W.gpart = reinterpret_cast<float *>(base + o_gp);
    W.fpart = reinterpret_cast<float *>(base + o_fp);     // one phase chunk
    W.ranges = reinterpret_cast<ushort4 *>(base + o_rg);
    W.counters = reinterpret_cast<int *>(base + o_cnt);   // zeroed by the sampling kernel
    W.gred = reinterpret_cast<double *>(base + o_gred);
    W.tickets = reinterpret_cast<int *>(base + o_tk);     // zeroed by the sampling kernel
    W.C = 1;
    W.chunk[0] = 0;
    W.chunk[1] = K;
    double *ent = reinterpret_cast<double *>(base + o_ent);

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool naive = (cfg->flags & XRDVI_FLAG_NAIVE_SUM) != 0;
    k_static_offsets<<<1, 1024, 0, st>>>(K, M_total, d_offsets, soff, err);
    const int work = std::max(M_total, N);
    k_static_prep<<<std::min((work + 255) / 256, 4 * sms), 256, 0, st>>>(
        K, M_total, N, soff, d_pos, d_inten, d_x, d_y, d_bg, (cfg->flags & XRDVI_FLAG_BF16_INT) ? 1 : 0, spos,
        sint, err);
    launch_sample(P, W, d_loc, d_raw, d_eps, cfg->seed, 0u, nullptr, 0u, nullptr, ent, st);
    launch_forward(P, W, nullptr, naive, st);
    launch_backward(P, W, st);
    launch_grad(P, W, d_loc, d_raw, nullptr, nullptr, d_grad, false, AdamConst{0.f, 0.f, 0.f, 0.f}, nullptr, nullptr,
                nullptr, nullptr, ent, d_elbo, nullptr, st);
    k_static_poison<<<(10 * K + 255) / 256, 256, 0, st>>>(err, d_elbo, d_grad, 10 * K);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("elbo_grad_static: ") + cudaGetErrorString(e));
    return XRDVI_OK;
}
