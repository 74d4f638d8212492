// C ABI of the xrdvi library: context lifetime, input validation, upload,
// the CUDA-graph fit loop, the single-step ELBO/gradient entry points, the
// posterior and checkpointing.  Host code only; the kernels live in
// xrdvi_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/xrdvi.h"
#include "xrdvi_internal.h"

using namespace xrdvi;

namespace {

thread_local std::string g_err;

xrdvi_status fail(xrdvi_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define XR_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? XRDVI_ENOMEM : XRDVI_ECUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

#define XR_TRY(expr)                          \
    do {                                      \
        xrdvi_status s_ = (expr);             \
        if (s_ != XRDVI_OK) return s_;        \
    } while (0)

constexpr int kUnroll = 16;          // fit steps per captured CUDA graph
constexpr uint32_t kStateMagic = 0x58524456u;  // "XRDV"

// Parameter-free part of ln p(theta) for one phase (Sec. 2.2, Appendix B.2):
// ln lambda - ln(mu_sd) - ln(alpha_sd) - ln(2 pi) + a ln b - lnGamma(a).
double prior_constant(const PriorConst &p) {
    return std::log(p.lambda) - std::log(p.mu_sd) - std::log(p.alpha_sd) - std::log(2.0 * M_PI) +
           p.w_shape * std::log(p.w_rate) - p.lgamma_w_shape;
}

float round_bf16(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    const uint32_t lsb = (b >> 16) & 1u;
    b += 0x7fffu + lsb;  // round to nearest even
    b &= 0xffff0000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

}  // namespace

namespace xrdvi {
// Error reporting for the other host translation units of the library.
xrdvi_status report_error(xrdvi_status st, const std::string &msg) { return fail(st, msg); }
}  // namespace xrdvi

namespace {
std::atomic<uint64_t> g_next_uid{1};

// The captured graphs of the last xrdvi_fit_batch call made with this context
// first in its array.  `key` holds each member's (uid, graph generation), in
// array order: a member that is destroyed, or whose captured arguments
// change, never matches again, so a stale entry is never launched.
struct BatchGraphs {
    std::vector<std::pair<uint64_t, uint64_t>> key;
    xrdvi::MultiStepPlan *plan = nullptr;   // host-side launch plan (null when every fit runs solo)
    std::vector<xrdvi_ctx *> solo;
    cudaStream_t cap = nullptr;             // private capture stream
    cudaGraphExec_t many = nullptr, one = nullptr;
    ~BatchGraphs() {
        if (many) cudaGraphExecDestroy(many);
        if (one) cudaGraphExecDestroy(one);
        if (cap) cudaStreamDestroy(cap);
        xrdvi::multi_plan_destroy(plan);
    }
};
}  // namespace

struct xrdvi_ctx {
    const uint64_t uid = g_next_uid.fetch_add(1);   // never reused within the process
    uint64_t graph_gen = 0;                         // bumped whenever captured arguments go stale
    std::unique_ptr<BatchGraphs> batch;             // see BatchGraphs
    int device = 0;
    cudaStream_t own_stream = nullptr;   // private stream (graph capture; default work stream)
    bool owns_stream = true;             // false when the stream was lent by a server slot
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;        // stream-ordered allocation from this pool when set
    xrdvi_config cfg{};
    Problem P;
    Workspace W;       // fit sample set (S)
    Workspace Wp;      // posterior sample set (S_post)
    PostBuffers B;
    float *loc = nullptr, *raw = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *eps_in = nullptr;   // injected noise [S*K*5]
    float *grad_beta = nullptr;   // [3] beta gradient of the last elbo_grad (fitted background)
    float *f_out = nullptr;    // profile output [S*N]
    double *ent = nullptr, *elbo = nullptr, *trace = nullptr;
    int *step = nullptr, *iter = nullptr;
    cudaGraphExec_t graph_many = nullptr, graph_one = nullptr;
    int64_t host_step = 0;
    double eta = 0.0;
    size_t bytes = 0;
    std::vector<void *> allocs;
    std::vector<void *> post_allocs;
    std::vector<int> host_off;   // CSR offsets (host copy, for work partitioning)

    template <class T>
    xrdvi_status alloc(T **p, size_t n, std::vector<void *> *list = nullptr) {
        if (n == 0) n = 1;
        void *q = nullptr;
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, n * sizeof(T), pool, own_stream)
                             : cudaMalloc(&q, n * sizeof(T));
        if (e != cudaSuccess) {
            return fail(e == cudaErrorMemoryAllocation ? XRDVI_ENOMEM : XRDVI_ECUDA,
                        std::string("device allocation: ") + cudaGetErrorString(e));
        }
        (list ? list : &allocs)->push_back(q);
        bytes += n * sizeof(T);
        *p = static_cast<T *>(q);
        return XRDVI_OK;
    }

    void drop_graphs() {
        if (graph_many) cudaGraphExecDestroy(graph_many);
        if (graph_one) cudaGraphExecDestroy(graph_one);
        graph_many = graph_one = nullptr;
        ++graph_gen;
        batch.reset();
    }

    void release(void *q) {
        if (pool)
            cudaFreeAsync(q, own_stream);
        else
            cudaFree(q);
    }

    void free_post() {
        for (void *q : post_allocs) release(q);
        post_allocs.clear();
        Wp = Workspace();
        B = PostBuffers();
    }

    ~xrdvi_ctx() {
        if (stream) cudaStreamSynchronize(stream);
        if (own_stream && own_stream != stream) cudaStreamSynchronize(own_stream);
        drop_graphs();
        free_post();
        for (void *q : allocs) release(q);
        if (own_stream && owns_stream) cudaStreamDestroy(own_stream);
    }
};

namespace {

// Far-field tables of each 2-theta tile: kFarNodes Chebyshev nodes of the
// first kind on the tile's span [x_lo, x_hi] (rounded to FP32, the positions
// the kernels evaluate at) and the Lagrange weights lam_p(x_i) of the tile's
// points for those nodes, by the barycentric formula (Berrut & Trefethen,
// "Barycentric Lagrange interpolation", SIAM Review 2004) in FP64.  Layout
// lam[(tile * kFarNodes + p) * kTile + j] for point tile * kTile + j (points
// past N repeat the last one).  A one-point tile gets equal weights 1/n
// (all its nodes are that point).
void far_tables(const float *x, int N, int T, bool sec, std::vector<float> &nx, std::vector<float> &nc,
                std::vector<float> &lam) {
    const int n = kFarNodes;
    nx.assign(static_cast<size_t>(T) * n, 0.f);
    if (sec) nc.assign(static_cast<size_t>(T) * n, 0.f);
    lam.assign(static_cast<size_t>(T) * n * kTile, 0.f);
    std::vector<double> z(n), bw(n), term(n);
    for (int t = 0; t < T; ++t) {
        const int i0 = t * kTile, i1 = std::min(i0 + kTile, N) - 1;
        const double lo = x[i0], hi = x[i1], c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
        for (int p = 0; p < n; ++p) {
            const float xp = static_cast<float>(c + h * std::cos(M_PI * (2 * p + 1) / (2.0 * n)));
            nx[static_cast<size_t>(t) * n + p] = xp;
            if (sec)
                nc[static_cast<size_t>(t) * n + p] = static_cast<float>(std::cos(static_cast<double>(xp) * M_PI / 360.0));
            z[p] = h > 0.0 ? (static_cast<double>(xp) - c) / h : 0.0;
        }
        float *L = lam.data() + static_cast<size_t>(t) * n * kTile;
        if (!(h > 0.0)) {
            for (int p = 0; p < n; ++p)
                for (int j = 0; j < kTile; ++j) L[p * kTile + j] = 1.f / n;
            continue;
        }
        // barycentric weights of the (rounded) nodes, scaled to max 1
        double wmax = 0.0;
        for (int p = 0; p < n; ++p) {
            double prod = 1.0;
            for (int q = 0; q < n; ++q)
                if (q != p) prod *= z[p] - z[q];
            bw[p] = 1.0 / prod;
            wmax = std::max(wmax, std::fabs(bw[p]));
        }
        for (int p = 0; p < n; ++p) bw[p] /= wmax;
        for (int j = 0; j < kTile; ++j) {
            const int i = std::min(i0 + j, N - 1);
            const double zi = (static_cast<double>(x[i]) - c) / h;
            int hit = -1;
            double den = 0.0;
            for (int p = 0; p < n && hit < 0; ++p) {
                const double d = zi - z[p];
                if (d == 0.0) hit = p;
                else den += (term[p] = bw[p] / d);
            }
            for (int p = 0; p < n; ++p)
                L[p * kTile + j] = hit >= 0 ? (p == hit ? 1.f : 0.f) : static_cast<float>(term[p] / den);
        }
    }
}

// Second far-field level: kFarNodes Chebyshev nodes on each super-tile's span
// (kSuperTiles tiles), the distance beyond it from which a peak is super-far
// (above every member tile's far gap, with a margin against rounding), and
// the super-level Lagrange weights at every tile's (FP32) nodes, as
// Mf[(t, P, p)] and Mb[(t, p, P)].
void far_tables2(const float *x, int N, int T, bool sec, const std::vector<float> &nx, std::vector<float> &nx2,
                 std::vector<float> &nc2, std::vector<float> &sgap, std::vector<float> &Mf, std::vector<float> &Mb) {
    const int n = kFarNodes, Tg = (T + kSuperTiles - 1) / kSuperTiles;
    nx2.assign(static_cast<size_t>(Tg) * n, 0.f);
    if (sec) nc2.assign(static_cast<size_t>(Tg) * n, 0.f);
    sgap.assign(Tg, 0.f);
    Mf.assign(static_cast<size_t>(T) * n * n, 0.f);
    Mb.assign(static_cast<size_t>(T) * n * n, 0.f);
    std::vector<double> z(n), bw(n), term(n);
    for (int g = 0; g < Tg; ++g) {
        const int i0 = g * kSuperTiles * kTile, i1 = std::min(i0 + kSuperTiles * kTile, N) - 1;
        const double lo = x[i0], hi = x[i1], c = 0.5 * (lo + hi), H = 0.5 * (hi - lo);
        double hmax = 0.0;
        for (int t = g * kSuperTiles; t < std::min((g + 1) * kSuperTiles, T); ++t) {
            const double tl = x[t * kTile], th = x[std::min(t * kTile + kTile, N) - 1];
            hmax = std::max(hmax, 0.5 * (th - tl));
        }
        sgap[g] = static_cast<float>(1.02 * std::max(0.5 * H, static_cast<double>(kFarGap) * hmax) + 2e-4);
        for (int p = 0; p < n; ++p) {
            const float xp = static_cast<float>(c + H * std::cos(M_PI * (2 * p + 1) / (2.0 * n)));
            nx2[static_cast<size_t>(g) * n + p] = xp;
            if (sec)
                nc2[static_cast<size_t>(g) * n + p] = static_cast<float>(std::cos(static_cast<double>(xp) * M_PI / 360.0));
            z[p] = H > 0.0 ? (static_cast<double>(xp) - c) / H : 0.0;
        }
        double wmax = 0.0;
        for (int p = 0; p < n; ++p) {
            double prod = 1.0;
            for (int q = 0; q < n; ++q)
                if (q != p) prod *= z[p] - z[q];
            bw[p] = 1.0 / prod;
            wmax = std::max(wmax, std::fabs(bw[p]));
        }
        for (int p = 0; p < n; ++p) bw[p] /= wmax;
        for (int t = g * kSuperTiles; t < std::min((g + 1) * kSuperTiles, T); ++t) {
            for (int q = 0; q < n; ++q) {   // tile node q
                double w[kFarNodes];
                if (!(H > 0.0)) {
                    for (int P = 0; P < n; ++P) w[P] = 1.0 / n;
                } else {
                    const double zi = (static_cast<double>(nx[static_cast<size_t>(t) * n + q]) - c) / H;
                    int hit = -1;
                    double den = 0.0;
                    for (int P = 0; P < n && hit < 0; ++P) {
                        const double d = zi - z[P];
                        if (d == 0.0) hit = P;
                        else den += (term[P] = bw[P] / d);
                    }
                    for (int P = 0; P < n; ++P) w[P] = hit >= 0 ? (P == hit ? 1.0 : 0.0) : term[P] / den;
                }
                for (int P = 0; P < n; ++P) {
                    Mf[(static_cast<size_t>(t) * n + P) * n + q] = static_cast<float>(w[P]);
                    Mb[(static_cast<size_t>(t) * n + q) * n + P] = static_cast<float>(w[P]);
                }
            }
        }
    }
}

xrdvi_status alloc_workspace(xrdvi_ctx *c, Workspace &W, int S, bool fit,
                             std::vector<void *> *list) {
    const Problem &P = c->P;
    const size_t SK = static_cast<size_t>(S) * P.K;
    const size_t before = c->bytes;
    W.S = S;
    XR_TRY(c->alloc(&W.eps, SK * 5, list));
    XR_TRY(c->alloc(&W.theta, SK * 5, list));
    XR_TRY(c->alloc(&W.cst, SK, list));
    XR_TRY(c->alloc(&W.lpj, static_cast<size_t>(S), list));
    XR_TRY(c->alloc(&W.ll, static_cast<size_t>(S), list));
    XR_TRY(c->alloc(&W.g, static_cast<size_t>(S) * P.Npad, list));
    XR_TRY(c->alloc(&W.llpart, static_cast<size_t>(S) * P.T, list));
    if (fit) {
        XR_TRY(c->alloc(&W.gpart, SK * P.T * kGradSums, list));
        XR_TRY(c->alloc(&W.gred, static_cast<size_t>(W.B) * P.K * kGradBlocks * kGredVals, list));
        XR_TRY(c->alloc(&W.tickets, static_cast<size_t>(W.B) * P.K, list));
        W.lq = nullptr;
        W.iw = nullptr;
        if (P.bgfit) XR_TRY(c->alloc(&W.bgpart, static_cast<size_t>(S) * P.T * 3, list));
        if (c->cfg.flags & XRDVI_FLAG_IW_ELBO) {   // ln q(u_s) and the normalised weights
            XR_TRY(c->alloc(&W.lq, static_cast<size_t>(S), list));
            XR_TRY(c->alloc(&W.iw, static_cast<size_t>(S), list));
        }
    } else {
        XR_TRY(c->alloc(&W.lq, static_cast<size_t>(S), list));
        W.gpart = nullptr;
    }
    if (P.gates) XR_TRY(c->alloc(&W.gzy, SK * 2, list));
    if (P.far) {   // far field: range ends, node weights of g (node sums below, sized with fpart)
        XR_TRY(c->alloc(&W.franges, SK * P.T, list));
        if (P.Tg) XR_TRY(c->alloc(&W.sranges, SK * P.Tg, list));
        if (fit) XR_TRY(c->alloc(&W.wfar, static_cast<size_t>(S) * P.T * kFarNodes, list));
        if (fit && P.Tg) XR_TRY(c->alloc(&W.wfar2, static_cast<size_t>(S) * P.T * kFarNodes, list));
    }
    choose_chunks(P, c->host_off.data(), S, W);
    W.fpart_cap = static_cast<size_t>(W.C) * S * P.Npad;
    XR_TRY(c->alloc(&W.fpart, W.fpart_cap, list));
    if (P.far) {   // per-chunk node sums: kFarNodes per kTile points, so any chunk count fpart holds fits
        XR_TRY(c->alloc(&W.fnode, W.fpart_cap / kTile * kFarNodes, list));
        if (P.Tg) XR_TRY(c->alloc(&W.fnode2, W.fpart_cap / kTile * kFarNodes, list));
    }
    XR_TRY(c->alloc(&W.ranges, SK * P.T, list));
    XR_TRY(c->alloc(&W.counters, kCounters, list));
    W.bytes = c->bytes - before;
    return XRDVI_OK;
}

xrdvi_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return XRDVI_OK;
}

// Reads and clears the flag the gradient reduction sets on a NaN or infinite
// gradient entry (in any step since the last check); synchronises the stream.
xrdvi_status check_gradients(xrdvi_ctx *c) {
    int bad = 0;
    XR_CUDA(cudaMemcpyAsync(&bad, c->P.nonfinite, 4, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaMemsetAsync(c->P.nonfinite, 0, 4, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    if (debug_build()) {   // bounds-check build: a violated check fails the call
        const int w = debug_word(false);
        if (w) return fail(XRDVI_ECUDA, "bounds check " + std::to_string(w) + " failed (XRDVI_DEBUG build)");
    }
    if (bad) return fail(XRDVI_ENONFINITE, "a gradient entry is not finite");
    return XRDVI_OK;
}

AdamConst adam_const(const xrdvi_config &cfg) {
    return AdamConst{cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps};
}

// Profile + likelihood, and the backward's gradient sums, of the fit's sample
// set: the dense profile kernels, or the tensor-core contractions of the
// shared-shape variant.
void fwd_pass(xrdvi_ctx *c, float *f_out, cudaStream_t st) {
    if (c->P.bgfit) launch_bg_curve(c->P, st);
    if (c->W.shared)
        launch_shared_forward(c->P, c->W, f_out, st);
    else
        launch_forward(c->P, c->W, f_out, (c->cfg.flags & XRDVI_FLAG_NAIVE_SUM) != 0, st);
}

void bwd_pass(xrdvi_ctx *c, cudaStream_t st) {
    if (c->W.shared)
        launch_shared_backward(c->P, c->W, st);
    else
        launch_backward(c->P, c->W, st);
}

// One SVI step: sample -> profile + likelihood -> backward -> Adam -> ELBO.
void enqueue_step(xrdvi_ctx *c, cudaStream_t st) {
    launch_sample(c->P, c->W, c->loc, c->raw, nullptr, c->cfg.seed, 0u, c->step, 0u, c->iter, c->ent, st);
    fwd_pass(c, nullptr, st);
    bwd_pass(c, st);
    launch_grad(c->P, c->W, c->loc, c->raw, c->loc, c->raw, nullptr, true, adam_const(c->cfg), c->m,
                c->v, c->iter, c->step, c->ent, c->elbo, c->trace, st);
    if (c->P.bgfit) launch_bg_grad(c->P, c->W, true, adam_const(c->cfg), c->iter, nullptr, st);
}

// Captured on the context's private stream (capturable in every case); the
// executable graph is then launched onto whichever stream the context uses.
xrdvi_status capture(xrdvi_ctx *c, int steps, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    XR_CUDA(cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < steps; ++i) enqueue_step(c, c->own_stream);
    cudaError_t e = cudaStreamEndCapture(c->own_stream, &g);
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    *out = x;   // set only on success
    return XRDVI_OK;
}

bool finite_all(const float *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

xrdvi_status validate(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg) {
    if (!pk || !pt || !cfg) return fail(XRDVI_EINVAL, "null argument");
    if (cfg->size != sizeof(xrdvi_config)) return fail(XRDVI_EINVAL, "config.size mismatch (call xrdvi_config_default)");
    if (pk->K < 1 || pk->K > kMaxK) return fail(XRDVI_EINVAL, "K must be in [1, 1024]");
    if (!pk->offsets || !pk->pos_deg || !pk->rel_int) return fail(XRDVI_EINVAL, "null peak arrays");
    if (pk->offsets[0] != 0) return fail(XRDVI_EINVAL, "offsets[0] must be 0");
    for (int k = 0; k < pk->K; ++k)
        if (pk->offsets[k + 1] - pk->offsets[k] < 1) return fail(XRDVI_EINVAL, "every phase needs at least one peak");
    const int M = pk->offsets[pk->K];
    if (M > kMaxPeaks) return fail(XRDVI_EINVAL, "total peaks above 24000");
    for (int i = 0; i < M; ++i) {
        const float p = pk->pos_deg[i], I = pk->rel_int[i];
        if (!(std::isfinite(p) && p > 0.f && p < 180.f)) return fail(XRDVI_EINVAL, "peak position outside (0, 180)");
        if (!(std::isfinite(I) && I >= 0.f && I <= 1.f)) return fail(XRDVI_EINVAL, "relative intensity outside [0, 1]");
    }
    if (pt->N < 1 || pt->N > kMaxN) return fail(XRDVI_EINVAL, "N must be in [1, 2^24]");
    if (!pt->x_deg || !pt->y_counts || !pt->bg) return fail(XRDVI_EINVAL, "null pattern arrays");
    for (int i = 0; i < pt->N; ++i) {
        const float x = pt->x_deg[i], y = pt->y_counts[i], b = pt->bg[i];
        if (!(std::isfinite(x) && x > 0.f && x < 180.f)) return fail(XRDVI_EINVAL, "2-theta outside (0, 180)");
        if (i > 0 && !(x > pt->x_deg[i - 1])) return fail(XRDVI_EINVAL, "x must be strictly increasing");
        if (!(std::isfinite(y) && y >= 0.f && std::floor(y) == y)) return fail(XRDVI_EINVAL, "counts must be non-negative integers");
        if (!(std::isfinite(b) && b >= 0.f)) return fail(XRDVI_EINVAL, "background must be finite and >= 0");
    }
    if (cfg->S < 1 || cfg->S > kMaxS) return fail(XRDVI_EINVAL, "S must be in [1, 65536]");
    if ((cfg->flags & XRDVI_FLAG_FIT_BACKGROUND) && !(std::isfinite(cfg->bg_prior_sd) && cfg->bg_prior_sd > 0.f))
        return fail(XRDVI_EINVAL, "bg_prior_sd must be positive");
    if ((cfg->flags & XRDVI_FLAG_FIX_R) && !(cfg->fix_r_value >= 0.f && cfg->fix_r_value <= 1.f))
        return fail(XRDVI_EINVAL, "fix_r_value must be in [0, 1]");
    if ((cfg->flags & XRDVI_FLAG_FIX_ALPHA) && !std::isfinite(cfg->fix_alpha_value))
        return fail(XRDVI_EINVAL, "fix_alpha_value must be finite");
    if ((cfg->flags & XRDVI_FLAG_GATES) &&
        !(cfg->gate_tau > 0.f && cfg->gate_tau < 100.f && cfg->gate_prior > 0.f && cfg->gate_prior < 1.f))
        return fail(XRDVI_EINVAL, "gates need gate_tau in (0, 100) and gate_prior in (0, 1)");
    const float pos_params[] = {cfg->prior_mu_sd, cfg->prior_alpha_sd, cfg->prior_w_shape, cfg->prior_w_rate,
                                cfg->alpha_min, cfg->init_h_frac, cfg->init_sigma, cfg->lr};
    for (float q : pos_params)
        if (!(std::isfinite(q) && q > 0.f)) return fail(XRDVI_EINVAL, "prior / optimiser parameters must be positive");
    if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->adam_eps > 0.f))
        return fail(XRDVI_EINVAL, "Adam betas must be in [0, 1) and eps > 0");
    return XRDVI_OK;
}

}  // namespace

namespace xrdvi {
xrdvi_status validate_problem(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg) {
    return validate(pk, pt, cfg);
}

xrdvi_status batch_set_tail(xrdvi_ctx *c, int tail_start) {
    if (!c || !c->W.tail_sum) return fail(XRDVI_EINVAL, "not a sub-model batch context");
    c->W.tail_start = tail_start;
    c->drop_graphs();   // kernel arguments are fixed at capture
    return XRDVI_OK;
}

xrdvi_status batch_tail_sums(xrdvi_ctx *c, double *host) {
    if (!c || !c->W.tail_sum || !host) return fail(XRDVI_EINVAL, "not a sub-model batch context");
    XR_CUDA(cudaMemcpyAsync(host, c->W.tail_sum, static_cast<size_t>(c->W.B) * 8, cudaMemcpyDeviceToHost,
                            c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    return XRDVI_OK;
}
}  // namespace xrdvi

namespace xrdvi {
// Access to a context's device state for the continuous-batching server.
void ctx_fit_step(xrdvi_ctx *c, FitStep *out) {
    out->P = &c->P;
    out->W = &c->W;
    out->loc = c->loc;
    out->raw = c->raw;
    out->m = c->m;
    out->v = c->v;
    out->iter = c->iter;
    out->step = c->step;
    out->ent = c->ent;
    out->elbo = c->elbo;
    out->trace = c->trace;
    out->seed = c->cfg.seed;
    out->ac = adam_const(c->cfg);
}

bool ctx_multi_eligible(const xrdvi_ctx *c) {
    return multi_fit_eligible(c->P, c->W, (c->cfg.flags & XRDVI_FLAG_NAIVE_SUM) != 0,
                              (c->cfg.flags & XRDVI_FLAG_IW_ELBO) != 0);
}

void ctx_enqueue_steps(xrdvi_ctx *c, int n, cudaStream_t st) {
    for (int i = 0; i < n; ++i) enqueue_step(c, st);
}

void ctx_advance(xrdvi_ctx *c, int n) { c->host_step += n; }

// Captures `steps` SVI steps of a batch (the plan's multi-fit launches, then
// each solo context's own kernels) on the private stream `cap` as one graph.
xrdvi_status capture_batch_steps(const MultiStepPlan *plan, xrdvi_ctx *const *solo, int nsolo, int steps,
                                 cudaStream_t cap, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    XR_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < steps; ++i) {
        if (plan) multi_plan_launch_step(plan, cap);
        for (int j = 0; j < nsolo; ++j) enqueue_step(solo[j], cap);
    }
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    *out = x;   // set only on success: callers destroy what they hold
    return XRDVI_OK;
}

cudaStream_t ctx_stream(const xrdvi_ctx *c) { return c->stream; }

// The ELBO estimates of the last n steps (host copy; synchronises the
// context's stream) and the last one's finiteness.
xrdvi_status ctx_read_trace(xrdvi_ctx *c, int n, double *host) {
    if (n <= 0) return XRDVI_OK;
    const int64_t s0 = c->host_step - n;
    for (int done = 0; done < n;) {
        const int64_t a = (s0 + done) & (kTraceCap - 1);
        const int64_t len = std::min<int64_t>(n - done, kTraceCap - a);
        XR_CUDA(cudaMemcpyAsync(host + done, c->trace + a, len * 8, cudaMemcpyDeviceToHost, c->stream));
        done += static_cast<int>(len);
    }
    XR_CUDA(cudaStreamSynchronize(c->stream));
    const xrdvi_status gs = check_gradients(c);
    if (!std::isfinite(host[n - 1])) return fail(XRDVI_ENONFINITE, "ELBO is not finite");
    return gs;
}
}  // namespace xrdvi

extern "C" {

const char *xrdvi_last_error(void) { return g_err.c_str(); }

const char *xrdvi_version(void) { return "xrdvi 0.1 (sm_103a)"; }

void xrdvi_config_default(xrdvi_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->size = sizeof(xrdvi_config);
    cfg->S = 256;
    cfg->lr = 0.01f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.999f;
    cfg->adam_eps = 1e-8f;
    cfg->seed = 0;
    cfg->prior_mu_sd = 0.03f;
    cfg->prior_alpha_mean = 1.0f;
    cfg->prior_alpha_sd = 0.2f;
    cfg->prior_w_shape = 3.0f;
    cfg->prior_w_rate = 100.0f;
    cfg->alpha_min = 1e-3f;
    cfg->init_h_frac = 0.1f;
    cfg->init_sigma = 0.1f;
    cfg->flags = 0;
    cfg->bg_prior_sd = 0.1f;
    cfg->fix_r_value = 0.5f;
    cfg->fix_alpha_value = 1.f;
    cfg->gate_tau = 2.f / 3.f;
    cfg->gate_prior = 0.5f;
}

xrdvi_status xrdvi_create(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                          xrdvi_ctx **out) {
    if (cfg && cfg->size == sizeof(xrdvi_config) && (cfg->flags & XRDVI_FLAG_DEVICE_PTRS) && pk && pt) {
        // device inputs: one read-back, then the host path
        if (pk->K < 1 || pk->K > kMaxK || pt->N < 1 || pt->N > kMaxN || !pk->offsets || !pk->pos_deg ||
            !pk->rel_int || !pt->x_deg || !pt->y_counts || !pt->bg)
            return fail(XRDVI_EINVAL, "bad sizes or null device arrays");
        std::vector<int32_t> off(pk->K + 1);
        XR_CUDA(cudaMemcpy(off.data(), pk->offsets, off.size() * 4, cudaMemcpyDeviceToHost));
        if (off[0] != 0 || off[pk->K] < 1 || off[pk->K] > kMaxPeaks) return fail(XRDVI_EINVAL, "bad offsets");
        const int M = off[pk->K], N = pt->N;
        std::vector<float> pos(M), inten(M), x(N), y(N), bg(N);
        XR_CUDA(cudaMemcpy(pos.data(), pk->pos_deg, M * 4, cudaMemcpyDeviceToHost));
        XR_CUDA(cudaMemcpy(inten.data(), pk->rel_int, M * 4, cudaMemcpyDeviceToHost));
        XR_CUDA(cudaMemcpy(x.data(), pt->x_deg, N * 4, cudaMemcpyDeviceToHost));
        XR_CUDA(cudaMemcpy(y.data(), pt->y_counts, N * 4, cudaMemcpyDeviceToHost));
        XR_CUDA(cudaMemcpy(bg.data(), pt->bg, N * 4, cudaMemcpyDeviceToHost));
        const xrdvi_peaks hpk{pk->K, off.data(), pos.data(), inten.data()};
        const xrdvi_pattern hpt{N, x.data(), y.data(), bg.data()};
        return xrdvi::create_context(&hpk, &hpt, cfg, nullptr, nullptr, out);
    }
    return xrdvi::create_context(pk, pt, cfg, nullptr, nullptr, out);
}

}  // extern "C"

xrdvi_status xrdvi::create_context(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                                   cudaMemPool_t pool, cudaStream_t stream, xrdvi_ctx **out) {
    return create_batch_context(pk, pt, cfg, 1, nullptr, pool, stream, out);
}

xrdvi_status xrdvi::create_batch_context(const xrdvi_peaks *pk, const xrdvi_pattern *pt, const xrdvi_config *cfg,
                                         int nsub, const uint32_t *masks, cudaMemPool_t pool, cudaStream_t stream,
                                         xrdvi_ctx **out) {
    NvtxRange nvtx("xrdvi_create");
    g_err.clear();
    if (!out) return fail(XRDVI_EINVAL, "null output pointer");
    *out = nullptr;
    XR_TRY(validate(pk, pt, cfg));
    const int K = pk->K, N = pt->N, M = pk->offsets[K];
    if (nsub < 1 || static_cast<int64_t>(nsub) * cfg->S > kMaxS)
        return fail(XRDVI_EINVAL, "sub-model batch: B * S must be in [1, 65536]");
    if (masks && (cfg->flags & (XRDVI_FLAG_SHARED_SHAPES | XRDVI_FLAG_FIT_BACKGROUND | XRDVI_FLAG_GATES)))
        return fail(XRDVI_EINVAL,
                    "the shared-shape, fitted-background and gate variants do not run in sub-model batches");
    if (masks) {
        if (K > 32) return fail(XRDVI_EINVAL, "sub-model batch: K must be <= 32");
        for (int b = 0; b < nsub; ++b)
            if (masks[b] == 0u || (K < 32 && (masks[b] >> K) != 0u))
                return fail(XRDVI_EINVAL, "sub-model batch: masks must be non-empty subsets of the K phases");
    } else if (nsub != 1) {
        return fail(XRDVI_EINVAL, "sub-model batch needs masks");
    }
    const size_t KB = static_cast<size_t>(K) * nsub;
    // host preparation: sort each phase by position, eta, data constant
    std::vector<float> pos(M), inten(M);
    std::vector<double> isum(K, 0.0);
    const bool bf16 = (cfg->flags & XRDVI_FLAG_BF16_INT) != 0;
    for (int k = 0; k < K; ++k) {
        const int b = pk->offsets[k], e = pk->offsets[k + 1];
        std::vector<int> idx(e - b);
        std::iota(idx.begin(), idx.end(), b);
        std::stable_sort(idx.begin(), idx.end(), [&](int i, int j) { return pk->pos_deg[i] < pk->pos_deg[j]; });
        for (int i = 0; i < e - b; ++i) {
            pos[b + i] = pk->pos_deg[idx[i]];
            const float I = bf16 ? round_bf16(pk->rel_int[idx[i]]) : pk->rel_int[idx[i]];
            inten[b + i] = I;
            isum[k] += I;
        }
    }
    double eta = -INFINITY, csum = 0.0;
    for (int i = 0; i < N; ++i) {
        const double y = pt->y_counts[i];
        eta = std::max(eta, y - static_cast<double>(pt->bg[i]));
        if (y > 0) csum += y * std::log(y) - y - std::lgamma(y + 1.0);
    }
    if (!(eta > 0.0)) return fail(XRDVI_EINVAL, "max(Y - B) must be positive (it sets the intensity prior)");
    const bool sec = (cfg->flags & XRDVI_FLAG_SEC_WIDTH) != 0;
    std::vector<float> csec;
    float sec_max = 1.f;
    if (sec) {   // angle-dependent width: cos(x/2) per point, x in degrees of 2-theta
        csec.resize(N);
        double mx = 1.0;
        for (int i = 0; i < N; ++i) {
            if (!(pt->x_deg[i] < 174.f)) return fail(XRDVI_EINVAL, "angle-dependent width needs every x < 174 deg");
            const double cv = std::cos(static_cast<double>(pt->x_deg[i]) * M_PI / 360.0);
            csec[i] = static_cast<float>(cv);
            mx = std::max(mx, 1.0 / cv);
        }
        sec_max = static_cast<float>(mx * (1.0 + 1e-6));   // reach bound, rounded up
    }
    const bool gauss = (cfg->flags & XRDVI_FLAG_GAUSS_LIK) != 0;
    if (gauss) {   // Gaussian variant: the data part is -ln(2 pi v_i)/2, v_i = max(y_i, 1)
        csum = 0.0;
        for (int i = 0; i < N; ++i)
            csum -= 0.5 * std::log(2.0 * M_PI * std::max(1.0, static_cast<double>(pt->y_counts[i])));
    }

    int dev = 0, sms = 0;
    XR_CUDA(cudaGetDevice(&dev));
    XR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    xrdvi_ctx *c = new xrdvi_ctx();
    c->device = dev;
    c->cfg = *cfg;
    c->eta = eta;
    auto bail = [&](xrdvi_status st) {
        std::string keep = g_err;
        delete c;
        g_err = keep;
        return st;
    };
    if (stream) {
        c->own_stream = stream;
        c->owns_stream = false;
    } else if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        return bail(fail(XRDVI_ECUDA, "cudaStreamCreate failed"));
    }
    c->stream = c->own_stream;
    c->pool = pool;

    Problem &P = c->P;
    P.K = K;
    P.N = N;
    P.Mtot = M;
    P.T = (N + kTile - 1) / kTile;
    P.Npad = P.T * kTile;
    P.csum = csum;
    P.gauss = gauss;
    P.sec = sec;
    P.sec_max = sec_max;
    P.prior.lambda = 1.0 / eta;
    P.prior.mu_sd = cfg->prior_mu_sd;
    P.prior.alpha_mean = cfg->prior_alpha_mean;
    P.prior.alpha_sd = cfg->prior_alpha_sd;
    P.prior.w_shape = cfg->prior_w_shape;
    P.prior.w_rate = cfg->prior_w_rate;
    P.prior.lgamma_w_shape = std::lgamma(static_cast<double>(cfg->prior_w_shape));
    P.prior.alpha_min = cfg->alpha_min;
    P.prior.lp_const = prior_constant(P.prior);
    P.area_norm = (cfg->flags & XRDVI_FLAG_AREA_NORM) != 0;
    P.gates = (cfg->flags & XRDVI_FLAG_GATES) != 0;
    P.gate_tau = cfg->gate_tau;
    P.gate_a0 = static_cast<float>(std::log(cfg->gate_prior / (1.0 - cfg->gate_prior)));
    P.fix_r = (cfg->flags & XRDVI_FLAG_FIX_R) != 0;
    P.fix_alpha = (cfg->flags & XRDVI_FLAG_FIX_ALPHA) != 0;
    P.r_value = cfg->fix_r_value;
    P.alpha_value = cfg->fix_alpha_value;
    if (P.fix_alpha)   // a fixed alpha has no prior: drop its normal's constant
        P.prior.lp_const += std::log(P.prior.alpha_sd) + 0.5 * std::log(2.0 * M_PI);

    xrdvi_status st;
#define XR_C(expr)                         \
    do {                                   \
        st = (expr);                       \
        if (st != XRDVI_OK) return bail(st); \
    } while (0)
    XR_C(c->alloc(&P.pos, M));
    XR_C(c->alloc(&P.inten, M));
    XR_C(c->alloc(&P.off, K + 1));
    XR_C(c->alloc(&P.x, N));
    XR_C(c->alloc(&P.y, N));
    XR_C(c->alloc(&P.bg, N));
    XR_C(c->alloc(&P.isum, K));
    XR_C(c->alloc(&P.nonfinite, 1));
    if (sec) XR_C(c->alloc(&P.csec, N));
    if (P.gates) {   // gate logits start at 0 (z = sigmoid(L / tau))
        XR_C(c->alloc(&P.gate_a, K));
        XR_C(c->alloc(&P.m_gate, K));
        XR_C(c->alloc(&P.v_gate, K));
        XR_C(c->alloc(&P.grad_gate, K));
    }
    std::vector<float> Tb;
    if (cfg->flags & XRDVI_FLAG_FIT_BACKGROUND) {
        // fitted background: Chebyshev terms of the grid mapped onto [-1, 1]
        P.bgfit = true;
        P.bg_sd = cfg->bg_prior_sd;
        Tb.resize(static_cast<size_t>(3) * N);
        const double x0 = pt->x_deg[0], x1 = pt->x_deg[N - 1];
        for (int i = 0; i < N; ++i) {
            const double z = N > 1 ? 2.0 * (pt->x_deg[i] - x0) / (x1 - x0) - 1.0 : 0.0;
            Tb[i] = 1.f;
            Tb[N + i] = static_cast<float>(z);
            Tb[2 * N + i] = static_cast<float>(2.0 * z * z - 1.0);
        }
        XR_C(c->alloc(&P.Tb, static_cast<size_t>(3) * N));
        XR_C(c->alloc(&P.Bb, N));
        XR_C(c->alloc(&P.beta, 3));
        XR_C(c->alloc(&P.m_beta, 3));
        XR_C(c->alloc(&P.v_beta, 3));
        XR_C(c->alloc(&c->grad_beta, 3));
    }
    // far field (off with the dense flag, the shared-shape variant and very
    // long patterns): Chebyshev nodes and Lagrange weights of every tile
    std::vector<float> nodex, nodec, lamh;
    P.far = !(cfg->flags & (XRDVI_FLAG_SHARED_SHAPES | XRDVI_FLAG_DENSE)) &&
            static_cast<size_t>(P.T) * kFarNodes * kTile * sizeof(float) <= kFarMaxLamBytes;
    std::vector<int> far_order(K);
    std::vector<float> nodex2, nodec2, sgaph, Mfh, Mbh;
    if (P.far) {
        far_tables(pt->x_deg, N, P.T, sec, nodex, nodec, lamh);
        if (P.T > kSuperTiles) {   // second level (with up to kSuperTiles tiles it would add nothing)
            far_tables2(pt->x_deg, N, P.T, sec, nodex, nodex2, nodec2, sgaph, Mfh, Mbh);
            P.Tg = (P.T + kSuperTiles - 1) / kSuperTiles;
            XR_C(c->alloc(&P.node_x2, nodex2.size()));
            if (sec) XR_C(c->alloc(&P.node_c2, nodec2.size()));
            XR_C(c->alloc(&P.sgap, sgaph.size()));
            XR_C(c->alloc(&P.Mf, Mfh.size()));
            XR_C(c->alloc(&P.Mb, Mbh.size()));
        }
        XR_C(c->alloc(&P.node_x, nodex.size()));
        XR_C(c->alloc(&P.lam, lamh.size()));
        if (sec) XR_C(c->alloc(&P.node_c, nodec.size()));
    }
    // phases by decreasing peak count (the shared-shape profile kernel starts the heaviest first)
    std::iota(far_order.begin(), far_order.end(), 0);
    std::stable_sort(far_order.begin(), far_order.end(), [&](int i, int j) {
        return pk->offsets[i + 1] - pk->offsets[i] > pk->offsets[j + 1] - pk->offsets[j];
    });
    XR_C(c->alloc(&P.far_order, static_cast<size_t>(K)));
    configure_grids(P, sms);
    c->host_off.assign(pk->offsets, pk->offsets + K + 1);
    c->W.B = nsub;
    c->W.S_sub = cfg->S;
    XR_C(alloc_workspace(c, c->W, cfg->S * nsub, true, nullptr));
    uint32_t *d_mask = nullptr;
    if (masks) {
        XR_C(c->alloc(&d_mask, static_cast<size_t>(nsub)));
        XR_C(c->alloc(&c->W.tail_sum, static_cast<size_t>(nsub)));
        c->W.mask = d_mask;
        c->cfg.S = cfg->S * nsub;
    }
    XR_C(c->alloc(&c->loc, KB * 5));
    XR_C(c->alloc(&c->raw, KB * 5));
    XR_C(c->alloc(&c->m, KB * 10));
    XR_C(c->alloc(&c->v, KB * 10));
    XR_C(c->alloc(&c->grad, KB * 10));
    XR_C(c->alloc(&c->ent, static_cast<size_t>(nsub)));
    XR_C(c->alloc(&c->elbo, static_cast<size_t>(nsub)));
    Workspace &W = c->W;
    if (cfg->flags & XRDVI_FLAG_SHARED_SHAPES) {
        // shared-shape variant: GEMM operands and scratch of the tensor-core contractions
        W.shared = true;
        W.Kpad = (K + 31) / 32 * 32;
        const int nk = K * kGradSums;
        W.gemm_splits = gemm_splits(W.S, nk, P.Npad, sms);
        XR_C(c->alloc(&W.H, static_cast<size_t>(2) * W.S * W.Kpad));      // TF32 hi + lo parts
        XR_C(c->alloc(&W.Ct, static_cast<size_t>(2) * P.Npad * W.Kpad));
        XR_C(c->alloc(&W.D, static_cast<size_t>(2) * nk * P.Npad));
        XR_C(c->alloc(&W.ghl, static_cast<size_t>(2) * W.S * P.Npad));
        XR_C(c->alloc(&W.gemm_work, gemm_workspace_floats(W.S, nk, W.gemm_splits)));
        XR_C(c->alloc(&W.gemm_err, 1));
        if (gemm_configure() != cudaSuccess) return bail(fail(XRDVI_ECUDA, "tensor-core GEMM set-up failed"));
        // the two contractions on fixed buffers: TMA descriptors built once
        const size_t nh = static_cast<size_t>(W.S) * W.Kpad, nc = static_cast<size_t>(P.Npad) * W.Kpad;
        const size_t ng = static_cast<size_t>(W.S) * P.Npad, nd = static_cast<size_t>(nk) * P.Npad;
        if (!gemm_plan(W.plan_fwd, W.S, N, W.Kpad, W.H, W.H + nh, W.Kpad, W.Ct, W.Ct + nc, W.Kpad, W.fpart, P.Npad,
                       1, nullptr, W.gemm_err) ||
            !gemm_plan(W.plan_bwd, W.S, nk, P.Npad, W.ghl, W.ghl + ng, P.Npad, W.D, W.D + nd, P.Npad, W.gpart, nk,
                       W.gemm_splits, W.gemm_work, W.gemm_err))
            return bail(fail(XRDVI_ECUDA, "tensor-core GEMM: TMA descriptor encoding failed"));
    }
    XR_C(c->alloc(&c->trace, kTraceCap));
    XR_C(c->alloc(&c->step, 1));
    XR_C(c->alloc(&c->iter, 1));

    // initial q (reading: loc at h = init_h_frac * eta, mu = 0, w at the prior
    // mean shape/rate, r = 1/2, alpha at its prior mean; sigma = init_sigma)
    std::vector<float> loc(KB * 5), raw(KB * 5);
    const double raw0 = std::log(std::expm1(static_cast<double>(cfg->init_sigma)));
    for (size_t k = 0; k < KB; ++k) {
        // area-normalised profiles start from the same curve: height times the initial shape's area
        const double a0 = 0.5 * (1.0 + std::max(static_cast<double>(cfg->prior_alpha_mean),
                                                 static_cast<double>(cfg->alpha_min))) *
                          (static_cast<double>(cfg->prior_w_shape) / cfg->prior_w_rate) *
                          (0.5 * 0.5 * std::sqrt(M_PI / std::log(2.0)) + 0.5 * 0.5 * M_PI);
        loc[k * 5 + 0] = static_cast<float>(std::log(cfg->init_h_frac * eta * ((cfg->flags & XRDVI_FLAG_AREA_NORM) ? a0 : 1.0)));
        loc[k * 5 + 1] = 0.f;
        loc[k * 5 + 2] = static_cast<float>(std::log(static_cast<double>(cfg->prior_w_shape) / cfg->prior_w_rate));
        loc[k * 5 + 3] = 0.f;
        loc[k * 5 + 4] = cfg->prior_alpha_mean;
        for (int j = 0; j < 5; ++j) raw[k * 5 + j] = static_cast<float>(raw0);
    }
    cudaStream_t s = c->stream;
    auto up = [&](void *dst, const void *src, size_t n) { return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s); };
    if (up(P.pos, pos.data(), M * 4) || up(P.inten, inten.data(), M * 4) ||
        up(P.off, pk->offsets, (K + 1) * 4) || up(P.x, pt->x_deg, N * 4) || up(P.y, pt->y_counts, N * 4) ||
        up(P.bg, pt->bg, N * 4) || up(P.isum, isum.data(), K * 8) ||
        up(P.far_order, far_order.data(), static_cast<size_t>(K) * 4) || (sec && up(P.csec, csec.data(), N * 4)) ||
        up(c->loc, loc.data(), KB * 20) ||
        up(c->raw, raw.data(), KB * 20) || cudaMemsetAsync(c->m, 0, KB * 40, s) ||
        cudaMemsetAsync(c->v, 0, KB * 40, s) || cudaMemsetAsync(c->step, 0, 4, s) ||
        cudaMemsetAsync(P.nonfinite, 0, 4, s) ||
        cudaMemsetAsync(c->trace, 0, kTraceCap * 8, s) ||
        (d_mask && (up(d_mask, masks, static_cast<size_t>(nsub) * 4) ||
                    cudaMemsetAsync(c->W.tail_sum, 0, static_cast<size_t>(nsub) * 8, s))) ||
        (P.gates && (cudaMemsetAsync(P.gate_a, 0, K * 4, s) || cudaMemsetAsync(P.m_gate, 0, K * 4, s) ||
                     cudaMemsetAsync(P.v_gate, 0, K * 4, s) || cudaMemsetAsync(P.grad_gate, 0, K * 4, s))) ||
        (P.far && (up(P.node_x, nodex.data(), nodex.size() * 4) || up(P.lam, lamh.data(), lamh.size() * 4) ||
                   (P.Tg && (up(P.node_x2, nodex2.data(), nodex2.size() * 4) || up(P.sgap, sgaph.data(), sgaph.size() * 4) ||
                             up(P.Mf, Mfh.data(), Mfh.size() * 4) || up(P.Mb, Mbh.data(), Mbh.size() * 4) ||
                             (sec && up(P.node_c2, nodec2.data(), nodec2.size() * 4)))) ||
                   (sec && up(P.node_c, nodec.data(), nodec.size() * 4)))) ||
        (P.bgfit && (up(P.Tb, Tb.data(), Tb.size() * 4) || cudaMemsetAsync(P.beta, 0, 12, s) ||
                     cudaMemsetAsync(P.m_beta, 0, 12, s) || cudaMemsetAsync(P.v_beta, 0, 12, s) ||
                     cudaMemsetAsync(c->grad_beta, 0, 12, s))) ||
        (W.shared && (cudaMemsetAsync(W.H, 0, static_cast<size_t>(2) * W.S * W.Kpad * 4, s) ||
                      cudaMemsetAsync(W.Ct, 0, static_cast<size_t>(2) * P.Npad * W.Kpad * 4, s) ||
                      cudaMemsetAsync(W.gemm_err, 0, 4, s))))
        return bail(fail(XRDVI_ECUDA, "upload failed"));
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(fail(XRDVI_ECUDA, "create: device error"));
#undef XR_C
    *out = c;
    return XRDVI_OK;
}

extern "C" {

void xrdvi_destroy(xrdvi_ctx *c) { delete c; }

xrdvi_status xrdvi_set_stream(xrdvi_ctx *c, void *stream) {
    if (!c) return fail(XRDVI_EINVAL, "null context");
    XR_CUDA(cudaStreamSynchronize(c->stream));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return XRDVI_OK;
}

xrdvi_status xrdvi_fit(xrdvi_ctx *c, int32_t iters, double *trace) {
    NvtxRange nvtx("xrdvi_fit");
    if (!c) return fail(XRDVI_EINVAL, "null context");
    if (iters < 0) return fail(XRDVI_EINVAL, "iters must be >= 0");
    if (iters == 0) return XRDVI_OK;
    if (c->host_step + iters > INT32_MAX) return fail(XRDVI_EINVAL, "step counter would overflow");
    if (!c->graph_many) XR_TRY(capture(c, kUnroll, &c->graph_many));
    if (!c->graph_one) XR_TRY(capture(c, 1, &c->graph_one));
    int done = 0;
    while (done < iters) {
        const int chunk = std::min(iters - done, kTraceCap / 2);
        int left = chunk;
        while (left >= kUnroll) {
            XR_CUDA(cudaGraphLaunch(c->graph_many, c->stream));
            left -= kUnroll;
        }
        while (left-- > 0) XR_CUDA(cudaGraphLaunch(c->graph_one, c->stream));
        if (trace) {
            const int64_t s0 = c->host_step + done;
            const int64_t a = s0 & (kTraceCap - 1);
            const int64_t n1 = std::min<int64_t>(chunk, kTraceCap - a);
            XR_CUDA(cudaMemcpyAsync(trace + done, c->trace + a, n1 * 8, cudaMemcpyDeviceToHost, c->stream));
            if (n1 < chunk)
                XR_CUDA(cudaMemcpyAsync(trace + done + n1, c->trace, (chunk - n1) * 8, cudaMemcpyDeviceToHost,
                                        c->stream));
        }
        done += chunk;
    }
    double last = 0.0;
    int gerr = 0;
    XR_CUDA(cudaMemcpyAsync(&last, c->elbo, 8, cudaMemcpyDeviceToHost, c->stream));
    if (c->W.gemm_err) XR_CUDA(cudaMemcpyAsync(&gerr, c->W.gemm_err, 4, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    c->host_step += iters;
    if (gerr) return fail(XRDVI_ETIMEOUT, "tensor-core pipeline wait gave up");
    const xrdvi_status gs = check_gradients(c);   // read and cleared in every case
    if (!std::isfinite(last)) return fail(XRDVI_ENONFINITE, "ELBO is not finite");
    return gs;
}

xrdvi_status xrdvi_fit_batch(xrdvi_ctx *const *ctxs, int32_t n, int32_t iters, double *last_elbo) {
    NvtxRange nvtx("xrdvi_fit_batch");
    if (!ctxs || n < 1 || n > kMaxBatch) return fail(XRDVI_EINVAL, "n must be in [1, 64] with a context array");
    if (iters < 0) return fail(XRDVI_EINVAL, "iters must be >= 0");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(XRDVI_EINVAL, "null context");
        if (ctxs[i]->device != ctxs[0]->device) return fail(XRDVI_EINVAL, "contexts on different devices");
        if (ctxs[i]->host_step + iters > INT32_MAX) return fail(XRDVI_EINVAL, "step counter would overflow");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(XRDVI_EINVAL, "a context appears twice");
    }
    for (int i = 0; i < n; ++i) XR_CUDA(cudaStreamSynchronize(ctxs[i]->stream));
    cudaStream_t st = ctxs[0]->stream;
    std::vector<std::pair<uint64_t, uint64_t>> key(n);
    for (int i = 0; i < n; ++i) key[i] = {ctxs[i]->uid, ctxs[i]->graph_gen};
    BatchGraphs *bg = ctxs[0]->batch.get();
    if (!bg || bg->key != key) {   // new member set, or a member's captured arguments changed
        ctxs[0]->batch.reset();
        auto fresh = std::make_unique<BatchGraphs>();
        std::vector<FitStep> fs;
        for (int i = 0; i < n; ++i) {
            if (ctx_multi_eligible(ctxs[i])) {
                FitStep f;
                ctx_fit_step(ctxs[i], &f);
                fs.push_back(f);
            } else {
                fresh->solo.push_back(ctxs[i]);
            }
        }
        if (!fs.empty()) {
            int sms = 0;
            XR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctxs[0]->device));
            fresh->plan = multi_plan_create(static_cast<int>(fs.size()));
            if (!fresh->plan || !multi_plan_set(fresh->plan, fs.data(), static_cast<int>(fs.size()), sms, st))
                return fail(XRDVI_ECUDA, "fit_batch: batch set-up failed");
        }
        if (cudaStreamCreateWithFlags(&fresh->cap, cudaStreamNonBlocking) != cudaSuccess)
            return fail(XRDVI_ECUDA, "fit_batch: cudaStreamCreate failed");
        fresh->key = key;
        bg = fresh.get();
        ctxs[0]->batch = std::move(fresh);
    }
    // kUnroll steps per captured graph (captured once per member set on the
    // private stream, then reused by later calls), the rest one by one
    xrdvi_status cs = XRDVI_OK;
    const int nsolo = static_cast<int>(bg->solo.size());
    if (iters >= kUnroll && !bg->many)
        cs = capture_batch_steps(bg->plan, bg->solo.data(), nsolo, kUnroll, bg->cap, &bg->many);
    if (cs == XRDVI_OK && iters % kUnroll && !bg->one)
        cs = capture_batch_steps(bg->plan, bg->solo.data(), nsolo, 1, bg->cap, &bg->one);
    if (cs == XRDVI_OK) {
        int left = iters;
        for (; left >= kUnroll && cs == XRDVI_OK; left -= kUnroll)
            if (cudaGraphLaunch(bg->many, st) != cudaSuccess) cs = fail(XRDVI_ECUDA, "fit_batch: graph launch failed");
        for (; left > 0 && cs == XRDVI_OK; --left)
            if (cudaGraphLaunch(bg->one, st) != cudaSuccess) cs = fail(XRDVI_ECUDA, "fit_batch: graph launch failed");
    }
    const xrdvi_status ls = cs != XRDVI_OK ? cs : check_launch("fit_batch");
    std::vector<double> last(n, 0.0);
    for (int i = 0; i < n; ++i) XR_CUDA(cudaMemcpyAsync(&last[i], ctxs[i]->elbo, 8, cudaMemcpyDeviceToHost, st));
    XR_CUDA(cudaStreamSynchronize(st));
    if (ls != XRDVI_OK) {
        ctxs[0]->batch.reset();   // a failed capture or launch is not reused
        return ls;
    }
    xrdvi_status out = XRDVI_OK;
    for (int i = 0; i < n; ++i) {
        ctxs[i]->host_step += iters;
        if (last_elbo) last_elbo[i] = last[i];
        const xrdvi_status gs = iters > 0 ? check_gradients(ctxs[i]) : XRDVI_OK;
        if (out == XRDVI_OK && iters > 0 && !std::isfinite(last[i]))
            out = fail(XRDVI_ENONFINITE, "ELBO is not finite (context " + std::to_string(i) + ")");
        if (out == XRDVI_OK && gs != XRDVI_OK) out = gs;
    }
    return out;
}

xrdvi_status xrdvi_elbo_grad(xrdvi_ctx *c, const float *eps, double *elbo, float *grad, float *f_out,
                             double *ll_out, double *lpj_out) {
    NvtxRange nvtx("xrdvi_elbo_grad");
    if (!c) return fail(XRDVI_EINVAL, "null context");
    const Problem &P = c->P;
    const int S = c->W.S;
    // injected noise: [S*K*5] normals, followed with gates by [S*K] logistic gate noise
    const size_t SK5 = static_cast<size_t>(S) * P.K * (P.gates ? 6 : 5);
    cudaStream_t st = c->stream;
    if (eps) {
        if (!finite_all(eps, SK5)) return fail(XRDVI_EINVAL, "eps must be finite");
        if (!c->eps_in) XR_TRY(c->alloc(&c->eps_in, SK5));
        XR_CUDA(cudaMemcpyAsync(c->eps_in, eps, SK5 * 4, cudaMemcpyHostToDevice, st));
    }
    if (f_out && !c->f_out) XR_TRY(c->alloc(&c->f_out, static_cast<size_t>(S) * P.N));
    launch_sample(P, c->W, c->loc, c->raw, eps ? c->eps_in : nullptr, c->cfg.seed, 0u, c->step, 0u, nullptr,
                  c->ent, st);
    fwd_pass(c, f_out ? c->f_out : nullptr, st);
    bwd_pass(c, st);
    launch_grad(P, c->W, c->loc, c->raw, nullptr, nullptr, c->grad, false, adam_const(c->cfg), nullptr, nullptr,
                nullptr, nullptr, c->ent, c->elbo, nullptr, st);
    if (P.bgfit) launch_bg_grad(P, c->W, false, adam_const(c->cfg), nullptr, c->grad_beta, st);
    XR_TRY(check_launch("elbo_grad"));
    double e = 0.0;
    XR_CUDA(cudaMemcpyAsync(&e, c->elbo, 8, cudaMemcpyDeviceToHost, st));
    if (grad) XR_CUDA(cudaMemcpyAsync(grad, c->grad, P.K * 10 * 4, cudaMemcpyDeviceToHost, st));
    if (f_out) XR_CUDA(cudaMemcpyAsync(f_out, c->f_out, static_cast<size_t>(S) * P.N * 4, cudaMemcpyDeviceToHost, st));
    if (ll_out) XR_CUDA(cudaMemcpyAsync(ll_out, c->W.ll, S * 8, cudaMemcpyDeviceToHost, st));
    if (lpj_out) XR_CUDA(cudaMemcpyAsync(lpj_out, c->W.lpj, S * 8, cudaMemcpyDeviceToHost, st));
    XR_CUDA(cudaStreamSynchronize(st));
    if (elbo) *elbo = e;
    const xrdvi_status gs = check_gradients(c);
    if (!std::isfinite(e)) return fail(XRDVI_ENONFINITE, "ELBO is not finite");
    return gs;
}

xrdvi_status xrdvi_forward_dev(xrdvi_ctx *c, const float *d_loc, const float *d_raw, const float *d_eps,
                               double *d_elbo) {
    if (!c || !d_loc || !d_raw || !d_eps || !d_elbo) return fail(XRDVI_EINVAL, "null argument");
    launch_sample(c->P, c->W, d_loc, d_raw, d_eps, c->cfg.seed, 0u, nullptr, 0u, nullptr, c->ent, c->stream);
    fwd_pass(c, nullptr, c->stream);
    launch_grad(c->P, c->W, d_loc, d_raw, nullptr, nullptr, nullptr, false, adam_const(c->cfg), nullptr, nullptr,
                nullptr, nullptr, c->ent, d_elbo, nullptr, c->stream);
    return check_launch("forward_dev");
}

xrdvi_status xrdvi_backward_dev(xrdvi_ctx *c, const float *d_loc, const float *d_raw, const float *d_eps,
                                float *d_grad) {
    if (!c || !d_loc || !d_raw || !d_eps || !d_grad) return fail(XRDVI_EINVAL, "null argument");
    launch_sample(c->P, c->W, d_loc, d_raw, d_eps, c->cfg.seed, 0u, nullptr, 0u, nullptr, c->ent, c->stream);
    fwd_pass(c, nullptr, c->stream);
    bwd_pass(c, c->stream);
    launch_grad(c->P, c->W, d_loc, d_raw, nullptr, nullptr, d_grad, false, adam_const(c->cfg), nullptr, nullptr,
                nullptr, nullptr, c->ent, nullptr, nullptr, c->stream);
    return check_launch("backward_dev");
}

xrdvi_status xrdvi_posterior(xrdvi_ctx *c, int32_t S_post, uint64_t seed, int32_t top_m, double *pi,
                             uint64_t *combos, double *combo_logp, double *log_evidence, double *ess,
                             double *coverage_log) {
    NvtxRange nvtx("xrdvi_posterior");
    if (!c) return fail(XRDVI_EINVAL, "null context");
    if (S_post < 1 || S_post > kMaxS) return fail(XRDVI_EINVAL, "S_post must be in [1, 65536]");
    if (top_m < 1 || top_m > 4096) return fail(XRDVI_EINVAL, "top_m must be in [1, 4096]");
    const Problem &P = c->P;
    const int K = P.K, W = (K + 63) / 64;
    if (c->B.cap_S < S_post || c->B.cap_M < top_m) {
        XR_CUDA(cudaStreamSynchronize(c->stream));
        c->bytes -= c->Wp.bytes;
        c->free_post();
        const int capS = std::max(S_post, c->B.cap_S), capM = std::max(top_m, 64);
        std::vector<void *> *L = &c->post_allocs;
        const size_t before = c->bytes;
        XR_TRY(alloc_workspace(c, c->Wp, capS, false, L));
        XR_TRY(c->alloc(&c->B.logw, capS, L));
        XR_TRY(c->alloc(&c->B.bits, static_cast<size_t>(capS) * K, L));
        XR_TRY(c->alloc(&c->B.pi, K, L));
        XR_TRY(c->alloc(&c->B.scalars, 4, L));
        XR_TRY(c->alloc(&c->B.combos, static_cast<size_t>(capM) * W, L));
        XR_TRY(c->alloc(&c->B.combo_logp, capM, L));
        XR_TRY(c->alloc(&c->B.order, K, L));
        XR_TRY(c->alloc(&c->B.cost, K, L));
        XR_TRY(c->alloc(&c->B.heap_cost, 2 * capM + 2, L));
        XR_TRY(c->alloc(&c->B.heap_node, 2 * capM + 2, L));
        XR_TRY(c->alloc(&c->B.node_mask, static_cast<size_t>(2 * capM + 2) * W, L));
        XR_TRY(c->alloc(&c->B.node_last, 2 * capM + 2, L));
        c->B.cap_S = capS;
        c->B.cap_M = capM;
        c->Wp.bytes = c->bytes - before;
    }
    c->Wp.S = S_post;
    {
        const size_t per_chunk = static_cast<size_t>(S_post) * P.Npad;
        choose_chunks(P, c->host_off.data(), S_post, c->Wp, static_cast<int>(c->Wp.fpart_cap / per_chunk));
    }
    cudaStream_t st = c->stream;
    const bool naive = (c->cfg.flags & XRDVI_FLAG_NAIVE_SUM) != 0;
    launch_sample(P, c->Wp, c->loc, c->raw, nullptr, seed, 1u, nullptr, 0u, nullptr, nullptr, st);
    if (P.bgfit) launch_bg_curve(P, st);
    launch_forward(P, c->Wp, nullptr, naive, st);
    launch_posterior(P, c->Wp, c->B, top_m, st);
    XR_TRY(check_launch("posterior"));
    double sc[4] = {0, 0, 0, 0};
    XR_CUDA(cudaMemcpyAsync(sc, c->B.scalars, 32, cudaMemcpyDeviceToHost, st));
    if (pi) XR_CUDA(cudaMemcpyAsync(pi, c->B.pi, K * 8, cudaMemcpyDeviceToHost, st));
    if (combos) XR_CUDA(cudaMemcpyAsync(combos, c->B.combos, static_cast<size_t>(top_m) * W * 8, cudaMemcpyDeviceToHost, st));
    if (combo_logp) XR_CUDA(cudaMemcpyAsync(combo_logp, c->B.combo_logp, top_m * 8, cudaMemcpyDeviceToHost, st));
    XR_CUDA(cudaStreamSynchronize(st));
    if (log_evidence) *log_evidence = sc[0];
    if (ess) *ess = sc[1];
    if (coverage_log) *coverage_log = sc[2];
    return XRDVI_OK;
}

xrdvi_status xrdvi_profile_steps(xrdvi_ctx *c, int32_t steps, float *kernel_ms) {
    if (!c || !kernel_ms) return fail(XRDVI_EINVAL, "null argument");
    if (steps < 1) return fail(XRDVI_EINVAL, "steps must be >= 1");
    if (c->host_step + steps > INT32_MAX) return fail(XRDVI_EINVAL, "step counter would overflow");
    cudaEvent_t ev[6];
    for (auto &e : ev) XR_CUDA(cudaEventCreate(&e));
    double acc[5] = {0, 0, 0, 0, 0};
    cudaStream_t st = c->stream;
    xrdvi_status rc = XRDVI_OK;
    for (int i = 0; i < steps && rc == XRDVI_OK; ++i) {
        cudaEventRecord(ev[0], st);
        launch_sample(c->P, c->W, c->loc, c->raw, nullptr, c->cfg.seed, 0u, c->step, 0u, c->iter, c->ent, st);
        cudaEventRecord(ev[1], st);
        fwd_pass(c, nullptr, st);
        cudaEventRecord(ev[2], st);
        bwd_pass(c, st);
        cudaEventRecord(ev[3], st);
        launch_grad(c->P, c->W, c->loc, c->raw, c->loc, c->raw, nullptr, true, adam_const(c->cfg), c->m, c->v,
                    c->iter, nullptr, c->ent, nullptr, nullptr, st);
        if (c->P.bgfit) launch_bg_grad(c->P, c->W, true, adam_const(c->cfg), c->iter, nullptr, st);
        cudaEventRecord(ev[4], st);
        launch_grad(c->P, c->W, c->loc, c->raw, nullptr, nullptr, nullptr, false, adam_const(c->cfg), nullptr,
                    nullptr, c->iter, c->step, c->ent, c->elbo, c->trace, st);
        cudaEventRecord(ev[5], st);
        if (cudaEventSynchronize(ev[5]) != cudaSuccess) {
            rc = fail(XRDVI_ECUDA, std::string("profile_steps: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        for (int k = 0; k < 5; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            acc[k] += ms;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc != XRDVI_OK) return rc;
    c->host_step += steps;
    for (int k = 0; k < 5; ++k) kernel_ms[k] = static_cast<float>(acc[k] / steps);
    return XRDVI_OK;
}

xrdvi_status xrdvi_profile_kernels(xrdvi_ctx *c, int32_t steps, float *kernel_ms, int64_t *work) {
    if (!c || !kernel_ms) return fail(XRDVI_EINVAL, "null argument");
    if (steps < 1) return fail(XRDVI_EINVAL, "steps must be >= 1");
    if (c->host_step + steps > INT32_MAX) return fail(XRDVI_EINVAL, "step counter would overflow");
    constexpr int nk = XRDVI_PROFILE_KERNELS;
    // one set of events per step, read after the last step: the steps run back
    // to back (no host round trip before a step's first kernel)
    std::vector<cudaEvent_t> evs(static_cast<size_t>(steps) * (nk + 1));
    for (auto &e : evs) XR_CUDA(cudaEventCreate(&e));
    double acc[nk] = {};
    cudaStream_t st = c->stream;
    const Problem &P = c->P;
    Workspace &W = c->W;
    const bool naive = (c->cfg.flags & XRDVI_FLAG_NAIVE_SUM) != 0;
    xrdvi_status rc = XRDVI_OK;
    for (int i = 0; i < steps; ++i) {
        cudaEvent_t *ev = evs.data() + static_cast<size_t>(i) * (nk + 1);
        cudaEventRecord(ev[0], st);
        launch_sample(P, W, c->loc, c->raw, nullptr, c->cfg.seed, 0u, c->step, 0u, c->iter, c->ent, st);
        cudaEventRecord(ev[1], st);
        if (P.bgfit) launch_bg_curve(P, st);
        if (W.shared) {   // one contraction: its time counts as the direct profile
            cudaEventRecord(ev[2], st);
            launch_shared_forward(P, W, nullptr, st);
            cudaEventRecord(ev[3], st);
            cudaEventRecord(ev[4], st);
        } else {
            launch_forward(P, W, nullptr, naive, st, &ev[2]);
        }
        cudaEventRecord(ev[5], st);
        if (W.shared) {
            launch_shared_backward(P, W, st);
            cudaEventRecord(ev[6], st);
            cudaEventRecord(ev[7], st);
        } else {
            launch_backward(P, W, st, &ev[6]);
        }
        cudaEventRecord(ev[8], st);
        launch_grad(P, W, c->loc, c->raw, c->loc, c->raw, nullptr, true, adam_const(c->cfg), c->m, c->v, c->iter,
                    nullptr, c->ent, nullptr, nullptr, st);
        if (P.bgfit) launch_bg_grad(P, W, true, adam_const(c->cfg), c->iter, nullptr, st);
        cudaEventRecord(ev[9], st);
        launch_grad(P, W, c->loc, c->raw, nullptr, nullptr, nullptr, false, adam_const(c->cfg), nullptr, nullptr,
                    c->iter, c->step, c->ent, c->elbo, c->trace, st);
        cudaEventRecord(ev[10], st);
    }
    if (cudaEventSynchronize(evs.back()) != cudaSuccess) {
        rc = fail(XRDVI_ECUDA, std::string("profile_kernels: ") + cudaGetErrorString(cudaGetLastError()));
    } else {
        for (int i = 0; i < steps; ++i) {
            const cudaEvent_t *ev = evs.data() + static_cast<size_t>(i) * (nk + 1);
            for (int k = 0; k < nk; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
                acc[k] += ms;
            }
        }
    }
    for (auto &e : evs) cudaEventDestroy(e);
    if (rc != XRDVI_OK) return rc;
    c->host_step += steps;
    for (int k = 0; k < nk; ++k) kernel_ms[k] = static_cast<float>(acc[k] / steps);
    if (work) {   // evaluation counts of the last step, from its peak ranges
        for (int j = 0; j < XRDVI_PROFILE_WORK; ++j) work[j] = 0;
        if (!W.shared) {
            const size_t nr = static_cast<size_t>(W.S) * P.K * P.T;
            std::vector<ushort4> rg(nr);
            std::vector<ushort2> fr(P.far ? nr : 0);
            const size_t ng = static_cast<size_t>(W.S) * P.K * P.Tg;
            std::vector<ushort2> sr(ng);
            XR_CUDA(cudaMemcpyAsync(rg.data(), W.ranges, nr * sizeof(ushort4), cudaMemcpyDeviceToHost, st));
            if (P.far) XR_CUDA(cudaMemcpyAsync(fr.data(), W.franges, nr * sizeof(ushort2), cudaMemcpyDeviceToHost, st));
            if (ng) XR_CUDA(cudaMemcpyAsync(sr.data(), W.sranges, ng * sizeof(ushort2), cudaMemcpyDeviceToHost, st));
            // the backward's Gaussian votes: per-(sample, phase) shift and reach,
            // peak positions and the grid
            std::vector<PhaseConst> cs(static_cast<size_t>(W.S) * P.K);
            std::vector<float> xs(P.N), ps(P.Mtot);
            XR_CUDA(cudaMemcpyAsync(cs.data(), W.cst, cs.size() * sizeof(PhaseConst), cudaMemcpyDeviceToHost, st));
            XR_CUDA(cudaMemcpyAsync(xs.data(), P.x, xs.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
            XR_CUDA(cudaMemcpyAsync(ps.data(), P.pos, ps.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
            XR_CUDA(cudaStreamSynchronize(st));
            constexpr int kBlk = 64;   // points of a warp's pair block
            for (size_t id = 0; id < nr; ++id) {
                const ushort4 r = rg[id];
                if (r.x == 0xffffu) continue;   // phase absent from this sample's sub-model
                const int k = static_cast<int>((id / P.T) % P.K);
                const int64_t me = c->host_off[k + 1] - c->host_off[k];
                const int64_t m1 = r.x, m2 = r.y, nb = r.z, ne = r.w;
                {   // pair blocks within a peak's Gaussian reach (p + mu - rl, p + mu + rr)
                    const PhaseConst &pc = cs[id / P.T];
                    const int i0 = static_cast<int>(id % P.T) * kTile;
                    const int mb = c->host_off[k];
                    for (int64_t m = std::min(nb, m1); m < std::max(ne, m2); ++m) {
                        const double cen = static_cast<double>(ps[mb + m]) + pc.mu;
                        int64_t blocks = 0;
                        for (int q = 0; q < kTile / kBlk; ++q) {
                            const double xa = xs[std::min(i0 + q * kBlk, P.N - 1)];
                            const double xb = xs[std::min(i0 + q * kBlk + kBlk - 1, P.N - 1)];
                            blocks += (xb > cen - pc.rl && xa < cen + pc.rr) ? 1 : 0;
                        }
                        work[(m >= m1 && m < m2) ? 4 : 5] += blocks * kBlk;
                    }
                }
                const int64_t fb = P.far ? fr[id].x : 0, fe = P.far ? fr[id].y : me;
                work[0] += ((m1 - fb) + (fe - m2)) * kTile;
                work[1] += (m2 - m1) * kTile;
                work[2] += ((m1 - std::min(nb, m1)) + (std::max(ne, m2) - m2)) * kTile;
                // far (peak, node) pairs: level 1 at the tile's nodes, level 2 once per super-tile
                const int tile = static_cast<int>(id % P.T);
                const size_t gid = (id / P.T) * P.Tg + tile / kSuperTiles;
                const int64_t sfb = ng ? sr[gid].x : 0, sfe = ng ? sr[gid].y : me;
                work[3] += ((fb - sfb) + (sfe - fe)) * kFarNodes;
                if (ng && tile % kSuperTiles == 0) work[3] += (sfb + (me - sfe)) * kFarNodes;
            }
        }
    }
    return XRDVI_OK;
}

xrdvi_status xrdvi_get_params(xrdvi_ctx *c, float *loc, float *raw) {
    if (!c) return fail(XRDVI_EINVAL, "null context");
    if (loc) XR_CUDA(cudaMemcpyAsync(loc, c->loc, c->P.K * 20, cudaMemcpyDeviceToHost, c->stream));
    if (raw) XR_CUDA(cudaMemcpyAsync(raw, c->raw, c->P.K * 20, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    return XRDVI_OK;
}

xrdvi_status xrdvi_set_params(xrdvi_ctx *c, const float *loc, const float *raw) {
    if (!c || !loc || !raw) return fail(XRDVI_EINVAL, "null argument");
    if (!finite_all(loc, c->P.K * 5) || !finite_all(raw, c->P.K * 5)) return fail(XRDVI_EINVAL, "params must be finite");
    XR_CUDA(cudaMemcpyAsync(c->loc, loc, c->P.K * 20, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaMemcpyAsync(c->raw, raw, c->P.K * 20, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    return XRDVI_OK;
}

namespace {
struct StateHeader {
    uint32_t magic, version;
    int32_t K, pad;
    int64_t step;
    uint64_t seed;
};
}  // namespace

xrdvi_status xrdvi_get_state(xrdvi_ctx *c, void *buf, size_t *len) {
    if (!c || !len) return fail(XRDVI_EINVAL, "null argument");
    const int K = c->P.K;
    // fitted background: beta and its Adam moments; gates: logits and their moments
    const int extra = (c->P.bgfit ? 9 : 0) + (c->P.gates ? 3 * K : 0);
    const size_t need = sizeof(StateHeader) + static_cast<size_t>(K) * (5 + 5 + 10 + 10) * 4 + extra * 4;
    if (!buf) {
        *len = need;
        return XRDVI_OK;
    }
    if (*len < need) return fail(XRDVI_EINVAL, "state buffer too small");
    StateHeader h{kStateMagic, 1u, K, extra, c->host_step, c->cfg.seed};
    char *p = static_cast<char *>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    XR_CUDA(cudaMemcpyAsync(p, c->loc, K * 20, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaMemcpyAsync(p + K * 20, c->raw, K * 20, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaMemcpyAsync(p + K * 40, c->m, K * 40, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaMemcpyAsync(p + K * 80, c->v, K * 40, cudaMemcpyDeviceToHost, c->stream));
    char *q = p + K * 120;
    if (c->P.bgfit) {
        XR_CUDA(cudaMemcpyAsync(q, c->P.beta, 12, cudaMemcpyDeviceToHost, c->stream));
        XR_CUDA(cudaMemcpyAsync(q + 12, c->P.m_beta, 12, cudaMemcpyDeviceToHost, c->stream));
        XR_CUDA(cudaMemcpyAsync(q + 24, c->P.v_beta, 12, cudaMemcpyDeviceToHost, c->stream));
        q += 36;
    }
    if (c->P.gates) {
        XR_CUDA(cudaMemcpyAsync(q, c->P.gate_a, K * 4, cudaMemcpyDeviceToHost, c->stream));
        XR_CUDA(cudaMemcpyAsync(q + K * 4, c->P.m_gate, K * 4, cudaMemcpyDeviceToHost, c->stream));
        XR_CUDA(cudaMemcpyAsync(q + K * 8, c->P.v_gate, K * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    XR_CUDA(cudaStreamSynchronize(c->stream));
    *len = need;
    return XRDVI_OK;
}

xrdvi_status xrdvi_set_state(xrdvi_ctx *c, const void *buf, size_t len) {
    if (!c || !buf) return fail(XRDVI_EINVAL, "null argument");
    const int K = c->P.K;
    const int extra = (c->P.bgfit ? 9 : 0) + (c->P.gates ? 3 * K : 0);
    const size_t need = sizeof(StateHeader) + static_cast<size_t>(K) * 120 + extra * 4;
    if (len < need) return fail(XRDVI_EINVAL, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1u || h.K != K || h.pad != extra)
        return fail(XRDVI_EINVAL, "state does not match this problem");
    if (h.step < 0 || h.step > INT32_MAX) return fail(XRDVI_EINVAL, "bad step counter");
    const char *p = static_cast<const char *>(buf) + sizeof(h);
    const int step = static_cast<int>(h.step);
    XR_CUDA(cudaMemcpyAsync(c->loc, p, K * 20, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaMemcpyAsync(c->raw, p + K * 20, K * 20, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaMemcpyAsync(c->m, p + K * 40, K * 40, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaMemcpyAsync(c->v, p + K * 80, K * 40, cudaMemcpyHostToDevice, c->stream));
    const char *q = p + K * 120;
    if (c->P.bgfit) {
        XR_CUDA(cudaMemcpyAsync(c->P.beta, q, 12, cudaMemcpyHostToDevice, c->stream));
        XR_CUDA(cudaMemcpyAsync(c->P.m_beta, q + 12, 12, cudaMemcpyHostToDevice, c->stream));
        XR_CUDA(cudaMemcpyAsync(c->P.v_beta, q + 24, 12, cudaMemcpyHostToDevice, c->stream));
        q += 36;
    }
    if (c->P.gates) {
        XR_CUDA(cudaMemcpyAsync(c->P.gate_a, q, K * 4, cudaMemcpyHostToDevice, c->stream));
        XR_CUDA(cudaMemcpyAsync(c->P.m_gate, q + K * 4, K * 4, cudaMemcpyHostToDevice, c->stream));
        XR_CUDA(cudaMemcpyAsync(c->P.v_gate, q + K * 8, K * 4, cudaMemcpyHostToDevice, c->stream));
    }
    XR_CUDA(cudaMemcpyAsync(c->step, &step, 4, cudaMemcpyHostToDevice, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    c->host_step = h.step;
    c->cfg.seed = h.seed;
    c->drop_graphs();  // the seed is a kernel argument of the captured step
    return XRDVI_OK;
}

xrdvi_status xrdvi_get_gates(xrdvi_ctx *c, float *logits, float *grad) {
    if (!c) return fail(XRDVI_EINVAL, "null context");
    if (!c->P.gates) return fail(XRDVI_EINVAL, "the context has no gates");
    const size_t n = static_cast<size_t>(c->P.K) * 4;
    if (logits) XR_CUDA(cudaMemcpyAsync(logits, c->P.gate_a, n, cudaMemcpyDeviceToHost, c->stream));
    if (grad) XR_CUDA(cudaMemcpyAsync(grad, c->P.grad_gate, n, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    return XRDVI_OK;
}

xrdvi_status xrdvi_get_background(xrdvi_ctx *c, float *beta, float *bg_curve, float *grad_beta) {
    if (!c) return fail(XRDVI_EINVAL, "null context");
    if (!c->P.bgfit) return fail(XRDVI_EINVAL, "the context does not fit the background");
    if (bg_curve) launch_bg_curve(c->P, c->stream);
    if (beta) XR_CUDA(cudaMemcpyAsync(beta, c->P.beta, 12, cudaMemcpyDeviceToHost, c->stream));
    if (bg_curve) XR_CUDA(cudaMemcpyAsync(bg_curve, c->P.Bb, static_cast<size_t>(c->P.N) * 4, cudaMemcpyDeviceToHost,
                                          c->stream));
    if (grad_beta) XR_CUDA(cudaMemcpyAsync(grad_beta, c->grad_beta, 12, cudaMemcpyDeviceToHost, c->stream));
    XR_CUDA(cudaStreamSynchronize(c->stream));
    return XRDVI_OK;
}

xrdvi_status xrdvi_philox4x32_10(int32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    if (n < 0 || n > (1 << 20)) return fail(XRDVI_EINVAL, "n must be in [0, 2^20]");
    if (n == 0) return XRDVI_OK;
    if (!ctr || !key || !out) return fail(XRDVI_EINVAL, "null argument");
    cudaStream_t s = nullptr;
    XR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    uint32_t *d = nullptr;
    const size_t nw = static_cast<size_t>(n) * 10;   // counters 4n, keys 2n, output 4n
    cudaError_t e = cudaMallocAsync(&d, nw * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, ctr, 16 * static_cast<size_t>(n), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 4 * n, key, 8 * static_cast<size_t>(n), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        launch_philox_words(n, d, d + 4 * n, d + 6 * n, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 6 * n, 16 * static_cast<size_t>(n), cudaMemcpyDeviceToHost, s);
    if (d) cudaFreeAsync(d, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("philox4x32_10: ") + cudaGetErrorString(e));
    return XRDVI_OK;
}

xrdvi_status xrdvi_debug_word(int32_t *word, int32_t reset) {
    if (!word) return fail(XRDVI_EINVAL, "null argument");
    if (!debug_build()) return fail(XRDVI_EINVAL, "not a bounds-check build (XRDVI_DEBUG)");
    *word = debug_word(reset != 0);
    return XRDVI_OK;
}

xrdvi_status xrdvi_debug_selftest(void) {
    if (!debug_build()) return fail(XRDVI_EINVAL, "not a bounds-check build (XRDVI_DEBUG)");
    float *d = nullptr;
    XR_CUDA(cudaMalloc(&d, sizeof(float)));
    const cudaError_t e = debug_selftest(d);
    cudaFree(d);
    if (e != cudaSuccess) return fail(XRDVI_ECUDA, std::string("debug self-test: ") + cudaGetErrorString(e));
    return XRDVI_OK;
}

xrdvi_status xrdvi_get_info(xrdvi_ctx *c, xrdvi_info *info) {
    if (!c || !info) return fail(XRDVI_EINVAL, "null argument");
    info->K = c->P.K;
    info->N = c->P.N;
    info->S = c->W.S;
    info->M_total = c->P.Mtot;
    info->step = c->host_step;
    info->eta = c->eta;
    info->lambda_ = c->P.prior.lambda;
    info->data_const = c->P.csum;
    info->device_bytes = c->bytes;
    info->point_tiles = c->P.T;
    return XRDVI_OK;
}

}  // extern "C"
