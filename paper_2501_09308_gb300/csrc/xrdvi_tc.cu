// Tensor-core kernels of the shared-shape variant: when every Monte-Carlo
// sample of a step shares the shape draw (mu, w, r, alpha) and only the
// intensities h differ, the profile of sample s is
//   f_s(x_i) = B(x_i) + sum_k h_sk C_k(x_i),
// a contraction over phases (the signal equation of Appendix A.2 with the
// phase profiles C_k = sum_m I_m V(x; p_m + mu_k, ...) factored out), and the
// backward's per-(sample, phase) sums are sum_i g_si D_jk(x_i) with
// sample-independent derivative profiles D_jk.  Both contractions run as
// GEMMs on the 5th-generation tensor cores (tcgen05, accumulators in TMEM)
// with a 3xTF32 split for FP32-level accuracy: a = a_hi + a_lo with a_hi the
// value truncated to TF32 and a_lo = a - a_hi, and
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/xrdvi.h"
#include "xrdvi_internal.h"

namespace xrdvi {
namespace {

constexpr int kGM = 128;        // tile rows (MMA M)
constexpr int kGKB = 16;        // reduction elements per stage (2 MMA steps of 8)
constexpr int kGThreads = 128;  // 4 warps: warp w reads TMEM lanes 32w..32w+31
constexpr int kStages = 3;      // stages in flight
constexpr uint32_t kSBO = 512;  // bytes between 8-row groups (4 cores of 128 B along K)
constexpr uint32_t kTileA = kGM * kGKB * 4;   // bytes of one A operand tile (8 KB)
constexpr uint32_t kWaitLimit = 1u << 22;     // mbarrier polls before giving up

// Per tile width kGN (MMA N, TMEM columns): B operand tile and stage bytes.
template <int kGN>
struct TileCfg {
    static constexpr uint32_t kTileB = kGN * kGKB * 4;
    static constexpr uint32_t kStage = 2 * kTileA + 2 * kTileB;   // hi + lo of A and B
    static constexpr uint32_t kSmem = kStages * kStage + 1024;
    // instruction descriptor of kind::tf32: D = F32, A = B = TF32, both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                       (static_cast<uint32_t>(kGN >> 3) << 17) |
                                       (static_cast<uint32_t>(kGM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row r, reduction index e < kGKB) in a K-major tile
// without swizzle built from core matrices of 8 rows x 16 bytes: the cores
// along K of one 8-row group are 128 bytes apart (leading byte offset), the
// 8-row groups kSBO bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t core_off(int r, int e) {
    return static_cast<uint32_t>((r >> 3) * kSBO + (e >> 2) * 128 + (r & 7) * 16 + (e & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
           (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (L2 only); src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kN>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kN) : "memory"); }

struct GemmArgs {
    int M, N, K;             // out[M x N] = A[M x K] . B[N x K]^T (row-major, K contiguous)
    const float *Ahi, *Alo, *Bhi, *Blo;   // TF32 hi and lo parts (tf32_split)
    int lda, ldb;
    float *out;              // split s writes out + s * split_stride (row stride ldo)
    int ldo;
    size_t split_stride;
    int kb_per_split, nkb;   // stages of kGKB per split, total
    int *err;                // set to 1 if an mbarrier wait gives up
};

// Issues the copies of reduction block kb (kGKB elements) of A (kGM rows) and
// B (kGN rows), hi and lo, into stage st in the core-matrix layout: one core
// row (4 elements, 16 bytes) per copy; rows beyond M / N and elements beyond
// K are zero-filled.
template <int kGN>
__device__ __forceinline__ void issue_stage(const GemmArgs &a, uint32_t st, int m0, int n0, int kb) {
    constexpr uint32_t kTileB = TileCfg<kGN>::kTileB;
    const int k0 = kb * kGKB;
    for (int idx = threadIdx.x; idx < (kGM + kGN) * (kGKB / 4); idx += kGThreads) {
        const bool isA = idx < kGM * (kGKB / 4);
        const int j = isA ? idx : idx - kGM * (kGKB / 4);
        const int r = j / (kGKB / 4), q = j % (kGKB / 4);
        const int row = (isA ? m0 : n0) + r, k = k0 + 4 * q;
        const bool ok = row < (isA ? a.M : a.N) && k < a.K;
        const size_t off = ok ? static_cast<size_t>(row) * (isA ? a.lda : a.ldb) + k : 0;
        const float *hi = (isA ? a.Ahi : a.Bhi) + off, *lo = (isA ? a.Alo : a.Blo) + off;
        const uint32_t o = core_off(r, 4 * q);
        const uint32_t base = isA ? st : st + 2 * kTileA;
        const uint32_t tile = isA ? kTileA : kTileB;
        cp_async16(base + o, hi, ok ? 16u : 0u);
        cp_async16(base + tile + o, lo, ok ? 16u : 0u);
    }
}

// One output tile of kGM x kGN per CTA over one split of the reduction.
// kStages stages of copies in flight; one thread issues 2 k-steps x 3 MMAs
// per stage (3xTF32) and commits them to the stage's mbarrier, which is
// awaited before the stage is refilled.
template <int kGN>
__global__ void __launch_bounds__(kGThreads) k_gemm_nt_tf32x3(GemmArgs a) {
    using Cfg = TileCfg<kGN>;
    constexpr uint32_t kTileB = Cfg::kTileB, kStage = Cfg::kStage;
    extern __shared__ uint8_t g_smem_raw[];
    __shared__ __align__(8) uint64_t s_mbar[kStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    uint8_t *smem = g_smem_raw + ((1024u - (smem_addr(g_smem_raw) & 1023u)) & 1023u);   // 1 KB aligned
    const uint32_t sbase = smem_addr(smem);
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN, split = blockIdx.z;
    const int kb0 = split * a.kb_per_split;
    const int kb1 = min(a.nkb, kb0 + a.kb_per_split);
    const int nk = kb1 - kb0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(smem_addr(&s_mbar[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(static_cast<uint32_t>(kGN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // prologue: the first kStages - 1 blocks in flight
#pragma unroll
    for (int i = 0; i < kStages - 1; ++i) {
        if (i < nk) issue_stage<kGN>(a, sbase + i * kStage, m0, n0, kb0 + i);
        cp_async_commit();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    for (int i = 0; i < nk; ++i) {
        const int st = i % kStages;
        cp_async_wait<kStages - 2>();   // this thread's copies of block i have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA operand reads
        __syncthreads();                // ... and every thread's
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t base = sbase + st * kStage;
#pragma unroll
            for (int t = 0; t < kGKB / 8; ++t) {
                const uint32_t off = static_cast<uint32_t>(t) * 256u;   // two 128-byte cores per k-step
                const uint64_t ahi = smem_desc(base + off, 128, kSBO), alo = smem_desc(base + kTileA + off, 128, kSBO);
                const uint64_t bhi = smem_desc(base + 2 * kTileA + off, 128, kSBO);
                const uint64_t blo = smem_desc(base + 2 * kTileA + kTileB + off, 128, kSBO);
                mma_tf32(tmem, alo, bhi, Cfg::kIdesc, (i > 0 || t > 0) ? 1u : 0u);
                mma_tf32(tmem, ahi, blo, Cfg::kIdesc, 1u);
                mma_tf32(tmem, ahi, bhi, Cfg::kIdesc, 1u);
            }
            mma_commit(smem_addr(&s_mbar[st]));
            // the stage refilled next held block i - 1: its MMAs must be done
            const int prev = i - 1;
            if (prev >= 0 && prev + kStages < nk &&
                !mbar_wait(smem_addr(&s_mbar[prev % kStages]), static_cast<uint32_t>((prev / kStages) & 1)))
                s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;   // uniform: read after the barrier
        const int nxt = i + kStages - 1;
        if (nxt < nk) issue_stage<kGN>(a, sbase + (nxt % kStages) * kStage, m0, n0, kb0 + nxt);
        cp_async_commit();
    }
    cp_async_wait<0>();
    // wait for the last block's MMAs (a commit tracks all earlier MMAs too);
    // one thread waits, the barrier publishes the outcome to all
    __syncthreads();
    if (threadIdx.x == 0 && !s_abort && nk > 0 &&
        !mbar_wait(smem_addr(&s_mbar[(nk - 1) % kStages]), static_cast<uint32_t>(((nk - 1) / kStages) & 1)))
        s_abort = 1;
    __syncthreads();
    const bool ok = !s_abort;
    if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
    tc_fence_after();
    if (ok) {
        // epilogue: warp w owns rows 32w..32w+31 of the tile (TMEM lanes)
        const int row = m0 + 32 * warp + lane;
        float *dst = a.out + static_cast<size_t>(split) * a.split_stride + static_cast<size_t>(row) * a.ldo;
#pragma unroll
        for (int c0 = 0; c0 < kGN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < a.M) {
                float f[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) f[j] = nk > 0 ? __uint_as_float(v[j]) : 0.f;
                const int n = n0 + c0;
                if (n + 16 <= a.N && (reinterpret_cast<uintptr_t>(dst + n) & 15u) == 0) {   // 16-byte stores
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(dst + n + j) = make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n + j < a.N) dst[n + j] = f[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(static_cast<uint32_t>(kGN)));
}

// out[m][n] = sum over the splits of part[s][m][n], in split order.
__global__ void k_splitk_reduce(const float *part, int splits, size_t split_stride, int M, int N, int ldp,
                                float *out, int ldo) {
    const size_t total = static_cast<size_t>(M) * N;
    for (size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx / N), n = static_cast<int>(idx - static_cast<size_t>(m) * N);
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += part[s * split_stride + static_cast<size_t>(m) * ldp + n];
        out[static_cast<size_t>(m) * ldo + n] = acc;
    }
}

// Element-wise 3xTF32 split of n floats: hi = a with the low 13 mantissa bits
// cleared, lo = a - hi (exact).
__global__ void k_tf32_split(const float *a, size_t n, float *hi, float *lo) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float v = a[i], h = tf32_hi(v);
        hi[i] = h;
        lo[i] = v - h;
    }
}

// Phase profiles and derivative profiles of the shared shapes (sample 0's
// draw), one thread per (phase k = blockIdx.y, point i).  With d = x - p - mu,
// s = 2 / w_side, t = s d, u = t^2, G = 2^-u, L = 1 / (1 + u), the ten sums
// over the phase's peaks, in the order of the backward's gradient sums, are
//   I G, I L, I G t, I L^2 t, I G |t|, I L^2 |t|, I G t^2, I L^2 t^2,
//   I G t|t|, I L^2 t|t|,
// and C_k = r sum I L + (1 - r) sum I G.  Beyond the Gaussian's reach
// (u >= 128) its terms are zero in FP32 and are skipped.
struct ShapeArgs {
    int N, Npad, K, Kpad;
    const float *x, *pos, *inten;
    const int *off;
    const float *csec;       // [N] cos(x/2) of the angle-dependent width (null: constant width)
    const PhaseConst *cst;   // sample 0's row [K]
    const float *theta;      // sample 0's row [K*5]
    float *D, *D_lo;         // [K*10*Npad] TF32 hi / lo parts
    float *Ct, *Ct_lo;       // [Npad*Kpad] TF32 hi / lo parts
};

constexpr int kShapeChunk = 512;   // peaks staged in shared memory at a time

__global__ void __launch_bounds__(256) k_shapes(ShapeArgs a) {
    __shared__ float2 sp[kShapeChunk];   // (p, I) of the phase's peaks
    const int k = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;   // blockDim.x * gridDim.x == Npad
    const PhaseConst c = a.cst[k];
    const float r = a.theta[k * 5 + 3];
    float acc[kGradSums];
#pragma unroll
    for (int j = 0; j < kGradSums; ++j) acc[j] = 0.f;
    const bool live = i < a.N;
    const float x = live ? a.x[i] : 0.f;
    const float cx = (a.csec && live) ? a.csec[i] : 1.f;   // t = s cos(x/2) d; mu sums take cos(x/2) once more
    for (int m0 = a.off[k]; m0 < a.off[k + 1]; m0 += kShapeChunk) {
        const int mn = min(kShapeChunk, a.off[k + 1] - m0);
        __syncthreads();
        for (int j = threadIdx.x; j < mn; j += blockDim.x) sp[j] = make_float2(a.pos[m0 + j], a.inten[m0 + j]);
        __syncthreads();
        if (!live) continue;
        for (int m = 0; m < mn; ++m) {
            const float2 pk = sp[m];
            const float d = (x - pk.x) - c.mu;
            const float t = (d >= 0.f ? c.sr : c.sl) * d * cx;
            const float at = fabsf(t), u = t * t;
            float L;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(L) : "f"(1.f + u));
            const float I = pk.y;
            const float IL = I * L, IL2 = IL * L;
            acc[1] += IL;
            acc[3] = fmaf(IL2, t, acc[3]);
            acc[5] = fmaf(IL2, at, acc[5]);
            acc[7] = fmaf(IL2, u, acc[7]);
            acc[9] = fmaf(IL2 * t, at, acc[9]);
            if (u < kGaussU) {
                float G;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G) : "f"(-u));
                const float IG = I * G;
                acc[0] += IG;
                acc[2] = fmaf(IG, t, acc[2]);
                acc[4] = fmaf(IG, at, acc[4]);
                acc[6] = fmaf(IG, u, acc[6]);
                acc[8] = fmaf(IG * t, at, acc[8]);
            }
        }
    }
    if (a.csec && live) {
        const float cx = a.csec[i];
        acc[2] *= cx; acc[3] *= cx; acc[4] *= cx; acc[5] *= cx;
    }
#pragma unroll
    for (int j = 0; j < kGradSums; ++j) {
        const size_t o = (static_cast<size_t>(k) * kGradSums + j) * a.Npad + i;
        const float h = tf32_hi(acc[j]);
        a.D[o] = h;
        a.D_lo[o] = acc[j] - h;
    }
    const float cv = fmaf(r, acc[1], (1.f - r) * acc[0]), ch = tf32_hi(cv);
    a.Ct[static_cast<size_t>(i) * a.Kpad + k] = ch;
    a.Ct_lo[static_cast<size_t>(i) * a.Kpad + k] = cv - ch;
}

}  // namespace

// Operands are stored split (TF32 hi part, then lo part, each of the sizes
// given in Workspace) by their producers: H by k_sample, Ct and D by
// k_shapes, g by k_lik.
void launch_shared_forward(const Problem &P, Workspace &W, float *f_out, cudaStream_t st) {
    ShapeArgs s;
    s.N = P.N; s.Npad = P.Npad; s.K = P.K; s.Kpad = W.Kpad;
    s.x = P.x; s.pos = P.pos; s.inten = P.inten; s.off = P.off;
    s.cst = W.cst; s.theta = W.theta; s.D = W.D; s.Ct = W.Ct; s.csec = P.csec;
    s.D_lo = W.D + static_cast<size_t>(P.K) * kGradSums * P.Npad;
    s.Ct_lo = W.Ct + static_cast<size_t>(P.Npad) * W.Kpad;
    k_shapes<<<dim3(P.T, P.K), 256, 0, st>>>(s);
    // f_s - B = sum_k h_sk C_k: [S x N] = H [S x Kpad] . Ct [N x Kpad]^T, into the first chunk slot
    const size_t nh = static_cast<size_t>(W.S) * W.Kpad;
    launch_gemm_nt_tf32x3(W.S, P.N, W.Kpad, W.H, W.H + nh, W.Kpad, W.Ct, s.Ct_lo, W.Kpad, W.fpart, P.Npad, 1,
                          nullptr, W.gemm_err, st);
    launch_lik(P, W, f_out, 1, st);
}

void launch_shared_backward(const Problem &P, Workspace &W, cudaStream_t st) {
    // per (s, k) sums: [S x 10K] = g [S x Npad] . D [10K x Npad]^T  (g = 0 on padding)
    const int nk = P.K * kGradSums;
    const size_t ng = static_cast<size_t>(W.S) * P.Npad, nd = static_cast<size_t>(nk) * P.Npad;
    launch_gemm_nt_tf32x3(W.S, nk, P.Npad, W.ghl, W.ghl + ng, P.Npad, W.D, W.D + nd, P.Npad, W.gpart, nk,
                          W.gemm_splits, W.gemm_work, W.gemm_err, st);
}

// Tile width: 128 columns where N is wide (fewer re-reads of A), 64 for
// narrow outputs.
static int tile_n(int N) { return N > 64 ? 128 : 64; }

size_t gemm_smem_bytes() { return TileCfg<128>::kSmem; }

int gemm_splits(int M, int N, int K, int sm_count) {
    const int tiles = ((M + kGM - 1) / kGM) * ((N + tile_n(N) - 1) / tile_n(N));
    const int nkb = (K + kGKB - 1) / kGKB;
    int s = (sm_count + tiles - 1) / tiles;   // about one CTA per SM
    s = s < nkb ? s : nkb;
    return s < 1 ? 1 : s;
}

size_t gemm_workspace_floats(int M, int N, int splits) {
    return splits > 1 ? static_cast<size_t>(splits) * M * N : 0;
}

cudaError_t gemm_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_nt_tf32x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(TileCfg<64>::kSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_nt_tf32x3<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(TileCfg<128>::kSmem));
    return e;
}

void launch_tf32_split(const float *a, size_t n, float *hi, float *lo, cudaStream_t st) {
    int blocks = static_cast<int>((n + 255) / 256);
    blocks = blocks < 4096 ? blocks : 4096;
    if (blocks > 0) k_tf32_split<<<blocks, 256, 0, st>>>(a, n, hi, lo);
}

void launch_gemm_nt_tf32x3(int M, int N, int K, const float *Ahi, const float *Alo, int lda, const float *Bhi,
                           const float *Blo, int ldb, float *out, int ldo, int splits, float *work, int *err,
                           cudaStream_t st) {
    GemmArgs a;
    a.M = M; a.N = N; a.K = K; a.Ahi = Ahi; a.Alo = Alo; a.Bhi = Bhi; a.Blo = Blo; a.lda = lda; a.ldb = ldb;
    a.err = err;
    a.nkb = (K + kGKB - 1) / kGKB;
    if (splits < 1) splits = 1;
    if (splits > a.nkb) splits = a.nkb > 0 ? a.nkb : 1;
    a.kb_per_split = (a.nkb + splits - 1) / splits;
    splits = a.nkb > 0 ? (a.nkb + a.kb_per_split - 1) / a.kb_per_split : 1;
    if (splits == 1) {
        a.out = out; a.ldo = ldo; a.split_stride = 0;
    } else {
        a.out = work; a.ldo = N; a.split_stride = static_cast<size_t>(M) * N;
    }
    const int tn = tile_n(N);
    dim3 grid((M + kGM - 1) / kGM, (N + tn - 1) / tn, splits);
    if (tn == 128)
        k_gemm_nt_tf32x3<128><<<grid, kGThreads, TileCfg<128>::kSmem, st>>>(a);
    else
        k_gemm_nt_tf32x3<64><<<grid, kGThreads, TileCfg<64>::kSmem, st>>>(a);
    if (splits > 1) {
        const size_t total = static_cast<size_t>(M) * N;
        int blocks = static_cast<int>((total + 255) / 256);
        blocks = blocks < 4096 ? blocks : 4096;
        k_splitk_reduce<<<blocks, 256, 0, st>>>(work, splits, a.split_stride, M, N, N, out, ldo);
    }
}

}  // namespace xrdvi

extern "C" xrdvi_status xrdvi_gemm_nt_tf32x3(int32_t M, int32_t N, int32_t K, const float *d_A, int32_t lda,
                                             const float *d_B, int32_t ldb, float *d_C, int32_t ldc,
                                             void *cuda_stream) {
    using xrdvi::report_error;
    if (M < 1 || N < 1 || K < 1 || !d_A || !d_B || !d_C) return report_error(XRDVI_EINVAL, "gemm: bad sizes");
    if (K % 4 || lda % 4 || ldb % 4 || lda < K || ldb < K || ldc < N)
        return report_error(XRDVI_EINVAL, "gemm: K, lda, ldb must be multiples of 4 with lda, ldb >= K, ldc >= N");
    if ((reinterpret_cast<uintptr_t>(d_A) | reinterpret_cast<uintptr_t>(d_B)) & 15u)
        return report_error(XRDVI_EINVAL, "gemm: A and B must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int splits = xrdvi::gemm_splits(M, N, K, sms);
    const size_t na = static_cast<size_t>(M) * lda, nb = static_cast<size_t>(N) * ldb;
    float *work = nullptr, *ahl = nullptr, *bhl = nullptr;
    int *err = nullptr;
    cudaError_t e = xrdvi::gemm_configure();
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ahl, 2 * na * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&bhl, 2 * nb * sizeof(float), st);
    const size_t wf = xrdvi::gemm_workspace_floats(M, N, splits);
    if (e == cudaSuccess && wf) e = cudaMallocAsync(&work, wf * sizeof(float), st);
    if (e == cudaSuccess) {
        xrdvi::launch_tf32_split(d_A, na, ahl, ahl + na, st);
        xrdvi::launch_tf32_split(d_B, nb, bhl, bhl + nb, st);
        xrdvi::launch_gemm_nt_tf32x3(M, N, K, ahl, ahl + na, lda, bhl, bhl + nb, ldb, d_C, ldc, splits, work, err,
                                     st);
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (work) cudaFreeAsync(work, st);
    if (ahl) cudaFreeAsync(ahl, st);
    if (bhl) cudaFreeAsync(bhl, st);
    if (err) cudaFreeAsync(err, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("gemm: ") + cudaGetErrorString(e));
    if (herr) return report_error(XRDVI_ETIMEOUT, "gemm: an mbarrier wait gave up");
    return XRDVI_OK;
}
