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
constexpr int kGN = 64;         // tile columns (MMA N)
constexpr int kGKB = 32;        // reduction elements per k-block (4 MMA steps of 8)
constexpr int kGThreads = 128;  // 4 warps: warp w reads TMEM lanes 32w..32w+31
constexpr uint32_t kTileA = kGM * kGKB * 4;   // bytes of one A operand tile (16 KB)
constexpr uint32_t kTileB = kGN * kGKB * 4;   // bytes of one B operand tile (8 KB)
constexpr uint32_t kStage = 2 * kTileA + 2 * kTileB;   // hi + lo of A and B (48 KB)
constexpr int kStages = 2;
constexpr uint32_t kWaitLimit = 1u << 22;     // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row r, reduction index e < 32) in a K-major tile
// without swizzle built from core matrices of 8 rows x 16 bytes: the 8 cores
// along K of one 8-row group are 128 bytes apart (leading byte offset), the
// 8-row groups 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t core_off(int r, int e) {
    return static_cast<uint32_t>((r >> 3) * 1024 + (e >> 2) * 128 + (r & 7) * 16 + (e & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
           (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(kGN >> 3) << 17) |
                            (static_cast<uint32_t>(kGM >> 4) << 24);

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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ float tf32_hi(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u); }

struct GemmArgs {
    int M, N, K;             // out[M x N] = A[M x K] . B[N x K]^T (both row-major, K contiguous)
    const float *A, *B;
    int lda, ldb;
    float *out;              // split s writes out + s * split_stride (row stride ldo)
    int ldo;
    size_t split_stride;
    int kb_per_split, nkb;   // k-blocks of kGKB per split, total
    int *err;                // set to 1 if an mbarrier wait gives up
};

// Loads one k-block of A (kGM rows) and B (kGN rows) from global memory,
// splits each element into TF32 hi / lo and stores them in the core-matrix
// layout.  Rows beyond M / N and reduction indices beyond K read as zero.
__device__ __forceinline__ void load_stage(const GemmArgs &a, uint8_t *st, int m0, int n0, int k0) {
    float *Ahi = reinterpret_cast<float *>(st), *Alo = reinterpret_cast<float *>(st + kTileA);
    float *Bhi = reinterpret_cast<float *>(st + 2 * kTileA), *Blo = reinterpret_cast<float *>(st + 2 * kTileA + kTileB);
    for (int idx = threadIdx.x; idx < kGM * (kGKB / 4); idx += kGThreads) {
        const int r = idx >> 3, q = idx & 7;
        const int row = m0 + r, k = k0 + 4 * q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < a.M && k < a.K) v = __ldg(reinterpret_cast<const float4 *>(a.A + static_cast<size_t>(row) * a.lda + k));
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        const uint32_t o = core_off(r, 4 * q) >> 2;
        *reinterpret_cast<float4 *>(Ahi + o) = h;
        *reinterpret_cast<float4 *>(Alo + o) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
    for (int idx = threadIdx.x; idx < kGN * (kGKB / 4); idx += kGThreads) {
        const int r = idx >> 3, q = idx & 7;
        const int row = n0 + r, k = k0 + 4 * q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < a.N && k < a.K) v = __ldg(reinterpret_cast<const float4 *>(a.B + static_cast<size_t>(row) * a.ldb + k));
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        const uint32_t o = core_off(r, 4 * q) >> 2;
        *reinterpret_cast<float4 *>(Bhi + o) = h;
        *reinterpret_cast<float4 *>(Blo + o) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
}

// One output tile of kGM x kGN per CTA over one split of the reduction.
// Double-buffered stages: all threads stage k-block kb while the MMAs of
// kb - 1 run; one thread issues 4 k-steps x 3 MMAs per block and commits
// them to the stage's mbarrier, which is awaited before the stage is reused.
__global__ void __launch_bounds__(kGThreads) k_gemm_nt_tf32x3(GemmArgs a) {
    extern __shared__ uint8_t g_smem_raw[];
    __shared__ __align__(8) uint64_t s_mbar[kStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    uint8_t *smem = g_smem_raw + ((1024u - (smem_addr(g_smem_raw) & 1023u)) & 1023u);   // 1 KB aligned
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN, split = blockIdx.z;
    const int kb0 = split * a.kb_per_split;
    const int kb1 = min(a.nkb, kb0 + a.kb_per_split);
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int nk = kb1 - kb0;
    for (int i = 0; i < nk; ++i) {
        const int buf = i & 1;
        uint8_t *st = smem + buf * kStage;
        if (i >= kStages && threadIdx.x == 0) {
            // the MMAs that read this stage (block i - 2) must be done
            if (!mbar_wait(smem_addr(&s_mbar[buf]), static_cast<uint32_t>(((i - kStages) >> 1) & 1))) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;   // uniform: read after the barrier
        load_stage(a, st, m0, n0, (kb0 + i) * kGKB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> MMA operand reads
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t base = smem_addr(st);
            for (int t = 0; t < kGKB / 8; ++t) {
                const uint32_t off = static_cast<uint32_t>(t) * 256u;   // two 128-byte cores per k-step
                const uint64_t ahi = smem_desc(base + off, 128, 1024), alo = smem_desc(base + kTileA + off, 128, 1024);
                const uint64_t bhi = smem_desc(base + 2 * kTileA + off, 128, 1024);
                const uint64_t blo = smem_desc(base + 2 * kTileA + kTileB + off, 128, 1024);
                mma_tf32(tmem, alo, bhi, (i > 0 || t > 0) ? 1u : 0u);
                mma_tf32(tmem, ahi, blo, 1u);
                mma_tf32(tmem, ahi, bhi, 1u);
            }
            mma_commit(smem_addr(&s_mbar[buf]));
        }
    }
    // wait for the last block's MMAs (a commit tracks all earlier MMAs too);
    // one thread waits, the barrier publishes the outcome to all
    __syncthreads();
    if (threadIdx.x == 0 && !s_abort && nk > 0 &&
        !mbar_wait(smem_addr(&s_mbar[(nk - 1) & 1]), static_cast<uint32_t>(((nk - 1) >> 1) & 1)))
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
            if (row < a.M && nk > 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n0 + c0 + j < a.N) dst[n0 + c0 + j] = __uint_as_float(v[j]);
            } else if (row < a.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n0 + c0 + j < a.N) dst[n0 + c0 + j] = 0.f;
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
    float *D;                // [K*10*Npad]
    float *Ct;               // [Npad*Kpad]
};

__global__ void __launch_bounds__(256) k_shapes(ShapeArgs a) {
    const int k = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.Npad) return;
    const PhaseConst c = a.cst[k];
    const float r = a.theta[k * 5 + 3];
    float acc[kGradSums];
#pragma unroll
    for (int j = 0; j < kGradSums; ++j) acc[j] = 0.f;
    if (i < a.N) {
        const float x = a.x[i];
        const float cx = a.csec ? a.csec[i] : 1.f;   // t = s cos(x/2) d; mu sums take cos(x/2) once more
        for (int m = a.off[k]; m < a.off[k + 1]; ++m) {
            const float d = (x - __ldg(&a.pos[m])) - c.mu;
            const float t = (d >= 0.f ? c.sr : c.sl) * d * cx;
            const float at = fabsf(t), u = t * t;
            float L;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(L) : "f"(1.f + u));
            const float I = __ldg(&a.inten[m]);
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
    if (a.csec && i < a.N) {
        const float cx = a.csec[i];
        acc[2] *= cx; acc[3] *= cx; acc[4] *= cx; acc[5] *= cx;
    }
#pragma unroll
    for (int j = 0; j < kGradSums; ++j) a.D[(static_cast<size_t>(k) * kGradSums + j) * a.Npad + i] = acc[j];
    a.Ct[static_cast<size_t>(i) * a.Kpad + k] = fmaf(r, acc[1], (1.f - r) * acc[0]);
}

}  // namespace

void launch_shared_forward(const Problem &P, Workspace &W, float *f_out, cudaStream_t st) {
    ShapeArgs s;
    s.N = P.N; s.Npad = P.Npad; s.K = P.K; s.Kpad = W.Kpad;
    s.x = P.x; s.pos = P.pos; s.inten = P.inten; s.off = P.off;
    s.cst = W.cst; s.theta = W.theta; s.D = W.D; s.Ct = W.Ct; s.csec = P.csec;
    k_shapes<<<dim3(P.T, P.K), 256, 0, st>>>(s);
    // f_s - B = sum_k h_sk C_k: [S x N] = H [S x Kpad] . Ct [N x Kpad]^T, into the first chunk slot
    launch_gemm_nt_tf32x3(W.S, P.N, W.Kpad, W.H, W.Kpad, W.Ct, W.Kpad, W.fpart, P.Npad, 1, nullptr, W.gemm_err, st);
    launch_lik(P, W, f_out, 1, st);
}

void launch_shared_backward(const Problem &P, Workspace &W, cudaStream_t st) {
    // per (s, k) sums: [S x 10K] = g [S x Npad] . D [10K x Npad]^T  (g = 0 on padding)
    const int nk = P.K * kGradSums;
    launch_gemm_nt_tf32x3(W.S, nk, P.Npad, W.g, P.Npad, W.D, P.Npad, W.gpart, nk, W.gemm_splits, W.gemm_work,
                          W.gemm_err, st);
}

size_t gemm_smem_bytes() { return kStages * kStage + 1024; }

int gemm_splits(int M, int N, int K, int sm_count) {
    const int tiles = ((M + kGM - 1) / kGM) * ((N + kGN - 1) / kGN);
    const int nkb = (K + kGKB - 1) / kGKB;
    int s = (sm_count + tiles - 1) / tiles;   // about one CTA per SM
    s = s < nkb ? s : nkb;
    return s < 1 ? 1 : s;
}

size_t gemm_workspace_floats(int M, int N, int splits) {
    return splits > 1 ? static_cast<size_t>(splits) * M * N : 0;
}

cudaError_t gemm_configure() {
    return cudaFuncSetAttribute(k_gemm_nt_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(gemm_smem_bytes()));
}

void launch_gemm_nt_tf32x3(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *out,
                           int ldo, int splits, float *work, int *err, cudaStream_t st) {
    GemmArgs a;
    a.M = M; a.N = N; a.K = K; a.A = A; a.B = B; a.lda = lda; a.ldb = ldb; a.err = err;
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
    dim3 grid((M + kGM - 1) / kGM, (N + kGN - 1) / kGN, splits);
    k_gemm_nt_tf32x3<<<grid, kGThreads, gemm_smem_bytes(), st>>>(a);
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
    float *work = nullptr;
    int *err = nullptr;
    cudaError_t e = xrdvi::gemm_configure();
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    const size_t wf = xrdvi::gemm_workspace_floats(M, N, splits);
    if (e == cudaSuccess && wf) e = cudaMallocAsync(&work, wf * sizeof(float), st);
    if (e == cudaSuccess) {
        xrdvi::launch_gemm_nt_tf32x3(M, N, K, d_A, lda, d_B, ldb, d_C, ldc, splits, work, err, st);
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (work) cudaFreeAsync(work, st);
    if (err) cudaFreeAsync(err, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return report_error(XRDVI_ECUDA, std::string("gemm: ") + cudaGetErrorString(e));
    if (herr) return report_error(XRDVI_ETIMEOUT, "gemm: an mbarrier wait gave up");
    return XRDVI_OK;
}
