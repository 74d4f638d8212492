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
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <string>

#include "../../include/xrdvi.h"
#include "xrdvi_internal.h"

namespace xrdvi {
namespace {

constexpr int kGM = 128;        // tile rows (MMA M)
constexpr int kGKB = 32;        // reduction elements per stage: one 128-byte row (4 MMA steps of 8)
constexpr int kGThreads = 128;  // warp 0: TMA producer, warp 1: MMA issuer, warp 2: TMEM owner; all: epilogue
constexpr int kStages = 3;      // stages in flight
constexpr uint32_t kTileA = kGM * kGKB * 4;   // bytes of one A operand tile (16 KB)
constexpr uint32_t kWaitLimit = 1u << 24;     // mbarrier polls before giving up

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

// Shared-memory matrix descriptor (tcgen05) of a K-major operand in the
// 128-byte swizzled layout that TMA writes: rows of 128 bytes, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1, layout type
// SWIZZLE_128B; the leading byte offset is unused for this layout (encoded 1).
// A k-step of 8 TF32 elements starts 32 bytes further along the row.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (static_cast<uint64_t>(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// TMA: 2D tile (x = reduction index, y = row) into shared memory, completion
// counted on the mbarrier in bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(y)
        : "memory");
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

struct GemmArgs {
    int M, N, K;             // out[M x N] = A[M x K] . B[N x K]^T (row-major, K contiguous)
    float *out;              // split s writes out + s * split_stride (row stride ldo)
    int ldo;
    size_t split_stride;
    int kb_per_split, nkb;   // stages of kGKB per split, total
    int *err;                // set to 1 if an mbarrier wait gives up
};

// One output tile of kGM x kGN per CTA over one split of the reduction.
// Warp-specialised pipeline over kStages shared-memory stages: the producer
// waits for a stage to be empty, arms its full barrier with the stage's bytes
// and issues four TMA tile loads (A and B, TF32 hi and lo parts); the MMA
// issuer waits for the full barrier, issues 4 k-steps x 3 MMAs (3xTF32) into
// the TMEM accumulator and commits them to the stage's empty barrier; after
// the last stage a commit to the done barrier releases the epilogue, in which
// every warp reads its 32 TMEM lanes.  Every wait is bounded.
template <int kGN>
__global__ void __launch_bounds__(kGThreads) k_gemm_nt_tf32x3(const __grid_constant__ CUtensorMap tAh,
                                                              const __grid_constant__ CUtensorMap tAl,
                                                              const __grid_constant__ CUtensorMap tBh,
                                                              const __grid_constant__ CUtensorMap tBl, GemmArgs a) {
    using Cfg = TileCfg<kGN>;
    constexpr uint32_t kTileB = Cfg::kTileB, kStage = Cfg::kStage;
    extern __shared__ uint8_t g_smem_raw[];
    __shared__ __align__(8) uint64_t s_full[kStages], s_empty[kStages], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    uint8_t *smem = g_smem_raw + ((1024u - (smem_addr(g_smem_raw) & 1023u)) & 1023u);   // 1 KB aligned (swizzle)
    const uint32_t sbase = smem_addr(smem);
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN, split = blockIdx.z;
    const int kb0 = split * a.kb_per_split;
    const int nk = min(a.nkb, kb0 + a.kb_per_split) - kb0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_addr(&s_full[i]), 1);
            mbar_init(smem_addr(&s_empty[i]), 1);
        }
        mbar_init(smem_addr(&s_done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(static_cast<uint32_t>(kGN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int i = 0; i < nk; ++i) {
            const int st = i % kStages, n = i / kStages;
            if (n > 0 && !mbar_wait(smem_addr(&s_empty[st]), static_cast<uint32_t>((n - 1) & 1))) {
                s_abort = 1;
                break;
            }
            if (*reinterpret_cast<volatile int *>(&s_abort)) break;
            const uint32_t full = smem_addr(&s_full[st]);
            const uint32_t base = sbase + st * kStage;
            const int k0 = (kb0 + i) * kGKB;
            mbar_expect_tx(full, kStage);
            tma_load_2d(base, &tAh, k0, m0, full);
            tma_load_2d(base + kTileA, &tAl, k0, m0, full);
            tma_load_2d(base + 2 * kTileA, &tBh, k0, n0, full);
            tma_load_2d(base + 2 * kTileA + kTileB, &tBl, k0, n0, full);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int i = 0; i < nk && ok; ++i) {
            const int st = i % kStages, n = i / kStages;
            if (!mbar_wait(smem_addr(&s_full[st]), static_cast<uint32_t>(n & 1))) {
                s_abort = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = sbase + st * kStage;
#pragma unroll
            for (int t = 0; t < kGKB / 8; ++t) {
                const uint32_t off = static_cast<uint32_t>(t) * 32u;   // 8 TF32 = 32 bytes along the row
                const uint64_t ahi = smem_desc_sw128(base + off), alo = smem_desc_sw128(base + kTileA + off);
                const uint64_t bhi = smem_desc_sw128(base + 2 * kTileA + off);
                const uint64_t blo = smem_desc_sw128(base + 2 * kTileA + kTileB + off);
                mma_tf32(tmem, alo, bhi, Cfg::kIdesc, (i > 0 || t > 0) ? 1u : 0u);
                mma_tf32(tmem, ahi, blo, Cfg::kIdesc, 1u);
                mma_tf32(tmem, ahi, bhi, Cfg::kIdesc, 1u);
            }
            mma_commit(smem_addr(&s_empty[st]));
        }
        if (ok && nk > 0)
            mma_commit(smem_addr(&s_done));
        else
            mbar_arrive(smem_addr(&s_done));   // nothing to wait for (no blocks, or aborted)
    }
    // epilogue: every thread waits for the accumulator
    const bool done = mbar_wait(smem_addr(&s_done), 0u);
    __syncthreads();
    const bool ok = done && !*reinterpret_cast<volatile int *>(&s_abort);
    if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
    tc_fence_after();
    if (ok) {
        // warp w owns rows 32w..32w+31 of the tile (TMEM lanes)
        const int row = m0 + 32 * warp + lane;
        float *dst = a.out + static_cast<size_t>(split) * a.split_stride + static_cast<size_t>(row) * a.ldo;
#pragma unroll 1
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
    if (warp == 2)
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
    const int *order;        // [K] phases by decreasing peak count: blockIdx.y -> phase
    const float *theta;      // sample 0's row [K*5]
    float *D, *D_lo;         // [K*10*Npad] TF32 hi / lo parts
    float *Ct, *Ct_lo;       // [Npad*Kpad] TF32 hi / lo parts
};

constexpr int kShapeChunk = 512;   // peaks staged in shared memory at a time

// The sums over one side's run of peaks [m0, m1) of the staged chunk at scale
// s (t = s d cos(x/2)): sum I L and sum I G (added to lS, gS in peak order),
// and the side's sum I L^2 t, I L^2 t^2, I G t, I G t^2.
__device__ __forceinline__ void shape_side(const float2 *sp, int m0, int m1, float x, float mu, float s, float cx,
                                           float &lS, float &gS, float &l1, float &l2, float &g1, float &g2) {
    for (int m = m0; m < m1; ++m) {
        const float2 pk = sp[m];
        const float d = (x - pk.x) - mu;
        const float t = s * d * cx, u = t * t;
        float L;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(L) : "f"(1.f + u));
        const float I = pk.y;
        const float IL = I * L, IL2 = IL * L;
        lS += IL;
        l1 = fmaf(IL2, t, l1);
        l2 = fmaf(IL2, u, l2);
        if (u < kGaussU) {
            float G;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G) : "f"(-u));
            const float IG = I * G;
            gS += IG;
            g1 = fmaf(IG, t, g1);
            g2 = fmaf(IG, u, g2);
        }
    }
}

__global__ void __launch_bounds__(256) k_shapes(ShapeArgs a) {
    __shared__ float2 sp[kShapeChunk];   // (p, I) of the phase's peaks
    // phase of this block row: the heaviest phases start first (blocks go out in
    // index order), so the kernel does not end on a phase of many peaks
    const int k = a.order[blockIdx.y], i = blockIdx.x * blockDim.x + threadIdx.x;   // blockDim.x * gridDim.x == Npad
    const PhaseConst c = a.cst[k];
    const float r = a.theta[k * 5 + 3];
    // A phase's peaks are sorted by position, so the peaks with d = x - p - mu
    // >= 0 (scale s_r, t >= 0) are a leading run and the rest (s_l, t < 0) the
    // trailing run: no per-peak side choice, and on each side |t| = +-t, so the
    // four sums in t, |t|, t^2, t|t| of each component come from two per side.
    float lS = 0.f, gS = 0.f;
    float l1[2] = {0.f, 0.f}, l2[2] = {0.f, 0.f}, g1[2] = {0.f, 0.f}, g2[2] = {0.f, 0.f};
    const bool live = i < a.N;
    const float x = live ? a.x[i] : 0.f;
    const float cx = (a.csec && live) ? a.csec[i] : 1.f;   // t = s cos(x/2) d; mu sums take cos(x/2) once more
    for (int m0 = a.off[k]; m0 < a.off[k + 1]; m0 += kShapeChunk) {
        const int mn = min(kShapeChunk, a.off[k + 1] - m0);
        __syncthreads();
        for (int j = threadIdx.x; j < mn; j += blockDim.x) sp[j] = make_float2(a.pos[m0 + j], a.inten[m0 + j]);
        __syncthreads();
        if (!live) continue;
        int lo = 0, hi = mn;   // first staged peak with d < 0 (d is non-increasing along the run)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((x - sp[mid].x) - c.mu >= 0.f)
                lo = mid + 1;
            else
                hi = mid;
        }
        shape_side(sp, 0, lo, x, c.mu, c.sr, cx, lS, gS, l1[0], l2[0], g1[0], g2[0]);
        shape_side(sp, lo, mn, x, c.mu, c.sl, cx, lS, gS, l1[1], l2[1], g1[1], g2[1]);
    }
    // the ten sums in the backward's order (t >= 0 on side 0, t < 0 on side 1)
    float acc[kGradSums];
    acc[0] = gS;
    acc[1] = lS;
    acc[2] = g1[0] + g1[1];
    acc[3] = l1[0] + l1[1];
    acc[4] = g1[0] - g1[1];
    acc[5] = l1[0] - l1[1];
    acc[6] = g2[0] + g2[1];
    acc[7] = l2[0] + l2[1];
    acc[8] = g2[0] - g2[1];
    acc[9] = l2[0] - l2[1];
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
    s.cst = W.cst; s.theta = W.theta; s.D = W.D; s.Ct = W.Ct; s.csec = P.csec; s.order = P.far_order;
    s.D_lo = W.D + static_cast<size_t>(P.K) * kGradSums * P.Npad;
    s.Ct_lo = W.Ct + static_cast<size_t>(P.Npad) * W.Kpad;
    k_shapes<<<dim3(P.T, P.K), 256, 0, st>>>(s);
    // f_s - B = sum_k h_sk C_k: [S x N] = H [S x Kpad] . Ct [N x Kpad]^T, into the first chunk slot
    launch_gemm(W.plan_fwd, st);
    launch_lik(P, W, f_out, 1, st);
}

void launch_shared_backward(const Problem &P, Workspace &W, cudaStream_t st) {
    // per (s, k) sums: [S x 10K] = g [S x Npad] . D [10K x Npad]^T  (g = 0 on padding)
    (void)P;
    launch_gemm(W.plan_bwd, st);
}

// Tile width: 128 columns where N is wide (fewer re-reads of A), 64 for
// narrow outputs (and, in gemm_plan, for short unsplit reductions).
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

// TMA descriptor of a row-major FP32 matrix [rows x K] (row stride ld
// elements) read in boxes of 32 reduction elements x box_rows rows with the
// 128-byte swizzle; out-of-range elements read as zero.
static bool encode_tmap(CUtensorMap *m, const float *ptr, int rows, int K, int ld, int box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f)
            return false;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(kGKB), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gemm_plan(GemmPlan &p, int M, int N, int K, const float *Ahi, const float *Alo, int lda, const float *Bhi,
               const float *Blo, int ldb, float *out, int ldo, int splits, float *work, int *err) {
    p.M = M; p.N = N; p.K = K; p.out = out; p.ldo = ldo; p.work = work; p.err = err;
    p.tn = tile_n(N);
    p.nkb = (K + kGKB - 1) / kGKB;
    if (splits < 1) splits = 1;
    // a short unsplit reduction (the forward's K = phases) is latency-bound per
    // tile: 64-wide tiles give twice the CTAs
    if (splits == 1 && p.nkb <= 4) p.tn = 64;
    if (splits > p.nkb) splits = p.nkb > 0 ? p.nkb : 1;
    p.kb_per_split = (p.nkb + splits - 1) / splits;
    p.splits = p.nkb > 0 ? (p.nkb + p.kb_per_split - 1) / p.kb_per_split : 1;
    return encode_tmap(&p.tAh, Ahi, M, K, lda, kGM) && encode_tmap(&p.tAl, Alo, M, K, lda, kGM) &&
           encode_tmap(&p.tBh, Bhi, N, K, ldb, p.tn) && encode_tmap(&p.tBl, Blo, N, K, ldb, p.tn);
}

void launch_gemm(const GemmPlan &p, cudaStream_t st) {
    GemmArgs a;
    a.M = p.M; a.N = p.N; a.K = p.K; a.err = p.err; a.nkb = p.nkb; a.kb_per_split = p.kb_per_split;
    if (p.splits == 1) {
        a.out = p.out; a.ldo = p.ldo; a.split_stride = 0;
    } else {
        a.out = p.work; a.ldo = p.N; a.split_stride = static_cast<size_t>(p.M) * p.N;
    }
    dim3 grid((p.M + kGM - 1) / kGM, (p.N + p.tn - 1) / p.tn, p.splits);
    if (p.tn == 128)
        k_gemm_nt_tf32x3<128><<<grid, kGThreads, TileCfg<128>::kSmem, st>>>(p.tAh, p.tAl, p.tBh, p.tBl, a);
    else
        k_gemm_nt_tf32x3<64><<<grid, kGThreads, TileCfg<64>::kSmem, st>>>(p.tAh, p.tAl, p.tBh, p.tBl, a);
    if (p.splits > 1) {
        const size_t total = static_cast<size_t>(p.M) * p.N;
        int blocks = static_cast<int>((total + 255) / 256);
        blocks = blocks < 4096 ? blocks : 4096;
        k_splitk_reduce<<<blocks, 256, 0, st>>>(p.work, p.splits, a.split_stride, p.M, p.N, p.N, p.out, p.ldo);
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
        xrdvi::GemmPlan plan;
        if (!xrdvi::gemm_plan(plan, M, N, K, ahl, ahl + na, lda, bhl, bhl + nb, ldb, d_C, ldc, splits, work, err)) {
            e = cudaErrorInvalidValue;
        } else {
            xrdvi::launch_gemm(plan, st);
            e = cudaGetLastError();
        }
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
