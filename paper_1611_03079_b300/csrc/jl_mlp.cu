// Learned screening surrogate on the sm_103a tensor cores.
//
// The network maps C to the normalised escape-count histogram of its Julia
// frame (128x128 over [-2,2]^2, limit 100), so that many C can be screened
// before any frame is rendered -- the paper's aim of sampling the parameter
// space quickly (Sec. 1) with the Mandelbrot set as the roadmap for C
// (Sec. 3).  Architecture (fixed): phi(C) = [sin 2piBC, cos 2piBC] (B: 32x2),
// Linear 64->256, ReLU, Linear 256->256, ReLU, Linear 256->101, softmax;
// bfloat16 weights and activations, binary32 accumulation, cross-entropy
// against the target histogram, Adam on binary32 master weights.
//
// Kernels:
//   train_step_kernel   one training step per 128-row tile of the batch in one
//                       launch: features, the three products with bias + ReLU,
//                       softmax and cross-entropy error, and the backward
//                       products (dX and the transposed dW) with activations
//                       in shared memory; per-tile gradient partials out
//   adam_kernel         sums the partials in a fixed order, Adam on binary32
//                       master weights, refreshes the packed bf16 images
//   fused_forward_kernel  screening forward (features -> softmax entropy)
//   tc_gemm_kernel      one product with a fused epilogue (bias + ReLU ->
//                       bf16, softmax, or plain fp32): the layered forward and
//                       the standalone product jl_gemm_bf16
// All products are tcgen05.mma issued by one thread, operands in shared
// memory in the no-swizzle core-matrix layouts (K-major, or MN-major where an
// operand is read transposed), accumulators in tensor memory read back with
// tcgen05.ld, completion tracked by tcgen05.commit on mbarriers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "jl_internal.h"
#include "jl_tc.cuh"

namespace jl {

static constexpr int kFreq = 32, kIn = 64, kHid = 256, kBins = 101;
static constexpr int kBinsPad = 112;  // N of the last product (multiple of 16)
static constexpr int kTrTP = 104;     // padded target row in training: 101 bins + 3 (16-byte rows)
// Parameter block (binary32, this order): W1[256x64] b1[256] W2[256x256] b2[256] W3[101x256] b3[101]
static constexpr int kOffW1 = 0;
static constexpr int kOffB1 = kOffW1 + kHid * kIn;
static constexpr int kOffW2 = kOffB1 + kHid;
static constexpr int kOffB2 = kOffW2 + kHid * kHid;
static constexpr int kOffW3 = kOffB2 + kHid;
static constexpr int kOffB3 = kOffW3 + kBins * kHid;
static constexpr int kNumParams = kOffB3 + kBins;  // 108,389

enum Epi { EPI_BIAS_ACT = 0, EPI_SOFTMAX = 1, EPI_F32 = 2 };

struct GemmArgs {
    const __nv_bfloat16 *A;  // trans 0: A[m * lda + k]; trans 1: A[k * lda + m]
    const __nv_bfloat16 *B;  // trans 0: B[n * ldb + k]; trans 1: B[k * ldb + n]
    int lda, ldb, a_trans, b_trans;
    int M, N, K, BN;         // BN: N rounded up to a multiple of 16 (<= 256)
    const float *bias;       // [N]
    int relu;
    __nv_bfloat16 *out_bf16; // EPI_BIAS_ACT: [M x ld_out], ld_out a multiple of 8, 16-byte aligned
    int ld_out;
    float *out_f32;          // EPI_F32: [M x ld_out32]
    int ld_out32;
    float *probs;            // EPI_SOFTMAX: [M x ldp] or NULL
    int ldp;
    float *score;            // EPI_SOFTMAX: [M] entropy of p or NULL
    int32_t *status;         // set to JL_ETIMEOUT if a wait gave up
    // B is not written by the preceding kernel of the stream: its chunks are
    // staged before waiting for it (programmatic dependent launch)
    int pre_b;
    // EPI_BIAS_ACT column split: CTA (x, z) computes columns
    // [z * n_per_cta, (z + 1) * n_per_cta) of its rows (a multiple of 64);
    // 0 = all BN columns in one CTA
    int n_per_cta;
};

static constexpr int kBM = 128, kBK = 64;
static constexpr int kTileA = kBM * kBK * 2;   // 16 KB
static constexpr int kTileB = 256 * kBK * 2;   // 32 KB
static constexpr int kStage = kTileA + kTileB;
static constexpr int kStages = 4;  // K chunks in flight (K <= 256 is staged in one go)
static constexpr int kGemmSmem = kStages * kStage + 4 * kBM * 4 + 128;  // stages + row exchange + barriers
static constexpr long long kWaitLimit = 2000000000ll;  // ~1 s at 2 GHz

// Stage rows [row0, row0 + nrows) x k [k0, k0 + 64) of an operand into the
// K-major core-matrix layout: piece (r, g) (8 consecutive k) at byte
// ((r/8)*8 + g)*128 + (r%8)*16.  Out-of-range elements are zero.  Each
// thread gathers up to eight pieces into registers before storing any, so
// their global-load latencies overlap.
__device__ __forceinline__ void stage_operand(uint8_t *dst, const __nv_bfloat16 *src, int ld, int trans, int row0,
                                              int nrows, int rlim, int k0, int klim)
{
    const int pieces = nrows * 8;
    const int step = blockDim.x;
    for (int base = threadIdx.x; base < pieces; base += 8 * step) {
        uint4 v[8];
        int off[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int p = base + u * step;
            v[u] = make_uint4(0, 0, 0, 0);
            off[u] = -1;
            if (p >= pieces)
                continue;
            int r, g;
            if (!trans) {
                // 8 consecutive threads fill one 128-byte core matrix (no bank conflicts)
                r = (p >> 6) * 8 + (p & 7);
                g = (p >> 3) & 7;
            } else {
                // consecutive threads take consecutive rows (contiguous in global)
                r = p % nrows;
                g = p / nrows;
            }
            off[u] = ((r >> 3) * 8 + g) * 128 + (r & 7) * 16;
            const int row = row0 + r;
            const int k = k0 + g * 8;
            if (row < rlim) {
                if (!trans) {
                    const __nv_bfloat16 *s = src + (size_t)row * ld + k;
                    if (k + 8 <= klim && ((reinterpret_cast<uintptr_t>(s) & 15) == 0)) {
                        v[u] = *reinterpret_cast<const uint4 *>(s);
                    } else {
                        uint16_t e[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            e[i] = (k + i < klim) ? __bfloat16_as_ushort(s[i]) : (uint16_t)0;
                        v[u] = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16),
                                          e[6] | (e[7] << 16));
                    }
                } else {
                    uint16_t e[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        e[i] = (k + i < klim) ? __bfloat16_as_ushort(src[(size_t)(k + i) * ld + row]) : (uint16_t)0;
                    v[u] = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16),
                                      e[6] | (e[7] << 16));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (off[u] >= 0)
                *reinterpret_cast<uint4 *>(dst + off[u]) = v[u];
    }
}

// Asynchronous form of stage_operand for 16-byte aligned operands (ld a
// multiple of 8 elements, 16-byte aligned base): every piece is one cp.async
// of up to 16 bytes, zero-filled past rlim / klim.  trans = 0 (stored
// rows x K): the K-major layout of stage_operand.  trans = 1 (stored K x rows,
// A[k * ld + row]): MN-major core matrices instead -- core matrix (r / 8, k / 8)
// at the same byte offset ((r / 8) * 8 + (k % 64) / 8) * 128, holding 8
// K-rows of 16 bytes (8 consecutive rows of the operand) -- so the pieces are
// contiguous in global memory and the MMA reads the operand as MN-major.
__device__ __forceinline__ void stage_async(uint8_t *dst, const __nv_bfloat16 *src, int ld, int trans, int row0,
                                            int nrows, int rlim, int k0, int klim)
{
    const int pieces = nrows * 8;
    const int nmg = nrows >> 3;
    for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
        int off;
        uint32_t bytes;
        const __nv_bfloat16 *sp = src;
        if (!trans) {
            // 8 consecutive threads fill one 128-byte core matrix
            const int r = (p >> 6) * 8 + (p & 7);
            const int g = (p >> 3) & 7;
            off = ((r >> 3) * 8 + g) * 128 + (r & 7) * 16;
            const int row = row0 + r, k = k0 + g * 8;
            const int nk = klim - k;
            bytes = (row < rlim && nk > 0) ? 2u * (uint32_t)min(nk, 8) : 0u;
            if (bytes)
                sp = src + (size_t)row * ld + k;
        } else {
            // 8 consecutive threads fill one core matrix (8 K-rows), and the
            // next 8 the core matrix of the next 8 operand rows, so a warp
            // reads 64 contiguous bytes from each of 8 K-rows
            const int kr = ((p >> 3) / nmg) * 8 + (p & 7);
            const int mg = (p >> 3) % nmg;
            off = (mg * 8 + (kr >> 3)) * 128 + (kr & 7) * 16;
            const int k = k0 + kr, m = row0 + mg * 8;
            const int nm = rlim - m;
            bytes = (k < klim && nm > 0) ? 2u * (uint32_t)min(nm, 8) : 0u;
            if (bytes)
                sp = src + (size_t)k * ld + m;
        }
        tc::cp_async16(dst + off, sp, bytes);
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 2^x with the hardware approximation (relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

static constexpr int kGemmThreads = 512;  // 16 warps: 4 per scheduler in the epilogue

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) tc_gemm_kernel(const __grid_constant__ GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *stage0 = sm;
    float *xch = reinterpret_cast<float *>(sm + kStages * kStage);                       // [4][128] row values
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kStages * kStage + 4 * kBM * 4);  // kStages + 1 mbarriers
    uint32_t *holder = reinterpret_cast<uint32_t *>(bars + kStages + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;

    if (warp == 0)
        tc::tmem_alloc(holder, 256);
    if (threadIdx.x == 0) {
        for (int b = 0; b <= kStages; ++b)
            tc::mbar_init(&bars[b], 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = *holder;

    // this CTA's columns [n0, n0 + nbn) (a multiple of 16 wide)
    const int npc = (EPI != EPI_SOFTMAX && g.n_per_cta > 0) ? g.n_per_cta : g.BN;
    const int n0 = (int)blockIdx.z * npc;
    const int nbn = min(npc, g.BN - n0);
    // Operands whose 16-byte pieces are aligned are staged with cp.async
    // (transposed ones MN-major, read as such by the MMA); others through
    // registers, K-major (transposed ones gathered element by element).
    const bool a_async = (g.lda & 7) == 0 && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0;
    const bool b_async = (g.ldb & 7) == 0 && (reinterpret_cast<uintptr_t>(g.B) & 15) == 0;
    const uint32_t idesc = tc::idesc_bf16_t(kBM, (uint32_t)nbn, a_async && g.a_trans, b_async && g.b_trans);
    const int nchunks = (g.K + kBK - 1) / kBK;
    const int nst = min(nchunks, kStages);
    // stage = A tile (128 x 64) + this CTA's B tile (nbn x 64)
    const int stage_bytes = kTileA + nbn * kBK * 2;
    auto stage = [&](int kc, bool do_a, bool do_b) {
        uint8_t *sA = stage0 + (kc % kStages) * stage_bytes;
        uint8_t *sB = sA + kTileA;
        if (do_a) {
            if (a_async)
                stage_async(sA, g.A, g.lda, g.a_trans, m0, kBM, g.M, kc * kBK, g.K);
            else
                stage_operand(sA, g.A, g.lda, g.a_trans, m0, kBM, g.M, kc * kBK, g.K);
        }
        if (do_b) {
            if (b_async)
                stage_async(sB, g.B, g.ldb, g.b_trans, n0, nbn, g.N, kc * kBK, g.K);
            else
                stage_operand(sB, g.B, g.ldb, g.b_trans, n0, nbn, g.N, kc * kBK, g.K);
        }
    };
    // the first chunks of B (not written by the preceding kernel), then,
    // once that kernel has completed, A; the copy groups are committed oldest
    // first, so waiting for chunk kc's second group covers its first
    const bool pb = g.pre_b != 0;
    if (pb) {
        for (int kc = 0; kc < nst; ++kc)
            stage(kc, false, true);
        tc::cp_async_commit();
    }
    tc::griddep_wait();
    tc::griddep_launch_dependents();
    for (int kc = 0; kc < nst; ++kc) {
        stage(kc, true, !pb);
        tc::cp_async_commit();
    }
    int committed = nst;
    bool ok = true;
    for (int kc = 0; kc < nchunks; ++kc) {
        const int s = kc % kStages;
        // this thread's copies of chunk kc have landed (later chunks may still fly)
        tc::cp_async_wait(min(committed - kc - 1, kStages - 1));
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(stage0 + s * stage_bytes), b0 = a0 + kTileA;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, 1024);
                const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, 1024);
                tc::mma_bf16(taddr, ad, bd, idesc, (kc | kk) != 0);
            }
            tc::mma_commit(&bars[s]);
        }
        if (kc + nst < nchunks) {
            // stage s is refilled with chunk kc + nst once chunk kc's MMAs are done
            if (!tc::mbar_wait(&bars[s], (kc / kStages) & 1, kWaitLimit))
                ok = false;
            stage(kc + nst, true, true);
            tc::cp_async_commit();
            ++committed;
        }
    }
    if (threadIdx.x == 0)
        tc::mma_commit(&bars[kStages]);
    if (!tc::mbar_wait(&bars[kStages], 0, kWaitLimit))
        ok = false;
    if (!ok && g.status)
        atomicExch(g.status, (int32_t)JL_ETIMEOUT);
    tc::tc_fence_after();

    // ---------------- epilogue: thread (row r, column quarter q) ----------------
    // Warp w reads tensor-memory lanes 32 (w % 4) .. +31 (rows) and takes the
    // column quarter q = w / 4 of them, so four threads share a row and four
    // warps share each scheduler.
    const int r = (warp & 3) * 32 + lane;
    const int q = warp >> 2;
    const int row = m0 + r;
    const bool in = row < g.M;
    const uint32_t tw = taddr + ((uint32_t)((warp & 3) * 32) << 16);

    if constexpr (EPI == EPI_SOFTMAX) {
        // the four quarters' values of each row, combined in quarter order
        auto row_combine = [&](float v, bool is_max) -> float {
            __syncthreads();
            xch[q * kBM + r] = v;
            __syncthreads();
            const float a = xch[r], b = xch[kBM + r], c = xch[2 * kBM + r], d = xch[3 * kBM + r];
            return is_max ? fmaxf(fmaxf(a, b), fmaxf(c, d)) : (a + b) + (c + d);
        };
        // quarter q holds logits q*32 .. q*32+31 of its row (BN <= 128)
        constexpr float kLog2e = 1.4426950408889634f;
        float z[32];
        float mq = -INFINITY;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c0 = q * 32 + h * 16;
            if (c0 < g.BN) {
                float v[16];
                tc::tmem_ld16(tw + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = c0 + j;
                    const float zz = col < g.N ? v[j] + g.bias[col] : -INFINITY;
                    z[h * 16 + j] = zz;
                    mq = fmaxf(mq, zz);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    z[h * 16 + j] = -INFINITY;
            }
        }
        const float mx = row_combine(mq, true);
        float sq = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (q * 32 + j < g.N)
                sq += ex2_approx((z[j] - mx) * kLog2e);
        const float sum = row_combine(sq, false);
        const float inv = 1.f / sum;
        const float lse = mx + logf(sum);
        float ent = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = q * 32 + j;
            if (col < g.N) {
                const float p = ex2_approx((z[j] - mx) * kLog2e) * inv;
                if (p > 0.f)
                    ent -= p * (z[j] - lse);
                if (g.probs && in)
                    g.probs[(size_t)row * g.ldp + col] = p;
            }
        }
        const float ent_row = row_combine(ent, false);
        if (in && g.score && q == 0)
            g.score[row] = ent_row;
    } else if constexpr (EPI == EPI_F32) {
        const bool vec_out = (g.ld_out32 & 3) == 0 && (reinterpret_cast<uintptr_t>(g.out_f32) & 15) == 0;
        for (int c0 = n0 + 16 * q; c0 < n0 + nbn; c0 += 64) {
            float v[16];
            tc::tmem_ld16(tw + (uint32_t)(c0 - n0), v);
            if (!in)
                continue;
            float *o = g.out_f32 + (size_t)row * g.ld_out32 + c0;
            if (vec_out && c0 + 16 <= g.N) {
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4)
                    reinterpret_cast<float4 *>(o)[k4] = make_float4(v[4 * k4], v[4 * k4 + 1], v[4 * k4 + 2],
                                                                    v[4 * k4 + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < g.N)
                        o[j] = v[j];
            }
        }
    } else {
        // quarter q takes columns n0 + 16 q (+ 64 k) of the CTA's nbn
        for (int c0 = n0 + 16 * q; c0 < n0 + nbn; c0 += 64) {
            float v[16];
            tc::tmem_ld16(tw + (uint32_t)(c0 - n0), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = c0 + j;
                float x = 0.f;
                if (col < g.N && in) {
                    x = v[j] + g.bias[col];
                    if (g.relu)
                        x = fmaxf(x, 0.f);
                }
                v[j] = x;
            }
            if (in) {
                if (c0 + 16 <= g.N) {
                    uint4 *op = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld_out + c0);
                    op[0] = make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]),
                                       tc::pack_bf16x2(v[4], v[5]), tc::pack_bf16x2(v[6], v[7]));
                    op[1] = make_uint4(tc::pack_bf16x2(v[8], v[9]), tc::pack_bf16x2(v[10], v[11]),
                                       tc::pack_bf16x2(v[12], v[13]), tc::pack_bf16x2(v[14], v[15]));
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < g.N)
                            g.out_bf16[(size_t)row * g.ld_out + c0 + j] = __float2bfloat16_rn(v[j]);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(taddr, 256);
}

// Fourier feature of frequency row (b0, b1): t = b0*cr + b1*ci turns,
// reduced to r = t - rint(t) in [-1/2, 1/2] (exact in binary32), then
// sin(2 pi r) and cos(2 pi r) with the hardware approximations on [-pi, pi]
// (absolute error ~1e-6, far below the bfloat16 rounding that follows).
__device__ __forceinline__ void fourier_pair(float b0, float b1, float cr, float ci, float &s, float &c)
{
    const float t = __fadd_rn(__fmul_rn(b0, cr), __fmul_rn(b1, ci));
    const float r = __fsub_rn(t, rintf(t));
    const float ang = __fmul_rn(6.28318530717958647692f, r);
    __sincosf(ang, &s, &c);
}

// ---------------------------------------------------------------------------
// Fused forward for screening: features -> three products -> softmax and
// entropy in one persistent kernel, activations kept on the SM.
// Weights are pre-packed in global memory as shared-memory images of the
// K-major core-matrix layout: W1 as two 256x32 K-chunks, W2 as eight 256x32
// and W3 as four 112x64, all fourteen streamed per tile through a four-slot
// ring of 16 KB slots with cp.async.bulk (completion as mbarrier transaction
// bytes); the four W3 chunks fit the ring at once, so they all arrive while
// the second epilogue runs.  The chunks stay L2-resident across CTAs.
// ---------------------------------------------------------------------------
static constexpr int kChK = 32;                              // K width of a weight chunk
static constexpr int kImgW = 256 * kChK * 2;                 // 16 KB: 256 rows x 32 k
static constexpr int kImgW3 = kBinsPad * 64 * 2;             // 14 KB: 112 rows x 64 k
static constexpr int kChunksPerTile = 2 + 8 + 4;             // W1, W2, W3 (the forward's chunks)
static constexpr int kRing = 4;                              // weight slots (16 KB)
static_assert((kRing & (kRing - 1)) == 0, "the ring size is a power of two");
// Packed images: chunks 0..13 as above, then for the training step's
// backward W3^T (14..17: 256 rows x 32 bins, zero past bin 101) and W2^T
// (18..25: 256 rows x 32 k).
static constexpr size_t kPackBytes = 22 * (size_t)kImgW + 4 * (size_t)kImgW3;
// shared-memory map of the fused kernel (bytes): two 128-row halves
static constexpr int kFsPhi = 0;                               // 2 x (128 x 64 bf16)
static constexpr int kFsH = kFsPhi + 2 * kBM * kIn * 2;        // 2 x (128 x 256 bf16)
static constexpr int kFsWB = kFsH + 2 * kBM * kHid * 2;        // kRing x 16 KB weight chunks
static constexpr int kFsB3 = kFsWB + kRing * kImgW;            // b3 (112 fp32), Fourier B (64 fp32)
static constexpr int kFsX = kFsB3 + (kBinsPad + 64) * 4;       // softmax partials: 256 rows x 2 fp32
static constexpr int kFsBar = kFsX + 2 * kBM * 2 * 4;          // mbarriers, TMEM holder, abort flag
static constexpr int kFusedSmem = kFsBar + 24 * 8;
static_assert(kFusedSmem <= 232448, "fused forward exceeds the shared-memory limit");
static constexpr int kFusedEpiWarps = 16;                      // two per row (column halves)
static constexpr int kFusedThreads = (kFusedEpiWarps + 2) * 32;  // + MMA warp + loader warp

// Byte offset and size of chunk j (0..25) in the packed images.
__host__ __device__ inline size_t chunk_offset(int j, uint32_t &bytes)
{
    if (j < 10) {
        bytes = kImgW;
        return (size_t)j * kImgW;
    }
    if (j < kChunksPerTile) {
        bytes = kImgW3;
        return 10 * (size_t)kImgW + (size_t)(j - 10) * kImgW3;
    }
    bytes = kImgW;
    return 10 * (size_t)kImgW + 4 * (size_t)kImgW3 + (size_t)(j - kChunksPerTile) * kImgW;
}

// bf16 of w at element (n, k) of the matrix that chunks j0.. hold as K-chunks
// of 8 G columns: chunk j0 + k / (8 G), core matrix (n / 8, (k % 8G) / 8) at
// ((n / 8) * G + (k % 8G) / 8) * 128, row n % 8 at 16 bytes, column k % 8 at 2.
__device__ __forceinline__ void put_image(uint8_t *pack, int j0, int G, int n, int k, float w)
{
    uint32_t bytes;
    const int kw = 8 * G;
    const size_t off = chunk_offset(j0 + k / kw, bytes);
    const int kk = k % kw;
    *reinterpret_cast<__nv_bfloat16 *>(pack + off + (((n >> 3) * G + (kk >> 3)) << 7) + ((n & 7) << 4) +
                                       ((kk & 7) << 1)) = __float2bfloat16_rn(w);
}

// The image positions of parameter i (value w): W1 once, W2 and W3 twice
// (as stored and transposed), biases none.
__device__ __forceinline__ void pack_param(uint8_t *pack, int i, float w)
{
    if (i < kOffB1) {
        const int o = (i - kOffW1) / kIn, k = (i - kOffW1) % kIn;
        put_image(pack, 0, 4, o, k, w);
    } else if (i >= kOffW2 && i < kOffB2) {
        const int o = (i - kOffW2) / kHid, k = (i - kOffW2) % kHid;
        put_image(pack, 2, 4, o, k, w);                 // W2[o][k]
        put_image(pack, 18, 4, k, o, w);                // W2^T[k][o]
    } else if (i >= kOffW3 && i < kOffB3) {
        const int b = (i - kOffW3) / kHid, h = (i - kOffW3) % kHid;
        put_image(pack, 10, 8, b, h, w);                // W3[b][h]
        put_image(pack, 14, 4, h, b, w);                // W3^T[h][b]
    }
}

// All image positions from the binary32 parameters (the padding stays as
// the zeros written when the images were allocated).
__global__ void pack_params_kernel(const float *__restrict__ p, uint8_t *__restrict__ pack)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNumParams)
        pack_param(pack, i, p[i]);
}

struct FusedArgs {
    const float *c;            // n x 2
    int64_t n;
    const uint8_t *pack;       // packed images
    const float *params;       // binary32 parameter block (biases)
    const float *B;            // Fourier matrix 32 x 2
    float *probs;              // n x 101 or NULL
    float *score;              // n or NULL
    int32_t *status;
};

// Warp-specialised fused forward over 256-row tiles (two 128-row halves,
// each with its own 256-column TMEM accumulator; 512 columns allocated).
//   loader (warp 17, one thread): streams the fourteen weight chunks of every
//     tile (W1 x 2 and W2 x 8 of 16 KB, W3 x 4 of 14 KB) into a four-slot ring
//     as soon as a slot's previous MMAs have completed;
//   MMA issuer (warp 16, one thread): issues each chunk's MMAs for both
//     halves, so every chunk is read from L2 once per 256 rows;
//   epilogue (warps 0..15): warp w serves TMEM lane quarter (w & 3) of half
//     (w >> 2) & 1 and column half w >> 3, so each row has two threads.  They
//     build Fourier features, turn accumulators into relu(D + b) bf16
//     activations in shared memory, and form softmax and entropy.
// Hand-offs are mbarriers: full / empty (ring slots), feat / h1 / h2 / tfree
// (one arrival per epilogue warp, waited by the MMA issuer) and acc (MMA
// completion, waited by the epilogue).  The next tile's features are built while product 2 runs, and
// its product 1 may start while the softmax of this tile is still computed.
// Every wait is bounded; a timeout sets a shared abort flag that ends all
// other waits, in-flight copies and MMAs are waited for, TMEM is freed and
// the status word reads JL_ETIMEOUT.  (One issuing thread that also refilled
// the ring waited for each chunk's MMAs before the next copy, which tied the
// products to MMA completion latency; the two roles are separate warps.)
__global__ void __launch_bounds__(kFusedThreads, 1) fused_forward_kernel(const __grid_constant__ FusedArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sPhi = sm + kFsPhi;
    uint8_t *sH = sm + kFsH;
    uint8_t *sWB = sm + kFsWB;
    float *b3 = reinterpret_cast<float *>(sm + kFsB3);
    float *Bs = b3 + kBinsPad;
    float2 *xbuf = reinterpret_cast<float2 *>(sm + kFsX);           // [256 rows]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kFsBar);
    uint64_t *full = bars, *empty = bars + kRing, *acc = bars + 2 * kRing, *feat = acc + 1, *h1b = acc + 2,
             *h2b = acc + 3, *tfree = acc + 4, *fin = acc + 5;
    uint32_t *holder = reinterpret_cast<uint32_t *>(acc + 6);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(acc + 7);
    uint64_t *pairb = acc + 8;  // [8]: the two warps serving the same rows (w, w + 8)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (a.n + 2 * kBM - 1) / (2 * kBM);
    if (blockIdx.x >= ntiles)
        return;
    const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);

    if (warp == 0)
        tc::tmem_alloc(holder, 512);
    for (int i = threadIdx.x; i < kBinsPad; i += blockDim.x)
        b3[i] = i < kBins ? a.params[kOffB3 + i] : 0.f;
    if (threadIdx.x < 64)
        Bs[threadIdx.x] = a.B[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRing; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(acc, 1);
        tc::mbar_init(feat, kFusedEpiWarps);
        tc::mbar_init(h1b, kFusedEpiWarps);
        tc::mbar_init(h2b, kFusedEpiWarps);
        tc::mbar_init(tfree, kFusedEpiWarps);
        tc::mbar_init(fin, 1);
        for (int i = 0; i < 8; ++i)
            tc::mbar_init(&pairb[i], 2);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = *holder;

    const uint8_t *gpack = reinterpret_cast<const uint8_t *>(a.pack);
    const int total_chunks = my_tiles * kChunksPerTile;
    if (warp == kFusedEpiWarps + 1) {
        // ------------------------------- loader -------------------------------
        // chunk q goes to slot q % kRing once the MMAs of chunk q - kRing have
        // completed (their commit arrives on empty[slot])
        if (lane == 0) {
            int issued = 0;
            for (int q = 0; q < total_chunks; ++q) {
                const int slot = q % kRing;
                if (q >= kRing && !tc::mbar_wait_or_abort(&empty[slot], ((q / kRing) - 1) & 1, kWaitLimit, abort_flag))
                    break;
                uint32_t bytes;
                const size_t off = chunk_offset(q % kChunksPerTile, bytes);
                tc::bulk_load(sWB + slot * kImgW, gpack + off, bytes, &full[slot]);
                ++issued;
            }
            // the last kRing copies issued sit in distinct slots: let them land
            for (int q = issued - kRing; q < issued; ++q)
                if (q >= 0)
                    tc::mbar_wait(&full[q % kRing], (q / kRing) & 1, kWaitLimit);
        }
    } else if (warp == kFusedEpiWarps) {
        // ------------------------------ MMA issuer ----------------------------
        if (lane == 0) {
            bool okp = true;
            // wait for chunk q, issue both halves' MMAs (two K-steps of 16) and
            // release the slot to the loader when they complete
            // ksteps: K steps of 16 in the chunk (2 for W1/W2, 4 for W3);
            // b_sbo: the chunk image's 8-row group stride (128 * K groups)
            // (descriptors are built once per call and advanced by adding
            // offsets / 16 to their start-address field; the wait probes the
            // barrier once before entering the bounded, abort-aware loop)
            auto run_chunk = [&](int q, uint32_t a0, uint32_t a1, uint32_t a_sbo, uint32_t n_rows, bool first,
                                 int ksteps, uint32_t b_sbo) -> bool {
                const int b = q & (kRing - 1);
                const uint32_t par = (uint32_t)(q / kRing) & 1u;
                if (!tc::mbar_try_wait(&full[b], par) &&
                    !tc::mbar_wait_or_abort(&full[b], par, kWaitLimit, abort_flag))
                    return false;
                tc::tc_fence_after();
                const uint32_t idesc = tc::idesc_bf16(kBM, n_rows);
                const uint64_t bd0 = tc::smem_desc(tc::smem_u32(sWB + b * kImgW), 128, b_sbo);
                const uint64_t ad0 = tc::smem_desc(a0, 128, a_sbo), ad1 = tc::smem_desc(a1, 128, a_sbo);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ab = h ? ad1 : ad0;
                    for (int kk = 0; kk < ksteps; ++kk)
                        tc::mma_bf16(taddr + (uint32_t)(h * 256), ab + (uint64_t)(16 * kk), bd0 + (uint64_t)(16 * kk),
                                     idesc, (first && kk == 0) ? 0u : 1u);
                }
                tc::mma_commit(&empty[b]);
                return true;
            };
            const uint32_t phi0 = tc::smem_u32(sPhi), phi1 = tc::smem_u32(sPhi + kBM * kIn * 2);
            const uint32_t hh0 = tc::smem_u32(sH), hh1 = tc::smem_u32(sH + kBM * kHid * 2);
            for (int it = 0; it < my_tiles && okp; ++it) {
                const int q0 = it * kChunksPerTile;
                // product 1: the tile's features are in place and the previous
                // tile's logits have been read out of TMEM
                okp = tc::mbar_wait_or_abort(feat, it & 1, kWaitLimit, abort_flag);
                if (okp && it > 0)
                    okp = tc::mbar_wait_or_abort(tfree, (it - 1) & 1, kWaitLimit, abort_flag);
                if (!okp)
                    break;
                tc::tc_fence_after();
                // K chunk j of Phi starts at core-matrix column 4 j (512 bytes)
                for (int j = 0; j < 2 && okp; ++j)
                    okp = run_chunk(q0 + j, phi0 + j * 512, phi1 + j * 512, 1024, kHid, j == 0, 2, 512);
                if (!okp)
                    break;
                tc::mma_commit(acc);
                // product 2: H1 written by every epilogue warp
                okp = tc::mbar_wait_or_abort(h1b, it & 1, kWaitLimit, abort_flag);
                if (!okp)
                    break;
                tc::tc_fence_after();
                for (int j = 0; j < 8 && okp; ++j)
                    okp = run_chunk(q0 + 2 + j, hh0 + j * 512, hh1 + j * 512, 4096, kHid, j == 0, 2, 512);
                if (!okp)
                    break;
                tc::mma_commit(acc);
                // product 3: H2 written
                okp = tc::mbar_wait_or_abort(h2b, it & 1, kWaitLimit, abort_flag);
                if (!okp)
                    break;
                tc::tc_fence_after();
                // W3 K chunk j (64 wide) starts at core-matrix column 8 j (1024 bytes)
                for (int j = 0; j < 4 && okp; ++j)
                    okp = run_chunk(q0 + 10 + j, hh0 + j * 1024, hh1 + j * 1024, 4096, kBinsPad, j == 0, 4, 1024);
                if (!okp)
                    break;
                tc::mma_commit(acc);
            }
            // every product issued has completed before TMEM is freed
            tc::mma_commit(fin);
            tc::mbar_wait(fin, 0, kWaitLimit);
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int quarter = warp & 3, half = (warp >> 2) & 1, ch = warp >> 3;
        const int r = quarter * 32 + lane;  // row within the half
        const uint32_t tw = taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 256);
        uint8_t *myPhi = sPhi + half * (kBM * kIn * 2);
        uint8_t *myH = sH + half * (kBM * kHid * 2);
        const float *b1g = a.params + kOffB1, *b2g = a.params + kOffB2;
        uint32_t acc_uses = 0;

        auto arrive = [&](uint64_t *bar) {
            __syncwarp();
            if (lane == 0)
                tc::mbar_arrive(bar);
        };
        auto wait_acc = [&]() -> bool {
            const bool w = tc::mbar_wait_or_abort(acc, acc_uses & 1, kWaitLimit, abort_flag);
            ++acc_uses;
            tc::tc_fence_after();
            return w;
        };
        // this thread's 16 Fourier frequencies (16 ch .. 16 ch + 15) of its row
        auto make_features = [&](int64_t tile) {
            const int64_t row = tile * (2 * kBM) + half * kBM + r;
            float cr = 0.f, ci = 0.f;
            if (row < a.n) {
                cr = a.c[2 * row];
                ci = a.c[2 * row + 1];
            }
            uint32_t sv[8], cv[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const int f0 = 16 * ch + j;
                float s0, c0, s1, c1;
                fourier_pair(Bs[2 * f0], Bs[2 * f0 + 1], cr, ci, s0, c0);
                fourier_pair(Bs[2 * f0 + 2], Bs[2 * f0 + 3], cr, ci, s1, c1);
                sv[j >> 1] = tc::pack_bf16x2(s0, s1);
                cv[j >> 1] = tc::pack_bf16x2(c0, c1);
            }
            if (row >= a.n) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    sv[j] = cv[j] = 0u;
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                *reinterpret_cast<uint4 *>(myPhi + ((r >> 3) * 8 + 2 * ch + g) * 128 + (r & 7) * 16) =
                    make_uint4(sv[4 * g], sv[4 * g + 1], sv[4 * g + 2], sv[4 * g + 3]);
                *reinterpret_cast<uint4 *>(myPhi + ((r >> 3) * 8 + 4 + 2 * ch + g) * 128 + (r & 7) * 16) =
                    make_uint4(cv[4 * g], cv[4 * g + 1], cv[4 * g + 2], cv[4 * g + 3]);
            }
            tc::fence_proxy_async_smem();
        };
        // relu(D + b) as bf16 into this half's H image, this thread's 128 columns
        auto hidden_epilogue = [&](const float *bias) {
#pragma unroll 1
            for (int c0 = 128 * ch; c0 < 128 * ch + 128; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tw + c0, v);
                uint32_t wv[16];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 bq = __ldg(reinterpret_cast<const float4 *>(bias + c0 + 4 * q));
                    wv[2 * q] = tc::pack_relu_bf16x2(__fadd_rn(v[4 * q], bq.x), __fadd_rn(v[4 * q + 1], bq.y));
                    wv[2 * q + 1] = tc::pack_relu_bf16x2(__fadd_rn(v[4 * q + 2], bq.z), __fadd_rn(v[4 * q + 3], bq.w));
                }
                const int g = c0 >> 3;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4 *>(myH + ((r >> 3) * 32 + g + q) * 128 + (r & 7) * 16) =
                        make_uint4(wv[4 * q], wv[4 * q + 1], wv[4 * q + 2], wv[4 * q + 3]);
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
        };

        // bounded rendezvous of warps w and w + 8 (never a hardware barrier:
        // a partner that gave up must not leave the other waiting forever)
        uint32_t pair_uses = 0;
        auto pair_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0)
                tc::mbar_arrive(&pairb[warp & 7]);
            const bool w = tc::mbar_wait_or_abort(&pairb[warp & 7], pair_uses & 1, kWaitLimit, abort_flag);
            ++pair_uses;
            return w;
        };

        make_features(blockIdx.x);
        arrive(feat);
        const float kLog2e = 1.4426950408889634f;
        for (int it = 0; it < my_tiles; ++it) {
            const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
            const int64_t row = tile * (2 * kBM) + half * kBM + r;
            const bool in = row < a.n;
            // ---- product 1 done: activations 1 ----
            if (!wait_acc())
                break;
            hidden_epilogue(b1g);
            arrive(h1b);
            // the Phi images were consumed by product 1: next tile's features
            if (it + 1 < my_tiles) {
                make_features(tile + gridDim.x);
                arrive(feat);
            }
            // ---- product 2 done: activations 2 ----
            if (!wait_acc())
                break;
            hidden_epilogue(b2g);
            arrive(h2b);
            // ---- product 3 done: logits of this thread's 56 columns ----
            if (!wait_acc())
                break;
            float z[56];
            const int cb = 56 * ch;
            tc::tmem_ld32(tw + cb, z);
            tc::tmem_ld16(tw + cb + 32, *reinterpret_cast<float(*)[16]>(z + 32));
            tc::tmem_ld8(tw + cb + 48, z + 48);
            tc::tc_fence_before();
            arrive(tfree);  // TMEM may now take the next tile's product 1
            // partial softmax over the valid columns of this thread:
            // m = max z, S = sum 2^((z - m) log2 e), T = sum e z;
            // sent as L = m + log S (log-sum-exp) and A = T / S (mean logit)
            const int nv = ch ? (kBins - 56) : 56;
            float mx = -INFINITY;
#pragma unroll
            for (int j = 0; j < 56; ++j) {
                z[j] = __fadd_rn(z[j], b3[cb + j]);
                if (j < nv)
                    mx = fmaxf(mx, z[j]);
            }
            const float mb = -__fmul_rn(mx, kLog2e);
            float S = 0.f, Tz = 0.f;
#pragma unroll
            for (int j = 0; j < 56; ++j) {
                if (j < nv) {
                    const float e = ex2_approx(__fmaf_rn(z[j], kLog2e, mb));
                    S = __fadd_rn(S, e);
                    Tz = __fmaf_rn(e, z[j], Tz);
                }
            }
            const float Lc = __fadd_rn(mx, logf(S));
            const float Ac = __fdiv_rn(Tz, S);
            const int xi = half * kBM + r;
            if (ch)
                xbuf[xi] = make_float2(Lc, Ac);
            if (!pair_sync())
                break;
            float L = 0.f;
            if (!ch) {
                const float2 o = xbuf[xi];
                // L = logaddexp(Lc, o.x); entropy = L - (w0 A0 + w1 A1), w = e^(Lc - L)
                const float hi = fmaxf(Lc, o.x), lo = fminf(Lc, o.x);
                L = __fadd_rn(hi, log1pf(expf(__fsub_rn(lo, hi))));
                const float w0 = expf(__fsub_rn(Lc, L)), w1 = expf(__fsub_rn(o.x, L));
                const float Am = __fadd_rn(__fmul_rn(w0, Ac), __fmul_rn(w1, o.y));
                if (in && a.score)
                    a.score[row] = __fsub_rn(L, Am);
                if (a.probs)
                    xbuf[xi].x = L;
            }
            if (a.probs) {
                if (!pair_sync())
                    break;
                if (ch)
                    L = xbuf[xi].x;
                if (in) {
                    const float lb = -__fmul_rn(L, kLog2e);
                    float *prow = a.probs + (size_t)row * kBins + cb;
#pragma unroll
                    for (int j = 0; j < 56; ++j)
                        if (j < nv)
                            prow[j] = ex2_approx(__fmaf_rn(z[j], kLog2e, lb));
                }
            }
        }
    }
    if (*abort_flag && a.status)
        atomicExch(a.status, (int32_t)JL_ETIMEOUT);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(taddr, 512);
}

// ---------------------------------------------------------------------------
// Small kernels: features, Adam, weight casts, histogram L1.
// ---------------------------------------------------------------------------
// phi[i] = [sin(2 pi t_j), cos(2 pi t_j)], t_j = B_j . C_i, j < 32 (bf16 out).
// Optional gather: row i takes C[idx[i]].
__global__ void features_kernel(const float *__restrict__ c, const int32_t *__restrict__ idx, int64_t n,
                                const float *__restrict__ Bm, __nv_bfloat16 *__restrict__ phi)
{
    tc::griddep_wait();
    tc::griddep_launch_dependents();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t >> 5;
    const int j = (int)(t & 31);
    if (i >= n)
        return;
    const int64_t src = idx ? idx[i] : i;
    const float cr = c[2 * src], ci = c[2 * src + 1];
    float s, co;
    fourier_pair(Bm[2 * j], Bm[2 * j + 1], cr, ci, s, co);
    phi[i * kIn + j] = __float2bfloat16_rn(s);
    phi[i * kIn + kFreq + j] = __float2bfloat16_rn(co);
}

// bf16 weight copies, contiguous: W1, W2, W3 as stored ([out][in]); the
// operands of the layered forward.
static constexpr int kWbW = kHid * kIn + kHid * kHid + kBins * kHid;  // W1 | W2 | W3

__global__ void cast_weights_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kIn)
        wb[i] = __float2bfloat16_rn(p[kOffW1 + i]);
    else if (i < kHid * kIn + kHid * kHid)
        wb[i] = __float2bfloat16_rn(p[kOffW2 + (i - kHid * kIn)]);
    else if (i < kWbW)
        wb[i] = __float2bfloat16_rn(p[kOffW3 + (i - kHid * kIn - kHid * kHid)]);
}

// Target histograms (n rows of 101) copied to rows of kTrTP floats, zero
// padded, so that the training step fetches each row with one bulk copy.
__global__ void pad_targets_kernel(const float *__restrict__ src, int64_t n, float *__restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * kTrTP) {
        const int64_t row = i / kTrTP;
        const int col = (int)(i - row * kTrTP);
        dst[i] = col < kBins ? src[row * kBins + col] : 0.f;
    }
}

// Where one batch's gradient partials live: the per-tile partials of the
// three weight gradients and the per-tile column sums of the bias gradients
// and of the losses (train_step_kernel writes one of each per 128-row tile).  They are summed in a fixed order wherever a
// gradient is needed (deterministic, so a resumed run continues bit for bit).
struct GradParts {
    const float *ws1, *ws2, *ws3;  // [S][256 x 64], [S][256 x 256], [S][101 x 256]
    const float *pb1, *pb2, *pb3;  // [ctas][256]
    const float *loss_part;        // [ctas]
    int S, ctas;
};

__device__ __forceinline__ float grad_of(const GradParts &q, int i)
{
    const float *src;
    int stride, nterm;
    if (i < kOffB1) {
        src = q.ws1 + (i - kOffW1), stride = kHid * kIn, nterm = q.S;
    } else if (i < kOffW2) {
        src = q.pb1 + (i - kOffB1), stride = 256, nterm = q.ctas;
    } else if (i < kOffB2) {
        src = q.ws2 + (i - kOffW2), stride = kHid * kHid, nterm = q.S;
    } else if (i < kOffW3) {
        src = q.pb2 + (i - kOffB2), stride = 256, nterm = q.ctas;
    } else if (i < kOffB3) {
        src = q.ws3 + (i - kOffW3), stride = kBins * kHid, nterm = q.S;
    } else {
        src = q.pb3 + (i - kOffB3), stride = 256, nterm = q.ctas;
    }
    // the terms in index order; loaded eight at a time so that their
    // latencies overlap (the sum itself stays sequential)
    float acc = 0.f;
    int r = 0;
    for (; r + 8 <= nterm; r += 8) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            t[u] = src[(size_t)(r + u) * stride];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            acc += t[u];
    }
    for (; r < nterm; ++r)
        acc += src[(size_t)r * stride];
    return acc;
}

__device__ __forceinline__ float loss_of(const GradParts &q)
{
    float acc = 0.f;
    for (int r = 0; r < q.ctas; ++r)
        acc += q.loss_part[r];
    return acc;
}

// The gradient of every parameter and the batch's loss sum, from the partials.
__global__ void grad_reduce_kernel(const __grid_constant__ GradParts q, float *__restrict__ grad, float *loss)
{
    tc::griddep_wait();
    tc::griddep_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNumParams)
        grad[i] = grad_of(q, i);
    if (i == 0 && loss)
        *loss = loss_of(q);
}

// Adam on the whole parameter block with each gradient summed from the
// batch's partials; bc1 = 1 - beta1^t and bc2 = 1 - beta2^t are the bias
// corrections of step t (1 for the first).  Also refreshes the packed bf16
// weight images (pack_param) and writes the batch's loss sum to *loss.
__global__ void adam_kernel(const __grid_constant__ GradParts q, float *__restrict__ p, float *__restrict__ m,
                            float *__restrict__ v, uint8_t *__restrict__ pack, float bc1, float bc2, float lr,
                            float beta1, float beta2, float eps, float *loss)
{
    // The next training step may be scheduled at once (its blocks take SMs
    // as this step's blocks leave them, and read nothing this kernel writes
    // before their own wait); the moments and parameters were final before
    // the training step this kernel follows began, so they are read before
    // waiting for it.
    tc::griddep_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float m0 = 0.f, v0 = 0.f, p0 = 0.f;
    if (i < kNumParams) {
        m0 = m[i];
        v0 = v[i];
        p0 = p[i];
    }
    tc::griddep_wait();
    if (i == 0 && loss)
        *loss = loss_of(q);
    if (i < kNumParams) {
        const float g = grad_of(q, i);
        const float mi = beta1 * m0 + (1.f - beta1) * g;
        const float vi = beta2 * v0 + (1.f - beta2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float upd = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        const float w = p0 - upd;
        p[i] = w;
        pack_param(pack, i, w);
    }
}

// ---------------------------------------------------------------------------
// Fused training step: one CTA per 128-row tile of the batch runs the forward
// and the backward of its rows with the activations kept on the SM, and
// leaves the tile's partial gradients for adam_kernel / grad_reduce_kernel.
//
// Shared memory holds the tile's features Phi (128 x 64), H1 and H2
// (128 x 256) and the logit error dZ (128 x 128, bins past 101 zero), each
// in the K-major core-matrix layout of the forward products with every
// column in one row group: core matrix (row / 8, column / 8) at byte
// ((row / 8) * G + column / 8) * 128, G = columns / 8.  The weight-gradient
// products contract over the rows and read the same buffers as MN-major
// operands (same core matrices; K-direction stride G * 128 in the LBO field,
// M/N-direction stride 128 in the SBO field).  They are computed transposed
// (dW^T = X^T dY, the input unit on the tensor-memory lanes) so that each
// warp stores 32 consecutive floats of a parameter row at a time.
//
// Weights arrive as the packed chunk images that adam_kernel maintains
// (pack_param), by cp.async.bulk into a ring of 16 KB slots: three of their
// own, plus two in the dZ buffer while dZ is not live.  Roles: thread 0
// issues the MMAs of a product as its chunks land (full barriers) and frees
// each slot by tcgen05.commit (empty barriers); thread 32 refills freed
// slots; the first chunks of each product are requested while the previous
// epilogue runs.  Phases:
//   P1  D = Phi W1^T        -> H1 = relu(D + b1)
//   P2  D = H1 W2^T         -> H2 = relu(D + b2)
//   P3  D = H2 W3^T         -> softmax; dZ = (p - t) / batch rows, loss, db3
//   P4  dW3^T = H2^T dZ;  P5  D = dZ W3 -> dZ2 = D * [H2 > 0] over H2, db2
//   P6  dW2^T = H1^T dZ2 (two halves of the input units)
//   P7  D = dZ2 W2          -> dZ1 = D * [H1 > 0] over H1, db1
//   P8  dW1^T = Phi^T dZ1   (M = 128 over Phi's 64 columns: lanes 64.. unused)
// Five CTAs share a tile (blockIdx.y = role): each runs P1..P3 for the
// tile's rows, then roles 0 and 2 take the chain P5, P7, P8 for hidden units
// 0..127 and 128..255 (each streams those rows of the W2^T chunks, and forms
// its half of dZ1, db1 and dW1), roles 1 and 3 their own P5 and dW2 for input
// units 0..127 and 128..255 (each with those units' db2), role 4 the loss,
// db3 and P4 (dW3) --
// so the long partial-gradient stores and the sums run beside the chain
// instead of on it, and the chain itself is halved.
// Bias gradients are column sums of the unrounded binary32 errors in a fixed
// order (a butterfly within each warp, then the four row groups in order).
// Every wait is bounded; one that gives up sets *status to JL_ETIMEOUT.
// ---------------------------------------------------------------------------
static constexpr int kTrThreads = 512;
static constexpr int kTrRoles = 5;  // CTAs per 128-row tile
static constexpr int kTrPhi = 0;
static constexpr int kTrH1 = kTrPhi + kBM * kIn * 2;
static constexpr int kTrH2 = kTrH1 + kBM * kHid * 2;
static constexpr int kTrDZ = kTrH2 + kBM * kHid * 2;     // dZ, or ring slots 3 and 4
static constexpr int kTrDZCols = 128;                     // dZ columns held (bins, zero past 101)
static constexpr int kTrRing = kTrDZ + kBM * kTrDZCols * 2;  // ring slots 0..2
static constexpr int kTrBar = kTrRing + 3 * kImgW;        // full[5], empty[5], acc, TMEM holder
static constexpr int kTrLw = kTrBar + 128;                // [16] per-warp loss sums
static constexpr int kTrB3 = kTrLw + 64;                  // b3 (112 fp32, zero past 101)
static constexpr int kTrScratch = kTrB3 + kBinsPad * 4;   // [4][128] fp32 exchange; b1 | b2 until P3
static constexpr int kTrSmem = kTrScratch + 4 * kBM * 4;
static_assert(kTrSmem <= 232448, "training step exceeds the shared-memory limit");
static_assert(kBM * kTrTP * 4 <= kBM * kHid * 2, "targets are staged in the H2 buffer");

struct TrainArgs {
    const float *c;          // C of batch row m at c[2 * idx[m]] (idx NULL: c[2 m])
    const int32_t *idx;
    int n;                   // batch rows
    const float *target;     // target histogram of batch row m: row trow[m] (NULL: m), kTrTP floats per
                             // row (101 bins, then padding; 16-byte aligned rows)
    const int32_t *trow;
    float inv_m;             // 1 / batch rows
    const float *B;          // Fourier matrix 32 x 2
    const float *params;     // binary32 parameters (the biases are read)
    const uint8_t *pack;     // packed weight images (chunk_offset)
    float *ws1, *ws2, *ws3;  // per-tile dW1 [256 x 64], dW2 [256 x 256], dW3 [101 x 256]
    float *pb1, *pb2, *pb3;  // per-tile bias-gradient sums [256]
    float *loss_part;        // per-tile loss sums
    int32_t *status;
    // the next step's batch (as c, idx, n, target, trow above; next_n = 0:
    // none): its rows are prefetched into L2 at the end of this step
    const float *next_c;
    const int32_t *next_idx;
    int next_n;
    const float *next_target;
    const int32_t *next_trow;
};

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Byte offset of element (row, col) in a full-width K-major buffer of G
// column groups.
__device__ __forceinline__ int tr_off(int row, int col, int G)
{
    return (((row >> 3) * G + (col >> 3)) << 7) + ((row & 7) << 4) + ((col & 7) << 1);
}

// bf16 of v[0..15] (with relu: of max(v, 0)) into columns col0 .. col0 + 15
// (col0 a multiple of 8) of row `row`: two 16-byte stores.
__device__ __forceinline__ void tr_store16(uint8_t *buf, int row, int col0, int G, const float (&v)[16], bool relu)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float *w = v + 8 * h;
        uint4 u;
        if (relu) {
            u = make_uint4(tc::pack_relu_bf16x2(w[0], w[1]), tc::pack_relu_bf16x2(w[2], w[3]),
                           tc::pack_relu_bf16x2(w[4], w[5]), tc::pack_relu_bf16x2(w[6], w[7]));
        } else {
            u = make_uint4(tc::pack_bf16x2(w[0], w[1]), tc::pack_bf16x2(w[2], w[3]), tc::pack_bf16x2(w[4], w[5]),
                           tc::pack_bf16x2(w[6], w[7]));
        }
        *reinterpret_cast<uint4 *>(buf + tr_off(row, col0 + 8 * h, G)) = u;
    }
}

// Column sums over a warp: lane L holds 32 values (its row, columns 0..31);
// afterwards lane L returns the sum of column L over the 32 lanes (a
// butterfly in a fixed order, 31 exchanges; v is overwritten).
__device__ __forceinline__ float tr_colsum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const float send = upper ? v[j] : v[j + s];
            const float keep = upper ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// One product's weight stream: chunks j0 .. j0 + n - 1 of the packed
// images, K-chunks of kw (32 or 64), N rows, through ns ring slots; with
// blen > 0, bytes [boff, boff + blen) of each chunk only (a block of its rows).
struct TrStream {
    int j0, n, kw, N, ns;
    int boff = 0, blen = 0;
};

__global__ void __launch_bounds__(kTrThreads, 1) train_step_kernel(const __grid_constant__ TrainArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sPhi = sm + kTrPhi, *sH1 = sm + kTrH1, *sH2 = sm + kTrH2, *sDZ = sm + kTrDZ;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + kTrBar);
    uint64_t *empty = full + 5;
    uint64_t *accbar = full + 10;
    uint64_t *tbar = full + 11;  // the tile's target rows
    uint32_t *holder = reinterpret_cast<uint32_t *>(full + 12);
    float *lw = reinterpret_cast<float *>(sm + kTrLw);
    float *b3s = reinterpret_cast<float *>(sm + kTrB3);
    float *scratch = reinterpret_cast<float *>(sm + kTrScratch);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int role = blockIdx.y;  // the share of the backward this CTA takes
    const int m0 = tile * kBM;
    // epilogue role: row r of the tile (tensor-memory lane), column quarter qd
    const int r = (warp & 3) * 32 + lane;
    const int qd = warp >> 2;
    const int row = m0 + r;
    const bool in = row < a.n;

    if (warp == 0)
        tc::tmem_alloc(holder, 512);
    const int nrows = max(0, min(kBM, a.n - m0));  // the tile's rows in the batch
    if (threadIdx.x == 0) {
        for (int i = 0; i < 12; ++i)
            tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        // the target rows' bytes, announced before any copy is issued
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(tbar)),
                     "r"((uint32_t)(nrows * kTrTP * 4))
                     : "memory");
    }
    __syncthreads();

    // ---- inputs of the call, read before waiting for the preceding kernel ----
    // targets of the tile's rows, staged through the (idle) H2 buffer: one
    // bulk copy of a padded row per thread, completing on tbar
    if ((int)threadIdx.x < nrows) {
        const int grow = m0 + threadIdx.x;
        const int64_t trw = a.trow ? (int64_t)a.trow[grow] : (int64_t)grow;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(sH2 + threadIdx.x * kTrTP * 4)),
                     "l"(a.target + trw * kTrTP), "r"((uint32_t)(kTrTP * 4)), "r"(tc::smem_u32(tbar))
                     : "memory");
    }
    // features: thread t takes row t / 4 and frequencies 8 (t % 4) .. + 7,
    // whose sines and cosines are one 16-byte core-matrix row each
    {
        const int rr = threadIdx.x >> 2, f0 = (threadIdx.x & 3) * 8;
        const int grow = m0 + rr;
        float sv[8], cv[8];
        if (grow < a.n) {
            const int64_t src = a.idx ? (int64_t)a.idx[grow] : (int64_t)grow;
            const float cr = a.c[2 * src], ci = a.c[2 * src + 1];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                fourier_pair(a.B[2 * (f0 + j)], a.B[2 * (f0 + j) + 1], cr, ci, sv[j], cv[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                sv[j] = cv[j] = 0.f;
        }
        const uint4 us = make_uint4(tc::pack_bf16x2(sv[0], sv[1]), tc::pack_bf16x2(sv[2], sv[3]),
                                    tc::pack_bf16x2(sv[4], sv[5]), tc::pack_bf16x2(sv[6], sv[7]));
        const uint4 uc = make_uint4(tc::pack_bf16x2(cv[0], cv[1]), tc::pack_bf16x2(cv[2], cv[3]),
                                    tc::pack_bf16x2(cv[4], cv[5]), tc::pack_bf16x2(cv[6], cv[7]));
        *reinterpret_cast<uint4 *>(sPhi + tr_off(rr, f0, kIn / 8)) = us;
        *reinterpret_cast<uint4 *>(sPhi + tr_off(rr, kFreq + f0, kIn / 8)) = uc;
    }
    bool ok = tc::mbar_wait(tbar, 0, kWaitLimit);
    float tg[32];  // targets of row `row`, bins 32 qd .. 32 qd + 31 (as 16-byte reads)
    {
        const float4 *T4 = reinterpret_cast<const float4 *>(sH2 + (size_t)r * kTrTP * 4 + 32 * qd * 4);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
            // quarter 3 reads past the row's 104 floats into the next row (or
            // the idle rest of the buffer); those bins are not used
            const float4 t4 = T4[j4];
            const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                tg[4 * j4 + e] = (in && 32 * qd + 4 * j4 + e < kBins) ? tv[e] : 0.f;
        }
    }

    // weights, biases and the partial buffers belong to the preceding kernel (Adam) until it completes
    tc::griddep_wait();
    tc::griddep_launch_dependents();

    uint32_t taddr = 0;
    // slot bookkeeping (each in the one thread that uses it): parity bits of
    // the loads issued per slot (loader), of the loads consumed (MMA issuer)
    uint32_t lpar = 0, lused = 0, fpar = 0;
    uint32_t accn = 0;  // completions of the accumulator barrier waited for
    const uint32_t aPhi = tc::smem_u32(sPhi), aH1 = tc::smem_u32(sH1), aH2 = tc::smem_u32(sH2),
                   aDZ = tc::smem_u32(sDZ);
    auto slot_addr = [&](int s) -> uint8_t * { return s < 3 ? sm + kTrRing + s * kImgW : sDZ + (s - 3) * kImgW; };

    // a wait whose phase has usually completed already: one probe, then the
    // bounded loop
    auto wait_phase = [&](uint64_t *bar, uint32_t parity) {
        if (!tc::mbar_try_wait(bar, parity) && !tc::mbar_wait(bar, parity, kWaitLimit))
            ok = false;
    };
    // loader: chunk c of stream w into slot s (= c mod w.ns), once the slot's
    // previous products have completed
    auto load = [&](const TrStream &w, int c, int s) {
        const uint32_t bit = 1u << s;
        if (lused & bit)
            wait_phase(&empty[s], ((lpar >> s) & 1u) ^ 1u);
        uint32_t bytes;
        size_t off = chunk_offset(w.j0 + c, bytes);
        if (w.blen > 0) {
            off += (size_t)w.boff;
            bytes = (uint32_t)w.blen;
        }
        tc::bulk_load(slot_addr(s), a.pack + off, bytes, &full[s]);
        lpar ^= bit;
        lused |= bit;
    };
    // the first chunks of w (their slots are free: every earlier product has completed)
    // (the other lanes of a warp whose lane 0 has a single-thread role wait
    // at __syncwarp rather than spin beside it, and the warp is converged
    // again before its next warp-wide tensor-memory access)
    auto prefetch = [&](const TrStream &w) {
        if (threadIdx.x == 32)
            for (int c = 0; c < min(w.n, w.ns); ++c)
                load(w, c, c);
        __syncwarp();
    };
    // D[dcol] = A x W^T over stream w: A the K-major activation buffer at
    // a_addr (aG column groups).  The MMA issuer consumes the chunks as they
    // land; the loader refills the slots they free.
    // (The issue loop is kept short: a descriptor's start-address field,
    // bits 0..13 = address / 16, is advanced by adding offsets / 16 to a
    // descriptor built once -- no carry, shared memory being below 256 KB --
    // and the slot index is a running counter.)
    auto run = [&](const TrStream &w, uint32_t a_addr, int aG, uint32_t dcol) {
        if (threadIdx.x == 0) {
            const uint32_t idesc = tc::idesc_bf16(kBM, (uint32_t)w.N);
            const int G = w.kw / 8;
            const uint64_t ad0 = tc::smem_desc(a_addr, 128, (uint32_t)aG * 128);
            const uint64_t bring = tc::smem_desc(tc::smem_u32(sm + kTrRing), 128, (uint32_t)G * 128);
            const uint64_t bdz = tc::smem_desc(tc::smem_u32(sDZ), 128, (uint32_t)G * 128);
            const uint32_t d = taddr + dcol;
            int s = 0;
            for (int c = 0; c < w.n; ++c) {
                wait_phase(&full[s], (fpar >> s) & 1u);
                fpar ^= 1u << s;
                tc::tc_fence_after();
                const uint64_t b0 = s < 3 ? bring + (uint64_t)(s * (kImgW >> 4)) : bdz + (uint64_t)((s - 3) * (kImgW >> 4));
                const uint64_t a0 = ad0 + (uint64_t)(c * G * 8);  // K columns 8 G c .. : (c G 128 bytes) / 16
                for (int kk = 0; kk < w.kw / 16; ++kk)
                    tc::mma_bf16(d, a0 + (uint64_t)(16 * kk), b0 + (uint64_t)(16 * kk), idesc, (c | kk) != 0);
                tc::mma_commit(&empty[s]);
                s = s + 1 == w.ns ? 0 : s + 1;
            }
        } else if (threadIdx.x == 32) {
            int s = 0;  // chunk w.ns goes to slot 0
            for (int c = w.ns; c < w.n; ++c) {
                load(w, c, s);
                s = s + 1 == w.ns ? 0 : s + 1;
            }
        }
        __syncwarp();
    };
    // every product issued so far has completed
    auto commit_wait = [&]() {
        if (threadIdx.x == 0)
            tc::mma_commit(accbar);
        __syncwarp();
        if (!tc::mbar_wait(accbar, accn & 1, kWaitLimit))
            ok = false;
        ++accn;
        __syncwarp();
        tc::tc_fence_after();
    };
    // shared-memory writes of an epilogue visible to the tensor core, its
    // tensor-memory reads finished, before the next product is issued
    auto epilogue_done = [&]() {
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();
    };
    // column sums of the tile for columns c0 .. c0 + 31 (this thread: row r,
    // v[j] = column c0 + j; the four quarters hold disjoint column ranges) to
    // out[c0 + j] for c0 + j < nvalid
    // (active false, uniform over the quarter: no sums for these columns;
    // the barriers are still taken)
    auto colsums32 = [&](float (&v)[32], int c0, int nvalid, float *out, bool active = true) {
        const float s = active ? tr_colsum32(v, lane) : 0.f;
        __syncthreads();
        scratch[(warp & 3) * kBM + qd * 32 + lane] = s;
        __syncthreads();
        if (active && (warp & 3) == 0 && c0 + lane < nvalid) {
            const int cc = qd * 32 + lane;
            out[c0 + lane] = (scratch[cc] + scratch[kBM + cc]) + (scratch[2 * kBM + cc] + scratch[3 * kBM + cc]);
        }
    };
    // the four quarters' values of each row, combined in quarter order
    auto row_combine = [&](float x, bool is_max) -> float {
        __syncthreads();
        scratch[qd * kBM + r] = x;
        __syncthreads();
        const float p0 = scratch[r], p1 = scratch[kBM + r], p2 = scratch[2 * kBM + r], p3 = scratch[3 * kBM + r];
        return is_max ? fmaxf(fmaxf(p0, p1), fmaxf(p2, p3)) : (p0 + p1) + (p2 + p3);
    };
    // one thread issues a weight-gradient product D[dcol] = X^T Y over the
    // tile's 128 rows: X (M side, columns xm0 ..) and Y (N side, columns
    // yn0 ..) are full-width buffers read MN-major
    auto issue_wgrad = [&](uint32_t x_addr, int xG, int xm0, uint32_t y_addr, int yG, int N, uint32_t dcol,
                           int yn0 = 0) {
        const uint32_t idesc = tc::idesc_bf16_t(kBM, (uint32_t)N, true, true);
#pragma unroll
        for (int kk = 0; kk < kBM / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(x_addr + (uint32_t)(kk * 2 * xG * 128 + (xm0 / 8) * 128),
                                              (uint32_t)xG * 128, 128);
            const uint64_t bd = tc::smem_desc(y_addr + (uint32_t)(kk * 2 * yG * 128 + (yn0 / 8) * 128),
                                              (uint32_t)yG * 128, 128);
            tc::mma_bf16(taddr + dcol, ad, bd, idesc, kk != 0);
        }
    };

    const TrStream w1{0, 2, 32, kHid, 5}, w2{2, 8, 32, kHid, 5}, w3{10, 4, 64, kBinsPad, 5};
    const TrStream w3t{14, 4, 32, kHid, 3};
    float *ws1 = a.ws1 + (size_t)tile * kHid * kIn;
    float *ws2 = a.ws2 + (size_t)tile * kHid * kHid;
    float *ws3 = a.ws3 + (size_t)tile * kBins * kHid;

    prefetch(w1);
    // biases: b1 | b2 in the exchange buffer (idle until the softmax), b3 apart
    for (int i = threadIdx.x; i < 2 * kHid; i += blockDim.x)
        scratch[i] = a.params[i < kHid ? kOffB1 + i : kOffB2 + (i - kHid)];
    if (threadIdx.x < kBinsPad)
        b3s[threadIdx.x] = threadIdx.x < kBins ? a.params[kOffB3 + threadIdx.x] : 0.f;
    tc::fence_proxy_async_smem();  // the features
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    taddr = *holder;
    const uint32_t tw = taddr + ((uint32_t)((warp & 3) * 32) << 16);

    // bias + relu of the accumulator at column dcol into the K-major buffer
    auto hidden_epilogue = [&](uint32_t dcol, const float *bias, uint8_t *dst) {
#pragma unroll 1
        for (int c0 = 64 * qd; c0 < 64 * qd + 64; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tw + dcol + (uint32_t)c0, v);
            // the 16 biases as four broadcast 16-byte reads
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
                const float4 b4 = reinterpret_cast<const float4 *>(bias + c0)[j4];
                v[4 * j4 + 0] = in ? v[4 * j4 + 0] + b4.x : 0.f;
                v[4 * j4 + 1] = in ? v[4 * j4 + 1] + b4.y : 0.f;
                v[4 * j4 + 2] = in ? v[4 * j4 + 2] + b4.z : 0.f;
                v[4 * j4 + 3] = in ? v[4 * j4 + 3] + b4.w : 0.f;
            }
            tr_store16(dst, r, c0, kHid / 8, v, true);
        }
    };
    // error through a ReLU: the accumulator at column 0 kept where the
    // activation in buf is > 0 (bf16 sign clear, not +0), written over the
    // activation as bf16; bias-gradient sums of the unrounded values to pb
    // (unless NULL)
    // (32 columns: accumulator column tcol, buffer column c0)
    auto mask_cols = [&](uint8_t *buf, float *pb, int tcol, int c0, int sum_lo = 0, int sum_hi = kHid) {
        {
            float v[32];
            tc::tmem_ld32(tw + (uint32_t)tcol, v);
#pragma unroll
            for (int g8 = 0; g8 < 4; ++g8) {
                const uint4 mq = *reinterpret_cast<const uint4 *>(buf + tr_off(r, c0 + 8 * g8, kHid / 8));
                const uint32_t mk[4] = {mq.x, mq.y, mq.z, mq.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t bits = (mk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                    float &x = v[8 * g8 + j];
                    x = (in && bits != 0u && bits < 0x8000u) ? x : 0.f;
                }
            }
            tr_store16(buf, r, c0, kHid / 8, *reinterpret_cast<const float(*)[16]>(v), false);
            tr_store16(buf, r, c0 + 16, kHid / 8, *reinterpret_cast<const float(*)[16]>(v + 16), false);
            if (pb)
                colsums32(v, c0, kHid, pb, c0 >= sum_lo && c0 < sum_hi);
        }
    };
    auto mask_epilogue = [&](uint8_t *buf, float *pb, int sum_lo = 0, int sum_hi = kHid) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h)
            mask_cols(buf, pb, 64 * qd + 32 * h, 64 * qd + 32 * h, sum_lo, sum_hi);
    };
    // transposed weight-gradient accumulator (lane = input unit u, column =
    // output unit o) to out[o * ld + u] for columns [c0, c0 + 16) below ncols:
    // each store instruction writes 32 consecutive floats
    auto store_wgrad32 = [&](uint32_t dcol, int c0, int ncols, float *out, int ld, int u) {
        float v[32];
        tc::tmem_ld32(tw + dcol + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < ncols)
                out[(size_t)(c0 + j) * ld + u] = v[j];
    };

    // ---------------- P1, P2: hidden layers ----------------
    run(w1, aPhi, kIn / 8, 0);
    commit_wait();
    prefetch(w2);
    hidden_epilogue(0, scratch, sH1);
    epilogue_done();
    run(w2, aH1, kHid / 8, 256);
    commit_wait();
    prefetch(w3);
    hidden_epilogue(256, scratch + kHid, sH2);
    epilogue_done();

    // ---------------- P3: logits, softmax, cross-entropy error ----------------
    run(w3, aH2, kHid / 8, 0);
    commit_wait();
    if (role != 4)
        prefetch(w3t);
    {
        constexpr float kLog2e = 1.4426950408889634f;
        float z[32];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c0 = 32 * qd + 16 * h;
            float v[16];
            if (c0 < kBinsPad) {
                tc::tmem_ld16(tw + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = 0.f;
            }
            if (c0 < kBinsPad) {
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) {
                    const float4 b4 = reinterpret_cast<const float4 *>(b3s + c0)[j4];
                    z[16 * h + 4 * j4 + 0] = c0 + 4 * j4 + 0 < kBins ? v[4 * j4 + 0] + b4.x : -INFINITY;
                    z[16 * h + 4 * j4 + 1] = c0 + 4 * j4 + 1 < kBins ? v[4 * j4 + 1] + b4.y : -INFINITY;
                    z[16 * h + 4 * j4 + 2] = c0 + 4 * j4 + 2 < kBins ? v[4 * j4 + 2] + b4.z : -INFINITY;
                    z[16 * h + 4 * j4 + 3] = c0 + 4 * j4 + 3 < kBins ? v[4 * j4 + 3] + b4.w : -INFINITY;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    z[16 * h + j] = -INFINITY;
            }
        }
        float mq = -INFINITY;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            mq = fmaxf(mq, z[j]);
        const float mx = row_combine(mq, true);
        // z - max and its exponential, each formed once
        float ez[32];
        float sq = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            z[j] = z[j] - mx;
            ez[j] = 32 * qd + j < kBins ? ex2_approx(z[j] * kLog2e) : 0.f;
            sq += ez[j];
        }
        const float sum = row_combine(sq, false);
        const float inv = __frcp_rn(sum);  // 1 / sum, correctly rounded
        // cross-entropy terms -t (z - max - log sum) for the loss (role 4 only)
        float ce = 0.f;
        if (role == 4) {
            const float lsum = logf(sum);
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (32 * qd + j < kBins && in)
                    ce -= tg[j] * (z[j] - lsum);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float d = 0.f;
            if (32 * qd + j < kBins && in)
                d = (ez[j] * inv - tg[j]) * a.inv_m;
            z[j] = d;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                v[j] = z[16 * h + j];
            tr_store16(sDZ, r, 32 * qd + 16 * h, kTrDZCols / 8, v, false);
        }
        if (role == 4) {
            const float sw = warp_sum(ce);
            if (lane == 0)
                lw[warp] = sw;
            colsums32(z, 32 * qd, kBins, a.pb3 + (size_t)tile * 256);
            if (threadIdx.x == 0) {
                float acc = 0.f;
                for (int i = 0; i < kTrThreads / 32; ++i)
                    acc += lw[i];
                a.loss_part[tile] = acc;
            }
        }
    }
    epilogue_done();

    if (role == 0 || role == 2) {
        // ---------- the chain for hidden units 128 h .. 128 h + 127 (h = role / 2):
        // P5 -> dZ2 (all columns); P7 on those units (rows 128 h.. of every
        // W2^T chunk) -> dZ1 over H1, db1; P8 dW1^T = Phi^T dZ1 for those units ----------
        const int half = role >> 1;
        const TrStream w2h{18, 8, 32, kBM, 5, half * (kImgW / 2), kImgW / 2};
        run(w3t, aDZ, kTrDZCols / 8, 0);
        commit_wait();
        prefetch(w2h);
        mask_epilogue(sH2, nullptr);
        epilogue_done();
        run(w2h, aH2, kHid / 8, 0);
        commit_wait();
        mask_cols(sH1, a.pb1 + (size_t)tile * 256, 32 * qd, kBM * half + 32 * qd);
        epilogue_done();
        if (threadIdx.x == 0) {
            tc::tc_fence_after();
            issue_wgrad(aPhi, kIn / 8, 0, aH1, kHid / 8, kBM, 0, kBM * half);
        }
        commit_wait();
        if ((warp & 3) < 2) {
            // lanes 0..63 hold the 64 input features; columns: the 128 units
            store_wgrad32(0, 32 * qd, kBM, ws1 + (size_t)kBM * half * kIn, kIn, r);
        }
    } else if (role == 1 || role == 3) {
        // ---------- P5 -> dZ2 and db2 for units 0..127 (role 1) or 128..255
        // (role 3); P6 dW2^T = H1^T dZ2 for input units 0..127 (role 1) or
        // 128..255 (role 3) ----------
        run(w3t, aDZ, kTrDZCols / 8, 0);
        commit_wait();
        mask_epilogue(sH2, a.pb2 + (size_t)tile * 256, role == 1 ? 0 : kBM, role == 1 ? kBM : kHid);
        epilogue_done();
        const int u0 = role == 1 ? 0 : kBM;
        if (threadIdx.x == 0) {
            tc::tc_fence_after();
            issue_wgrad(aH1, kHid / 8, u0, aH2, kHid / 8, kHid, 0);
        }
        commit_wait();
#pragma unroll 1
        for (int c0 = 64 * qd; c0 < 64 * qd + 64; c0 += 32)
            store_wgrad32(0, c0, kHid, ws2, kHid, u0 + r);
    } else {
        // ---------- role 4: P4 dW3^T = H2^T dZ (input units in two halves, columns 256 and 384) ----------
        if (threadIdx.x == 0) {
            tc::tc_fence_after();
            issue_wgrad(aH2, kHid / 8, 0, aDZ, kTrDZCols / 8, kBinsPad, 256);
            issue_wgrad(aH2, kHid / 8, kBM, aDZ, kTrDZCols / 8, kBinsPad, 384);
        }
        commit_wait();
        // dW3[b][u]: lanes over the hidden unit u, quarters over the bins
        // (quarter 3 reads columns 96..127 of an accumulator 112 wide: the
        // last 16 lie in the next accumulator or unused columns, and are not
        // stored)
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh)
            store_wgrad32((uint32_t)(256 + hh * 128), 32 * qd, kBins, ws3, kHid, hh * kBM + r);
        // (the shortest share) the next step's C values and target rows of
        // this tile's rows into L2, so that its input phase, which starts
        // when Adam's blocks leave the SM, reads them from there
        if (threadIdx.x < kBM && m0 + (int)threadIdx.x < a.next_n) {
            const int grow = m0 + threadIdx.x;
            const int64_t src = a.next_idx ? (int64_t)a.next_idx[grow] : (int64_t)grow;
            const int64_t trw = a.next_trow ? (int64_t)a.next_trow[grow] : (int64_t)grow;
            prefetch_l2(a.next_c + 2 * src);
            const char *t = reinterpret_cast<const char *>(a.next_target + trw * kTrTP);
#pragma unroll
            for (int b = 0; b < kTrTP * 4; b += 128)
                prefetch_l2(t + b);
            prefetch_l2(t + kTrTP * 4 - 1);
        }
    }

    if (!ok && a.status)
        atomicExch(a.status, (int32_t)JL_ETIMEOUT);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(taddr, 512);
}

// L1[i] = sum_b |p[i][b] - q[i][b]| over `bins` columns.
__global__ void hist_l1_kernel(const float *__restrict__ p, int ldp, const float *__restrict__ q, int ldq, int n,
                               int bins, float *__restrict__ out)
{
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n)
        return;
    float s = 0.f;
    for (int b = lane; b < bins; b += 32)
        s += fabsf(p[(size_t)i * ldp + b] - q[(size_t)i * ldq + b]);
    s = warp_sum(s);
    if (lane == 0)
        out[i] = s;
}

// ---------------------------------------------------------------------------
// Device top-k: k largest non-negative binary32 scores, ties by smaller index.
// Exact radix select on the float bits (ordered like the values for x >= 0)
// in three digit levels (11, 11, 10 bits), then all keys above the threshold
// plus the first `need` ties in index order, then each of the k survivors
// placed at its rank by (score desc, index asc).
// ---------------------------------------------------------------------------
struct TopkState {
    uint32_t prefix;     // fixed high bits of the threshold so far
    uint32_t k_rem;      // rank still to find inside the current prefix
    uint32_t count_gt;   // keys strictly above the final threshold
    uint32_t need;       // ties to take
    uint32_t n_sel;      // selected so far (atomic)
    uint32_t pad[3];
};

__device__ __forceinline__ uint32_t score_key(float s) { return __float_as_uint(fmaxf(s, 0.f)); }

__global__ void topk_hist_kernel(const float *__restrict__ score, int64_t n, const TopkState *st, int level,
                                 uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        h[i] = 0;
    __syncthreads();
    const int shift = level == 0 ? 21 : (level == 1 ? 10 : 0);
    const uint32_t dmask = level == 2 ? 0x3FFu : 0x7FFu;
    const int hi_bits = level == 0 ? 0 : (level == 1 ? 11 : 22);
    const uint32_t prefix = st->prefix;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = score_key(score[i]);
        if (hi_bits == 0 || (key >> (32 - hi_bits)) == prefix)
            atomicAdd(&h[(key >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (h[i])
            atomicAdd(&hist[i], h[i]);
}

// Initial state (rank k, empty prefix), a zeroed digit histogram and zeroed
// output ranks.
__global__ void topk_init_kernel(uint32_t *hist, TopkState *st, uint32_t k, uint32_t *rank)
{
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        hist[i] = 0;
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
        rank[i] = 0;
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->k_rem = k;
        st->count_gt = 0;
        st->need = 0;
        st->n_sel = 0;
    }
}

// Find the digit bin holding rank k_rem counted from the top: the bins in
// descending digit order, an inclusive prefix sum over them (one CTA of 1024
// threads, two bins each), and the bin where the running count reaches k_rem.
// The histogram is zeroed for the next level.
__global__ void __launch_bounds__(1024) topk_scan_kernel(uint32_t *hist, TopkState *st, int level)
{
    __shared__ uint32_t v[2048];
    __shared__ uint32_t wsum[32];
    __shared__ int found;
    const int nb = level == 2 ? 1024 : 2048;
    const int bits = level == 2 ? 10 : 11;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    // element e = bin nb - 1 - e (descending digits)
    const uint32_t a0 = (2 * t < nb) ? hist[nb - 1 - 2 * t] : 0u;
    const uint32_t a1 = (2 * t + 1 < nb) ? hist[nb - 2 - 2 * t] : 0u;
    if (t == 0)
        found = -1;
    __syncthreads();
    hist[2 * t] = 0;
    hist[2 * t + 1] = 0;
    // inclusive scan of the pair sums across the CTA
    uint32_t x = a0 + a1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t z = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o)
                z += y;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    const uint32_t incl1 = x + (w > 0 ? wsum[w - 1] : 0u);  // through element 2t + 1
    const uint32_t incl0 = incl1 - a1;                       // through element 2t
    const uint32_t k_rem = st->k_rem;
    // the first element whose running count reaches k_rem (unique)
    if (incl0 >= k_rem && incl0 - a0 < k_rem)
        found = 2 * t;
    else if (incl1 >= k_rem && incl1 - a1 < k_rem)
        found = 2 * t + 1;
    v[2 * t] = incl0;
    v[2 * t + 1] = incl1;
    __syncthreads();
    if (t == 0) {
        // no bin reaches k_rem (cannot happen for a consistent state): bin 0
        const int e = found >= 0 ? found : nb - 1;
        const uint32_t above = e > 0 ? v[e - 1] : 0u;  // elements before e: bins strictly above
        st->count_gt += above;
        st->k_rem = k_rem - above;
        st->prefix = (st->prefix << bits) | (uint32_t)(nb - 1 - e);
        if (level == 2)
            st->need = k_rem - above;
    }
}

// Keys above the threshold: appended in any order (sorted afterwards).
__global__ void topk_collect_gt_kernel(const float *__restrict__ score, int64_t n, TopkState *st,
                                       uint32_t *__restrict__ sel_key, uint32_t *__restrict__ sel_idx)
{
    const uint32_t thr = st->prefix;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = score_key(score[i]);
        if (key > thr) {
            const uint32_t pos = atomicAdd(&st->n_sel, 1u);
            sel_key[pos] = key;
            sel_idx[pos] = (uint32_t)i;
        }
    }
}

// Ties (key == threshold): count per block of a fixed index range.
__global__ void topk_tie_count_kernel(const float *__restrict__ score, int64_t n, const TopkState *st,
                                      int64_t per_block, uint32_t *__restrict__ counts)
{
    const uint32_t thr = st->prefix;
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(n, b0 + per_block);
    uint32_t c = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
        c += (score_key(score[i]) == thr) ? 1u : 0u;
    __shared__ uint32_t red[32];
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += red[w];
        counts[blockIdx.x] = s;
    }
}

// Ties in index order: block-exclusive prefix of the per-block counts, then
// each block writes its ties whose global tie rank is below `need`.
__global__ void topk_tie_select_kernel(const float *__restrict__ score, int64_t n, TopkState *st, int64_t per_block,
                                       const uint32_t *__restrict__ counts, uint32_t *__restrict__ sel_key,
                                       uint32_t *__restrict__ sel_idx)
{
    // a block without ties in its range selects nothing
    if (counts[blockIdx.x] == 0)
        return;
    const uint32_t thr = st->prefix;
    __shared__ uint32_t base_s;
    __shared__ uint32_t warp_tot[32];
    {
        // ties in the blocks before this one (block-wide sum of their counts)
        uint32_t b = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x)
            b += counts[i];
        b = __reduce_add_sync(0xffffffffu, b);
        if ((threadIdx.x & 31) == 0)
            warp_tot[threadIdx.x >> 5] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                t += warp_tot[w];
            base_s = t;
        }
        __syncthreads();
    }
    const uint32_t need = st->need;
    const uint32_t gt = st->count_gt;
    uint32_t run = base_s;
    if (run >= need)
        return;
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(n, b0 + per_block);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t s0 = b0; s0 < b1; s0 += blockDim.x) {
        const int64_t i = s0 + threadIdx.x;
        const bool tie = i < b1 && score_key(score[i]) == thr;
        const unsigned bal = __ballot_sync(0xffffffffu, tie);
        if (lane == 0)
            warp_tot[w] = __popc(bal);
        __syncthreads();
        uint32_t off = 0, tot = 0;
        for (int q = 0; q < nw; ++q) {
            if (q < w)
                off += warp_tot[q];
            tot += warp_tot[q];
        }
        const uint32_t rank = run + off + __popc(bal & ((1u << lane) - 1u));
        if (tie && rank < need) {
            sel_key[gt + rank] = thr;
            sel_idx[gt + rank] = (uint32_t)i;
        }
        run += tot;
        __syncthreads();
        if (run >= need)
            break;
    }
}

// Sort of the k selected (key, index) pairs, key descending then index
// ascending, by ranks: the position of a pair is the number of pairs that
// precede it (composite keys are unique, so the positions are a permutation).
// Grid (pair blocks of 256, splits of the pairs compared against); partial
// ranks are added atomically into `rank` (zeroed by topk_init_kernel).
static constexpr int kRankSplit = 32;
static constexpr int kRankTile = 1024;

__device__ __forceinline__ uint64_t topk_comp(uint32_t key, uint32_t idx)
{
    return ((uint64_t)(~key) << 32) | idx;  // ascending = score descending, then index ascending
}

__global__ void __launch_bounds__(256) topk_rank_kernel(const uint32_t *__restrict__ sel_key,
                                                         const uint32_t *__restrict__ sel_idx, int k,
                                                         uint32_t *__restrict__ rank)
{
    __shared__ uint64_t tile[kRankTile];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t ci = i < k ? topk_comp(sel_key[i], sel_idx[i]) : ~0ull;
    const int per = (k + kRankSplit - 1) / kRankSplit;
    const int j0 = blockIdx.y * per, j1 = min(k, j0 + per);
    uint32_t r = 0;
    for (int base = j0; base < j1; base += kRankTile) {
        const int nt = min(kRankTile, j1 - base);
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += blockDim.x)
            tile[t] = topk_comp(sel_key[base + t], sel_idx[base + t]);
        __syncthreads();
        int t = 0;
        for (; t + 8 <= nt; t += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                r += (tile[t + u] < ci) ? 1u : 0u;
        }
        for (; t < nt; ++t)
            r += (tile[t] < ci) ? 1u : 0u;
    }
    if (i < k && r)
        atomicAdd(&rank[i], r);
}

__global__ void topk_scatter_kernel(const uint32_t *__restrict__ sel_key, const uint32_t *__restrict__ sel_idx,
                                    const uint32_t *__restrict__ rank, int k, int32_t *__restrict__ out_idx,
                                    float *__restrict__ out_score)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k)
        return;
    const uint32_t r = rank[i];
    if (r >= (uint32_t)k)
        return;  // cannot happen for unique keys; never write out of range
    out_idx[r] = (int32_t)sel_idx[i];
    if (out_score)
        out_score[r] = __uint_as_float(sel_key[i]);
}

}  // namespace jl

// ---------------------------------------------------------------------------
// Model object and host orchestration
// ---------------------------------------------------------------------------
struct jl_model {
    int device = -1;
    float *params = nullptr;   // binary32 master [kNumParams]
    float *grads = nullptr;
    float *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;  // bf16 W1 | W2 | W3 for the layered forward (refreshed by it)
    uint8_t *wpack = nullptr;        // packed bf16 weight images (chunk_offset), kept current by Adam
    float *B = nullptr;        // Fourier matrix 32 x 2
    int32_t *step = nullptr;   // Adam step counter (device)
    float *loss = nullptr;     // device accumulator
    int32_t *status = nullptr;
    // layered-forward work buffers for up to `cap` rows
    int cap = 0;
    __nv_bfloat16 *phi = nullptr, *h1 = nullptr, *h2 = nullptr;  // layered forward activations
    // training partials for a batch of up to `tcap` rows, per 128-row tile
    int tcap = 0;
    float *pb = nullptr;        // column sums of the three bias gradients [3][tiles x 256]
    float *loss_part = nullptr; // loss sums [tiles]
    float *ws = nullptr;        // dW1 | dW2 | dW3 partials [tiles blocks each]
    int tiles = 0;              // tiles of the last training step
    float *tpad = nullptr;      // padded copy of the targets of a call [tpad_rows x kTrTP]
    int64_t tpad_rows = 0;
    // screening as one CUDA graph (forward + top-k), captured on an internal
    // stream for the last (c, n, k, outputs) seen and replayed on the caller's
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t survey_exec = nullptr;
    const void *sk_c = nullptr, *sk_idx = nullptr, *sk_val = nullptr, *sk_score = nullptr;
    int64_t sk_n = 0;
    int32_t sk_k = 0;
};

namespace jl {

static bool g_gemm_attr_set[4] = {false, false, false, false};

// Launch with programmatic stream serialization: the kernel may start while
// the preceding kernel of the stream finishes (each kernel waits for it with
// griddep_wait before using its results or writing anything).
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

template <int EPI>
static cudaError_t launch_gemm(const GemmArgs &a, cudaStream_t st)
{
    auto kern = tc_gemm_kernel<EPI>;
    if (!g_gemm_attr_set[EPI]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
        if (e != cudaSuccess)
            return e;
        g_gemm_attr_set[EPI] = true;
    }
    const int grid = (a.M + kBM - 1) / kBM;
    // columns in blocks of 64 per CTA (a few row tiles would leave most SMs
    // idle with whole rows per CTA); the softmax needs every column of a row
    GemmArgs b = a;
    b.n_per_cta = EPI == EPI_SOFTMAX ? 0 : 64;
    const int nz = b.n_per_cta ? (a.BN + b.n_per_cta - 1) / b.n_per_cta : 1;
    return launch_pdl(kern, dim3(grid, 1, nz), dim3(kGemmThreads), (size_t)kGemmSmem, st, b);
}

static GemmArgs gemm_args(const __nv_bfloat16 *A, int lda, int at, const __nv_bfloat16 *B, int ldb, int bt, int M,
                          int N, int K, int32_t *status)
{
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.A = A;
    a.lda = lda;
    a.a_trans = at;
    a.B = B;
    a.ldb = ldb;
    a.b_trans = bt;
    a.M = M;
    a.N = N;
    a.K = K;
    a.BN = (N + 15) / 16 * 16;
    a.status = status;
    return a;
}

static constexpr size_t kWs1 = (size_t)kHid * kIn, kWs2 = (size_t)kHid * kHid, kWs3 = (size_t)kBins * kHid;

static void free_work(jl_model *md)
{
    cudaFree(md->phi);
    cudaFree(md->h1);
    cudaFree(md->h2);
    cudaFree(md->pb);
    cudaFree(md->loss_part);
    cudaFree(md->ws);
    md->phi = md->h1 = md->h2 = nullptr;
    md->pb = md->loss_part = md->ws = nullptr;
    md->cap = md->tcap = 0;
}

// Work buffers for `rows` rows: layered-forward activations (train false) or
// the per-tile gradient partials of a training batch (train true).
static int ensure_work(jl_model *md, int rows, bool train)
{
    if (train ? rows <= md->tcap : rows <= md->cap)
        return JL_OK;
    const size_t r = (size_t)rows;
    cudaError_t e = cudaSuccess;
    if (!train) {
        cudaFree(md->phi);
        cudaFree(md->h1);
        cudaFree(md->h2);
        md->phi = md->h1 = md->h2 = nullptr;
        md->cap = 0;
        e = cudaMalloc(&md->phi, r * kIn * 2);
        if (e == cudaSuccess)
            e = cudaMalloc(&md->h1, r * kHid * 2);
        if (e == cudaSuccess)
            e = cudaMalloc(&md->h2, r * kHid * 2);
        if (e == cudaSuccess)
            md->cap = rows;
    } else {
        cudaFree(md->pb);
        cudaFree(md->loss_part);
        cudaFree(md->ws);
        md->pb = md->loss_part = md->ws = nullptr;
        md->tcap = 0;
        const size_t tiles = (r + kBM - 1) / kBM;
        e = cudaMalloc(&md->pb, 3 * tiles * 256 * 4);
        if (e == cudaSuccess)
            e = cudaMalloc(&md->loss_part, tiles * 4);
        if (e == cudaSuccess)
            e = cudaMalloc(&md->ws, tiles * (kWs1 + kWs2 + kWs3) * 4);
        if (e == cudaSuccess)
            md->tcap = rows;
    }
    if (e != cudaSuccess) {
        free_work(md);
        return cuda_fail(e, "cudaMalloc(surrogate work buffers)");
    }
    return JL_OK;
}

// The partials of the last training step, for grad_of / adam_kernel.
static GradParts grad_parts(const jl_model *md)
{
    GradParts q;
    const size_t cs = (size_t)md->tiles * 256;
    q.ws1 = md->ws;
    q.ws2 = md->ws + (size_t)md->tiles * kWs1;
    q.ws3 = md->ws + (size_t)md->tiles * (kWs1 + kWs2);
    q.pb1 = md->pb;
    q.pb2 = md->pb + cs;
    q.pb3 = md->pb + 2 * cs;
    q.loss_part = md->loss_part;
    q.S = md->tiles;
    q.ctas = md->tiles;
    return q;
}

// Layered forward of n rows (n <= cap): phi, h1, h2 and the softmax
// epilogue (probs and / or entropy score).
static cudaError_t forward_rows(jl_model *md, const float *c, int64_t n, float *probs, float *score, cudaStream_t st)
{
    const int64_t threads = n * 32;
    cudaError_t e = launch_pdl(features_kernel, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, st, c,
                               (const int32_t *)nullptr, n, (const float *)md->B, md->phi);
    if (e != cudaSuccess)
        return e;
    const __nv_bfloat16 *W1 = md->wb, *W2 = md->wb + kHid * kIn, *W3 = md->wb + kHid * kIn + kHid * kHid;
    // each product follows the kernel that wrote its A operand; the weights
    // (B) were written earlier
    GemmArgs a = gemm_args(md->phi, kIn, 0, W1, kIn, 0, (int)n, kHid, kIn, md->status);
    a.pre_b = 1;
    a.bias = md->params + kOffB1;
    a.relu = 1;
    a.out_bf16 = md->h1;
    a.ld_out = kHid;
    if ((e = launch_gemm<EPI_BIAS_ACT>(a, st)) != cudaSuccess)
        return e;
    a = gemm_args(md->h1, kHid, 0, W2, kHid, 0, (int)n, kHid, kHid, md->status);
    a.pre_b = 1;
    a.bias = md->params + kOffB2;
    a.relu = 1;
    a.out_bf16 = md->h2;
    a.ld_out = kHid;
    if ((e = launch_gemm<EPI_BIAS_ACT>(a, st)) != cudaSuccess)
        return e;
    a = gemm_args(md->h2, kHid, 0, W3, kHid, 0, (int)n, kBins, kHid, md->status);
    a.pre_b = 1;
    a.bias = md->params + kOffB3;
    a.probs = probs;
    a.ldp = kBins;
    a.score = score;
    if ((e = launch_gemm<EPI_SOFTMAX>(a, st)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

// One fused training step over n batch rows (n <= cap): forward, softmax
// error and backward of every 128-row tile in one launch (train_step_kernel),
// leaving one partial per tile in md's gradient buffers for grad_of.
static cudaError_t train_rows(jl_model *md, const float *c, const int32_t *idx, int n, const float *target,
                              const int32_t *trow, float inv_m, cudaStream_t st, const float *next_c = nullptr,
                              const int32_t *next_idx = nullptr, int next_n = 0, const float *next_target = nullptr,
                              const int32_t *next_trow = nullptr)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(train_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem);
        if (e != cudaSuccess)
            return e;
        attr_set = true;
    }
    const int tiles = (n + kBM - 1) / kBM;
    md->tiles = tiles;
    const GradParts q = grad_parts(md);
    TrainArgs a;
    a.c = c;
    a.idx = idx;
    a.n = n;
    a.target = target;
    a.trow = trow;
    a.inv_m = inv_m;
    a.B = md->B;
    a.params = md->params;
    a.pack = md->wpack;
    a.ws1 = const_cast<float *>(q.ws1);
    a.ws2 = const_cast<float *>(q.ws2);
    a.ws3 = const_cast<float *>(q.ws3);
    a.pb1 = const_cast<float *>(q.pb1);
    a.pb2 = const_cast<float *>(q.pb2);
    a.pb3 = const_cast<float *>(q.pb3);
    a.loss_part = md->loss_part;
    a.status = md->status;
    a.next_c = next_c;
    a.next_idx = next_idx;
    a.next_n = next_n;
    a.next_target = next_target;
    a.next_trow = next_trow;
    return launch_pdl(train_step_kernel, dim3((unsigned)tiles, kTrRoles), dim3(kTrThreads), (size_t)kTrSmem, st, a);
}

// The targets of a call (n rows of 101) as padded rows in md->tpad.
static int pad_targets(jl_model *md, const float *target, int64_t n, cudaStream_t st)
{
    if (n > md->tpad_rows) {
        cudaFree(md->tpad);
        md->tpad = nullptr;
        md->tpad_rows = 0;
        cudaError_t e = cudaMalloc(&md->tpad, (size_t)n * kTrTP * 4);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(padded targets)");
        md->tpad_rows = n;
    }
    const int64_t total = n * kTrTP;
    pad_targets_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(target, n, md->tpad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "pad targets");
}

static void destroy_model(jl_model *md)
{
    if (!md)
        return;
    free_work(md);
    cudaFree(md->tpad);
    if (md->survey_exec)
        cudaGraphExecDestroy(md->survey_exec);
    if (md->cap_stream)
        cudaStreamDestroy(md->cap_stream);
    cudaFree(md->params);
    cudaFree(md->grads);
    cudaFree(md->m);
    cudaFree(md->v);
    cudaFree(md->wb);
    cudaFree(md->wpack);
    cudaFree(md->B);
    cudaFree(md->step);
    cudaFree(md->loss);
    cudaFree(md->status);
    delete md;
}

static int refresh_bf16(jl_model *md, cudaStream_t st)
{
    cast_weights_kernel<<<(kWbW + 255) / 256, 256, 0, st>>>(md->params, md->wb);
    pack_params_kernel<<<(kNumParams + 255) / 256, 256, 0, st>>>(md->params, md->wpack);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "cast weights");
}

static int check_status(jl_model *md, cudaStream_t st)
{
    int32_t s = 0;
    cudaError_t e = cudaMemcpyAsync(&s, md->status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate status");
    if (s != 0)
        return fail(s, "a tensor-core wait gave up (status " + std::to_string(s) + ")");
    return JL_OK;
}

}  // namespace jl

using namespace jl;

extern "C" {

int jl_model_num_params(void) { return kNumParams; }

int jl_model_create(const float *fourier_B, const float *init_params, jl_model **out)
{
    if (!out || !fourier_B || !init_params)
        return fail(JL_EINVAL, "fourier_B, init_params and out must not be NULL");
    *out = nullptr;
    jl_model *md = new jl_model();
    cudaError_t e = cudaGetDevice(&md->device);
    const size_t pb = (size_t)kNumParams * 4;
    if (e == cudaSuccess) e = cudaMalloc(&md->params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&md->grads, pb);
    if (e == cudaSuccess) e = cudaMalloc(&md->m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&md->v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&md->wb, (size_t)kWbW * 2);
    if (e == cudaSuccess) e = cudaMalloc(&md->wpack, kPackBytes);
    if (e == cudaSuccess) e = cudaMemset(md->wpack, 0, kPackBytes);
    if (e == cudaSuccess) e = cudaMalloc(&md->B, kFreq * 2 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&md->step, 4);
    if (e == cudaSuccess) e = cudaMalloc(&md->loss, 4);
    if (e == cudaSuccess) e = cudaMalloc(&md->status, 4);
    if (e == cudaSuccess) e = cudaMemcpy(md->params, init_params, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(md->B, fourier_B, kFreq * 2 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(md->m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(md->v, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(md->grads, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(md->step, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(md->status, 0, 4);
    if (e != cudaSuccess) {
        destroy_model(md);
        return cuda_fail(e, "jl_model_create");
    }
    int rc = refresh_bf16(md, nullptr);
    if (rc == JL_OK && (e = cudaDeviceSynchronize()) != cudaSuccess)
        rc = cuda_fail(e, "jl_model_create");
    if (rc != JL_OK) {
        destroy_model(md);
        return rc;
    }
    *out = md;
    return JL_OK;
}

void jl_model_destroy(jl_model *md) { destroy_model(md); }

int jl_model_get_state(const jl_model *md, float *params, float *m, float *v, int32_t *step)
{
    if (!md)
        return fail(JL_EINVAL, "invalid model");
    const size_t pb = (size_t)kNumParams * 4;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpy(params, md->params, pb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && m) e = cudaMemcpy(m, md->m, pb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemcpy(v, md->v, pb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && step) e = cudaMemcpy(step, md->step, 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "jl_model_get_state");
}

int jl_model_set_state(jl_model *md, const float *params, const float *m, const float *v, const int32_t *step)
{
    if (!md)
        return fail(JL_EINVAL, "invalid model");
    const size_t pb = (size_t)kNumParams * 4;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpy(md->params, params, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(md->m, m, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && v) e = cudaMemcpy(md->v, v, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && step) e = cudaMemcpy(md->step, step, 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(e, "jl_model_set_state");
    int rc = refresh_bf16(md, nullptr);
    if (rc == JL_OK && (e = cudaDeviceSynchronize()) != cudaSuccess)
        rc = cuda_fail(e, "jl_model_set_state");
    return rc;
}

int jl_model_forward(jl_model *md, const float *c, int64_t n, float *probs, float *score, void *stream)
{
    if (!md || !c || n < 1)
        return fail(JL_EINVAL, "invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    static bool attr_set = false;
    if (!attr_set) {
        e = cudaFuncSetAttribute(fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
        if (e != cudaSuccess)
            return cuda_fail(e, "fused forward attribute");
        attr_set = true;
    }
    FusedArgs a;
    a.c = c;
    a.n = n;
    a.pack = md->wpack;
    a.params = md->params;
    a.B = md->B;
    a.probs = probs;
    a.score = score;
    a.status = md->status;
    const int64_t tiles = (n + 2 * kBM - 1) / (2 * kBM);
    const int sms = device_sm_count();
    const int grid = (int)std::min<int64_t>(tiles, sms > 0 ? sms : 148);
    fused_forward_kernel<<<grid, kFusedThreads, kFusedSmem, st>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "fused forward");
}

// The forward built from one launch of the general product kernel per layer;
// kept as a reference for the fused kernel.
int jl_model_forward_layered(jl_model *md, const float *c, int64_t n, float *probs, float *score, void *stream)
{
    if (!md || !c || n < 1)
        return fail(JL_EINVAL, "invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t chunk = 1 << 16;
    int rc = ensure_work(md, (int)std::min<int64_t>(n, chunk), false);
    if (rc != JL_OK)
        return rc;
    // the plain bf16 weights this path reads, from the current parameters
    cast_weights_kernel<<<(kWbW + 255) / 256, 256, 0, st>>>(md->params, md->wb);
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min<int64_t>(chunk, n - r0);
        cudaError_t e = forward_rows(md, c + 2 * r0, rows, probs ? probs + r0 * kBins : nullptr,
                                     score ? score + r0 : nullptr, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "surrogate forward");
    }
    return JL_OK;
}

int jl_model_grads(jl_model *md, const float *c, const float *target, int32_t n, float *loss_host, float *grads_host,
                   void *stream)
{
    if (!md || !c || !target || n < 1 || n > 65536)
        return fail(JL_EINVAL, "invalid arguments (1 <= n <= 65536)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(md, n, true);
    if (rc == JL_OK)
        rc = pad_targets(md, target, n, st);
    if (rc != JL_OK)
        return rc;
    cudaError_t e = train_rows(md, c, nullptr, n, md->tpad, nullptr, 1.f / (float)n, st);
    if (e == cudaSuccess) {
        e = launch_pdl(grad_reduce_kernel, dim3((kNumParams + 255) / 256), dim3(256), 0, st, grad_parts(md), md->grads,
                       md->loss);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate gradients");
    rc = check_status(md, st);
    if (rc != JL_OK)
        return rc;
    if (loss_host) {
        float s = 0.f;
        if ((e = cudaMemcpy(&s, md->loss, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "loss copy");
        *loss_host = s / (float)n;
    }
    if (grads_host && (e = cudaMemcpy(grads_host, md->grads, (size_t)kNumParams * 4, cudaMemcpyDeviceToHost)) !=
                          cudaSuccess)
        return cuda_fail(e, "gradient copy");
    return JL_OK;
}

int jl_train(jl_model *md, const float *c, const float *hist, int32_t n, const int32_t *order, int32_t epochs,
             int32_t batch, float lr, float lr_final, float *loss_curve, void *stream)
{
    if (!md || !c || !hist || n < 1 || epochs < 1 || batch < 1 || batch > n || !(lr > 0.f) || !(lr_final > 0.f))
        return fail(JL_EINVAL, "invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(md, batch, true);
    if (rc == JL_OK)
        rc = pad_targets(md, hist, n, st);
    if (rc != JL_OK)
        return rc;
    const int steps = n / batch;  // the last partial batch of an epoch is dropped
    const int nparam_blocks = (kNumParams + 255) / 256;
    // batch losses of every step, read back once at the end (no per-epoch drain)
    const size_t nsteps = (size_t)epochs * steps;
    float *loss_steps = nullptr;
    cudaError_t e = cudaMalloc(&loss_steps, nsteps * 4);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(loss per step)");
    const double total = (double)epochs * steps;
    // Adam's step count: read once, advanced on the host, written back at the end
    int32_t step0 = 0;
    e = cudaMemcpyAsync(&step0, md->step, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(loss_steps);
        return cuda_fail(e, "step counter");
    }
    int32_t done = 0;  // steps launched
    for (int ep = 0; ep < epochs && rc == JL_OK; ++ep) {
        for (int s = 0; s < steps; ++s) {
            // batch (ep, s): C of batch row m and its target row idx[m] (of the
            // padded copy of hist, gathered by the training-step kernel), or
            // rows s * batch + m
            auto batch_of = [&](int bep, int bs, const int32_t *&bidx, const float *&bc, const float *&bt) {
                bidx = order ? order + (size_t)bep * n + (size_t)bs * batch : nullptr;
                bc = order ? c : c + 2 * (size_t)bs * batch;
                bt = order ? md->tpad : md->tpad + (size_t)bs * batch * kTrTP;
            };
            const int32_t *idx, *nidx = nullptr;
            const float *cb, *tb, *ncb = nullptr, *ntb = nullptr;
            batch_of(ep, s, idx, cb, tb);
            const bool last = ep == epochs - 1 && s == steps - 1;
            if (!last)
                batch_of(s + 1 < steps ? ep : ep + 1, s + 1 < steps ? s + 1 : 0, nidx, ncb, ntb);
            e = train_rows(md, cb, idx, batch, tb, idx, 1.f / (float)batch, st, ncb, nidx, last ? 0 : batch, ntb,
                           nidx);
            if (e == cudaSuccess) {
                // cosine schedule from lr to lr_final over the steps of this call
                const double t = ((double)ep * steps + s) / total;
                const float lr_t = (float)(lr_final + 0.5 * (lr - lr_final) * (1.0 + cos(3.141592653589793 * t)));
                const int step_t = step0 + ep * steps + s + 1;
                const float b1 = 0.9f, b2 = 0.999f;
                // the bias corrections in binary32, as 1 - powf(beta, t)
                const float bc1 = 1.f - powf(b1, (float)step_t), bc2 = 1.f - powf(b2, (float)step_t);
                e = launch_pdl(adam_kernel, dim3(nparam_blocks), dim3(256), 0, st, grad_parts(md), md->params, md->m,
                               md->v, md->wpack, bc1, bc2, lr_t, b1, b2, 1e-8f, loss_steps + (size_t)ep * steps + s);
                if (e == cudaSuccess)
                    ++done;
            }
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "training step");
                break;
            }
        }
    }
    const int32_t step_end = step0 + done;
    cudaError_t e2 = cudaMemcpyAsync(md->step, &step_end, 4, cudaMemcpyHostToDevice, st);
    std::vector<float> hl;
    if (rc == JL_OK && loss_curve && e2 == cudaSuccess) {
        hl.resize(nsteps);
        e2 = cudaMemcpyAsync(hl.data(), loss_steps, nsteps * 4, cudaMemcpyDeviceToHost, st);
    }
    cudaError_t e3 = cudaStreamSynchronize(st);
    if (e2 == cudaSuccess)
        e2 = e3;
    cudaFree(loss_steps);
    if (rc == JL_OK && e2 == cudaSuccess && loss_curve) {
        for (int ep = 0; ep < epochs; ++ep) {
            double acc = 0.0;
            for (int s = 0; s < steps; ++s)
                acc += hl[(size_t)ep * steps + s] / (double)batch;
            loss_curve[ep] = (float)(acc / steps);
        }
    }
    if (rc == JL_OK && e2 != cudaSuccess)
        rc = cuda_fail(e2, "training");
    if (rc != JL_OK)
        return rc;
    return check_status(md, st);
}

int jl_topk(const float *score, int64_t n, int32_t k, int32_t *out_idx, float *out_score, void *stream)
{
    if (!score || !out_idx || n < 1 || k < 1 || k > n || k > 16384 || n > (int64_t)0x7fffffff)
        return fail(JL_EINVAL, "jl_topk: need 1 <= k <= min(n, 16384), n < 2^31");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t per_block = 8192;
    const int nblk = (int)((n + per_block - 1) / per_block);
    const size_t bytes = 2048 * 4 + sizeof(TopkState) + (size_t)nblk * 4 + 3 * (size_t)k * 4 + 256;
    uint8_t *w = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&w), bytes, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(topk)");
    uint32_t *hist = reinterpret_cast<uint32_t *>(w);
    TopkState *state = reinterpret_cast<TopkState *>(w + 2048 * 4);
    uint32_t *counts = reinterpret_cast<uint32_t *>(w + 2048 * 4 + sizeof(TopkState));
    uint32_t *sel_key = counts + nblk;
    uint32_t *sel_idx = sel_key + k;
    uint32_t *rank = sel_idx + k;
    int rc = JL_OK;
    do {
        topk_init_kernel<<<1, 1024, 0, st>>>(hist, state, (uint32_t)k, rank);
        const int grid = 148 * 4;
        for (int level = 0; level < 3 && e == cudaSuccess; ++level) {
            topk_hist_kernel<<<grid, 256, 0, st>>>(score, n, state, level, hist);
            topk_scan_kernel<<<1, 1024, 0, st>>>(hist, state, level);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        topk_collect_gt_kernel<<<grid, 256, 0, st>>>(score, n, state, sel_key, sel_idx);
        topk_tie_count_kernel<<<nblk, 256, 0, st>>>(score, n, state, per_block, counts);
        topk_tie_select_kernel<<<nblk, 256, 0, st>>>(score, n, state, per_block, counts, sel_key, sel_idx);
        topk_rank_kernel<<<dim3((unsigned)((k + 255) / 256), kRankSplit), 256, 0, st>>>(sel_key, sel_idx, k, rank);
        topk_scatter_kernel<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(sel_key, sel_idx, rank, k, out_idx,
                                                                       out_score);
        e = cudaGetLastError();
    } while (0);
    if (e != cudaSuccess)
        rc = cuda_fail(e, "jl_topk");
    cudaError_t e2 = cudaFreeAsync(w, st);
    if (rc == JL_OK && e2 != cudaSuccess)
        rc = cuda_fail(e2, "cudaFreeAsync(topk)");
    return rc;
}

int jl_survey(jl_model *md, const float *c, int64_t n, int32_t k, int32_t *top_idx, float *top_score, float *score,
              void *stream)
{
    if (!md || !c || n < 1 || !top_idx || !score)
        return fail(JL_EINVAL, "invalid arguments");
    if (k < 1 || k > n || k > 16384 || n > (int64_t)0x7fffffff)
        return fail(JL_EINVAL, "jl_survey: need 1 <= k <= min(n, 16384), n < 2^31");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a caller that is capturing its own graph gets the launches themselves
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) {
        int rc = jl_model_forward(md, c, n, nullptr, score, stream);
        return rc != JL_OK ? rc : jl_topk(score, n, k, top_idx, top_score, stream);
    }
    // the ~14 launches of a screening call as one graph launch, captured the
    // second time in a row that a call has the same pointers and sizes (a
    // one-off call runs its launches directly)
    const bool key = md->sk_c == c && md->sk_n == n && md->sk_k == k && md->sk_idx == top_idx &&
                     md->sk_val == top_score && md->sk_score == score;
    if (!key) {
        if (md->survey_exec) {
            cudaGraphExecDestroy(md->survey_exec);
            md->survey_exec = nullptr;
        }
        md->sk_c = c;
        md->sk_n = n;
        md->sk_k = k;
        md->sk_idx = top_idx;
        md->sk_val = top_score;
        md->sk_score = score;
        int rc = jl_model_forward(md, c, n, nullptr, score, stream);
        return rc != JL_OK ? rc : jl_topk(score, n, k, top_idx, top_score, stream);
    }
    if (!md->survey_exec) {
        if (md->survey_exec) {
            cudaGraphExecDestroy(md->survey_exec);
            md->survey_exec = nullptr;
        }
        if (!md->cap_stream) {
            e = cudaStreamCreateWithFlags(&md->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate(survey capture)");
        }
        e = cudaStreamBeginCapture(md->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture(survey)");
        int rc = jl_model_forward(md, c, n, nullptr, score, md->cap_stream);
        if (rc == JL_OK)
            rc = jl_topk(score, n, k, top_idx, top_score, md->cap_stream);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(md->cap_stream, &g);
        if (rc == JL_OK && e != cudaSuccess)
            rc = cuda_fail(e, "cudaStreamEndCapture(survey)");
        if (rc == JL_OK) {
            e = cudaGraphInstantiate(&md->survey_exec, g, 0);
            if (e != cudaSuccess) {
                md->survey_exec = nullptr;
                rc = cuda_fail(e, "cudaGraphInstantiate(survey)");
            }
        }
        if (g)
            cudaGraphDestroy(g);
        if (rc != JL_OK) {
            md->sk_c = nullptr;  // capture again next time
            return rc;
        }
    }
    e = cudaGraphLaunch(md->survey_exec, st);
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "cudaGraphLaunch(survey)");
}

int jl_gemm_bf16(const void *A, int32_t lda, int32_t a_trans, const void *B, int32_t ldb, int32_t b_trans, int32_t M,
                 int32_t N, int32_t K, float *C, int32_t ldc, int32_t *status, void *stream)
{
    if (!A || !B || !C || M < 1 || N < 1 || N > 256 || K < 1 || ldc < N || lda < 1 || ldb < 1)
        return fail(JL_EINVAL, "jl_gemm_bf16: need M, K >= 1, 1 <= N <= 256, ldc >= N");
    GemmArgs a = gemm_args(static_cast<const __nv_bfloat16 *>(A), lda, a_trans ? 1 : 0,
                           static_cast<const __nv_bfloat16 *>(B), ldb, b_trans ? 1 : 0, M, N, K, status);
    a.out_f32 = C;
    a.ld_out32 = ldc;
    cudaError_t e = launch_gemm<EPI_F32>(a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "jl_gemm_bf16");
}

int jl_hist_l1(const float *p, int32_t ldp, const float *q, int32_t ldq, int32_t n, int32_t bins, float *out,
               void *stream)
{
    if (!p || !q || !out || n < 1 || bins < 1 || ldp < bins || ldq < bins)
        return fail(JL_EINVAL, "invalid arguments");
    hist_l1_kernel<<<(n + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(p, ldp, q, ldq, n, bins, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JL_OK : cuda_fail(e, "jl_hist_l1");
}

// Checkpoint: little-endian binary with a header; params, Adam m and v, step,
// Fourier matrix.  Resuming from it continues training bit-identically.
int jl_model_save(const jl_model *md, const char *path)
{
    if (!md || !path)
        return fail(JL_EINVAL, "invalid arguments");
    std::vector<float> p(kNumParams), m(kNumParams), v(kNumParams), B(kFreq * 2);
    int32_t step = 0;
    int rc = jl_model_get_state(md, p.data(), m.data(), v.data(), &step);
    if (rc != JL_OK)
        return rc;
    cudaError_t e = cudaMemcpy(B.data(), md->B, B.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "save: Fourier matrix");
    FILE *fp = fopen(path, "wb");
    if (!fp)
        return fail(JL_EINVAL, std::string("cannot open ") + path);
    const char magic[8] = {'J', 'L', 'M', 'L', 'P', '0', '0', '1'};
    const int32_t hdr[4] = {kNumParams, kFreq, step, 0};
    bool okw = fwrite(magic, 1, 8, fp) == 8 && fwrite(hdr, 4, 4, fp) == 4 &&
               fwrite(B.data(), 4, B.size(), fp) == B.size() && fwrite(p.data(), 4, p.size(), fp) == p.size() &&
               fwrite(m.data(), 4, m.size(), fp) == m.size() && fwrite(v.data(), 4, v.size(), fp) == v.size();
    fclose(fp);
    return okw ? JL_OK : fail(JL_EINVAL, "short write");
}

int jl_model_load(const char *path, jl_model **out)
{
    if (!path || !out)
        return fail(JL_EINVAL, "invalid arguments");
    *out = nullptr;
    FILE *fp = fopen(path, "rb");
    if (!fp)
        return fail(JL_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    std::vector<float> p(kNumParams), m(kNumParams), v(kNumParams), B(kFreq * 2);
    bool okr = fread(magic, 1, 8, fp) == 8 && memcmp(magic, "JLMLP001", 8) == 0 && fread(hdr, 4, 4, fp) == 4 &&
               hdr[0] == kNumParams && hdr[1] == kFreq && fread(B.data(), 4, B.size(), fp) == B.size() &&
               fread(p.data(), 4, p.size(), fp) == p.size() && fread(m.data(), 4, m.size(), fp) == m.size() &&
               fread(v.data(), 4, v.size(), fp) == v.size();
    fclose(fp);
    if (!okr)
        return fail(JL_EINVAL, "not a jl surrogate checkpoint (or truncated)");
    jl_model *md = nullptr;
    int rc = jl_model_create(B.data(), p.data(), &md);
    if (rc != JL_OK)
        return rc;
    rc = jl_model_set_state(md, nullptr, m.data(), v.data(), &hdr[2]);
    if (rc != JL_OK) {
        destroy_model(md);
        return rc;
    }
    *out = md;
    return JL_OK;
}

}  // extern "C"
