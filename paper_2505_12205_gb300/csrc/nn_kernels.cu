// Kernels of the learned fast-forward (include/lbm_nn.h): a convolutional
// encoder-decoder on coarse-grained (phi, u, v) fields, trained and run on the
// GPU.  Activations are bfloat16 in channels-last layout, x[m * stride + c]
// with m = (b * H + y) * W + x; weights are bfloat16 [co][taps * ci] (k = tap
// * ci + c, tap = 3 ky + kx); accumulation is float32.
//
// The convolutions are implicit GEMMs on the tensor cores (warp-level
// mma.sync m16n8k16, bfloat16 operands, float32 accumulators): forward
// Y[m][co] = sum_k A[m][k] W[co][k] with A the patches of X gathered on the
// fly; backward-data is the forward kernel with the weights flipped in space
// and transposed in channels; the weight gradient dW[co][k] = sum_m dZ[m][co]
// A[m][k] reduces over the spatial positions, split over blocks whose
// partial sums are added in a fixed order (no atomics: training gives the
// same weights on every run).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lbm_nn.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;   // tile sizes; smem row pitch (bf16)

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t lds32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// One 64 x 64 x 32 step of the block tile from As[row m][k] and Bs[col n][k]
// (both k-contiguous): 4 warps in 2 x 2, each 32 x 32 = 2 x 4 mma tiles.
__device__ __forceinline__ void tile_mma(const bf16 (*As)[LDS], const bf16 (*Bs)[LDS], float (&acc)[2][4][4],
                                         int wm, int wn, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
        uint32_t a[2][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm * 32 + i * 16 + g;
            a[i][0] = lds32(&As[r][kk + 2 * t]);
            a[i][1] = lds32(&As[r + 8][kk + 2 * t]);
            a[i][2] = lds32(&As[r][kk + 2 * t + 8]);
            a[i][3] = lds32(&As[r + 8][kk + 2 * t + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = wn * 32 + j * 8 + g;
            b[j][0] = lds32(&Bs[n][kk + 2 * t]);
            b[j][1] = lds32(&Bs[n][kk + 2 * t + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
}

// 8 consecutive k of row m of the patch matrix A of X (zero outside the image
// and beyond K); k is a multiple of 8 and ci a multiple of 8, so the 8 values
// are one tap and one 16-byte vector.
__device__ __forceinline__ uint4 patch8(const bf16* __restrict__ X, int xs, int ci, int taps, int m, int k, int M,
                                        int K, int H, int W)
{
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (m >= M || k >= K) return v;
    const int tap = taps == 9 ? k / ci : 0, c = k - tap * ci;
    const int x = m % W, r = m / W, y = r % H, b = r / H;
    const int yy = y + (taps == 9 ? tap / 3 - 1 : 0), xx = x + (taps == 9 ? tap % 3 - 1 : 0);
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) return v;
    return *reinterpret_cast<const uint4*>(X + int64_t((b * H + yy) * W + xx) * xs + c);
}

// Y[m][yo + co] (bf16, optional) and Yf[m][co] (f32, optional) =
// relu?(sum_k A[m][k] Wt[co][k] + bias[co])
// Block tile TM x TN (64 x 64, or 128 x 32 for layers with at most 32 output
// channels), four warps of 32 x 32 each.
template <int TM, int TN>
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ X, int xs, int ci, int taps,
                                                  const bf16* __restrict__ Wt, const float* __restrict__ bias,
                                                  int co, bf16* __restrict__ Y, int ys, int yo,
                                                  float* __restrict__ Yf, int yfs, int relu, int M, int H, int W,
                                                  int kchunk, float* __restrict__ part)
{
    static_assert((TM / 32) * (TN / 32) == 4, "four warps of 32 x 32");
    constexpr int WN = TN / 32;
    __shared__ __align__(16) bf16 As[TM][LDS];
    __shared__ __align__(16) bf16 Bs[TN][LDS];
    const int K = taps * ci;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    // this block's range of k: all of it, or split z of a split-K launch
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, wm = warp / WN, wn = warp % WN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
    // the next k tile's 16-byte vectors are loaded into registers while the
    // tensor cores work on the current one
    constexpr int NA = TM * (BK / 8) / 128, NB = TN * (BK / 8) / 128;
    uint4 ra[NA], rb[NB];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int v = tid + i * 128, r = v / (BK / 8), q = v % (BK / 8);
            ra[i] = patch8(X, xs, ci, taps, m0 + r, k0 + q * 8, M, K, H, W);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int v = tid + i * 128, r = v / (BK / 8), q = v % (BK / 8), n = n0 + r, k = k0 + q * 8;
            rb[i] = (n < co && k < K) ? *reinterpret_cast<const uint4*>(Wt + int64_t(n) * K + k)
                                      : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    load(kb);
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int v = tid + i * 128, r = v / (BK / 8), q = v % (BK / 8);
            *reinterpret_cast<uint4*>(&As[r][q * 8]) = ra[i];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int v = tid + i * 128, r = v / (BK / 8), q = v % (BK / 8);
            *reinterpret_cast<uint4*>(&Bs[r][q * 8]) = rb[i];
        }
        __syncthreads();
        if (k0 + BK < ke) load(k0 + BK);
        tile_mma(As, Bs, acc, wm, wn, lane);
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm * 32 + i * 16 + g + (e >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * t + (e & 1);
                if (m >= M || n >= co) continue;
                if (part) {                   // split-K: the raw partial sum of this k range
                    part[(int64_t(blockIdx.z) * M + m) * co + n] = acc[i][j][e];
                    continue;
                }
                float v = acc[i][j][e] + (bias ? bias[n] : 0.0f);
                if (relu) v = fmaxf(v, 0.0f);
                if (Y) Y[int64_t(m) * ys + yo + n] = __float2bfloat16_rn(v);
                if (Yf) Yf[int64_t(m) * yfs + n] = v;
            }
}

// ---------------------------------------------------------- tcgen05 path
//
// The forward convolution as an implicit GEMM on the fifth-generation tensor
// cores: a block computes a 128-position x TN-channel tile of
// Y[m][co] = sum_k A[m][k] W[co][k] with one tcgen05.mma (M = 128, N = TN,
// K = 16, bfloat16 operands, float32 accumulator in tensor memory) per 16 k,
// issued by one thread.  The operand tiles of 64 k are gathered by all 128
// threads with 16-byte asynchronous copies (zero-filled outside the image and
// the matrices) into shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices; core matrices adjacent in k 128
// bytes apart, 8-row groups 1024 bytes apart), in a ring of three stages: the
// copies of stages k + 1 and k + 2 are in flight while the tensor cores work
// on stage k, and an mbarrier that the MMA unit's commit arrives on says when
// a slot may be refilled.  The
// accumulator is read back by the four warps with tcgen05.ld (warp w owns
// tensor-memory lanes 32 w .. 32 w + 31 = the tile's rows) for the epilogue
// (bias, ReLU, bfloat16 / float32 outputs, or split-K partial sums).  Every
// wait on an mbarrier is bounded: on timeout the block records an error flag
// and leaves after a bounded wait for its own MMAs, freeing its tensor memory.

constexpr int TC_TM = 128, TC_BK = 64, TC_STAGES = 3;
constexpr uint32_t TC_SBO = 1024, TC_LBO = 128;       // bytes: 8-row groups, k-adjacent core matrices

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address,
// leading (k) and stride (m/n) byte offsets, each >> 4; descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((TC_LBO >> 4) & 0x3FFFu) << 16) |
           (uint64_t((TC_SBO >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: float32 accumulator,
// bfloat16 A and B, both K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(TC_TM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait for the phase `parity` of the mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

template <int TN>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(const bf16* __restrict__ X, int xs, int ci, int taps,
                                                     const bf16* __restrict__ Wt, const float* __restrict__ bias,
                                                     int co, bf16* __restrict__ Y, int ys, int yo,
                                                     float* __restrict__ Yf, int yfs, int relu, int M, int H, int W,
                                                     int kchunk, float* __restrict__ part, int* __restrict__ err)
{
    static_assert(TN % 16 == 0 && TN >= 32 && TN <= 256, "N of an M = 128 MMA");
    constexpr int NS = TC_STAGES;
    constexpr int A_BYTES = TC_TM * TC_BK * 2, B_BYTES = TN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t NCOL = TN;                          // float32 accumulator columns (a power of two)
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + NS * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + NS * STAGE + 8 * NS);
    int* s_ok = reinterpret_cast<int*>(tc_smem + NS * STAGE + 8 * NS + 4);     // one thread waits, all read
    const int K = taps * ci;
    const int m0 = blockIdx.x * TC_TM, n0 = blockIdx.y * TN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_addr(tc_smem), bar0 = smem_addr(bars);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int j = 0; j < NS; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8 * j) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;

    // the rows this thread gathers: rq + 16 i, i = 0 .. 7, at the 8-k vector q8;
    // their pixel index m (-1 beyond M) and coordinates
    const int rq = tid >> 3, q8 = tid & 7;
    int pm[8], py[8], px[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + rq + 16 * i;
        pm[i] = m < M ? m : -1;
        const int mm = m < M ? m : 0;
        px[i] = mm % W;
        py[i] = (mm / W) % H;
    }
    const int nk = (ke - kb + TC_BK - 1) / TC_BK;
    // stage kt's operands (A 128 rows, B TN rows, k0 .. k0 + 63, zero outside)
    // into ring slot kt mod NS by asynchronous copies; one commit group per stage
    auto gather = [&](int kt) {
        if (kt < nk) {
            const uint32_t As = sbase + (kt % NS) * STAGE, Bs = As + A_BYTES;
            const int k = kb + kt * TC_BK + q8 * 8;
            const int tap = taps == 9 ? k / ci : 0, c = k - tap * ci;
            const int dy = taps == 9 ? tap / 3 - 1 : 0, dx = taps == 9 ? tap % 3 - 1 : 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = rq + 16 * i, yy = py[i] + dy, xx = px[i] + dx;
                const bool in = k < ke && pm[i] >= 0 && yy >= 0 && yy < H && xx >= 0 && xx < W;
                const bf16* src = in ? X + int64_t(pm[i] + dy * W + dx) * xs + c : X;
                cp_async16(As + (r >> 3) * TC_SBO + q8 * TC_LBO + (r & 7) * 16, src, in ? 16u : 0u);
            }
#pragma unroll
            for (int i = 0; i < TN / 16; ++i) {
                const int r = rq + 16 * i, n = n0 + r;
                const bool in = n < co && k < ke;
                const bf16* src = in ? Wt + int64_t(n) * K + k : Wt;
                cp_async16(Bs + (r >> 3) * TC_SBO + q8 * TC_LBO + (r & 7) * 16, src, in ? 16u : 0u);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int kt = 0; kt < NS - 1; ++kt) gather(kt);

    bool ok = true;
    int kl = -1;                                          // the last stage whose MMAs were committed
    for (int kt = 0; kt < nk; ++kt) {
        // this thread's copies of stage kt are in; make them visible to the
        // tensor cores' (async proxy) reads
        asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        // the MMAs of stage kt - 1 must be done before its slot is refilled
        // below (thread 0 waits; the block learns the outcome at the barrier)
        if (tid == 0)
            *s_ok = kt == 0 || mbar_wait(bar0 + 8 * ((kt - 1) % NS), uint32_t(((kt - 1) / NS) & 1)) ? 1 : 0;
        __syncthreads();
        ok = *s_ok != 0;
        if (!ok) break;                                   // the same for every thread
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = sbase + (kt % NS) * STAGE, b0 = a0 + A_BYTES;
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j) {
                const uint64_t ad = tc_desc(a0 + j * 2 * TC_LBO), bd = tc_desc(b0 + j * 2 * TC_LBO);
                const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(tc_idesc(TN)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar0 + 8 * (kt % NS))
                         : "memory");
        }
        kl = kt;
        gather(kt + NS - 1);                              // into the slot of stage kt - 1
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // the last commit covers every MMA of the block
    if (tid == 0) {
        const uint32_t bl = bar0 + 8 * ((kl < 0 ? 0 : kl) % NS), pl = uint32_t(((kl < 0 ? 0 : kl) / NS) & 1);
        if (ok && kl >= 0) ok = mbar_wait(bl, pl);
        if (!ok) {
            atomicExch(err, 1);
            // drain: give the MMAs in flight a bounded time before the memory goes
            if (kl >= 0) mbar_wait(bl, pl);
        }
        *s_ok = ok ? 1 : 0;
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    __syncthreads();
    ok = *s_ok != 0;
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int m = m0 + warp * 32 + lane;               // this thread's row of the tile
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (m >= M) continue;
            const int nb0 = n0 + c0;
            if (!part && Y && !Yf && nb0 + 16 <= co && ((ys | (yo + nb0)) & 7) == 0) {
                // 16 channels of one position: two 16-byte stores
                uint32_t h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float v0 = __uint_as_float(r[2 * e]) + (bias ? bias[nb0 + 2 * e] : 0.0f);
                    float v1 = __uint_as_float(r[2 * e + 1]) + (bias ? bias[nb0 + 2 * e + 1] : 0.0f);
                    if (relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
                    h[e] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                uint4* dst = reinterpret_cast<uint4*>(Y + int64_t(m) * ys + yo + nb0);
                dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
                dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
                continue;
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n = nb0 + e;
                if (n >= co) continue;
                const float a = __uint_as_float(r[e]);
                if (part) {                   // split-K: the raw partial sum of this k range
                    part[(int64_t(blockIdx.z) * M + m) * co + n] = a;
                    continue;
                }
                float v = a + (bias ? bias[n] : 0.0f);
                if (relu) v = fmaxf(v, 0.0f);
                if (Y) Y[int64_t(m) * ys + yo + n] = __float2bfloat16_rn(v);
                if (Yf) Yf[int64_t(m) * yfs + n] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
    }
}

template <int TN>
constexpr int tc_smem_bytes() { return TC_STAGES * (TC_TM * TC_BK * 2 + TN * TC_BK * 2) + 8 * TC_STAGES + 16; }

// Sum of the split-K partial sums part[z][m][n] in the order z = 0, 1, ...
// (deterministic), then bias, ReLU and the outputs of k_conv_fwd.
__global__ void k_conv_reduce(const float* __restrict__ part, int splits, int M, int co,
                              const float* __restrict__ bias, int relu, bf16* __restrict__ Y, int ys, int yo,
                              float* __restrict__ Yf, int yfs)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(M) * co) return;
    const int m = int(i / co), n = int(i % co);
    float v = part[i];
    for (int z = 1; z < splits; ++z) v += part[int64_t(z) * M * co + i];
    v += bias ? bias[n] : 0.0f;
    if (relu) v = fmaxf(v, 0.0f);
    if (Y) Y[int64_t(m) * ys + yo + n] = __float2bfloat16_rn(v);
    if (Yf) Yf[int64_t(m) * yfs + n] = v;
}

// Sum over this block's chunk of positions of dZ[m][co] A[m][k]: added to
// dWt[co][k] when there is one chunk, else written to the chunk's slice
// part[chunk][co][k] (grid: co tiles x k tiles x position chunks)
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ X, int xs, int ci, int taps,
                                                    const bf16* __restrict__ dZ, int zs, int co,
                                                    float* __restrict__ dW, int M, int H, int W, int mchunk,
                                                    float* __restrict__ part)
{
    __shared__ __align__(16) bf16 As[BM][LDS];   // [co][m]
    __shared__ __align__(16) bf16 Bs[BN][LDS];   // [k][m]
    const int K = taps * ci;
    const int c0 = blockIdx.x * BM, k0 = blockIdx.y * BN;
    const int mb = blockIdx.z * mchunk, me = min(M, mb + mchunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, wm = warp >> 1, wn = warp & 1;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
    for (int mm = mb; mm < me; mm += BK) {
        // BK positions x 64 channels of dZ, stored transposed
        for (int v = tid; v < BK * (BM / 8); v += 128) {
            const int r = v / (BM / 8), q = v % (BM / 8), m = mm + r, c = c0 + q * 8;
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (m < me && c < co) w = *reinterpret_cast<const uint4*>(dZ + int64_t(m) * zs + c);
            const bf16* e8 = reinterpret_cast<const bf16*>(&w);
#pragma unroll
            for (int e = 0; e < 8; ++e) As[q * 8 + e][r] = e8[e];
        }
        // BK positions x 64 k of the patch matrix, stored transposed
        for (int v = tid; v < BK * (BN / 8); v += 128) {
            const int r = v / (BN / 8), q = v % (BN / 8), m = mm + r;
            const uint4 w = m < me ? patch8(X, xs, ci, taps, m, k0 + q * 8, M, K, H, W) : make_uint4(0u, 0u, 0u, 0u);
            const bf16* e8 = reinterpret_cast<const bf16*>(&w);
#pragma unroll
            for (int e = 0; e < 8; ++e) Bs[q * 8 + e][r] = e8[e];
        }
        __syncthreads();
        tile_mma(As, Bs, acc, wm, wn, lane);
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + wm * 32 + i * 16 + g + (e >= 2 ? 8 : 0);
                const int k = k0 + wn * 32 + j * 8 + 2 * t + (e & 1);
                if (c >= co || k >= K) continue;
                if (part) part[(int64_t(blockIdx.z) * co + c) * K + k] = acc[i][j][e];
                else dW[int64_t(c) * K + k] += acc[i][j][e];      // one chunk: the only writer
            }
}

// dbias[c] += sum_m dZ[m][c]
// part[chunk][ch] = sum over the chunk's positions of dZ[m][ch]
__global__ void k_bias_grad(const bf16* __restrict__ dZ, int zs, int c, int M, int mchunk, float* __restrict__ part)
{
    const int ch = blockIdx.x * blockDim.x + threadIdx.x;
    if (ch >= c) return;
    const int mb = blockIdx.y * mchunk, me = min(M, mb + mchunk);
    float s = 0.0f;
    for (int m = mb; m < me; ++m) s += __bfloat162float(dZ[int64_t(m) * zs + ch]);
    part[int64_t(blockIdx.y) * c + ch] = s;
}

// acc[i] += sum_z part[z][i], z = 0, 1, ... in order (n values per slice)
__global__ void k_sum_slices(const float* __restrict__ part, int nz, int64_t n, float* __restrict__ acc)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = part[i];
    for (int z = 1; z < nz; ++z) v += part[int64_t(z) * n + i];
    acc[i] += v;
}

// Wflip[c][tap' * co + o] = Wt[o][(taps - 1 - tap') * ci + c]
__global__ void k_flip(const bf16* __restrict__ Wt, int ci, int co, int taps, bf16* __restrict__ Wf)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t n = int64_t(ci) * co * taps;
    if (i >= n) return;
    const int c = int(i / (int64_t(taps) * co)), rem = int(i % (int64_t(taps) * co));
    const int tp = rem / co, o = rem % co;
    Wf[i] = Wt[int64_t(o) * taps * ci + int64_t(taps - 1 - tp) * ci + c];
}

// dZ[m][c] = dY[m][c] (Y[m][yo + c] > 0), dY read at dy_stride / dy_offset
__global__ void k_relu_bwd(const bf16* __restrict__ dY, int dys, int dyo, const bf16* __restrict__ Y, int ys, int yo,
                           bf16* __restrict__ dZ, int zs, int c, int64_t M)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M * c) return;
    const int64_t m = i / c;
    const int ch = int(i % c);
    const float y = __bfloat162float(Y[m * ys + yo + ch]);
    dZ[m * zs + ch] = y > 0.0f ? dY[m * dys + dyo + ch] : __float2bfloat16_rn(0.0f);
}

// 2 x 2 average pooling: Y[b][y][x][c] = mean of X[b][2y..2y+1][2x..2x+1][c]
__global__ void k_pool(const bf16* __restrict__ X, int xs, int xo, bf16* __restrict__ Y, int ys, int yo, int c, int nb,
                       int H, int W)
{
    const int Ho = H / 2, Wo = W / 2;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nb) * Ho * Wo * c) return;
    const int ch = int(i % c);
    const int64_t mo = i / c;
    const int x = int(mo % Wo), r = int(mo / Wo), y = r % Ho, b = r / Ho;
    float s = 0.0f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            s += __bfloat162float(X[int64_t((b * H + 2 * y + dy) * W + 2 * x + dx) * xs + xo + ch]);
    Y[mo * ys + yo + ch] = __float2bfloat16_rn(0.25f * s);
}

// adjoint of k_pool, accumulated: dX[b][y][x][c] += dY[b][y/2][x/2][c] / 4
__global__ void k_pool_bwd(const bf16* __restrict__ dY, int dys, bf16* __restrict__ dX, int dxs, int dxo, int c, int nb,
                           int H, int W)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nb) * H * W * c) return;
    const int ch = int(i % c);
    const int64_t m = i / c;
    const int x = int(m % W), r = int(m / W), y = r % H, b = r / H;
    const float g = __bfloat162float(dY[int64_t((b * (H / 2) + y / 2) * (W / 2) + x / 2) * dys + ch]);
    bf16* p = dX + m * dxs + dxo + ch;
    *p = __float2bfloat16_rn(__bfloat162float(*p) + 0.25f * g);
}

// nearest 2x upsampling: Y[b][y][x][yo + c] = X[b][y/2][x/2][c] (Y is H x W)
__global__ void k_up(const bf16* __restrict__ X, int xs, bf16* __restrict__ Y, int ys, int yo, int c, int nb, int H,
                     int W)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nb) * H * W * c) return;
    const int ch = int(i % c);
    const int64_t m = i / c;
    const int x = int(m % W), r = int(m / W), y = r % H, b = r / H;
    Y[m * ys + yo + ch] = X[int64_t((b * (H / 2) + y / 2) * (W / 2) + x / 2) * xs + ch];
}

// adjoint of k_up: dX[b][y][x][c] = sum of dY over the 2 x 2 children (dY channels at dyo)
__global__ void k_up_bwd(const bf16* __restrict__ dY, int dys, int dyo, bf16* __restrict__ dX, int dxs, int c, int nb,
                         int H, int W)
{
    const int Ho = H / 2, Wo = W / 2;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nb) * Ho * Wo * c) return;
    const int ch = int(i % c);
    const int64_t mo = i / c;
    const int x = int(mo % Wo), r = int(mo / Wo), y = r % Ho, b = r / Ho;
    float s = 0.0f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            s += __bfloat162float(dY[int64_t((b * H + 2 * y + dy) * W + 2 * x + dx) * dys + dyo + ch]);
    dX[mo * dxs + ch] = __float2bfloat16_rn(s);
}

// residual head and loss: pred = x[:, :c] + d, r = pred - target;
// loss += sum r^2 / n (atomic); dd = 2 r / n (bf16, the gradient of the head)
__global__ void k_mse(const float* __restrict__ d, int dstr, const bf16* __restrict__ x, int xs, const float* __restrict__ target,
                      int c, int64_t M, float inv_n, float* __restrict__ pred, bf16* __restrict__ dd, int dds,
                      float* __restrict__ loss)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    float r2 = 0.0f;
    if (i < M * c) {
        const int64_t m = i / c;
        const int ch = int(i % c);
        const float p = __bfloat162float(x[m * xs + ch]) + d[m * dstr + ch];
        if (pred) pred[i] = p;
        if (target) {
            const float r = p - target[i];
            r2 = r * r * inv_n;
            if (dd) dd[m * dds + ch] = __float2bfloat16_rn(2.0f * r * inv_n);
        }
    }
    if (loss) {
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, r2);
    }
}

// Adam on float32 master weights; writes the bf16 copy the kernels read
__global__ void k_adam(float* __restrict__ w, float* __restrict__ mo, float* __restrict__ ve, const float* __restrict__ g,
                       bf16* __restrict__ wb, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float m = b1 * mo[i] + (1.0f - b1) * gi;
    const float v = b2 * ve[i] + (1.0f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    const float wi = w[i] - lr * (m * c1) / (sqrtf(v * c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, int64_t n)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// dA += dB over c channels (bf16 tensors with strides/offsets)
__global__ void k_add(const bf16* __restrict__ s, int ss, int so, bf16* __restrict__ d, int ds, int dof, int c, int64_t M)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= M * c) return;
    const int64_t m = i / c;
    const int ch = int(i % c);
    bf16* p = d + m * ds + dof + ch;
    *p = __float2bfloat16_rn(__bfloat162float(*p) + __bfloat162float(s[m * ss + so + ch]));
}

// Coarse input of the network from solver fields (planes [H][W] of phi, u, v
// at the fine resolution): mean over f x f cells, scaled, channels-last bf16
// x[b][y][x][c] with c = 0 phi, 1 u * su, 2 v * su, 3 cond, 4..cs-1 zero.
__global__ void k_coarsen(const float* __restrict__ phi, const float* __restrict__ u, const float* __restrict__ v,
                          int Hf, int Wf, int f, float su, float cond, bf16* __restrict__ x, int cs, float* __restrict__ xf)
{
    const int Hc = Hf / f, Wc = Wf / f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Hc * Wc) return;
    const int cx = i % Wc, cy = i / Wc;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    for (int dy = 0; dy < f; ++dy)
        for (int dx = 0; dx < f; ++dx) {
            const int64_t j = int64_t(cy * f + dy) * Wf + cx * f + dx;
            s0 += phi[j];
            s1 += u[j];
            s2 += v[j];
        }
    const float inv = 1.0f / float(f * f);
    const float vals[4] = {s0 * inv, s1 * inv * su, s2 * inv * su, cond};
    for (int c = 0; c < cs; ++c) {
        const float val = c < 4 ? vals[c] : 0.0f;
        if (x) x[int64_t(i) * cs + c] = __float2bfloat16_rn(val);
        if (xf && c < 3) xf[int64_t(i) * 3 + c] = val;
    }
}

// Fine fields from a coarse prediction pred[y][x][3] (phi, u su, v su):
// bilinear interpolation between coarse cell centres (clamped at the edges);
// phi clamped to [0, 1] and the speed to umax.
__global__ void k_refine(const float* __restrict__ pred, int Hc, int Wc, int f, float inv_su, float umax,
                         float* __restrict__ phi, float* __restrict__ u, float* __restrict__ v)
{
    const int Hf = Hc * f, Wf = Wc * f;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(Hf) * Wf) return;
    const int x = int(i % Wf), y = int(i / Wf);
    const float cx = (x + 0.5f) / f - 0.5f, cy = (y + 0.5f) / f - 0.5f;
    const int x0 = min(max(int(floorf(cx)), 0), Wc - 1), y0 = min(max(int(floorf(cy)), 0), Hc - 1);
    const int x1 = min(x0 + 1, Wc - 1), y1 = min(y0 + 1, Hc - 1);
    const float tx = fminf(fmaxf(cx - x0, 0.0f), 1.0f), ty = fminf(fmaxf(cy - y0, 0.0f), 1.0f);
    float out[3];
    for (int c = 0; c < 3; ++c) {
        const float a = pred[(int64_t(y0) * Wc + x0) * 3 + c], b = pred[(int64_t(y0) * Wc + x1) * 3 + c];
        const float d = pred[(int64_t(y1) * Wc + x0) * 3 + c], e = pred[(int64_t(y1) * Wc + x1) * 3 + c];
        out[c] = (1.0f - ty) * ((1.0f - tx) * a + tx * b) + ty * ((1.0f - tx) * d + tx * e);
    }
    const float uu = out[1] * inv_su, vv = out[2] * inv_su;
    const float sp = sqrtf(uu * uu + vv * vv), k = sp > umax ? umax / sp : 1.0f;
    phi[i] = fminf(fmaxf(out[0], 0.0f), 1.0f);
    u[i] = uu * k;
    v[i] = vv * k;
}

// part[block] = (sum phi, sum 4 q (1 - q)) over the block's 256 x 16 values
// (fixed order: per thread, then a shuffle tree, then the warps in order)
constexpr int kMassPer = 256 * 16;
__global__ void __launch_bounds__(256) k_mass_sums(const float* __restrict__ phi, int64_t n, double2* __restrict__ part)
{
    __shared__ double2 ws[8];
    const int64_t base = int64_t(blockIdx.x) * kMassPer;
    double a = 0.0, b = 0.0;
    for (int j = 0; j < 16; ++j) {
        const int64_t i = base + j * 256 + threadIdx.x;
        if (i < n) {
            const double p = phi[i], q = fmin(fmax(p, 0.0), 1.0);
            a += p;
            b += 4.0 * q * (1.0 - q);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_double2(a, b);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = ws[0];
        for (int w = 1; w < 8; ++w) {
            t.x += ws[w].x;
            t.y += ws[w].y;
        }
        part[blockIdx.x] = t;
    }
}

// sums = the block partials added in block order (one thread)
__global__ void k_mass_final(const double2* __restrict__ part, int nb, double* __restrict__ sums)
{
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
        a += part[i].x;
        b += part[i].y;
    }
    sums[0] = a;
    sums[1] = b;
}

// phi += c 4 phi (1 - phi), c = (target - sums[0]) / sums[1] (no change where sums[1] == 0)
__global__ void k_mass_apply(float* __restrict__ phi, int64_t n, double target, const double* __restrict__ sums)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n || !(sums[1] > 0.0)) return;
    const float c = float((target - sums[0]) / sums[1]);
    const float p = phi[i], q = fminf(fmaxf(p, 0.0f), 1.0f);
    phi[i] = p + c * 4.0f * q * (1.0f - q);
}

// Re-sharpening of a phase field whose interface profile is wider than the
// equilibrium one (a field refined from a coarse grid): phi <- 1/2 +
// 1/2 tanh(ratio atanh(2 q - 1)), q = phi clamped to [eps, 1 - eps].  On the
// profile 1/2 + 1/2 tanh(2 x / W') this gives the profile of width W' / ratio
// with the same phi = 1/2 crossing.
__global__ void k_sharpen(float* __restrict__ phi, int64_t n, float ratio)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float q = fminf(fmaxf(phi[i], 1e-6f), 1.0f - 1e-6f);
    phi[i] = 0.5f + 0.5f * tanhf(ratio * atanhf(2.0f * q - 1.0f));
}

// Interface comparison of two phase fields on an ny x nx grid:
// out[0] += cells where (a > 1/2) != (b > 1/2); out[1] += grid edges
// (x- and y-neighbours, periodic in x) across which b crosses 1/2;
// out[2] += sum a; out[3] += sum b.
__global__ void k_interface(const float* __restrict__ a, const float* __restrict__ b, int ny, int nx,
                            double* __restrict__ out)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double d = 0.0, e = 0.0, sa = 0.0, sb = 0.0;
    if (i < int64_t(ny) * nx) {
        const int x = int(i % nx), y = int(i / nx);
        const bool ia = a[i] > 0.5f, ib = b[i] > 0.5f;
        d = ia != ib ? 1.0 : 0.0;
        const int64_t ir = int64_t(y) * nx + (x + 1) % nx;
        e = ((b[ir] > 0.5f) != ib) ? 1.0 : 0.0;
        if (y + 1 < ny) e += ((b[i + nx] > 0.5f) != ib) ? 1.0 : 0.0;
        sa = a[i];
        sb = b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_down_sync(0xffffffffu, d, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], d);
        atomicAdd(&out[1], e);
        atomicAdd(&out[2], sa);
        atomicAdd(&out[3], sb);
    }
}

// Intact length of a jet issued along y from y = 0: per column x of
// [x0, x1), the number of cells from y = 0 up to the first phi <= 1/2;
// out[0] / out[1] = the largest over the columns, for a / b.
__global__ void k_jet_length(const float* __restrict__ a, const float* __restrict__ b, int ny, int nx, int x0, int x1,
                             int* __restrict__ out)
{
    const int x = x0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= x1) return;
    int la = 0, lb = 0;
    while (la < ny && a[int64_t(la) * nx + x] > 0.5f) ++la;
    while (lb < ny && b[int64_t(lb) * nx + x] > 0.5f) ++lb;
    atomicMax(&out[0], la);
    atomicMax(&out[1], lb);
}

thread_local std::string g_nn_err;

int nn_fail(int code, const std::string& msg)
{
    g_nn_err = msg;
    return code;
}

int nn_launch_status(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LBM_NN_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

unsigned blocks_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

constexpr int kTargetBlocks = 2 * 152;                  // two 128-thread blocks per SM of a GB300
constexpr int64_t kConvWsFloats = int64_t(1) << 22;     // largest split-K workspace (16 MB)

// forward convolution contraction: 0 tcgen05 (tensor memory), 1 warp-level
// mma.sync, 2 (default) by the call's work: tcgen05 for calls of at least
// 4 GFLOP (the tcgen05 blocks pay a fixed set-up -- tensor-memory allocation,
// barriers -- that a call of a few short k loops does not amortise; measured:
// the network's ~1.2 GFLOP layers of one input are faster on mma.sync, its
// ~19 GFLOP layers of 16 inputs on tcgen05), else mma.sync
int g_conv_path = 2;
constexpr double kTcMinFlop = 4e9;
// per-device error flag of the tcgen05 kernels (a bounded wait gave up)
int* g_tc_err[64] = {};

int tc_err_flag(int** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return nn_fail(LBM_NN_ERR_CUDA, "conv_fwd: no device");
    if (!g_tc_err[dev]) {
        e = cudaMalloc(reinterpret_cast<void**>(&g_tc_err[dev]), sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(g_tc_err[dev], 0, sizeof(int));
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_fwd: error flag: ") + cudaGetErrorString(e));
    }
    *out = g_tc_err[dev];
    return LBM_NN_OK;
}

template <int TN>
cudaError_t launch_tc(dim3 grid, cudaStream_t s, const bf16* X, int xs, int ci, int taps, const bf16* Wt,
                      const float* bias, int co, bf16* Y, int ys, int yo, float* Yf, int yfs, int relu, int M, int H,
                      int W, int kchunk, float* part, int* err)
{
    constexpr int smem = tc_smem_bytes<TN>();
    cudaError_t e = cudaFuncSetAttribute(k_conv_fwd_tc<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_conv_fwd_tc<TN><<<grid, 128, smem, s>>>(X, xs, ci, taps, Wt, bias, co, Y, ys, yo, Yf, yfs, relu, M, H, W, kchunk,
                                             part, err);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

const char* lbm_nn_last_error(void) { return g_nn_err.c_str(); }

int lbm_nn_conv_fwd(const void* x, int32_t x_stride, int32_t ci, int32_t taps, const void* wt, const float* bias,
                    int32_t co, void* y, int32_t y_stride, int32_t y_offset, float* yf, int32_t yf_stride, int32_t relu,
                    int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!x || !wt || (!y && !yf) || nb < 1 || h < 1 || w < 1 || co < 1) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: bad arguments");
    if (taps != 9 && taps != 1) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: taps must be 9 or 1");
    if (ci < 8 || ci % 8 || x_stride % 8 || x_stride < ci) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: ci and the input stride must be multiples of 8");
    if (!aligned16(x) || !aligned16(wt)) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: x and wt must be 16-byte aligned");
    if (y && (y_offset < 0 || y_offset + co > y_stride)) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: output channels exceed the stride");
    if (yf && yf_stride < co) return nn_fail(LBM_NN_ERR_ARG, "conv_fwd: f32 output stride below co");
    const int M = nb * h * w, K = taps * ci;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double flop = 2.0 * double(M) * double(co) * double(K);
    const bool tc = g_conv_path == 0 || (g_conv_path == 2 && flop >= kTcMinFlop);
    // tcgen05: 128 x 32 / 64 / 128 tiles by the channel count; mma.sync:
    // 128 x 32 tiles (no idle half of a 64-wide tile) or 64 x 64
    const bool narrow = co <= 32;
    const int TM = tc ? TC_TM : (narrow ? 128 : BM);
    const int TN = tc ? (co <= 32 ? 32 : co <= 64 ? 64 : 128) : (narrow ? 32 : BN);
    const int tiles = blocks_for(M, TM) * blocks_for(co, TN);
    // Split-K when the output tiles alone leave the GPU mostly idle (the deep,
    // coarse levels of the network): each split writes its partial sums to a
    // workspace slice, and k_conv_reduce adds them in split order.
    int splits = 1;
    if (tiles < kTargetBlocks && K >= 4 * BK) {
        splits = std::min((kTargetBlocks + tiles - 1) / tiles, K / (2 * BK));
        while (splits > 1 && int64_t(splits) * M * co > kConvWsFloats) --splits;
    }
    float* ws = nullptr;
    if (splits > 1) {
        // stream-ordered scratch: concurrent calls on other streams get their own
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), size_t(splits) * M * co * sizeof(float), s);
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_fwd: workspace: ") + cudaGetErrorString(e));
    }
    const int kstep = tc ? TC_BK : BK;
    const int kchunk = splits > 1 ? blocks_for(blocks_for(K, splits), kstep) * kstep : K;
    splits = blocks_for(K, kchunk);
    dim3 grid(blocks_for(M, TM), blocks_for(co, TN), splits);
    if (tc) {
        int* err = nullptr;
        const int r = tc_err_flag(&err);
        if (r != LBM_NN_OK) return r;
        const bf16* X = static_cast<const bf16*>(x);
        const bf16* Wt = static_cast<const bf16*>(wt);
        bf16* Y = static_cast<bf16*>(y);
        float* part = splits > 1 ? ws : nullptr;
        cudaError_t e;
        if (TN == 32) e = launch_tc<32>(grid, s, X, x_stride, ci, taps, Wt, bias, co, Y, y_stride, y_offset, yf, yf_stride, relu, M, h, w, kchunk, part, err);
        else if (TN == 64) e = launch_tc<64>(grid, s, X, x_stride, ci, taps, Wt, bias, co, Y, y_stride, y_offset, yf, yf_stride, relu, M, h, w, kchunk, part, err);
        else e = launch_tc<128>(grid, s, X, x_stride, ci, taps, Wt, bias, co, Y, y_stride, y_offset, yf, yf_stride, relu, M, h, w, kchunk, part, err);
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_fwd: ") + cudaGetErrorString(e));
    } else {
        auto kern = narrow ? k_conv_fwd<128, 32> : k_conv_fwd<BM, BN>;
        kern<<<grid, 128, 0, s>>>(static_cast<const bf16*>(x), x_stride, ci, taps, static_cast<const bf16*>(wt), bias,
                                  co, static_cast<bf16*>(y), y_stride, y_offset, yf, yf_stride, relu, M, h, w, kchunk,
                                  splits > 1 ? ws : nullptr);
    }
    if (ws) {
        k_conv_reduce<<<blocks_for(int64_t(M) * co, 256), 256, 0, s>>>(ws, splits, M, co, bias, relu,
                                                                       static_cast<bf16*>(y), y_stride, y_offset, yf,
                                                                       yf_stride);
        const cudaError_t e = cudaFreeAsync(ws, s);
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_fwd: workspace: ") + cudaGetErrorString(e));
    }
    return nn_launch_status("conv_fwd");
}

int lbm_nn_conv_wgrad(const void* x, int32_t x_stride, int32_t ci, int32_t taps, const void* dz, int32_t dz_stride,
                      int32_t co, float* dwt, float* dbias, int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!x || !dz || !dwt || nb < 1 || h < 1 || w < 1 || co < 1) return nn_fail(LBM_NN_ERR_ARG, "conv_wgrad: bad arguments");
    if (taps != 9 && taps != 1) return nn_fail(LBM_NN_ERR_ARG, "conv_wgrad: taps must be 9 or 1");
    if (ci < 8 || ci % 8 || x_stride % 8 || co % 8 || dz_stride % 8) return nn_fail(LBM_NN_ERR_ARG, "conv_wgrad: channels and strides must be multiples of 8");
    if (x_stride < ci || dz_stride < co) return nn_fail(LBM_NN_ERR_ARG, "conv_wgrad: strides below the channel counts");
    if (!aligned16(x) || !aligned16(dz)) return nn_fail(LBM_NN_ERR_ARG, "conv_wgrad: x and dz must be 16-byte aligned");
    const int M = nb * h * w, K = taps * ci;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // positions split into chunks of at least 1024 (fewer when the partial
    // tiles would not fit the scratch cap); each chunk's partial weight
    // gradient goes to its own slice, and the slices are added to dwt in
    // chunk order: no atomics, the same result on every run
    int nchunk = int(blocks_for(M, 1024));
    while (nchunk > 1 && int64_t(nchunk) * co * K > kConvWsFloats) nchunk = (nchunk + 1) / 2;
    const int mchunk = int(blocks_for(M, nchunk));
    nchunk = int(blocks_for(M, mchunk));
    const int bchunk = 4096, nbc = dbias ? int(blocks_for(M, bchunk)) : 0;
    const size_t wfl = nchunk > 1 ? size_t(nchunk) * co * K : 0, bfl = size_t(nbc) * co;
    float* ws = nullptr;
    if (wfl + bfl > 0) {
        const cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), (wfl + bfl) * sizeof(float), s);
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_wgrad: workspace: ") + cudaGetErrorString(e));
    }
    dim3 grid(blocks_for(co, BM), blocks_for(K, BN), nchunk);
    k_conv_wgrad<<<grid, 128, 0, s>>>(static_cast<const bf16*>(x), x_stride, ci, taps, static_cast<const bf16*>(dz),
                                      dz_stride, co, dwt, M, h, w, mchunk, nchunk > 1 ? ws : nullptr);
    if (nchunk > 1)
        k_sum_slices<<<blocks_for(int64_t(co) * K, 256), 256, 0, s>>>(ws, nchunk, int64_t(co) * K, dwt);
    if (dbias) {
        dim3 gb(blocks_for(co, 64), nbc);
        k_bias_grad<<<gb, 64, 0, s>>>(static_cast<const bf16*>(dz), dz_stride, co, M, bchunk, ws + wfl);
        k_sum_slices<<<blocks_for(co, 256), 256, 0, s>>>(ws + wfl, nbc, co, dbias);
    }
    if (ws) {
        const cudaError_t e = cudaFreeAsync(ws, s);
        if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_wgrad: workspace: ") + cudaGetErrorString(e));
    }
    return nn_launch_status("conv_wgrad");
}

int lbm_nn_set_conv_path(int32_t path)
{
    if (path < 0 || path > 2) return nn_fail(LBM_NN_ERR_ARG, "conv path must be 0 (tcgen05), 1 (mma.sync) or 2 (by size)");
    g_conv_path = path;
    return LBM_NN_OK;
}

int lbm_nn_conv_status(int32_t* timed_out)
{
    if (!timed_out) return nn_fail(LBM_NN_ERR_ARG, "conv_status: NULL");
    int* err = nullptr;
    const int r = tc_err_flag(&err);
    if (r != LBM_NN_OK) return r;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("conv_status: ") + cudaGetErrorString(e));
    *timed_out = h;
    return LBM_NN_OK;
}

int lbm_nn_flip_weights(const void* wt, int32_t ci, int32_t co, int32_t taps, void* wflip, void* stream)
{
    if (!wt || !wflip || ci < 1 || co < 1 || (taps != 9 && taps != 1)) return nn_fail(LBM_NN_ERR_ARG, "flip: bad arguments");
    const int64_t n = int64_t(ci) * co * taps;
    k_flip<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(wt), ci, co, taps,
                                                                              static_cast<bf16*>(wflip));
    return nn_launch_status("flip");
}

int lbm_nn_relu_bwd(const void* dy, int32_t dy_stride, int32_t dy_offset, const void* y, int32_t y_stride,
                    int32_t y_offset, void* dz, int32_t dz_stride, int32_t c, int64_t m, void* stream)
{
    if (!dy || !y || !dz || c < 1 || m < 1) return nn_fail(LBM_NN_ERR_ARG, "relu_bwd: bad arguments");
    k_relu_bwd<<<blocks_for(m * c, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(dy), dy_stride, dy_offset, static_cast<const bf16*>(y), y_stride, y_offset,
        static_cast<bf16*>(dz), dz_stride, c, m);
    return nn_launch_status("relu_bwd");
}

int lbm_nn_pool(const void* x, int32_t x_stride, int32_t x_offset, void* y, int32_t y_stride, int32_t y_offset,
                int32_t c, int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!x || !y || c < 1 || h % 2 || w % 2) return nn_fail(LBM_NN_ERR_ARG, "pool: bad arguments");
    const int64_t n = int64_t(nb) * (h / 2) * (w / 2) * c;
    k_pool<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(x), x_stride, x_offset, static_cast<bf16*>(y), y_stride, y_offset, c, nb, h, w);
    return nn_launch_status("pool");
}

int lbm_nn_pool_bwd(const void* dy, int32_t dy_stride, void* dx, int32_t dx_stride, int32_t dx_offset, int32_t c,
                    int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!dy || !dx || c < 1 || h % 2 || w % 2) return nn_fail(LBM_NN_ERR_ARG, "pool_bwd: bad arguments");
    const int64_t n = int64_t(nb) * h * w * c;
    k_pool_bwd<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(dy), dy_stride, static_cast<bf16*>(dx), dx_stride, dx_offset, c, nb, h, w);
    return nn_launch_status("pool_bwd");
}

int lbm_nn_upsample(const void* x, int32_t x_stride, void* y, int32_t y_stride, int32_t y_offset, int32_t c,
                    int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!x || !y || c < 1 || h % 2 || w % 2) return nn_fail(LBM_NN_ERR_ARG, "upsample: bad arguments");
    const int64_t n = int64_t(nb) * h * w * c;
    k_up<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(x), x_stride, static_cast<bf16*>(y), y_stride, y_offset, c, nb, h, w);
    return nn_launch_status("upsample");
}

int lbm_nn_upsample_bwd(const void* dy, int32_t dy_stride, int32_t dy_offset, void* dx, int32_t dx_stride, int32_t c,
                        int32_t nb, int32_t h, int32_t w, void* stream)
{
    if (!dy || !dx || c < 1 || h % 2 || w % 2) return nn_fail(LBM_NN_ERR_ARG, "upsample_bwd: bad arguments");
    const int64_t n = int64_t(nb) * (h / 2) * (w / 2) * c;
    k_up_bwd<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(dy), dy_stride, dy_offset, static_cast<bf16*>(dx), dx_stride, c, nb, h, w);
    return nn_launch_status("upsample_bwd");
}

int lbm_nn_mse(const float* d, int32_t d_stride, const void* x, int32_t x_stride, const float* target, int32_t c,
               int64_t m, float* pred, void* dd, int32_t dd_stride, float* loss, void* stream)
{
    if (!d || !x || c < 1 || m < 1 || d_stride < c || x_stride < c) return nn_fail(LBM_NN_ERR_ARG, "mse: bad arguments");
    const int64_t n = m * c;
    k_mse<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d, d_stride, static_cast<const bf16*>(x), x_stride, target, c, m, 1.0f / float(n), pred, static_cast<bf16*>(dd),
        dd_stride, loss);
    return nn_launch_status("mse");
}

int lbm_nn_adam(float* w, float* m, float* v, const float* g, void* w_bf16, int64_t n, float lr, float beta1,
                float beta2, float eps, int32_t t, void* stream)
{
    if (!w || !m || !v || !g || n < 1 || t < 1) return nn_fail(LBM_NN_ERR_ARG, "adam: bad arguments");
    const float c1 = 1.0f / (1.0f - powf(beta1, float(t))), c2 = 1.0f / (1.0f - powf(beta2, float(t)));
    k_adam<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(w, m, v, g, static_cast<bf16*>(w_bf16), n,
                                                                             lr, beta1, beta2, eps, c1, c2);
    return nn_launch_status("adam");
}

int lbm_nn_to_bf16(const float* a, void* b, int64_t n, void* stream)
{
    if (!a || !b || n < 1) return nn_fail(LBM_NN_ERR_ARG, "to_bf16: bad arguments");
    k_to_bf16<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, static_cast<bf16*>(b), n);
    return nn_launch_status("to_bf16");
}

int lbm_nn_add(const void* src, int32_t src_stride, int32_t src_offset, void* dst, int32_t dst_stride,
               int32_t dst_offset, int32_t c, int64_t m, void* stream)
{
    if (!src || !dst || c < 1 || m < 1) return nn_fail(LBM_NN_ERR_ARG, "add: bad arguments");
    k_add<<<blocks_for(m * c, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(src), src_stride, src_offset, static_cast<bf16*>(dst), dst_stride, dst_offset, c, m);
    return nn_launch_status("add");
}

int lbm_nn_coarsen(const float* phi, const float* u, const float* v, int32_t hf, int32_t wf, int32_t factor,
                   float u_scale, float cond, void* x, int32_t x_channels, float* xf, void* stream)
{
    if (!phi || !u || !v || factor < 1 || hf % factor || wf % factor || (!x && !xf) || (x && x_channels < 4))
        return nn_fail(LBM_NN_ERR_ARG, "coarsen: bad arguments");
    const int n = (hf / factor) * (wf / factor);
    k_coarsen<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(phi, u, v, hf, wf, factor, u_scale, cond,
                                                                                 static_cast<bf16*>(x), x_channels, xf);
    return nn_launch_status("coarsen");
}

int lbm_nn_refine(const float* pred, int32_t hc, int32_t wc, int32_t factor, float u_scale, float u_max, float* phi,
                  float* u, float* v, void* stream)
{
    if (!pred || !phi || !u || !v || factor < 1 || hc < 1 || wc < 1 || !(u_scale > 0.0f) || !(u_max > 0.0f))
        return nn_fail(LBM_NN_ERR_ARG, "refine: bad arguments");
    const int64_t n = int64_t(hc) * factor * wc * factor;
    k_refine<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(pred, hc, wc, factor, 1.0f / u_scale,
                                                                               u_max, phi, u, v);
    return nn_launch_status("refine");
}

int lbm_nn_sharpen(float* phi, int64_t n, float ratio, void* stream)
{
    if (!phi || n < 1 || !(ratio > 0.0f)) return nn_fail(LBM_NN_ERR_ARG, "sharpen: bad arguments");
    k_sharpen<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(phi, n, ratio);
    return nn_launch_status("sharpen");
}

int lbm_nn_mass_project(float* phi, int64_t n, double target, double* sums, void* stream)
{
    if (!phi || !sums || n < 1) return nn_fail(LBM_NN_ERR_ARG, "mass_project: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = int(blocks_for(n, kMassPer));
    double2* part = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&part), size_t(nb) * sizeof(double2), s);
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("mass_project: ") + cudaGetErrorString(e));
    k_mass_sums<<<nb, 256, 0, s>>>(phi, n, part);
    k_mass_final<<<1, 1, 0, s>>>(part, nb, sums);
    k_mass_apply<<<blocks_for(n, 256), 256, 0, s>>>(phi, n, target, sums);
    e = cudaFreeAsync(part, s);
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("mass_project: ") + cudaGetErrorString(e));
    return nn_launch_status("mass_project");
}

int lbm_nn_interface_stats(const float* a, const float* b, int32_t ny, int32_t nx, double* out, void* stream)
{
    if (!a || !b || !out || ny < 1 || nx < 1) return nn_fail(LBM_NN_ERR_ARG, "interface_stats: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(double), s);
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("interface_stats: ") + cudaGetErrorString(e));
    k_interface<<<blocks_for(int64_t(ny) * nx, 256), 256, 0, s>>>(a, b, ny, nx, out);
    return nn_launch_status("interface_stats");
}

int lbm_nn_jet_length(const float* a, const float* b, int32_t ny, int32_t nx, int32_t x0, int32_t x1, int32_t* out,
                      void* stream)
{
    if (!a || !b || !out || ny < 1 || nx < 1 || x0 < 0 || x1 > nx || x0 >= x1)
        return nn_fail(LBM_NN_ERR_ARG, "jet_length: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return nn_fail(LBM_NN_ERR_CUDA, std::string("jet_length: ") + cudaGetErrorString(e));
    k_jet_length<<<blocks_for(x1 - x0, 128), 128, 0, s>>>(a, b, ny, nx, x0, x1, out);
    return nn_launch_status("jet_length");
}

}  // extern "C"
