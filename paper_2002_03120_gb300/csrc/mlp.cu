// mlp.cu -- the apparent-viscosity surrogate network on GB300 tensor cores.
//
// Network (a build component, not in the paper): 3 -> 128 -> 128 -> 128 ->
// 128 -> 1, GELU (erf form) after every hidden layer, MSE loss, Adam.  The
// three 128 x 128 layers run as tcgen05 MMAs (kind::f16, BF16 operands for
// both A and B, FP32 accumulators in tensor memory); the 3 -> 128 input layer,
// the 128 -> 1 output layer and all element-wise work run in FP32 on the CUDA
// cores.  One MMA tile is M = 128 rows x N = 128 x K = 128 (eight K = 16
// steps), issued by one thread; completion is signalled through an mbarrier
// by tcgen05.commit; the epilogue reads the accumulator rows with tcgen05.ld
// (thread t of the 128 owns row t = TMEM lane t).
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, core (row group g, K chunk c) at byte offset
// (16 g + c) * 128 of a 32 KB tile; descriptor leading-dimension offset 128 B
// (next K chunk), stride-dimension offset 2048 B (next 8-row group).  Every
// address an MMA can touch lies inside its 32 KB tile.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace sdpd {
namespace mlp {

constexpr int WID = 128;
constexpr int NIN = 3;
constexpr int TILE_BYTES = WID * WID * 2;  // one 128 x 128 bf16 operand
constexpr int NPARAM = WID * NIN + WID + 3 * (WID * WID + WID) + WID + 1;
// flat parameter offsets: W0 [128][3], b0, W1 [128][128], b1, W2, b2, W3, b3, W4 [128], b4
constexpr int OFF_W0 = 0, OFF_B0 = OFF_W0 + WID * NIN;
__host__ __device__ constexpr int off_W(int l) { return OFF_B0 + WID + (l - 1) * (WID * WID + WID); }
__host__ __device__ constexpr int off_b(int l) { return off_W(l) + WID * WID; }
constexpr int OFF_W4 = OFF_B0 + WID + 3 * (WID * WID + WID), OFF_B4 = OFF_W4 + WID;
static_assert(OFF_B4 + 1 == NPARAM, "parameter layout");

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A BF16 (bits
// 7-9 = 1), B BF16 (bits 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(WID >> 3) << 17) |
                           ((uint32_t)(WID >> 4) << 24);
constexpr long long WAIT_LIMIT = 1LL << 22;   // bounded mbarrier wait (iterations)
constexpr int ERR_MMA_TIMEOUT = 1;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a 128 x 128 operand in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (uint32_t)(((r >> 3) * 16 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;    // leading dimension byte offset: next K chunk
    d |= (uint64_t)(2048u >> 4) << 32;   // stride dimension byte offset: next 8-row group
    d |= (uint64_t)1 << 46;              // descriptor version
    return d;                            // base offset 0, no swizzle
}

__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
}

// Bounded wait for the phase with parity `par`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t par)
{
    const uint32_t a = smem_u32(mbar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(par)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive accumulator columns of this thread's lane (row).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// exp2 on the special-function unit (relative error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erf by Abramowitz & Stegun, Handbook of Mathematical Functions, formula
// 7.1.26 (Hastings' rational approximation), |error| <= 1.5e-7: one
// reciprocal, one exponential, no branch.
__device__ __forceinline__ float erf_as(float x)
{
    const float a = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, a, 1.0f));
    float p = fmaf(1.061405429f, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    p *= t;
    const float r = fmaf(-p, ex2_approx(-a * a * 1.44269504088896341f), 1.0f);
    return copysignf(r, x);
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU, erf form: 0.5 z (1 + erf(z / sqrt 2)) = z (1 - h) for z >= 0 and
// z h for z < 0, with h = 0.5 erfc(|z| / sqrt 2) = 0.5 P(t) exp(-z^2 / 2) from
// the same Abramowitz & Stegun 7.1.26 polynomial (coefficients halved).
__device__ __forceinline__ float gelu(float z)
{
    const float a = fabsf(z) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.3275911f, a, 1.0f));
    float p = fmaf(0.5f * 1.061405429f, t, 0.5f * -1.453152027f);
    p = fmaf(p, t, 0.5f * 1.421413741f);
    p = fmaf(p, t, 0.5f * -0.284496736f);
    p = fmaf(p, t, 0.5f * 0.254829592f);
    const float h = (p * t) * ex2_approx(z * z * -0.72134752044448170f);
    return z * (z >= 0.0f ? 1.0f - h : h);
}
__device__ __forceinline__ float gelu_prime(float z)
{
    return 0.5f * (1.0f + erf_as(z * 0.70710678118654752f)) +
           z * ex2_approx(-0.5f * 1.44269504088896341f * z * z) * 0.39894228040143268f;
}

// Eight values of one row, written as one 16-byte core-matrix row.
__device__ __forceinline__ void put8(uint8_t *tile, int r, int k0, const float *v)
{
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(tile + core_off(r, k0)) = *reinterpret_cast<uint4 *>(h);
}

__device__ __forceinline__ void put1(uint8_t *tile, int r, int k, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(tile + core_off(r, k)) = __float2bfloat16_rn(v);
}

// D(128 x 128, TMEM) (+)= A(tile) . B(tile)^T over K = 128 in eight K = 16
// steps, issued by thread 0; every thread waits for completion.  Returns
// false if the wait timed out (error recorded).
__device__ bool gemm_128(uint8_t *A, uint8_t *B, uint32_t dtmem, bool accumulate, uint64_t *mbar,
                         uint32_t &parity, int *err)
{
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
        for (int s = 0; s < 8; ++s)
            mma_bf16(dtmem, make_desc(a0 + s * 256), make_desc(b0 + s * 256), (accumulate || s > 0) ? 1 : 0);
        mma_commit(mbar);
    }
    const bool ok = mbar_wait(mbar, parity);
    if (!ok) {
        // record the failure, then give the MMAs in flight one more bounded
        // wait before the caller frees tensor memory
        if (threadIdx.x == 0) atomicOr(err, ERR_MMA_TIMEOUT);
        (void)mbar_wait(mbar, parity);
    }
    parity ^= 1u;
    tc_fence_after();
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Row t (= this thread) of the accumulator, column chunk c (16 values).
__device__ __forceinline__ void acc_row16(uint32_t taddr, int c, float v[16])
{
    const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) * 32) << 16;
    tc_ld16(taddr + lane_base + (uint32_t)(c * 16), v);
}

struct Net {
    float *P;            // FP32 master parameters [NPARAM]
    float *G;            // gradients [NPARAM]
    float *M, *V;        // Adam moments
    __nv_bfloat16 *Wb;   // BF16 copies of W1..W3 [3][128][128]
    float *Z, *H0, *D;   // training scratch: Z [4][Bmax][128], first-layer input copy, dz buffers
    float *Gp, *Lp;      // per-tile gradient shares [Bmax/128][NPARAM] and squared-error sums
    float *Y, *DY, *loss;
    int *err;
    int bmax;
    long long step;
    cudaStream_t own;
};

// Stage the BF16 weights of layer l (as B operand: rows = out, K = in) or
// its transpose (rows = in, K = out).
__device__ void stage_weights(uint8_t *tile, const __nv_bfloat16 *W, bool transpose)
{
    const int t = threadIdx.x;
    if (!transpose) {
        float v[8];
        for (int c = 0; c < 16; ++c) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __bfloat162float(W[t * WID + 8 * c + i]);
            put8(tile, t, 8 * c, v);
        }
    } else {
        // row i = t of W^T: column t of W
        float v[8];
        for (int c = 0; c < 16; ++c) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __bfloat162float(W[(8 * c + i) * WID + t]);
            put8(tile, t, 8 * c, v);
        }
    }
}

// ------------------------------------------------------------- inference
// Persistent over 128-row tiles with NWG warpgroups per CTA: each warpgroup
// owns one tile at a time (its own activation operand in shared memory and
// its own 128 accumulator columns in tensor memory) and synchronises only
// with itself (named barrier g + 1), so the MMAs of one warpgroup overlap
// the GELU epilogues of the others.  The three hidden weight tiles are
// staged once per CTA and shared.
constexpr int NWG = 4;
constexpr size_t FWD_SMEM = (size_t)(3 + NWG) * TILE_BYTES + 128;

__device__ __forceinline__ void wg_bar(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }

// Row r (output unit) of one hidden weight tile, as the B operand.
__device__ __forceinline__ void stage_row(uint8_t *tile, const __nv_bfloat16 *W, int r)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(W + r * WID);
#pragma unroll
    for (int c = 0; c < 16; ++c) *reinterpret_cast<uint4 *>(tile + core_off(r, 8 * c)) = __ldg(src + c);
}

// D(128 x 128) = A . B^T for warpgroup g; thread tt == 0 of the warpgroup
// issues, all 128 threads wait.  A timeout in any thread is seen by all
// (flag in shared memory read after the barrier), so the warpgroup leaves
// its loop together.
__device__ bool wg_gemm(uint8_t *A, uint8_t *B, uint32_t dtmem, uint64_t *mbar, uint32_t &parity, int g,
                        int tt, volatile int *flag, int *err)
{
    proxy_fence();
    tc_fence_before();
    wg_bar(g);
    if (tt == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
        for (int s = 0; s < 8; ++s) mma_bf16(dtmem, make_desc(a0 + s * 256), make_desc(b0 + s * 256), s > 0 ? 1 : 0);
        mma_commit(mbar);
    }
    if (!mbar_wait(mbar, parity)) {
        *flag = 1;
        atomicOr(err, ERR_MMA_TIMEOUT);
        (void)mbar_wait(mbar, parity);
    }
    parity ^= 1u;
    tc_fence_after();
    wg_bar(g);
    return *flag == 0;
}

__global__ void __launch_bounds__(128 * NWG, 1) k_mlp_forward(const float *__restrict__ P,
                                                              const __nv_bfloat16 *__restrict__ Wb,
                                                              const float *__restrict__ X, float *__restrict__ Y,
                                                              long long n, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;                                        // 3 weight tiles
    const int g = threadIdx.x >> 7, tt = threadIdx.x & 127;
    uint8_t *sA = smem + (3 + g) * TILE_BYTES;                 // this warpgroup's activations
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (3 + NWG) * TILE_BYTES) + g;
    volatile int *flag = reinterpret_cast<int *>(smem + (3 + NWG) * TILE_BYTES + 64) + g;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + (3 + NWG) * TILE_BYTES + 96);
    for (int r = threadIdx.x; r < 3 * WID; r += blockDim.x)
        stage_row(sB + (r >> 7) * TILE_BYTES, Wb + (r >> 7) * WID * WID, r & 127);
    if (tt == 0) {
        mbar_init(mbar);
        *flag = 0;
    }
    if (threadIdx.x < 32) tc_alloc(slot, 128 * NWG);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tcols = *slot + (uint32_t)(g * WID);                         // this warpgroup's columns
    const uint32_t tl = tcols + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16);  // + this warp's lanes
    const float4 *P4 = reinterpret_cast<const float4 *>(P);
    uint32_t parity = 0;
    bool ok = true;
    for (long long tile = (long long)blockIdx.x * NWG + g; ok && tile * WID < n; tile += (long long)gridDim.x * NWG) {
        const long long row = tile * WID + tt;
        const bool valid = row < n;
        const float x0 = valid ? X[3 * row] : 0.f, x1 = valid ? X[3 * row + 1] : 0.f,
                    x2 = valid ? X[3 * row + 2] : 0.f;
        // input layer 3 -> 128 (FP32), W0 rows 8c..8c+7 = 24 floats = 6 float4
#pragma unroll 2
        for (int c = 0; c < 16; ++c) {
            float w[24], bb[8], h[8];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float4 q = __ldg(P4 + (OFF_W0 / 4) + 6 * c + k);
                w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float4 q = __ldg(P4 + (OFF_B0 / 4) + 2 * c + k);
                bb[4 * k] = q.x; bb[4 * k + 1] = q.y; bb[4 * k + 2] = q.z; bb[4 * k + 3] = q.w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) h[i] = gelu(fmaf(w[3 * i], x0, fmaf(w[3 * i + 1], x1, fmaf(w[3 * i + 2], x2, bb[i]))));
            put8(sA, tt, 8 * c, h);
        }
        float y = 0.f;
        for (int l = 1; l <= 3; ++l) {
            ok = wg_gemm(sA, sB + (l - 1) * TILE_BYTES, tcols, mbar, parity, g, tt, flag, err);
            if (!ok) break;
            for (int c = 0; c < 8; ++c) {
                float v[16];
                tc_ld16(tl + (uint32_t)(c * 16), v);
                float bb[16];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 q = __ldg(P4 + off_b(l) / 4 + 4 * c + k);
                    bb[4 * k] = q.x; bb[4 * k + 1] = q.y; bb[4 * k + 2] = q.z; bb[4 * k + 3] = q.w;
                }
                if (l < 3) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = gelu(v[i] + bb[i]);
                    put8(sA, tt, 16 * c, v);
                    put8(sA, tt, 16 * c + 8, v + 8);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 q = __ldg(P4 + OFF_W4 / 4 + 4 * c + k);
                        y = fmaf(gelu(v[4 * k] + bb[4 * k]), q.x, y);
                        y = fmaf(gelu(v[4 * k + 1] + bb[4 * k + 1]), q.y, y);
                        y = fmaf(gelu(v[4 * k + 2] + bb[4 * k + 2]), q.z, y);
                        y = fmaf(gelu(v[4 * k + 3] + bb[4 * k + 3]), q.w, y);
                    }
                }
            }
        }
        if (valid && ok) Y[row] = y + P[OFF_B4];
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc_dealloc(*slot, 128 * NWG);
}

// ------------------------------------------------------------- training
// One CTA per 128-row tile of the batch: forward (pre-activations kept in Z),
// backward through every layer for the tile's rows, the tile's share of each
// gradient into its row of Gp [ntile][NPARAM] and its squared-error sum into
// Lp[tile]; k_mlp_reduce adds the tiles in a fixed order.  The output
// gradient dy = 2 (y - t) / B needs no sum across tiles, so the tiles are
// independent.  Thread t owns batch row tile * 128 + t (TMEM lane t) in the
// row-wise steps and output unit t in the column-wise sums.
__global__ void __launch_bounds__(128, 1) k_mlp_grad(Net net, const float *__restrict__ X,
                                                     const float *__restrict__ T, int B)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;                       // A operand
    uint8_t *sB = smem + TILE_BYTES;          // B operand
    uint8_t *sC = smem + 2 * TILE_BYTES;      // second A (weight-gradient GEMM)
    uint8_t *sD = smem + 3 * TILE_BYTES;      // second B
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 4 * TILE_BYTES);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 4 * TILE_BYTES + 16);
    float *red = reinterpret_cast<float *>(smem + 4 * TILE_BYTES + 32);   // 4 floats
    const int t = threadIdx.x;
    const int tile = blockIdx.x;
    const int r0 = tile * WID;                // first batch row of the tile
    const int nrow = min(WID, B - r0);        // rows of this tile
    const int row = r0 + t;
    const bool valid = t < nrow;
    const int bm = net.bmax;
    float *Z = net.Z;                         // [4][bmax][128]
    float *Dc = net.D, *Dn = net.D + (size_t)bm * WID;   // dz of the current / next layer
    float *Gp = net.Gp + (size_t)tile * NPARAM;
    const float *P = net.P;
    if (t == 0) mbar_init(mbar);
    if (t < 32) tc_alloc(slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *slot;             // columns [0,128): activations; [128,256): weight gradients
    uint32_t parity = 0;
    bool ok = true;
    float v[16];
    // ---------------- forward, keeping the pre-activations
    const float x0 = valid ? X[3 * row] : 0.f, x1 = valid ? X[3 * row + 1] : 0.f, x2 = valid ? X[3 * row + 2] : 0.f;
    for (int c = 0; c < 16; ++c) {
        float h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int o = 8 * c + i;
            const float z = P[OFF_W0 + 3 * o] * x0 + P[OFF_W0 + 3 * o + 1] * x1 + P[OFF_W0 + 3 * o + 2] * x2 +
                            P[OFF_B0 + o];
            Z[(0 * bm + row) * WID + o] = valid ? z : 0.f;
            h[i] = valid ? gelu(z) : 0.f;
        }
        put8(sA, t, 8 * c, h);
    }
    float y = 0.f;
    for (int l = 1; l <= 3 && ok; ++l) {
        stage_weights(sB, net.Wb + (l - 1) * WID * WID, false);
        ok = gemm_128(sA, sB, taddr, false, mbar, parity, net.err);
        if (!ok) break;
        for (int c = 0; c < 8; ++c) {
            acc_row16(taddr, c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int o = 16 * c + i;
                const float z = v[i] + P[off_b(l) + o];
                Z[(l * bm + row) * WID + o] = valid ? z : 0.f;
                const float h = valid ? gelu(z) : 0.f;
                if (l < 3) v[i] = h;
                else y += h * P[OFF_W4 + o];
            }
            if (l < 3) {
                put8(sA, t, 16 * c, v);
                put8(sA, t, 16 * c + 8, v + 8);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) goto done;
    {
        float dy = 0.f, sq = 0.f;
        if (valid) {
            y += P[OFF_B4];
            net.Y[row] = y;
            dy = 2.0f * (y - T[row]) / (float)B;
            sq = (y - T[row]) * (y - T[row]);
        }
        net.DY[row] = dy;   // 0 on the rows past B (the scratch holds whole tiles)
        // the tile's squared-error sum, fixed order: warps, then warps 0..3
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if ((t & 31) == 0) red[t >> 5] = sq;
        __syncthreads();
        if (t == 0) net.Lp[tile] = (red[0] + red[1]) + (red[2] + red[3]);
        // output layer (thread t = unit o): gW4 = sum_rows dy gelu(z3), gb4 = sum_rows dy
        float gw = 0.f, gb = 0.f;
        for (int r = 0; r < nrow; ++r) {
            const float d = net.DY[r0 + r];
            gw += d * gelu(Z[(3 * bm + r0 + r) * WID + t]);
            gb += d;
        }
        Gp[OFF_W4 + t] = gw;
        if (t == 0) Gp[OFF_B4] = gb;
        // dz of the last hidden layer for this thread's row
        for (int o = 0; o < WID; ++o)
            Dc[row * WID + o] = valid ? dy * P[OFF_W4 + o] * gelu_prime(Z[(3 * bm + row) * WID + o]) : 0.f;
    }
    __syncthreads();
    // ---------------- hidden layers l = 3, 2, 1 (z_l = W_l a_{l-1} + b_l)
    for (int l = 3; l >= 1 && ok; --l) {
        // weight gradient over the tile: A = dz^T (rows = unit o, K = row), B = a^T (rows = input i, K = row)
        for (int o = 0; o < WID; ++o) {
            put1(sC, o, t, Dc[row * WID + o]);
            put1(sD, o, t, valid ? gelu(Z[((l - 1) * bm + row) * WID + o]) : 0.f);
        }
        ok = gemm_128(sC, sD, taddr + 128, false, mbar, parity, net.err);
        if (!ok) break;
        for (int c = 0; c < 8; ++c) {
            acc_row16(taddr + 128, c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) Gp[off_W(l) + t * WID + 16 * c + i] = v[i];
        }
        {
            float gb = 0.f;
            for (int r = 0; r < nrow; ++r) gb += Dc[(r0 + r) * WID + t];
            Gp[off_b(l) + t] = gb;
        }
        tc_fence_before();
        __syncthreads();
        // input gradient: dh = dz W_l (A = dz rows, B = W_l^T), dz_{l-1} = dh gelu'(z_{l-1})
        stage_weights(sB, net.Wb + (l - 1) * WID * WID, true);
        for (int c = 0; c < 16; ++c) put8(sA, t, 8 * c, Dc + row * WID + 8 * c);
        ok = gemm_128(sA, sB, taddr, false, mbar, parity, net.err);
        if (!ok) break;
        for (int c = 0; c < 8; ++c) {
            acc_row16(taddr, c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int o = 16 * c + i;
                Dn[row * WID + o] = valid ? v[i] * gelu_prime(Z[((l - 1) * bm + row) * WID + o]) : 0.f;
            }
        }
        tc_fence_before();
        __syncthreads();
        float *tmp = Dc;
        Dc = Dn;
        Dn = tmp;
    }
    if (ok) {
        // input layer (thread t = unit o): gW0 = dz_0^T x, gb0 = sum dz_0
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, gb = 0.f;
        for (int r = 0; r < nrow; ++r) {
            const float d = Dc[(r0 + r) * WID + t];
            g0 += d * X[3 * (r0 + r)];
            g1 += d * X[3 * (r0 + r) + 1];
            g2 += d * X[3 * (r0 + r) + 2];
            gb += d;
        }
        Gp[OFF_W0 + 3 * t] = g0;
        Gp[OFF_W0 + 3 * t + 1] = g1;
        Gp[OFF_W0 + 3 * t + 2] = g2;
        Gp[OFF_B0 + t] = gb;
    }
done:
    tc_fence_before();
    __syncthreads();
    if (t < 32) tc_dealloc(taddr, 256);
}

// Gradient and loss of the batch: the tiles' shares added in tile order.
__global__ void k_mlp_reduce(Net net, int ntile, int B)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) {
        float g = 0.f;
        for (int i = 0; i < ntile; ++i) g += net.Gp[(size_t)i * NPARAM + k];
        net.G[k] = g;
    }
    if (k == 0) {
        float l = 0.f;
        for (int i = 0; i < ntile; ++i) l += net.Lp[i];
        *net.loss = l / (float)B;
    }
}

// Adam (Kingma & Ba) on the FP32 masters; refreshes the BF16 copies.
__global__ void k_mlp_adam(Net net, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float g = net.G[k];
    const float m = b1 * net.M[k] + (1.f - b1) * g;
    const float v = b2 * net.V[k] + (1.f - b2) * g * g;
    net.M[k] = m;
    net.V[k] = v;
    const float p = net.P[k] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    net.P[k] = p;
    for (int l = 1; l <= 3; ++l)
        if (k >= off_W(l) && k < off_W(l) + WID * WID) net.Wb[(l - 1) * WID * WID + (k - off_W(l))] = __float2bfloat16_rn(p);
}

__global__ void k_mlp_refresh(Net net)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * WID * WID) return;
    const int l = k / (WID * WID) + 1, e = k % (WID * WID);
    net.Wb[k] = __float2bfloat16_rn(net.P[off_W(l) + e]);
}

}  // namespace mlp
}  // namespace sdpd

// ======================================================================= ABI
using namespace sdpd::mlp;

struct sdpd_mlp {
    Net net;
};

namespace {
constexpr size_t SMEM_BYTES = 4 * TILE_BYTES + 64;

sdpd_status mlp_fail(sdpd_status s, const std::string &m)
{
    sdpd::set_last_error(m.c_str());
    return s;
}

sdpd_status mlp_err(sdpd_mlp *h)
{
    int e = 0;
    if (cudaMemcpy(&e, h->net.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(SDPD_E_CUDA, "mlp: reading the error word");
    if (e) return mlp_fail(SDPD_E_TIMEOUT, "mlp: tensor-core completion wait timed out");
    return SDPD_OK;
}
}  // namespace

extern "C" {

void mlp_destroy(sdpd_mlp *h);

sdpd_status mlp_init(int in, int width, int depth, unsigned long long seed, int batch_max, sdpd_mlp **out)
{
    if (!out) return mlp_fail(SDPD_E_INVALID, "mlp_init: out is NULL");
    *out = nullptr;
    if (in != NIN || width != WID || depth != 4) return mlp_fail(SDPD_E_INVALID, "mlp_init: network is 3 -> 4 x 128 -> 1");
    if (batch_max < 1 || batch_max > 4096) return mlp_fail(SDPD_E_INVALID, "mlp_init: batch_max must be 1..4096");
    sdpd_mlp *h = new sdpd_mlp();
    Net &n = h->net;
    n.bmax = (batch_max + WID - 1) / WID * WID;
    auto A = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = A((void **)&n.P, NPARAM * 4) && A((void **)&n.G, NPARAM * 4) && A((void **)&n.M, NPARAM * 4) &&
              A((void **)&n.V, NPARAM * 4) && A((void **)&n.Wb, 3 * WID * WID * 2) &&
              A((void **)&n.Z, (size_t)4 * n.bmax * WID * 4) && A((void **)&n.D, (size_t)2 * n.bmax * WID * 4) &&
              A((void **)&n.Gp, (size_t)(n.bmax / WID) * NPARAM * 4) && A((void **)&n.Lp, (size_t)(n.bmax / WID) * 4) &&
              A((void **)&n.Y, (size_t)n.bmax * 4) && A((void **)&n.DY, (size_t)n.bmax * 4) &&
              A((void **)&n.loss, 4) && A((void **)&n.err, 4);
    if (!ok) {
        delete h;
        return mlp_fail(SDPD_E_OOM, "mlp_init: cudaMalloc failed");
    }
    // He-uniform initial weights from a splitmix64 stream of the seed
    std::vector<float> P(NPARAM, 0.f);
    uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
    auto rnd = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int count, int fan_in) {
        const double lim = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < count; ++k) P[off + k] = (float)((2.0 * rnd() - 1.0) * lim);
    };
    fill(OFF_W0, WID * NIN, NIN);
    for (int l = 1; l <= 3; ++l) fill(off_W(l), WID * WID, WID);
    fill(OFF_W4, WID, WID);
    cudaMemcpy(n.P, P.data(), NPARAM * 4, cudaMemcpyHostToDevice);
    cudaMemset(n.M, 0, NPARAM * 4);
    cudaMemset(n.V, 0, NPARAM * 4);
    cudaMemset(n.G, 0, NPARAM * 4);
    cudaMemset(n.err, 0, 4);
    n.step = 0;
    k_mlp_refresh<<<(3 * WID * WID + 255) / 256, 256>>>(n);
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM);
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        mlp_destroy(h);
        return mlp_fail(SDPD_E_CUDA, "mlp_init: initialisation failed");
    }
    *out = h;
    return SDPD_OK;
}

void mlp_destroy(sdpd_mlp *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    Net &n = h->net;
    void *ps[] = { n.P, n.G, n.M, n.V, n.Wb, n.Z, n.D, n.Gp, n.Lp, n.Y, n.DY, n.loss, n.err };
    for (void *p : ps) cudaFree(p);
    delete h;
}

sdpd_status mlp_set_params(sdpd_mlp *h, const float *params)
{
    if (!h || !params) return mlp_fail(SDPD_E_INVALID, "mlp_set_params: NULL argument");
    if (cudaMemcpy(h->net.P, params, NPARAM * 4, cudaMemcpyDefault) != cudaSuccess)
        return mlp_fail(SDPD_E_CUDA, "mlp_set_params: copy");
    k_mlp_refresh<<<(3 * WID * WID + 255) / 256, 256>>>(h->net);
    cudaMemset(h->net.M, 0, NPARAM * 4);
    cudaMemset(h->net.V, 0, NPARAM * 4);
    h->net.step = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? SDPD_OK : mlp_fail(SDPD_E_CUDA, "mlp_set_params");
}

sdpd_status mlp_get_params(sdpd_mlp *h, float *params, float *grads)
{
    if (!h) return mlp_fail(SDPD_E_INVALID, "mlp_get_params: NULL argument");
    if (cudaDeviceSynchronize() != cudaSuccess) return mlp_fail(SDPD_E_CUDA, "mlp_get_params");
    if (params && cudaMemcpy(params, h->net.P, NPARAM * 4, cudaMemcpyDefault) != cudaSuccess)
        return mlp_fail(SDPD_E_CUDA, "mlp_get_params: copy");
    if (grads && cudaMemcpy(grads, h->net.G, NPARAM * 4, cudaMemcpyDefault) != cudaSuccess)
        return mlp_fail(SDPD_E_CUDA, "mlp_get_params: copy");
    return SDPD_OK;
}

int mlp_param_count(void) { return NPARAM; }

sdpd_status mlp_gradients(sdpd_mlp *h, const float *X, const float *T, int batch, float *loss, void *stream)
{
    if (!h || !X || !T) return mlp_fail(SDPD_E_INVALID, "mlp_gradients: NULL argument");
    if (batch < 1 || batch > h->net.bmax) return mlp_fail(SDPD_E_INVALID, "mlp_gradients: batch out of range");
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const int ntile = (batch + WID - 1) / WID;
    k_mlp_grad<<<ntile, 128, SMEM_BYTES, st>>>(h->net, X, T, batch);
    k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(h->net, ntile, batch);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(SDPD_E_CUDA, "mlp_gradients: launch");
    if (loss) {
        if (cudaMemcpyAsync(loss, h->net.loss, 4, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return mlp_fail(SDPD_E_CUDA, "mlp_gradients: loss");
        return mlp_err(h);
    }
    return SDPD_OK;
}

sdpd_status mlp_train_step(sdpd_mlp *h, const float *X, const float *T, int batch, float lr, float *loss,
                           void *stream)
{
    sdpd_status s = mlp_gradients(h, X, T, batch, nullptr, stream);
    if (s != SDPD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    h->net.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)h->net.step));
    const float c2 = (float)(1.0 - std::pow(b2, (double)h->net.step));
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(h->net, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(SDPD_E_CUDA, "mlp_train_step: launch");
    if (loss) {
        if (cudaMemcpyAsync(loss, h->net.loss, 4, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return mlp_fail(SDPD_E_CUDA, "mlp_train_step: loss");
        return mlp_err(h);
    }
    return SDPD_OK;
}

sdpd_status mlp_infer(sdpd_mlp *h, const float *X, float *Y, long long n, void *stream)
{
    if (!h || (n && (!X || !Y))) return mlp_fail(SDPD_E_INVALID, "mlp_infer: NULL argument");
    if (n <= 0) return SDPD_OK;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (n + WID - 1) / WID;
    const int grid = (int)std::min<long long>((tiles + NWG - 1) / NWG, (long long)nsm);
    (void)cudaGetLastError();
    k_mlp_forward<<<grid, 128 * NWG, FWD_SMEM, (cudaStream_t)stream>>>(h->net.P, h->net.Wb, X, Y, n, h->net.err);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(SDPD_E_CUDA, "mlp_infer: launch");
    return SDPD_OK;
}

sdpd_status mlp_check(sdpd_mlp *h)
{
    if (!h) return mlp_fail(SDPD_E_INVALID, "mlp_check: NULL");
    if (cudaDeviceSynchronize() != cudaSuccess) return mlp_fail(SDPD_E_CUDA, "mlp_check: device error");
    return mlp_err(h);
}

}  // extern "C"
