// labs_net.cu -- the learned proposal network (the library's addition: the paper has no
// learned component).  BF16 operands with FP32 accumulation on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in TMEM, operands staged by TMA), hand-written
// forward, backward, loss and AdamW kernels.
//
// Network, per state of n free variables (positions p = 0..n-1):
//   x (3 features per position, padded to 16 channels)
//   a1..a3 = relu(conv(a_{l-1}) + b_l): Conv1d, 64 output channels, 7 taps, zero padding 3
//   h      = relu(W4 a3 + b4) per position;  score_p = w5 . h_p + b5   (flip score)
//   restart = w6 . mean_p(a3_p) + b6                                   (restart score)
// Loss per sample: wf * CE(softmax(score), t) + 0.5 (restart - y)^2, batch mean.
//
// Layouts.  Activations are bf16 [B][P][C] with P = ceil16(n) + 6 rows per sample:
// row r holds position r-3, rows outside 3..n+2 stay zero (the convolution's padding
// and the tile tail).  Convolution weights are packed bf16 [64 out][taps x Cin]
// (tap-major, channel fastest), the layout the products' K-major weight operand takes;
// the backward-data pass uses the tap-reversed transpose.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "labs_internal.cuh"
#include "labs_tc.cuh"
#include "labs_nvtx.h"

namespace labsgpu {
namespace net {

using bf16 = __nv_bfloat16;

constexpr int kC = 64, kTaps = 7, kCin = 16;
constexpr int oW1 = 0, oB1 = oW1 + kC * kCin * kTaps, oW2 = oB1 + kC, oB2 = oW2 + kC * kC * kTaps, oW3 = oB2 + kC,
              oB3 = oW3 + kC * kC * kTaps, oW4 = oB3 + kC, oB4 = oW4 + kC * kC, oW5 = oB4 + kC, oB5 = oW5 + kC,
              oW6 = oB5 + 1, oB6 = oW6 + kC, kParams = oB6 + 1;
// packed bf16 operand copies (element offsets)
constexpr int pWf1 = 0, pWf2 = pWf1 + kC * kTaps * kCin, pWf3 = pWf2 + kC * kTaps * kC, pWf4 = pWf3 + kC * kTaps * kC,
              pWb2 = pWf4 + kC * kC, pWb3 = pWb2 + kC * kTaps * kC, pWb4 = pWb3 + kC * kTaps * kC, pW5 = pWb4 + kC * kC,
              pW6 = pW5 + kC, kPacked = pW6 + kC;

__host__ __device__ inline int rows_per_sample(int n)
{
    return ((n + 15) & ~15) + 6;
}

namespace {

enum { EPI_BIAS_RELU = 0, EPI_MASK = 1, EPI_MASK_POOL = 2 };

// out[b][3+p][o] = epi(sum_{k<TAPS, c<CIN} in[b][p+k+RO][c] * Wt[o][k*CIN+c]) for p < n, on
// the 5th-generation tensor cores.  The B*P activation rows form
// one long sequence (the zero rows around each sample keep the samples apart), so output
// row G (sample b = G / P, position G % P - 3) takes input rows G - 3 + RO + k, k < TAPS:
// a tile of 128 output rows reads 128 + TAPS - 1 consecutive input rows.  TMA stages them
// once, in the K-major layout without swizzling (16-byte rows back to back, one column
// of rows per 8 input channels, kRowsPad rows apart), and tap k is the same operand with
// its start address 16 k bytes further.  The weights (64 outputs x TAPS CIN) are staged
// once per CTA in the same layout (64 rows per column of 8 K values).  One thread issues
// TAPS * CIN/16 MMAs of M = 128, N = 64, K = 16 into 64 TMEM columns; every warp reads
// its 32 rows back (tcgen05.ld) for the epilogue, which writes only rows of real
// positions (the zero rows stay zero).
constexpr int kTcThreads = 128;
constexpr int kTcTile = 128;  // output rows per tile (the MMA's M)

template <int CIN, int TAPS>
struct TcShape {
    static constexpr int KK = TAPS * CIN;
    static constexpr int RO = 3 - (TAPS - 1) / 2;
    static constexpr int ROWS = kTcTile + TAPS - 1;              // input rows per tile
    static constexpr int ROWS_PAD = (ROWS + 7) & ~7;              // 128-byte aligned columns
    static constexpr int A_COL = ROWS_PAD * 16;                   // bytes per 8-channel column
    static constexpr int A_BYTES = (CIN / 8) * A_COL;
    static constexpr int W_BYTES = (KK / 8) * 1024;               // 64 rows x 16 bytes per column
    static constexpr int BAR_OFF = W_BYTES + A_BYTES;             // three barriers, the TMEM slot
    static constexpr int BIAS_OFF = BAR_OFF + 32;
    static constexpr int SMEM = BIAS_OFF + 2 * kC * 4 + 128;       // + alignment slack
};

template <int CIN, int TAPS, int EPI>
__global__ void __launch_bounds__(kTcThreads) rows_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmW,
                                                             const float* __restrict__ bias,
                                                             const bf16* __restrict__ mask,
                                                             const float* __restrict__ pool_dr,
                                                             const bf16* __restrict__ pool_w, bf16* __restrict__ out,
                                                             int n, int64_t rows_total, int* __restrict__ err)
{
    using S = TcShape<CIN, TAPS>;
    extern __shared__ unsigned char tc_smem_raw[];
    // 128-byte aligned base for the TMA destinations
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~uintptr_t(127));
    const uint32_t sW = smem_addr(sm), sA = sW + S::W_BYTES;
    const uint32_t bar_w = sW + S::BAR_OFF, bar_a = bar_w + 8, bar_m = bar_w + 16, slot = bar_w + 24;
    float* sbias = reinterpret_cast<float*>(sm + S::BIAS_OFF);
    float* spool = sbias + kC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = rows_per_sample(n);
    const int64_t tiles = (rows_total + kTcTile - 1) / kTcTile;
    if (threadIdx.x < kC) {
        sbias[threadIdx.x] = (EPI == EPI_BIAS_RELU) ? bias[threadIdx.x] : 0.f;
        spool[threadIdx.x] = (EPI == EPI_MASK_POOL) ? __bfloat162float(pool_w[threadIdx.x]) / (float)n : 0.f;
    }
    if (warp == 0) tmem_alloc(slot, 64);
    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_a, 1);
        mbar_init(bar_m, 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + S::BAR_OFF + 24);
    bool ok = true;
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar_w, S::W_BYTES);
        for (int j = 0; j < S::KK / 8; ++j) tma_load_2d(sW + 1024 * j, &tmW, 8 * j, 0, bar_w);
        ok = mbar_wait(bar_w, 0);
    }
    constexpr uint32_t idesc = idesc_bf16_f32(kTcTile, kC);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
        const int64_t G0 = tile * kTcTile;
        if (threadIdx.x == 0 && ok) {
            mbar_arrive_expect_tx(bar_a, S::A_BYTES / S::ROWS_PAD * S::ROWS);
            for (int j = 0; j < CIN / 8; ++j)
                tma_load_2d(sA + S::A_COL * j, &tmA, 8 * j, (int)(G0 - 3 + S::RO), bar_a);
            ok = mbar_wait(bar_a, it & 1);
            if (ok) {
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < TAPS; ++k)
#pragma unroll
                    for (int s2 = 0; s2 < CIN / 16; ++s2) {
                        const uint64_t ad = smem_desc(sA + 16 * k + 2 * s2 * S::A_COL, S::A_COL, 128);
                        const uint64_t bd = smem_desc(sW + (k * (CIN / 8) + 2 * s2) * 1024, 1024, 128);
                        tc_mma_bf16(tmem, ad, bd, idesc, (k | s2) != 0);
                    }
                tc_commit(bar_m);
            }
        }
        // every thread waits for the accumulator (a failed copy or wait skips the tile)
        ok = __syncthreads_and(ok) && mbar_wait(bar_m, it & 1);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            break;
        }
        tc_fence_after();
        float acc[64];
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[16];
            tmem_ld16(trow + 16 * q, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[16 * q + i] = v[i];
        }
        tc_wait_ld();
        const int64_t G = G0 + 32 * warp + lane;
        const int b = (int)(G / P), p = (int)(G % P) - 3;
        if (G < rows_total && p >= 0 && p < n) {
            bf16* dst = out + G * kC;
            const float pdr = (EPI == EPI_MASK_POOL) ? pool_dr[b] : 0.f;
#pragma unroll
            for (int c8 = 0; c8 < kC / 8; ++c8) {
                uint4 mk = make_uint4(0u, 0u, 0u, 0u);
                if (EPI != EPI_BIAS_RELU) mk = *reinterpret_cast<const uint4*>(mask + G * kC + 8 * c8);
                const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
                uint32_t pk[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int o = 8 * c8 + 2 * h;
                    float v0 = acc[o], v1 = acc[o + 1];
                    if (EPI == EPI_BIAS_RELU) {
                        v0 = fmaxf(v0 + sbias[o], 0.f);
                        v1 = fmaxf(v1 + sbias[o + 1], 0.f);
                    } else {
                        if (EPI == EPI_MASK_POOL) {
                            v0 += spool[o] * pdr;
                            v1 += spool[o + 1] * pdr;
                        }
                        const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[h]);
                        if (!(__bfloat162float(m2.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(m2.y) > 0.f)) v1 = 0.f;
                    }
                    const __nv_bfloat162 r2 = __floats2bfloat162_rn(v0, v1);
                    pk[h] = *reinterpret_cast<const uint32_t*>(&r2);
                }
                *reinterpret_cast<uint4*>(dst + 8 * c8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        // the next tile's copy overwrites the operand and its MMAs the accumulator
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
}

// Weight gradients on the tensor cores: dW[o][c][k] = sum over the B*P rows r of
// G[r][o] * IN[r - 3 + RO + k][c] (rows of G outside the positions are zero).  The
// reduction dimension is the rows, so both operands are MN-major: a staged column of 16-
// byte rows (8 channels or 8 outputs per row) is the MN-major core-matrix layout without
// swizzling (8 K rows of 16 bytes each, the next 8 rows 128 bytes further), and columns
// lie kWgCol bytes apart along M (or N).  M = 128 covers 16 columns of (tap, 8-channel
// block) pairs: column c holds channels 8 (c % (CIN/8)) .. +7 of tap c / (CIN/8), loaded
// with that tap's row offset, so every column's shift is in its TMA coordinate; columns
// past the last tap load tap 0 and their rows of the result are dropped.  N = 64
// outputs (the 8 columns of G).  A CTA walks blocks of kWgRows rows, accumulating
// ceil(TAPS CIN / 128) tiles of 128 x 64 in TMEM, and writes its partial sums; a second
// kernel adds the partials of all CTAs into the gradient.
constexpr int kWgRows = 64;                 // rows (K) per staged block
constexpr int kWgCol = kWgRows * 16;        // bytes per staged column
constexpr int kWgCtasPerSm = 2;

template <int CIN, int TAPS>
struct WgShape {
    static constexpr int KK = TAPS * CIN;
    static constexpr int RO = 3 - (TAPS - 1) / 2;
    static constexpr int NT = (KK + 127) / 128;           // M tiles
    static constexpr int NCOL = 16 * NT;                  // staged columns of IN
    static constexpr int IN_BYTES = NCOL * kWgCol;
    static constexpr int G_BYTES = 8 * kWgCol;
    static constexpr int BAR_OFF = IN_BYTES + G_BYTES;
    static constexpr int TMEM_COLS = NT * 64 <= 64 ? 64 : (NT * 64 <= 128 ? 128 : 256);
    // a CTA holding 256 of the SM's 512 TMEM columns asks for enough shared memory that
    // no third CTA fits beside two (its allocation would wait for theirs to end)
    static constexpr int SMEM_NEED = BAR_OFF + 32 + 128;
    static constexpr int SMEM = TMEM_COLS > 128 && SMEM_NEED < 80 * 1024 ? 80 * 1024 : SMEM_NEED;
};

// Instruction descriptor of kind::f16 with both operands MN-major (bits 15 and 16).
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N)
{
    return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

template <int CIN, int TAPS>
__global__ void __launch_bounds__(kTcThreads) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmIN,
                                                              const __grid_constant__ CUtensorMap tmG,
                                                              float* __restrict__ part, int64_t rows,
                                                              int* __restrict__ err)
{
    using S = WgShape<CIN, TAPS>;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~uintptr_t(127));
    const uint32_t sIN = smem_addr(sm), sG = sIN + S::IN_BYTES;
    const uint32_t bar_a = sIN + S::BAR_OFF, bar_m = bar_a + 8, slot = bar_a + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tmem_alloc(slot, S::TMEM_COLS);
    if (threadIdx.x == 0) {
        mbar_init(bar_a, 1);
        mbar_init(bar_m, 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + S::BAR_OFF + 16);
    constexpr uint32_t idesc = idesc_bf16_f32_mn(128, kC);
    const int64_t blocks = (rows + kWgRows - 1) / kWgRows;
    bool ok = true;
    int it = 0;
    for (int64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x, ++it) {
        if (threadIdx.x == 0 && ok) {
            const int R0 = (int)(blk * kWgRows);
            mbar_arrive_expect_tx(bar_a, (uint32_t)(S::IN_BYTES + S::G_BYTES));
            for (int c = 0; c < S::NCOL; ++c) {
                const int tap = c / (CIN / 8), ch = c % (CIN / 8);
                tma_load_2d(sIN + c * kWgCol, &tmIN, 8 * ch, R0 - 3 + S::RO + (tap < TAPS ? tap : 0), bar_a);
            }
            for (int j = 0; j < 8; ++j) tma_load_2d(sG + j * kWgCol, &tmG, 8 * j, R0, bar_a);
            ok = mbar_wait(bar_a, it & 1);
            if (ok) {
                tc_fence_after();
#pragma unroll
                for (int t = 0; t < S::NT; ++t)
#pragma unroll
                    for (int ks = 0; ks < kWgRows / 16; ++ks) {
                        // MN-major without swizzling: the leading byte offset steps along K
                        // (the next 8 rows, 128 bytes on), the stride byte offset along M or
                        // N (the next column of 8 values)
                        const uint64_t ad = smem_desc(sIN + t * 16 * kWgCol + 256 * ks, 128, kWgCol);
                        const uint64_t bd = smem_desc(sG + 256 * ks, 128, kWgCol);
                        tc_mma_bf16(tmem + 64 * t, ad, bd, idesc, it > 0 || ks > 0);
                    }
                tc_commit(bar_m);
                // the next block's copies overwrite the operands: wait for these MMAs
                ok = mbar_wait(bar_m, it & 1);
            }
        }
    }
    tc_fence_before();
    ok = __syncthreads_and(ok);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    tc_fence_after();
    // partial sums of this CTA: row m of tile t is (tap, channel) = ((128 t + m) / CIN,
    // (128 t + m) % CIN); columns are the 64 outputs
    if (ok && it > 0) {
        float* dst = part + (int64_t)blockIdx.x * S::NT * 128 * kC;
        for (int t = 0; t < S::NT; ++t) {
            const int m = 128 * t + 32 * warp + lane;
            float4* d4 = reinterpret_cast<float4*>(dst + (int64_t)m * kC);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 64 * t + 16 * q, v);
                tc_wait_ld();
                if (m < S::KK) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        d4[4 * q + i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
        }
    } else if (ok) {
        // no block for this CTA: zero partials
        float* dst = part + (int64_t)blockIdx.x * S::NT * 128 * kC;
        for (int i = threadIdx.x; i < S::KK * kC; i += blockDim.x) dst[i] = 0.f;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

// dW[o][c][k] += sum over CTAs of part[cta][k CIN + c][o].
template <int CIN, int TAPS>
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int ctas, float* __restrict__ dW)
{
    using S = WgShape<CIN, TAPS>;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S::KK * kC; i += gridDim.x * blockDim.x) {
        const int m = i / kC, o = i % kC;
        float t = 0.f;
        for (int c = 0; c < ctas; ++c) t += part[(int64_t)c * S::NT * 128 * kC + i];
        const int k = m / CIN, ch = m % CIN;
        dW[((int64_t)o * CIN + ch) * TAPS + k] += t;
    }
}

// Bias gradient: db[o] += sum_{b, p<n} G[b][p+3][o], summed over all B*P rows (the rows
// outside 0 <= p < n hold zeros).  Thread t reads channels 8 (t % 8) .. +7 of rows
// t / 8, t / 8 + 32, ... as one 16-byte load; the CTA's 32 row lanes are added in shared
// memory and each CTA adds its 64 sums to db.
__global__ void __launch_bounds__(256) colsum_kernel(const bf16* __restrict__ G, float* __restrict__ db,
                                                     int64_t rows)
{
    __shared__ float part[32][kC + 1];
    const int cg = threadIdx.x & 7, rl = threadIdx.x >> 3;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t r = (int64_t)blockIdx.x * 32 + rl; r < rows; r += (int64_t)gridDim.x * 32) {
        const uint4 v = *reinterpret_cast<const uint4*>(G + r * kC + 8 * cg);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
            acc[2 * h] += __bfloat162float(b2.x);
            acc[2 * h + 1] += __bfloat162float(b2.y);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) part[rl][8 * cg + i] = acc[i];
    __syncthreads();
    if (threadIdx.x < kC) {
        float t = 0.f;
        for (int k = 0; k < 32; ++k) t += part[k][threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

// x (float32 [B][3][n]) -> bf16 input rows [B][P][16].
__global__ void input_kernel(const float* __restrict__ x, bf16* __restrict__ X0, int B, int n)
{
    const int P = rows_per_sample(n);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * n * 3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / (3 * n)), rem = (int)(t % (3 * n)), f = rem / n, p = rem % n;
        X0[((int64_t)b * P + p + 3) * kCin + f] = __float2bfloat16_rn(x[t]);
    }
}

// Heads: score[b][p] = b5 + sum_j h[b][p][j] w5[j]; pooled[b][c] = mean_p a3[b][p][c];
// restart[b] = b6 + sum_c pooled[b][c] w6[c].  One warp per sample: lane l scores
// positions l, l+32, ... (its row of h as 16-byte loads) and sums channels 2l, 2l+1 of a3
// over the positions (one 4-byte load per row).
__global__ void head_kernel(const bf16* __restrict__ H, const bf16* __restrict__ A3, const bf16* __restrict__ wpk,
                            const float* __restrict__ params, float* __restrict__ score,
                            float* __restrict__ pooled, float* __restrict__ restart, int B, int n)
{
    __shared__ float w5[kC];
    for (int j = threadIdx.x; j < kC; j += blockDim.x) w5[j] = __bfloat162float(wpk[pW5 + j]);
    __syncthreads();
    const int P = rows_per_sample(n);
    const int lane = threadIdx.x & 31;
    const float b5 = params[oB5], b6 = params[oB6];
    const float w6a = __bfloat162float(wpk[pW6 + 2 * lane]), w6b = __bfloat162float(wpk[pW6 + 2 * lane + 1]);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const bf16* hb = H + b * P * kC;
        for (int p = lane; p < n; p += 32) {
            const uint4* row = reinterpret_cast<const uint4*>(hb + (int64_t)(p + 3) * kC);
            float sacc = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < kC / 8; ++c8) {
                const uint4 v = row[c8];
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
                    sacc += __bfloat162float(b2.x) * w5[8 * c8 + 2 * h] + __bfloat162float(b2.y) * w5[8 * c8 + 2 * h + 1];
                }
            }
            score[b * n + p] = sacc + b5;
        }
        const bf16* ab = A3 + b * P * kC + 2 * lane;
        float ma = 0.f, mb = 0.f;
        for (int p = 0; p < n; ++p) {
            const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(ab + (int64_t)(p + 3) * kC);
            ma += __bfloat162float(v.x);
            mb += __bfloat162float(v.y);
        }
        ma /= (float)n;
        mb /= (float)n;
        pooled[b * kC + 2 * lane] = ma;
        pooled[b * kC + 2 * lane + 1] = mb;
        float r = ma * w6a + mb * w6b;
#pragma unroll
        for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, off);
        if (lane == 0) restart[b] = r + b6;
    }
}

// Loss and its gradients w.r.t. the scores and the restart output (batch mean).
__global__ void loss_kernel(const float* __restrict__ score, const float* __restrict__ restart,
                            const int32_t* __restrict__ target, const float* __restrict__ y,
                            const float* __restrict__ wf, float* __restrict__ ds, float* __restrict__ dr,
                            float* __restrict__ loss, int B, int n)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float inv = 1.f / (float)B;
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const float* s = score + b * n;
        float m = -INFINITY;
        for (int p = lane; p < n; p += 32) m = fmaxf(m, s[p]);
#pragma unroll
        for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
        float z = 0.f;
        for (int p = lane; p < n; p += 32) z += expf(s[p] - m);
#pragma unroll
        for (int off = 16; off; off >>= 1) z += __shfl_xor_sync(0xFFFFFFFFu, z, off);
        const int t = min(max(target[b], 0), n - 1);
        const float w = wf[b];
        for (int p = lane; p < n; p += 32) ds[b * n + p] = w * (expf(s[p] - m) / z - (p == t ? 1.f : 0.f)) * inv;
        if (lane == 0) {
            const float e = restart[b] - y[b];
            dr[b] = e * inv;
            const float ce = logf(z) + m - s[t];
            atomicAdd(loss, (w * ce + 0.5f * e * e) * inv);
        }
    }
}

// Head backward: dh = bf16(w5 ds (h > 0)); dw5, db5, dw6, db6 accumulated.
__global__ void head_back_kernel(const bf16* __restrict__ H, const float* __restrict__ pooled,
                                 const bf16* __restrict__ wpk, const float* __restrict__ ds,
                                 const float* __restrict__ dr, bf16* __restrict__ dH, float* __restrict__ grad,
                                 int B, int n)
{
    const int P = rows_per_sample(n);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    float gw5a = 0.f, gw5b = 0.f, gw6a = 0.f, gw6b = 0.f, gb5 = 0.f, gb6 = 0.f;
    const float w5a = __bfloat162float(wpk[pW5 + lane]), w5b = __bfloat162float(wpk[pW5 + lane + 32]);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const bf16* hb = H + b * P * kC;
        bf16* db = dH + b * P * kC;
        for (int p = 0; p < n; ++p) {
            const float d = ds[b * n + p];
            const float ha = __bfloat162float(hb[(int64_t)(p + 3) * kC + lane]);
            const float hbv = __bfloat162float(hb[(int64_t)(p + 3) * kC + lane + 32]);
            gw5a += ha * d;
            gw5b += hbv * d;
            if (lane == 0) gb5 += d;
            db[(int64_t)(p + 3) * kC + lane] = __float2bfloat16_rn(ha > 0.f ? w5a * d : 0.f);
            db[(int64_t)(p + 3) * kC + lane + 32] = __float2bfloat16_rn(hbv > 0.f ? w5b * d : 0.f);
        }
        const float r = dr[b];
        gw6a += pooled[b * kC + lane] * r;
        gw6b += pooled[b * kC + lane + 32] * r;
        if (lane == 0) gb6 += r;
    }
    atomicAdd(grad + oW5 + lane, gw5a);
    atomicAdd(grad + oW5 + lane + 32, gw5b);
    atomicAdd(grad + oW6 + lane, gw6a);
    atomicAdd(grad + oW6 + lane + 32, gw6b);
    if (lane == 0) {
        atomicAdd(grad + oB5, gb5);
        atomicAdd(grad + oB6, gb6);
    }
}

// bf16 operand copies of the float32 master weights.
__global__ void pack_kernel(const float* __restrict__ prm, bf16* __restrict__ wpk)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kPacked; t += gridDim.x * blockDim.x) {
        float v;
        if (t < pWf2) {  // Wf1[o][k*16+c] = W1[o][c][k]
            const int o = t / (kTaps * kCin), kk = t % (kTaps * kCin), k = kk / kCin, c = kk % kCin;
            v = prm[oW1 + (o * kCin + c) * kTaps + k];
        } else if (t < pWf4) {  // Wf2 / Wf3
            const int base = t < pWf3 ? oW2 : oW3, u = t - (t < pWf3 ? pWf2 : pWf3);
            const int o = u / (kTaps * kC), kk = u % (kTaps * kC), k = kk / kC, c = kk % kC;
            v = prm[base + (o * kC + c) * kTaps + k];
        } else if (t < pWb2) {  // Wf4[j][c] = W4[j][c]
            v = prm[oW4 + (t - pWf4)];
        } else if (t < pWb4) {  // Wb[c][k'*64+o] = W[o][c][6-k']
            const int base = t < pWb3 ? oW2 : oW3, u = t - (t < pWb3 ? pWb2 : pWb3);
            const int c = u / (kTaps * kC), kk = u % (kTaps * kC), kr = kk / kC, o = kk % kC;
            v = prm[base + (o * kC + c) * kTaps + (kTaps - 1 - kr)];
        } else if (t < pW5) {  // Wb4[c][j] = W4[j][c]
            const int u = t - pWb4, c = u / kC, j = u % kC;
            v = prm[oW4 + j * kC + c];
        } else if (t < pW6) {
            v = prm[oW5 + (t - pW5)];
        } else {
            v = prm[oW6 + (t - pW6)];
        }
        wpk[t] = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ bool is_weight(int i)
{
    return (i >= oW1 && i < oB1) || (i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || (i >= oW4 && i < oB4) ||
           (i >= oW5 && i < oB5) || (i >= oW6 && i < oB6);
}

__global__ void adamw_kernel(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                             float* __restrict__ v, float lr, float wd, float c1, float c2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        const float decay = is_weight(i) ? wd : 0.f;
        prm[i] = prm[i] - lr * (mh / (sqrtf(vh) + eps) + decay * prm[i]);
    }
}

// He-uniform weights from Philox (key = seed, counter = (index, 0, 0, 3)), zero biases.
__global__ void init_kernel(float* __restrict__ prm, uint64_t seed)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        int fan = 0;
        if (i >= oW1 && i < oB1) fan = 3 * kTaps;
        else if ((i >= oW2 && i < oB2) || (i >= oW3 && i < oB3)) fan = kC * kTaps;
        else if ((i >= oW4 && i < oB4) || (i >= oW5 && i < oB5) || (i >= oW6 && i < oB6)) fan = kC;
        if (fan == 0) {
            prm[i] = 0.f;
            continue;
        }
        uint32_t c0 = (uint32_t)i, c1 = 0, c2 = 0, c3 = 3u, k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            if (r) {
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
            const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
            const uint32_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
            c0 = y0;
            c1 = lo1;
            c2 = y2;
            c3 = lo0;
        }
        const float u = (float)(c0 >> 8) * (1.f / 16777216.f) * 2.f - 1.f;
        prm[i] = u * sqrtf(6.f / (float)fan);
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the
// library links no driver library of its own).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// Row-major BF16 matrix [outer][inner] (rows 2 inner bytes apart, a multiple of 16), read
// in boxes of box_outer rows x box_inner values; reads outside the matrix give zeros.
bool map_rows(CUtensorMap* m, const bf16* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
              uint32_t box_outer)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * sizeof(bf16)};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CIN, int TAPS, int EPI>
int launch_rows_tc(const bf16* in, const bf16* Wt, const float* bias, const bf16* mask, const float* pdr,
                   const bf16* pw, bf16* out, int B, int n, int sms, int* err, cudaStream_t s)
{
    using S = TcShape<CIN, TAPS>;
    const int64_t rows = (int64_t)B * rows_per_sample(n);
    CUtensorMap ma, mw;
    if (!map_rows(&ma, in, CIN, (uint64_t)rows, 8, S::ROWS) || !map_rows(&mw, Wt, S::KK, kC, 8, kC))
        return LABS_ECUDA;
    auto fn = rows_tc_kernel<CIN, TAPS, EPI>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) != cudaSuccess)
        return LABS_ECUDA;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, S::SMEM) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t tiles = (rows + kTcTile - 1) / kTcTile;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms * per_sm);
    fn<<<grid, kTcThreads, S::SMEM, s>>>(ma, mw, bias, mask, pdr, pw, out, n, rows, err);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

template <int CIN, int TAPS>
int launch_wgrad_tc(const bf16* G, const bf16* IN, float* dW, float* part, int B, int n, int sms, int* err,
                    cudaStream_t s)
{
    using S = WgShape<CIN, TAPS>;
    const int64_t rows = (int64_t)B * rows_per_sample(n);
    CUtensorMap mi, mg;
    if (!map_rows(&mi, IN, CIN, (uint64_t)rows, 8, kWgRows) || !map_rows(&mg, G, kC, (uint64_t)rows, 8, kWgRows))
        return LABS_ECUDA;
    auto fn = wgrad_tc_kernel<CIN, TAPS>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) != cudaSuccess)
        return LABS_ECUDA;
    const int ctas = sms * kWgCtasPerSm;
    fn<<<ctas, kTcThreads, S::SMEM, s>>>(mi, mg, part, rows, err);
    wgrad_reduce_kernel<CIN, TAPS><<<(S::KK * kC + 255) / 256, 256, 0, s>>>(part, ctas, dW);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

}  // namespace

// Workspace carve-up for a batch of B states of n free variables.
struct NetWs {
    bf16 *X0, *A1, *A2, *A3, *H, *dH, *dA3, *dA2, *dA1, *wpk;
    float *score, *restart, *pooled, *ds, *dr, *loss;
    int* err;  // set by a tensor-core kernel whose copy or MMA wait gave up
    float* part;  // per-CTA partial weight gradients
    size_t bytes;
};

static size_t align256(size_t x)
{
    return (x + 255) & ~(size_t)255;
}

static int sm_count();

NetWs carve(void* base, int64_t B, int n)
{
    NetWs w;
    const size_t P = (size_t)rows_per_sample(n);
    const size_t act = align256((size_t)B * P * kC * sizeof(bf16));
    char* p = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* q = p ? p + off : nullptr;
        off += align256(bytes);
        return q;
    };
    w.X0 = (bf16*)take((size_t)B * P * kCin * sizeof(bf16));
    w.A1 = (bf16*)take(act);
    w.A2 = (bf16*)take(act);
    w.A3 = (bf16*)take(act);
    w.H = (bf16*)take(act);
    w.dH = (bf16*)take(act);
    w.dA3 = (bf16*)take(act);
    w.dA2 = (bf16*)take(act);
    w.dA1 = (bf16*)take(act);
    w.wpk = (bf16*)take(kPacked * sizeof(bf16));
    w.score = (float*)take((size_t)B * n * 4);
    w.ds = (float*)take((size_t)B * n * 4);
    w.restart = (float*)take((size_t)B * 4);
    w.dr = (float*)take((size_t)B * 4);
    w.pooled = (float*)take((size_t)B * kC * 4);
    w.loss = (float*)take(4);
    w.err = (int*)take(4);
    // per-CTA partial weight gradients (the largest product's M tiles x 64 outputs)
    w.part = (float*)take((size_t)sm_count() * kWgCtasPerSm * WgShape<kC, kTaps>::NT * 128 * kC * 4);
    w.bytes = off;
    return w;
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Forward of a batch whose inputs are already in w.X0 (activations zeroed by the caller).
int forward(const float* prm, const NetWs& w, int B, int n, cudaStream_t s)
{
    const int sms = sm_count();
    pack_kernel<<<64, 256, 0, s>>>(prm, w.wpk);
    int rc = launch_rows_tc<kCin, kTaps, EPI_BIAS_RELU>(w.X0, w.wpk + pWf1, prm + oB1, nullptr, nullptr, nullptr, w.A1,
                                                        B, n, sms, w.err, s);
    if (!rc) rc = launch_rows_tc<kC, kTaps, EPI_BIAS_RELU>(w.A1, w.wpk + pWf2, prm + oB2, nullptr, nullptr, nullptr,
                                                           w.A2, B, n, sms, w.err, s);
    if (!rc) rc = launch_rows_tc<kC, kTaps, EPI_BIAS_RELU>(w.A2, w.wpk + pWf3, prm + oB3, nullptr, nullptr, nullptr,
                                                           w.A3, B, n, sms, w.err, s);
    if (!rc) rc = launch_rows_tc<kC, 1, EPI_BIAS_RELU>(w.A3, w.wpk + pWf4, prm + oB4, nullptr, nullptr, nullptr, w.H,
                                                       B, n, sms, w.err, s);
    if (rc) return rc;
    head_kernel<<<std::min(B, sms * 8), 128, 0, s>>>(w.H, w.A3, w.wpk, prm, w.score, w.pooled, w.restart, B, n);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int zero_acts(const NetWs& w, int B, int n, cudaStream_t s)
{
    // X0 .. dA1 are contiguous at the start of the workspace
    const size_t bytes = (size_t)((char*)w.wpk - (char*)w.X0);
    return cudaMemsetAsync(w.X0, 0, bytes, s) == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int backward(const float* prm, const NetWs& w, const int32_t* target, const float* y, const float* wf, float* grad,
             int B, int n, cudaStream_t s)
{
    const int sms = sm_count();
    if (cudaMemsetAsync(grad, 0, kParams * sizeof(float), s) != cudaSuccess) return LABS_ECUDA;
    if (cudaMemsetAsync(w.loss, 0, sizeof(float), s) != cudaSuccess) return LABS_ECUDA;
    loss_kernel<<<std::min(B, sms * 8), 128, 0, s>>>(w.score, w.restart, target, y, wf, w.ds, w.dr, w.loss, B, n);
    head_back_kernel<<<std::min(B, sms * 4), 128, 0, s>>>(w.H, w.pooled, w.wpk, w.ds, w.dr, w.dH, grad, B, n);
    int rc = cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
    // h = relu(W4 a3 + b4): dW4, db4, then da3 = (W4^T dh + w6 dr / n) * (a3 > 0)
    if (!rc) rc = launch_wgrad_tc<kC, 1>(w.dH, w.A3, grad + oW4, w.part, B, n, sms, w.err, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dH, grad + oB4, (int64_t)B * rows_per_sample(n));
    if (!rc) rc = launch_rows_tc<kC, 1, EPI_MASK_POOL>(w.dH, w.wpk + pWb4, nullptr, w.A3, w.dr, w.wpk + pW6, w.dA3,
                                                       B, n, sms, w.err, s);
    // conv3
    if (!rc) rc = launch_wgrad_tc<kC, kTaps>(w.dA3, w.A2, grad + oW3, w.part, B, n, sms, w.err, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA3, grad + oB3, (int64_t)B * rows_per_sample(n));
    if (!rc) rc = launch_rows_tc<kC, kTaps, EPI_MASK>(w.dA3, w.wpk + pWb3, nullptr, w.A2, nullptr, nullptr, w.dA2, B,
                                                      n, sms, w.err, s);
    // conv2
    if (!rc) rc = launch_wgrad_tc<kC, kTaps>(w.dA2, w.A1, grad + oW2, w.part, B, n, sms, w.err, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA2, grad + oB2, (int64_t)B * rows_per_sample(n));
    if (!rc) rc = launch_rows_tc<kC, kTaps, EPI_MASK>(w.dA2, w.wpk + pWb2, nullptr, w.A1, nullptr, nullptr, w.dA1, B,
                                                      n, sms, w.err, s);
    // conv1
    if (!rc) rc = launch_wgrad_tc<kCin, kTaps>(w.dA1, w.X0, grad + oW1, w.part, B, n, sms, w.err, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA1, grad + oB1, (int64_t)B * rows_per_sample(n));
    if (!rc && cudaGetLastError() != cudaSuccess) rc = LABS_ECUDA;
    return rc;
}

int load_inputs(const float* x, const NetWs& w, int B, int n, cudaStream_t s)
{
    input_kernel<<<std::min<int64_t>(((int64_t)B * n * 3 + 255) / 256, sm_count() * 16), 256, 0, s>>>(x, w.X0, B, n);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int init_params(float* prm, uint64_t seed, cudaStream_t s)
{
    init_kernel<<<64, 256, 0, s>>>(prm, seed);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int adamw(float* prm, const float* grad, float* m, float* v, int64_t t, float lr, float wd, cudaStream_t s)
{
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    adamw_kernel<<<64, 256, 0, s>>>(prm, grad, m, v, lr, wd, c1, c2);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

}  // namespace net
}  // namespace labsgpu

namespace labsgpu {

size_t net_workspace_bytes(int64_t B, int n)
{
    return net::carve(nullptr, B, n).bytes;
}

int net_forward_ws(const float* params, const float* x, int64_t B, int n, void* ws, const float** scores,
                   const float** restart, void* stream)
{
    const net::NetWs w = net::carve(ws, B, n);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = net::zero_acts(w, (int)B, n, s);
    if (!rc) rc = net::load_inputs(x, w, (int)B, n, s);
    if (!rc) rc = net::forward(params, w, (int)B, n, s);
    if (scores) *scores = w.score;
    if (restart) *restart = w.restart;
    return rc;
}

}  // namespace labsgpu

using namespace labsgpu;

extern "C" {

int labs_net_sizes(int32_t n, int64_t batch, size_t* param_count, size_t* workspace_bytes)
{
    if (n < 2 || n > kMaxN || batch < 0) return LABS_EINVAL;
    if (param_count) *param_count = net::kParams;
    if (workspace_bytes) *workspace_bytes = net::carve(nullptr, batch, n).bytes;
    return LABS_OK;
}

int labs_net_init(float* dev_params, uint64_t seed, void* cuda_stream)
{
    LABS_API_RANGE();
    if (!dev_params) return LABS_EINVAL;
    return net::init_params(dev_params, seed, (cudaStream_t)cuda_stream);
}

int labs_net_forward(const float* dev_params, const float* dev_x, int64_t batch, int32_t n, float* dev_scores,
                     float* dev_restart, void* dev_ws, size_t ws_bytes, void* cuda_stream)
{
    LABS_API_RANGE();
    if (!dev_params || !dev_x || n < 2 || n > kMaxN || batch < 0 || batch > INT32_MAX) return LABS_EINVAL;
    if (batch == 0) return LABS_OK;
    const net::NetWs w = net::carve(dev_ws, batch, n);
    if (!dev_ws || ws_bytes < w.bytes) return LABS_ENOMEM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = net::zero_acts(w, (int)batch, n, s);
    if (!rc) rc = net::load_inputs(dev_x, w, (int)batch, n, s);
    if (!rc) rc = net::forward(dev_params, w, (int)batch, n, s);
    if (!rc && dev_scores)
        rc = cudaMemcpyAsync(dev_scores, w.score, (size_t)batch * n * 4, cudaMemcpyDeviceToDevice, s) ? LABS_ECUDA : 0;
    if (!rc && dev_restart)
        rc = cudaMemcpyAsync(dev_restart, w.restart, (size_t)batch * 4, cudaMemcpyDeviceToDevice, s) ? LABS_ECUDA : 0;
    return rc;
}

int labs_net_gradients(const float* dev_params, const float* dev_x, const int32_t* dev_target, const float* dev_y,
                       const float* dev_wf, int64_t batch, int32_t n, float* dev_grads, float* dev_loss, void* dev_ws,
                       size_t ws_bytes, void* cuda_stream)
{
    LABS_API_RANGE();
    if (!dev_params || !dev_x || !dev_target || !dev_y || !dev_wf || !dev_grads || n < 2 || n > kMaxN || batch < 1 ||
        batch > INT32_MAX)
        return LABS_EINVAL;
    const net::NetWs w = net::carve(dev_ws, batch, n);
    if (!dev_ws || ws_bytes < w.bytes) return LABS_ENOMEM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = net::zero_acts(w, (int)batch, n, s);
    if (!rc) rc = net::load_inputs(dev_x, w, (int)batch, n, s);
    if (!rc) rc = net::forward(dev_params, w, (int)batch, n, s);
    if (!rc) rc = net::backward(dev_params, w, dev_target, dev_y, dev_wf, dev_grads, (int)batch, n, s);
    if (!rc && dev_loss) rc = cudaMemcpyAsync(dev_loss, w.loss, 4, cudaMemcpyDeviceToDevice, s) ? LABS_ECUDA : 0;
    return rc;
}

int labs_net_adamw(float* dev_params, const float* dev_grads, float* dev_m, float* dev_v, int64_t t, float lr,
                   float weight_decay, void* cuda_stream)
{
    LABS_API_RANGE();
    if (!dev_params || !dev_grads || !dev_m || !dev_v || t < 1) return LABS_EINVAL;
    return net::adamw(dev_params, dev_grads, dev_m, dev_v, t, lr, weight_decay, (cudaStream_t)cuda_stream);
}

}  // extern "C"
