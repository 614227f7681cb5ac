// labs_net.cu -- the learned proposal network (the library's addition: the paper has no
// learned component).  BF16 operands with FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), hand-written forward, backward, loss and AdamW kernels.
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
// (tap-major, channel fastest) so that every tensor-core fragment element pair is one
// 32-bit load; the backward-data pass uses the tap-reversed transpose.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "labs_internal.cuh"
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

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void st2(bf16* p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

enum { EPI_BIAS_RELU = 0, EPI_MASK = 1, EPI_MASK_POOL = 2 };

// out[b][3+p][o] = epi(sum_{k<TAPS, c<CIN} in[b][p+k+RO][c] * Wt[o][k*CIN+c]) for p < n.
// One warp computes 16 positions x 64 outputs; the CTA (4 warps) keeps Wt in shared
// memory with a padded row stride (conflict-free fragment loads).
template <int CIN, int TAPS, int EPI>
__global__ void __launch_bounds__(128) rows_gemm_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Wt,
                                                        const float* __restrict__ bias,
                                                        const bf16* __restrict__ mask,
                                                        const float* __restrict__ pool_dr,
                                                        const bf16* __restrict__ pool_w, bf16* __restrict__ out,
                                                        int B, int n)
{
    constexpr int KK = TAPS * CIN;
    constexpr int KS = KK + 8;  // padded smem row stride (elements)
    constexpr int RO = 3 - (TAPS - 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16* ws = reinterpret_cast<bf16*>(smem_raw);
    for (int t = threadIdx.x; t < kC * KK / 2; t += blockDim.x) {
        const int o = (2 * t) / KK, kk = (2 * t) % KK;
        *reinterpret_cast<uint32_t*>(ws + o * KS + kk) = ld32(Wt + 2 * t);
    }
    __syncthreads();
    const int P = rows_per_sample(n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int mtiles = (n + 15) >> 4;
    const int64_t total = (int64_t)B * mtiles;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < total; tile += (int64_t)gridDim.x * 4) {
        const int b = (int)(tile / mtiles), p0 = (int)(tile % mtiles) * 16;
        const bf16* src = in + (int64_t)b * P * CIN;
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int k = 0; k < TAPS; ++k) {
            const bf16* r0 = src + (int64_t)(p0 + g + k + RO) * CIN + tig * 2;
            const bf16* r1 = r0 + 8 * CIN;
#pragma unroll
            for (int c0 = 0; c0 < CIN; c0 += 16) {
                const uint32_t a0 = ld32(r0 + c0), a1 = ld32(r1 + c0), a2 = ld32(r0 + c0 + 8), a3 = ld32(r1 + c0 + 8);
                const bf16* wb = ws + g * KS + k * CIN + c0 + tig * 2;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bf16* w = wb + j * 8 * KS;
                    mma16816(acc[j], a0, a1, a2, a3, ld32(w), ld32(w + 8));
                }
            }
        }
        bf16* dst = out + (int64_t)b * P * kC;
        const bf16* msk = mask ? mask + (int64_t)b * P * kC : nullptr;
        const float pdr = (EPI == EPI_MASK_POOL) ? pool_dr[b] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int p = p0 + g + 8 * h;
            if (p >= n) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int o = 8 * j + tig * 2;
                float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
                if (EPI == EPI_BIAS_RELU) {
                    v0 = fmaxf(v0 + bias[o], 0.f);
                    v1 = fmaxf(v1 + bias[o + 1], 0.f);
                } else {
                    if (EPI == EPI_MASK_POOL) {
                        v0 += __bfloat162float(pool_w[o]) * pdr / (float)n;
                        v1 += __bfloat162float(pool_w[o + 1]) * pdr / (float)n;
                    }
                    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(msk + (int64_t)(p + 3) * kC + o);
                    if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
                }
                st2(dst + (int64_t)(p + 3) * kC + o, v0, v1);
            }
        }
    }
}

// dW[o][c][k] += sum_{b, p<n} G[b][p+3][o] * IN[b][p+k+RO][c]  (fp32 atomics into the
// gradient in canonical [o][c][k] order).  CTA = 4 warps = all 64 o x 64 (k,c) columns;
// blockIdx.y splits the batch.
template <int CIN, int TAPS>
__global__ void __launch_bounds__(128) wgrad_kernel(const bf16* __restrict__ G, const bf16* __restrict__ IN,
                                                    float* __restrict__ dW, int B, int n)
{
    constexpr int KK = TAPS * CIN;
    constexpr int RO = 3 - (TAPS - 1) / 2;
    const int P = rows_per_sample(n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int o0 = warp * 16;
    const int kkb = blockIdx.x * 64;
    const int bsplit = gridDim.y;
    const int b_lo = (int)((int64_t)B * blockIdx.y / bsplit), b_hi = (int)((int64_t)B * (blockIdx.y + 1) / bsplit);
    int kcol[8], ccol[8];
    bool valid[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int kk = kkb + 8 * j + g;
        valid[j] = kk < KK;
        kcol[j] = valid[j] ? kk / CIN : 0;
        ccol[j] = valid[j] ? kk % CIN : 0;
    }
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int mtiles = (n + 15) >> 4;
    for (int b = b_lo; b < b_hi; ++b) {
        const bf16* gs = G + (int64_t)b * P * kC;
        const bf16* is = IN + (int64_t)b * P * CIN;
        for (int mt = 0; mt < mtiles; ++mt) {
            const int p = mt * 16 + tig * 2;
            const bf16* gp = gs + (int64_t)(p + 3) * kC + o0 + g;
            const uint32_t a0 = pack2(gp[0], gp[kC]);
            const uint32_t a1 = pack2(gp[8], gp[kC + 8]);
            const uint32_t a2 = pack2(gp[8 * kC], gp[9 * kC]);
            const uint32_t a3 = pack2(gp[8 * kC + 8], gp[9 * kC + 8]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bf16* ip = is + (int64_t)(p + kcol[j] + RO) * CIN + ccol[j];
                const uint32_t b0 = pack2(ip[0], ip[CIN]);
                const uint32_t b1 = pack2(ip[8 * CIN], ip[9 * CIN]);
                mma16816(acc[j], a0, a1, a2, a3, b0, b1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        // acc[j][0..1]: o = o0+g, cols 8j+tig*2+{0,1}; acc[j][2..3]: o = o0+g+8
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int o = o0 + g + (e >= 2 ? 8 : 0);
            const int kk = kkb + 8 * j + tig * 2 + (e & 1);
            if (kk >= KK) continue;
            const int k = kk / CIN, c = kk % CIN;
            atomicAdd(dW + ((int64_t)o * CIN + c) * TAPS + k, acc[j][e]);
        }
    }
}

// Bias gradient: db[o] += sum_{b, p<n} G[b][p+3][o].
__global__ void colsum_kernel(const bf16* __restrict__ G, float* __restrict__ db, int B, int n)
{
    const int P = rows_per_sample(n);
    const int o = threadIdx.x & 63, part = threadIdx.x >> 6;  // 4 parts x 64 channels
    float s = 0.f;
    for (int64_t r = (int64_t)blockIdx.x * 4 + part; r < (int64_t)B * n; r += (int64_t)gridDim.x * 4) {
        const int b = (int)(r / n), p = (int)(r % n);
        s += __bfloat162float(G[((int64_t)b * P + p + 3) * kC + o]);
    }
    atomicAdd(db + o, s);
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
// restart[b] = b6 + sum_c pooled[b][c] w6[c].  One warp per sample.
__global__ void head_kernel(const bf16* __restrict__ H, const bf16* __restrict__ A3, const bf16* __restrict__ wpk,
                            const float* __restrict__ params, float* __restrict__ score,
                            float* __restrict__ pooled, float* __restrict__ restart, int B, int n)
{
    const int P = rows_per_sample(n);
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const bf16* hb = H + b * P * kC;
        for (int p = lane; p < n; p += 32) {
            float s = 0.f;
            for (int j = 0; j < kC; ++j)
                s += __bfloat162float(hb[(int64_t)(p + 3) * kC + j]) * __bfloat162float(wpk[pW5 + j]);
            score[b * n + p] = s + params[oB5];
        }
        const bf16* ab = A3 + b * P * kC;
        float r = 0.f;
        for (int c = lane; c < kC; c += 32) {
            float m = 0.f;
            for (int p = 0; p < n; ++p) m += __bfloat162float(ab[(int64_t)(p + 3) * kC + c]);
            m /= (float)n;
            pooled[b * kC + c] = m;
            r += m * __bfloat162float(wpk[pW6 + c]);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, off);
        if (lane == 0) restart[b] = r + params[oB6];
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

template <int CIN, int TAPS, int EPI>
int launch_rows(const bf16* in, const bf16* Wt, const float* bias, const bf16* mask, const float* pdr,
                const bf16* pw, bf16* out, int B, int n, int sms, cudaStream_t s)
{
    const size_t smem = (size_t)kC * (TAPS * CIN + 8) * sizeof(bf16);
    auto fn = rows_gemm_kernel<CIN, TAPS, EPI>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LABS_ECUDA;
    const int64_t tiles = (int64_t)B * ((n + 15) >> 4);
    const int grid = (int)std::min<int64_t>((tiles + 3) / 4, (int64_t)sms * 8);
    fn<<<grid, 128, smem, s>>>(in, Wt, bias, mask, pdr, pw, out, B, n);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

template <int CIN, int TAPS>
int launch_wgrad(const bf16* G, const bf16* IN, float* dW, int B, int n, int sms, cudaStream_t s)
{
    constexpr int KK = TAPS * CIN;
    dim3 grid((KK + 63) / 64, (unsigned)std::min<int64_t>(B, std::max(1, sms * 4 / ((KK + 63) / 64))));
    wgrad_kernel<CIN, TAPS><<<grid, 128, 0, s>>>(G, IN, dW, B, n);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

}  // namespace

// Workspace carve-up for a batch of B states of n free variables.
struct NetWs {
    bf16 *X0, *A1, *A2, *A3, *H, *dH, *dA3, *dA2, *dA1, *wpk;
    float *score, *restart, *pooled, *ds, *dr, *loss;
    size_t bytes;
};

static size_t align256(size_t x)
{
    return (x + 255) & ~(size_t)255;
}

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
    int rc = launch_rows<kCin, kTaps, EPI_BIAS_RELU>(w.X0, w.wpk + pWf1, prm + oB1, nullptr, nullptr, nullptr, w.A1, B,
                                                     n, sms, s);
    if (!rc) rc = launch_rows<kC, kTaps, EPI_BIAS_RELU>(w.A1, w.wpk + pWf2, prm + oB2, nullptr, nullptr, nullptr, w.A2,
                                                        B, n, sms, s);
    if (!rc) rc = launch_rows<kC, kTaps, EPI_BIAS_RELU>(w.A2, w.wpk + pWf3, prm + oB3, nullptr, nullptr, nullptr, w.A3,
                                                        B, n, sms, s);
    if (!rc) rc = launch_rows<kC, 1, EPI_BIAS_RELU>(w.A3, w.wpk + pWf4, prm + oB4, nullptr, nullptr, nullptr, w.H, B, n,
                                                    sms, s);
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
    if (!rc) rc = launch_wgrad<kC, 1>(w.dH, w.A3, grad + oW4, B, n, sms, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dH, grad + oB4, B, n);
    if (!rc) rc = launch_rows<kC, 1, EPI_MASK_POOL>(w.dH, w.wpk + pWb4, nullptr, w.A3, w.dr, w.wpk + pW6, w.dA3, B, n,
                                                    sms, s);
    // conv3
    if (!rc) rc = launch_wgrad<kC, kTaps>(w.dA3, w.A2, grad + oW3, B, n, sms, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA3, grad + oB3, B, n);
    if (!rc) rc = launch_rows<kC, kTaps, EPI_MASK>(w.dA3, w.wpk + pWb3, nullptr, w.A2, nullptr, nullptr, w.dA2, B, n,
                                                   sms, s);
    // conv2
    if (!rc) rc = launch_wgrad<kC, kTaps>(w.dA2, w.A1, grad + oW2, B, n, sms, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA2, grad + oB2, B, n);
    if (!rc) rc = launch_rows<kC, kTaps, EPI_MASK>(w.dA2, w.wpk + pWb2, nullptr, w.A1, nullptr, nullptr, w.dA1, B, n,
                                                   sms, s);
    // conv1
    if (!rc) rc = launch_wgrad<kCin, kTaps>(w.dA1, w.X0, grad + oW1, B, n, sms, s);
    colsum_kernel<<<sms * 4, 256, 0, s>>>(w.dA1, grad + oB1, B, n);
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
