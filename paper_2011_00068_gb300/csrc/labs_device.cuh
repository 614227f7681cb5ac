// labs_device.cuh -- device code of the walk shared by the kernel translation units
// (included by labs_kernels.cu, labs_long.cu and the walk-instantiation units
// labs_walk8a/8b.cu, labs_walk16a/16b.cu and labs_walk32*.cu).  Not part of the
// public ABI.
//
// A tile of lanes owns one walker (or one input row): the whole warp, or half of it when
// two walkers share a warp.  A walker's sequence is kept in shared
// memory split by parity, because for even lags every term of the neighbourhood
// evaluation pairs positions of equal parity:
//   A0[u] = s_{2u}   (u = 0..n-1),   A1[u] = s_{2u+1}   (u = 0..n-2),
// and its even-lag autocorrelations (odd lags vanish by Eq. 4) as the symmetric table
//   E[d] = C_{2|d|}  (0 < |d| < n),  E[0] = 0.
//
// dISL of free variable i = 2v+p (class p, index v), q = L-1-i its mirror, c = n-1:
//   flipping {i, q} changes C_k, k even, by dC_k = -4 s_i u_k with
//   u_k = s_{i+k}[i+k != q] + s_{i-k} (out-of-range s = 0; the pair (i,q) is excluded
//   because both of its ends flip), so with Eq. 2
//   dISL_i = sum_k dC_k (2 C_k + dC_k)
//          = -8 s_i (X_i - s_q C_{q-i}) + 16 (N_i - 1) + 32 (P_i - [3i >= L-1] s_q s_{3i-L+1})
//   X_i = sum_{j != i, j = i mod 2} s_j C_{|j-i|}      (a Toeplitz product: X_v = sum_u A_p[u] E[u-v])
//   P_i = sum_{k even, 2 <= k <= i} s_{i+k} s_{i-k}
//   N_i = number of positions of the parity of i, minus one (n-1 for even i, n-2 for odd i).
//   The centre flips alone: dC_k = -2 s_c (s_{c+k} + s_{c-k}), so
//   dISL_c = -4 s_c X_c + 16 floor(c/2).
// X costs n(n-1)/2 multiply-adds per class, i.e. about one per (flip, even lag) pair of
// the neighbourhood (Algorithm 1's loop over the (L+1)/2 free variables), and is the hot
// loop.  The first half of a tile holds the even class, the second half the odd class;
// each lane owns R consecutive outputs v0..v0+R-1 and slides a window of R values of E
// along u.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "labs_internal.cuh"

namespace labsgpu {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

#ifndef LABS_TOEPLITZ_UNROLL
#define LABS_TOEPLITZ_UNROLL 2  // u-blocks of the Toeplitz loop unrolled together
#endif
constexpr int kToeplitzUnroll = LABS_TOEPLITZ_UNROLL;

#ifndef LABS_WALK_MIN_BLOCKS
#define LABS_WALK_MIN_BLOCKS 2  // CTAs of 8 warps per SM the walk kernel is compiled for (2 measured fastest)
#endif

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ void philox(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                       uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
        uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
        uint32_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0;
        c1 = lo1;
        c2 = y2;
        c3 = lo0;
    }
}

// Word j (j < 8) of the free-variable bits of start r of walker g: Philox block
// (g, r, j/4, 0) under key (seed lo, seed hi), word j%4; bits >= n cleared.
__device__ __forceinline__ uint32_t start_word(uint64_t seed, uint32_t g, uint32_t r, int j, int n)
{
    uint32_t c0 = g, c1 = r, c2 = (uint32_t)(j >> 2), c3 = 0u;
    philox(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint32_t w = (j & 3) == 0 ? c0 : (j & 3) == 1 ? c1 : (j & 3) == 2 ? c2 : c3;
    int lo = 32 * j;
    if (n <= lo) return 0u;
    if (n - lo >= 32) return w;
    return w & ((1u << (n - lo)) - 1u);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int detail)
{
    if (atomicCAS(&st->error, 0, code) == 0) st->error_detail = detail;
}

// A group of TILE lanes that runs one walker (or one row): the whole warp (TILE = 32)
// or a half warp (TILE = 16, two walkers per warp).  Every warp-level primitive of the
// walk goes through it with the tile's own lane mask, so the two halves of a warp may
// take different paths.
template <int TILE>
struct Tile {
    static constexpr int kSize = TILE;
    static constexpr int kHalf = TILE / 2;  // lanes per parity class
    static constexpr unsigned kLow = TILE == 32 ? 0xFFFFFFFFu : ((1u << TILE) - 1u);
    int lane;       // 0 .. TILE-1
    int base;       // warp lane of the tile's lane 0
    unsigned mask;  // the tile's lanes
    __device__ explicit Tile(int warp_lane)
        : lane(warp_lane & (TILE - 1)), base(warp_lane & ~(TILE - 1)), mask(kLow << (warp_lane & ~(TILE - 1)))
    {
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ unsigned ballot(bool p) const { return (__ballot_sync(mask, p) >> base) & kLow; }
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(mask, v, base + src); }
    __device__ __forceinline__ uint32_t shfl(uint32_t v, int src) const { return __shfl_sync(mask, v, base + src); }
    __device__ __forceinline__ int rmin(int v) const { return __reduce_min_sync(mask, v); }
    __device__ __forceinline__ int rmax(int v) const { return __reduce_max_sync(mask, v); }
    __device__ __forceinline__ int radd(int v) const { return __reduce_add_sync(mask, v); }
    __device__ __forceinline__ uint32_t rxor(uint32_t v) const { return __reduce_xor_sync(mask, v); }
    __device__ __forceinline__ unsigned rminu(unsigned v) const { return __reduce_min_sync(mask, v); }
};

// Two walkers per warp advancing in lockstep (lanes 16h..16h+15 belong to walker h):
// the same interface as Tile<16>, built from full-warp collectives in which each half
// contributes the neutral value to the other half's reduction.  Only for converged
// code: both halves must reach every call.
struct Pair {
    static constexpr int kSize = 16;
    static constexpr int kHalf = 8;
    int lane;  // 0 .. 15
    int h;     // which walker of the warp
    int base;  // 16 h
    __device__ explicit Pair(int warp_lane) : lane(warp_lane & 15), h(warp_lane >> 4), base(warp_lane & 16) {}
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ unsigned ballot(bool p) const { return (__ballot_sync(kFull, p) >> base) & 0xFFFFu; }
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(kFull, v, base + src); }
    __device__ __forceinline__ uint32_t shfl(uint32_t v, int src) const { return __shfl_sync(kFull, v, base + src); }
    __device__ __forceinline__ int rmin(int v) const
    {
        const int a = __reduce_min_sync(kFull, h ? INT_MAX : v), b = __reduce_min_sync(kFull, h ? v : INT_MAX);
        return h ? b : a;
    }
    __device__ __forceinline__ unsigned rminu(unsigned v) const
    {
        const unsigned a = __reduce_min_sync(kFull, h ? 0xFFFFFFFFu : v), b = __reduce_min_sync(kFull, h ? v : 0xFFFFFFFFu);
        return h ? b : a;
    }
    __device__ __forceinline__ int rmax(int v) const
    {
        const int a = __reduce_max_sync(kFull, h ? INT_MIN : v), b = __reduce_max_sync(kFull, h ? v : INT_MIN);
        return h ? b : a;
    }
    __device__ __forceinline__ int radd(int v) const
    {
        const int a = __reduce_add_sync(kFull, h ? 0 : v), b = __reduce_add_sync(kFull, h ? v : 0);
        return h ? b : a;
    }
    __device__ __forceinline__ uint32_t rxor(uint32_t v) const
    {
        const uint32_t a = __reduce_xor_sync(kFull, h ? 0u : v), b = __reduce_xor_sync(kFull, h ? v : 0u);
        return h ? b : a;
    }
};

// Four walkers per warp advancing in lockstep (lanes 8h..8h+7 belong to walker h): the
// reductions are butterflies of xor-shuffles that stay inside each group of 8 lanes, so
// one sequence serves all four walkers.  Only for converged code.
struct Quad {
    static constexpr int kSize = 8;
    static constexpr int kHalf = 4;
    int lane;  // 0 .. 7
    int h;     // which walker of the warp
    int base;  // 8 h
    __device__ explicit Quad(int warp_lane) : lane(warp_lane & 7), h(warp_lane >> 3), base(warp_lane & 24) {}
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ unsigned ballot(bool p) const { return (__ballot_sync(kFull, p) >> base) & 0xFFu; }
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(kFull, v, base + src); }
    __device__ __forceinline__ uint32_t shfl(uint32_t v, int src) const { return __shfl_sync(kFull, v, base + src); }
    __device__ __forceinline__ int rmin(int v) const
    {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
    __device__ __forceinline__ unsigned rminu(unsigned v) const
    {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
    __device__ __forceinline__ int rmax(int v) const
    {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
    __device__ __forceinline__ int radd(int v) const
    {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        return v;
    }
    __device__ __forceinline__ uint32_t rxor(uint32_t v) const
    {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
        return v;
    }
};

// Per-walker views of the shared-memory layout.
struct View {
    float* A0;    // A0[-apad .. alen-apad)
    float* A1;
    float2* G;    // G[y] = (E[y], E[y+1]), y in [-gpad, glen-gpad)
    uint32_t* B;  // bit-packed classes and reversals, 4 x bvec words
    __half* H0;   // FP16 copies of A0 and A1 for the tensor-core Toeplitz product (null:
    __half* H1;   // none); every write of a row entry writes its copy too
    int gpad;
    int bvec;
};

__device__ __forceinline__ View make_view(int* base, const WarpSmem& L)
{
    View v;
    v.A0 = reinterpret_cast<float*>(base) + L.apad;
    v.A1 = reinterpret_cast<float*>(base) + L.alen + L.apad;
    v.G = reinterpret_cast<float2*>(base + L.goff) + L.gpad;
    v.B = reinterpret_cast<uint32_t*>(base + L.boff);
    v.H0 = L.hlen ? reinterpret_cast<__half*>(base + L.hoff) + L.hpad : nullptr;
    v.H1 = L.hlen ? reinterpret_cast<__half*>(base + L.hoff + L.hlen) + L.hpad : nullptr;
    v.gpad = L.gpad;
    v.bvec = L.bvec;
    return v;
}

// Row entry u of class p (and its FP16 copy, when the layout keeps one).
__device__ __forceinline__ void set_row(const View& V, int p, int u, float s)
{
    (p ? V.A1 : V.A0)[u] = s;
    if (V.H0 != nullptr) (p ? V.H1 : V.H0)[u] = __float2half_rn(s);
}

// E[m] = e (m >= 1) in every pair of G that holds it, mirrored to E[-m].
__device__ __forceinline__ void set_E(const View& V, int m, float e)
{
    V.G[m].x = e;
    V.G[m - 1].y = e;
    if (m <= V.gpad) V.G[-m].x = e;
    if (m < V.gpad) V.G[-m - 1].y = e;
}

// Zeroes the walker's rows, table and bit vectors.
template <class TL>
__device__ __forceinline__ void clear_rows(int* base, const WarpSmem& L, const TL& t)
{
    int4* b4 = reinterpret_cast<int4*>(base);
    for (int i = t.lane; i < L.words / 4; i += TL::kSize) b4[i] = make_int4(0, 0, 0, 0);
    t.sync();
}

// Fills A0/A1 from the free-variable bits (word j of the bits lives in tile lane j's
// `word`), by Eq. 4: s_j = x_j for j <= c, s_{c+t} = (-1)^t x_{c-t}.
template <class TL>
__device__ __forceinline__ void rows_from_bits(const View& V, uint32_t word, int L, int n, const TL& t)
{
    const int c = n - 1;
    for (int j0 = 0; j0 < L; j0 += TL::kSize) {
        const int j = j0 + t.lane;
        int f = j <= c ? j : 2 * c - j;
        if (j >= L) f = 0;
        const uint32_t w = t.shfl(word, f >> 5);
        if (j < L) {
            const int x = ((w >> (f & 31)) & 1u) ? -1 : 1;
            const int s = (j > c && ((j - c) & 1)) ? -x : x;
            set_row(V, j & 1, j >> 1, (float)s);
        }
    }
    t.sync();
}

// Bit-packed classes: B[p*bvec + k] holds bits 32k..32k+31 of class p (bit u set
// <=> A_p[u] = -1); B[(2+p)*bvec + k] the same for the reversed class (bit u is
// class entry n_p-1-u).  Zero beyond the class length.  A lane group wider than a warp
// (one walker per CTA) builds one word per warp and round.
template <class TL>
__device__ __forceinline__ void bits_from_rows(const View& V, int n, const TL& t)
{
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float* A = p ? V.A1 : V.A0;
        const int np = p ? n - 1 : n;
        if constexpr (TL::kSize > 32) {
            const int wl = t.lane & 31;
            for (int k = t.lane >> 5; k < V.bvec; k += TL::kSize / 32) {
                const int u = 32 * k + wl;
                const uint32_t w = __ballot_sync(kFull, u < np && A[u] < 0.f);
                const uint32_t r = __ballot_sync(kFull, u < np && A[np - 1 - u] < 0.f);
                if (wl == 0) {
                    V.B[p * V.bvec + k] = w;
                    V.B[(2 + p) * V.bvec + k] = r;
                }
            }
        } else {
            // words beyond the class (and its zero word) stay zero: every caller cleared
            // them and no walker of another length shares this walker's memory since
            const int nwd = min(V.bvec, (np + 31) / 32 + 1);
            for (int k = 0; k < nwd; ++k) {
                uint32_t w = 0, r = 0;
#pragma unroll
                for (int h = 0; h < 32 / TL::kSize; ++h) {
                    const int u = 32 * k + TL::kSize * h + t.lane;
                    const uint32_t bw = t.ballot(u < np && A[u] < 0.f);
                    const uint32_t br = t.ballot(u < np && A[np - 1 - u] < 0.f);
                    w |= (TL::kSize == 32) ? bw : (bw << (TL::kSize * h));
                    r |= (TL::kSize == 32) ? br : (br << (TL::kSize * h));
                }
                if (t.lane == 0) {
                    V.B[p * V.bvec + k] = w;
                    V.B[(2 + p) * V.bvec + k] = r;
                }
            }
        }
    }
    t.sync();
}

// Even-lag autocorrelations (Eq. 1) into E and the ISL (Eq. 2) from the bit-packed
// classes: for each class, sum_u a_u a_{u+m} = (n_p - m) - 2 #{u : a_u != a_{u+m}}.
template <class TL>
__device__ __forceinline__ int build_table(const View& V, int n, const TL& t)
{
    bits_from_rows(V, n, t);
    int part = 0;
    const uint32_t* x0 = V.B;
    const uint32_t* x1 = V.B + V.bvec;
    // lags m = mb + g kSize, g < 4, together (eight independent counts), both classes in
    // one pass over the words (lengths n - m and n - 1 - m, same shift)
    constexpr int kG = 4;
    for (int mb = 1 + t.lane; mb < n; mb += kG * TL::kSize) {
        int c0[kG], c1[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) c0[g] = c1[g] = 0;
        for (int k = 0; 32 * k < n - mb; ++k) {
#pragma unroll
            for (int g = 0; g < kG; ++g) {
                const int m = mb + g * TL::kSize, len0 = n - m, v0 = len0 - 32 * k, v1 = v0 - 1;
                if (v0 > 0) {
                    const int q = m >> 5, r = m & 31;
                    const uint32_t m0 = v0 >= 32 ? ~0u : (1u << v0) - 1u;
                    const uint32_t m1 = v1 >= 32 ? ~0u : (v1 > 0 ? (1u << v1) - 1u : 0u);
                    c0[g] += __popc((x0[k] ^ __funnelshift_r(x0[k + q], x0[k + q + 1], r)) & m0);
                    c1[g] += __popc((x1[k] ^ __funnelshift_r(x1[k + q], x1[k + q + 1], r)) & m1);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const int m = mb + g * TL::kSize;
            if (m < n) {
                const int len0 = n - m, len1 = len0 - 1;
                const int d = len0 - 2 * c0[g] + (len1 > 0 ? len1 - 2 * c1[g] : 0);
                set_E(V, m, (float)d);
                part += d * d;
            }
        }
    }
    t.sync();
    return t.radd(part);
}

// Lane layout of the neighbourhood: the first half of the tile holds the even class,
// the second half the odd class; lane l of a half owns outputs v0 .. v0+R-1.
template <class TL, int R>
struct Outs {
    int p, v0;
    __device__ explicit Outs(const TL& t) : p(t.lane / TL::kHalf), v0((t.lane % TL::kHalf) * R) {}
};

// X_v = sum_u A_p[u] E[u-v] for the lane's R outputs v = v0..v0+R-1 (the Toeplitz
// product), on the FP32 pipes with packed pairs: accumulator r holds the partial sums
// of X_{v0+r} over even u (.x) and odd u (.y), so one __ffma2_rn multiplies the pair
// (A[u], A[u+1]) by G[u-v] = (E[u-v], E[u+1-v]).  The window win[j] = G[u-v0-j] slides
// two positions per pair of u: two 8-byte loads per R packed FMAs.  All operands and
// partial sums are integers below 2^24, so the result is exact.
// Outputs C0 .. C0+RC-1 of the lane's block (G already offset by -v0).
template <int R, int C0, int RC>
__device__ __forceinline__ void toeplitz_part(const float* A, const float2* G, int nu, float (&X)[R])
{
    float2 acc[RC], win[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        acc[r] = make_float2(0.f, 0.f);
        win[r] = G[-C0 - r];
    }
#pragma unroll kToeplitzUnroll
    for (int u = 0; u < nu; u += 8) {
        const float4 a0 = *reinterpret_cast<const float4*>(A + u);
        const float4 a1 = *reinterpret_cast<const float4*>(A + u + 4);
        const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                              make_float2(a1.z, a1.w)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = __ffma2_rn(ap[q], win[r], acc[r]);
#pragma unroll
            for (int j = RC - 1; j >= 2; --j) win[j] = win[j - 2];
            if (RC >= 2) win[1] = G[u + 2 * q + 1 - C0];
            win[0] = G[u + 2 * q + 2 - C0];
        }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) X[C0 + r] = acc[r].x + acc[r].y;
}

// All R outputs in one pass over u (a two-pass split of a 13-output block, fewer
// registers, ran the four-walker step 13-29% slower than one pass).
template <class TL, int R>
__device__ __forceinline__ void toeplitz(const View& V, int n, const Outs<TL, R>& o, float (&X)[R])
{
    const float* A = o.p ? V.A1 : V.A0;
    toeplitz_part<R, 0, R>(A, V.G - o.v0, (n + 7) & ~7, X);
}

// The Toeplitz products of both walkers of a warp (two walkers per warp) on the tensor
// cores, for n <= 128.  In blocks of 16, u = 16 s + j and v = 16 t + i, the product is
//   X_t = sum_d T_d A_{t+d},   T_d[i][j] = E[16 d + j - i],   A_s[j] = A_p[16 s + j],
// a sum over the block diagonals d of a 16 x 16 Toeplitz block of the table times the
// row blocks d further.  One mma.sync.m16n8k16 per diagonal takes T_d (rows i, columns
// j) and, as its 8 columns, the row blocks of output blocks t = 0..3 of both classes
// (columns 0-3 class 0, 4-7 class 1); d runs from -(T-1) to S-1 for the T output and S
// row blocks.  The table's entries are rounded to FP16 as they are loaded (|E| < 2^11
// is exact), the rows come from their FP16 copies (A = 0, +-1), and the products
// accumulate in FP32: every partial sum is an integer below 2^24, so the result equals
// the FP32 product's.  Reads outside the class meet the rows' zero padding, and E is
// finite (zero) beyond the table.  The warp writes each walker's results to its
// scratch X[2][xp], and every lane then reads its R outputs.
__device__ __forceinline__ uint32_t half2_bits(float2 v)
{
    const __half2 h = __float22half2_rn(v);  // .x in the low half
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One block diagonal of one walker: T_d from the table pairs at gy (and the pair 8 below,
// carried in am8), the row blocks' FP16 pairs at ab.
__device__ __forceinline__ void tc_diag(float (&d)[4], const float2* gy, const uint32_t* ab, uint32_t& am8)
{
    const uint32_t a0 = half2_bits(gy[0]), a2 = half2_bits(gy[8]);
    mma_16816(d, a0, am8, a2, a0, ab[0], ab[4]);
    am8 = a2;
}

template <int R>
__device__ __forceinline__ void toeplitz_tc(const View& V, const WarpSmem& SL, int n, const Outs<Pair, R>& o, int h,
                                            float (&X)[R])
{
    const int l = threadIdx.x & 31, g = l >> 2, tq = l & 3;
    const int S = (n + 15) >> 4;               // row blocks
    const int T = (((n + 1) >> 1) + 15) >> 4;  // output blocks per class (<= 4)
    const int pb = g >> 2, tb = g & 3;         // this lane's operand column: class, block
    const int px = tq >> 1, tx = 2 * (tq & 1); // its accumulator columns: class, first block
    int* const own = reinterpret_cast<int*>(V.A0) - SL.apad;
    int* const base0 = own - h * SL.words;     // walker 0 of the warp; walker 1 follows
    const float2* gy = reinterpret_cast<const float2*>(base0 + SL.goff) + SL.gpad + (2 * tq - g - 16 * (T - 1));
    const uint32_t* ab = reinterpret_cast<const uint32_t*>(base0 + SL.hoff + pb * SL.hlen) + (SL.hpad >> 1) +
                         8 * (tb - (T - 1)) + tq;
    const int nd = S + T - 1, w1 = SL.words, g1 = SL.words >> 1;
    // two independent accumulator chains, one per walker
    float d0[4] = {0.f, 0.f, 0.f, 0.f}, e0[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t am0 = half2_bits(gy[-8]), am1 = half2_bits(gy[g1 - 8]);
    for (int k = 0; k < nd; ++k) {
        tc_diag(d0, gy, ab, am0);
        tc_diag(e0, gy + g1, ab + w1, am1);
        gy += 16;
        ab += 8;
    }
    float* xp = reinterpret_cast<float*>(base0 + SL.roff) + px * SL.xp + 16 * tx + g;
    float* xq = xp + w1;
    if (tx < T) {
        xp[0] = d0[0];
        xp[8] = d0[2];
        xq[0] = e0[0];
        xq[8] = e0[2];
    }
    if (tx + 1 < T) {
        xp[16] = d0[1];
        xp[24] = d0[3];
        xq[16] = e0[1];
        xq[24] = e0[3];
    }
    __syncwarp();
    const float* xr = reinterpret_cast<const float*>(own + SL.roff) + o.p * SL.xp + o.v0;
#pragma unroll
    for (int r = 0; r < R; ++r) X[r] = xr[r];
}

// The same product for one walker whose lane group spans W whole warps (one walker per
// warp, W = 1, or per CTA): the output blocks form ceil(T/4) column groups of 4 blocks
// per class, warp w takes groups w, w + W, ..., and for group m the block diagonals run
// from -(4m+3) (or -(T-1)) up to S-1-4m.  Two accumulator chains per warp (two groups,
// or the even and odd diagonals of a lone group; integer partial sums, so the split does
// not change the result).  The results go through the walker's scratch X[2][xp] to the
// lanes' R outputs; the group's barrier orders them.
template <class LG, int R>
__device__ __forceinline__ void toeplitz_tc1(const View& V, const WarpSmem& SL, int n, const Outs<LG, R>& o,
                                             const LG& t, float (&X)[R])
{
    constexpr int W = LG::kSize / 32;
    const int warp = W == 1 ? 0 : (int)(threadIdx.x >> 5), l = threadIdx.x & 31, g = l >> 2, tq = l & 3;
    const int S = (n + 15) >> 4, T = (((n + 1) >> 1) + 15) >> 4, M = (T + 3) >> 2;
    const int pb = g >> 2, tb = g & 3, px = tq >> 1, tx = 2 * (tq & 1);
    int* const base = reinterpret_cast<int*>(V.A0) - SL.apad;
    const float2* G = reinterpret_cast<const float2*>(base + SL.goff) + SL.gpad + (2 * tq - g);
    const uint32_t* H = reinterpret_cast<const uint32_t*>(base + SL.hoff + pb * SL.hlen) + (SL.hpad >> 1) + 8 * tb + tq;
    float* xs = reinterpret_cast<float*>(base + SL.roff) + px * SL.xp + g;
    // warp w takes groups m and m + W together: a diagonal's table fragment is loaded
    // once for both (their diagonal ranges are shifted by 4W); a group without a partner
    // runs alone with two chains (even and odd diagonals)
    for (int m = warp; m < M; m += 2 * W) {
        const int mb = m + W;
        const int dloA = -min(4 * m + 3, T - 1), dhi = S - 1 - 4 * m;  // group m: d = dloA .. dhi
        if (mb < M) {
            const int dlo = -min(4 * mb + 3, T - 1), dhiB = dhi - 4 * W;  // group mb: d = dlo .. dhiB
            const float2* gy = G + 16 * dlo;
            const uint32_t* ab = H + 8 * (4 * m + dlo);  // group m's operand; mb's is 32 W words further
            float dA[4] = {0.f, 0.f, 0.f, 0.f}, dB[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t am = half2_bits(gy[-8]);
            for (int d = dlo; d <= dhi; ++d) {
                const uint32_t a0 = half2_bits(gy[0]), a2 = half2_bits(gy[8]);
                if (d >= dloA) mma_16816(dA, a0, am, a2, a0, ab[0], ab[4]);
                if (d <= dhiB) mma_16816(dB, a0, am, a2, a0, ab[32 * W], ab[32 * W + 4]);
                am = a2;
                gy += 16;
                ab += 8;
            }
            const int tA = tx + 4 * m, tB = tx + 4 * mb;
            if (tA < T) {
                xs[16 * tA] = dA[0];
                xs[16 * tA + 8] = dA[2];
            }
            if (tA + 1 < T) {
                xs[16 * tA + 16] = dA[1];
                xs[16 * tA + 24] = dA[3];
            }
            if (tB < T) {
                xs[16 * tB] = dB[0];
                xs[16 * tB + 8] = dB[2];
            }
            if (tB + 1 < T) {
                xs[16 * tB + 16] = dB[1];
                xs[16 * tB + 24] = dB[3];
            }
        } else {
            const int nd = dhi - dloA + 1;
            const float2* gy = G + 16 * dloA;
            const uint32_t* ab = H + 8 * (4 * m + dloA);
            float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t am = half2_bits(gy[-8]);
            int k = 0;
            for (; k + 1 < nd; k += 2) {
                tc_diag(d0, gy, ab, am);
                tc_diag(d1, gy + 16, ab + 8, am);
                gy += 32;
                ab += 16;
            }
            if (k < nd) tc_diag(d0, gy, ab, am);
            const int t0 = tx + 4 * m;
            if (t0 < T) {
                xs[16 * t0] = d0[0] + d1[0];
                xs[16 * t0 + 8] = d0[2] + d1[2];
            }
            if (t0 + 1 < T) {
                xs[16 * t0 + 16] = d0[1] + d1[1];
                xs[16 * t0 + 24] = d0[3] + d1[3];
            }
        }
    }
    t.sync();
    const float* xr = reinterpret_cast<const float*>(base + SL.roff) + o.p * SL.xp + o.v0;
#pragma unroll
    for (int r = 0; r < R; ++r) X[r] = xr[r];
}

// The Toeplitz product of a lane group that owns one walker: on the tensor cores when
// the layout holds the FP16 rows and the results' scratch, else on the FP32 pipes.
template <class LG, int R>
__device__ __forceinline__ void toeplitz_one(const View& V, const WarpSmem& SL, int n, const Outs<LG, R>& o,
                                             const LG& t, float (&X)[R])
{
    if constexpr (LG::kSize >= 32) {
        if (SL.xp != 0) {
            toeplitz_tc1(V, SL, n, o, t, X);
            return;
        }
    }
    toeplitz(V, n, o, X);
}

// P_v = sum_{m=1}^{v} A_p[v+m] A_p[v-m] from scratch for the lane's outputs, from the
// bit-packed classes (built by build_table): the pairs compare bits v+1.. of the
// class with bits n_p-v.. of the reversed class, P_v = v - 2 #{mismatches}.
template <class TL, int R>
__device__ __forceinline__ void p_direct(const View& V, int n, const Outs<TL, R>& o, float (&P)[R])
{
    const int np = o.p ? n - 1 : n;
    const int nv = o.p ? (n >> 1) : ((n + 1) >> 1);
    const uint32_t* x = V.B + o.p * V.bvec;
    const uint32_t* xr = V.B + (2 + o.p) * V.bvec;
    // the R outputs word by word (independent chains); output v compares v bits
    int cnt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) cnt[r] = 0;
    const int vtop = min(o.v0 + R - 1, nv - 1);
    for (int k = 0; 32 * k < vtop; ++k) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = o.v0 + r;
            const int valid = v - 32 * k;
            if (v < nv && valid > 0) {
                const uint32_t a = __funnelshift_r(x[k + ((v + 1) >> 5)], x[k + ((v + 1) >> 5) + 1], (v + 1) & 31);
                const uint32_t b = __funnelshift_r(xr[k + ((np - v) >> 5)], xr[k + ((np - v) >> 5) + 1], (np - v) & 31);
                const uint32_t mk = valid >= 32 ? ~0u : (1u << valid) - 1u;
                cnt[r] += __popc((a ^ b) & mk);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = o.v0 + r;
        P[r] = (v >= nv || v == 0) ? 0.f : (float)(v - 2 * cnt[r]);
    }
}

// Change of P for a move that negates class-pb entries w1 and w2 (w2 < 0: centre, one
// entry).  A pair (v+m, v-m) with exactly one negated end changes by -2 x its old
// product; pairs with both ends negated are unchanged.  Reads A before the flip.
template <class TL, int R>
__device__ __forceinline__ void p_update(const View& V, int n, const Outs<TL, R>& o, float (&P)[R], int pb, int w1,
                                         int w2)
{
    if (o.p != pb) return;
    const float* A = pb ? V.A1 : V.A0;
    const int nv = pb ? (n >> 1) : ((n + 1) >> 1);
    const float a1 = A[w1];
    const float a2 = w2 >= 0 ? A[w2] : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = o.v0 + r;
        if (v >= nv) continue;
        float d = 0.f;
        const int t1 = 2 * v - w1;
        if (v != w1 && t1 != w2) d = a1 * A[t1];
        if (w2 >= 0) {
            const int t2 = 2 * v - w2;
            if (v != w2 && t2 != w1) d = fmaf(a2, A[t2], d);
        }
        P[r] = fmaf(-2.f, d, P[r]);
    }
}

// dl[r] = dISL of free variable i = 2(v0+r)+p, or INT_MAX where that output does not
// exist.  Formula in the header comment; evaluated in exact float arithmetic (all
// terms are integers below 2^24) and converted once.
template <class TL, int R>
__device__ __forceinline__ void assemble(const View& V, int n, const Outs<TL, R>& o, const float (&X)[R],
                                         const float (&P)[R], int (&dl)[R])
{
    const int p = o.p;
    const float* A = p ? V.A1 : V.A0;
    const int nv = p ? (n >> 1) : ((n + 1) >> 1);
    const int c = n - 1;
    const float base = (float)(16 * ((p ? n - 2 : n - 1) - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = o.v0 + r;
        if (v >= nv) {
            dl[r] = INT_MAX;
            continue;
        }
        const int i = 2 * v + p;
        const float av = A[v];
        if (i == c) {
            dl[r] = __float2int_rn(fmaf(-4.f * av, X[r], (float)(16 * (c >> 1))));
            continue;
        }
        const float sq = A[n - 1 - v - p];
        const float ck0 = V.G[c - i].x;
        const int t = 3 * v + p - n + 1;
        const float corr = t >= 0 ? sq * A[t] : 0.f;
        dl[r] = __float2int_rn(fmaf(-8.f * av, fmaf(-sq, ck0, X[r]), fmaf(32.f, P[r] - corr, base)));
    }
}

// Rebuilds the walker's rows and table from its bits; returns the ISL.
template <class TL>
__device__ __forceinline__ int load_rows(int* base, const WarpSmem& SL, const View& V, uint32_t word, int L, int n,
                                         const TL& t)
{
    clear_rows(base, SL, t);
    rows_from_bits(V, word, L, n, t);
    return build_table(V, n, t);
}

// HT fingerprint (Zobrist): XOR of the keys of the free variables equal to -1.
template <class TL>
__device__ __forceinline__ uint64_t fingerprint_all(uint32_t word, const uint64_t* zk, int n, const TL& t)
{
    uint64_t f = 0;
    const int nr = (n + TL::kSize - 1) & ~(TL::kSize - 1);
    for (int i0 = 0; i0 < nr; i0 += TL::kSize) {
        const int i = i0 + t.lane;
        const uint32_t w = t.shfl(word, i0 >> 5);
        if (i < n && ((w >> (i & 31)) & 1u)) f ^= __ldg(zk + i);
    }
    const uint32_t lo = t.rxor((uint32_t)f);
    const uint32_t hi = t.rxor((uint32_t)(f >> 32));
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Registers of one walker while its tile runs it.
struct Walker {
    uint32_t word;   // tile lane j < 8: bits word j
    uint64_t fp;
    int isl, best_isl, since, stag;
    uint32_t restart_idx, gen;
    int restarts, overflows, blocked;
    int64_t steps, best_step, target_step;
};

struct WalkEnv {
    const KParams* p;
    uint64_t* T;       // this walker's HT
    uint64_t tmask;
    const uint64_t* zk;
    WalkerState* st;
    int L, n, patience;
    uint32_t g;
    // learned mode (null when off): proposed restart state and its flag
    uint32_t* slot;
    int32_t* slot_valid;
    // replay dumps of a traced walker in learned mode (null when off)
    uint32_t* rdump;   // [cap][8]
    int64_t* rdump_idx;
    int32_t* rdump_count;
    int dump_cap;
};

__device__ __forceinline__ bool target_met(const KParams& p, int L, int isl)
{
    if (p.target_num <= 0 || p.target_den <= 0) return false;
    return (int64_t)p.target_den * L * L >= 2 * (int64_t)p.target_num * isl;
}

// PSL objective: the current sequence's PSL, and the PSL halves of the (PSL, ISL)
// pairs of the best sequence and of the best since the last (re)start.
struct PslTrack {
    int psl, best_psl, since_psl;
};

// Lower (PSL, ISL) pair, compared lexicographically.
__device__ __forceinline__ bool psl_better(int psl, int isl, int psl0, int isl0)
{
    return psl < psl0 || (psl == psl0 && isl < isl0);
}

// max |C_{2m}| over m = 1..n-1 from the table: the PSL of a skew-symmetric sequence
// (Section 1; its odd-lag C_k vanish).
template <class TL>
__device__ __forceinline__ int table_psl(const View& V, int n, const TL& t)
{
    int mx = 0;
    for (int m = 1 + t.lane; m < n; m += TL::kSize) mx = max(mx, abs(__float2int_rn(V.G[m].x)));
    return t.rmax(mx);
}

// Best-sequence update: strictly lower ISL, or under the PSL objective (ps != null) a
// strictly lower (PSL, ISL) pair.
template <class TL>
__device__ __forceinline__ void note_best(const WalkEnv& env, Walker& w, const TL& t, PslTrack* ps = nullptr)
{
    const bool better = ps ? psl_better(ps->psl, w.isl, ps->best_psl, w.best_isl) : w.isl < w.best_isl;
    if (better) {
        w.best_isl = w.isl;
        if (ps) ps->best_psl = ps->psl;
        w.best_step = w.steps;
        if (t.lane < kBitWords) env.st->best[t.lane] = w.word;
    }
    if (w.target_step < 0 && target_met(*env.p, env.L, w.isl)) w.target_step = w.steps;
}

// Algorithm 1 start: random skew-symmetric S (restart index w.restart_idx), its ISL,
// insert it into HT (a fresh generation: its home slot is free), best update.
template <class TL>
__device__ void start_walker(const WalkEnv& env, Walker& w, int* base, const WarpSmem& SL, const View& V,
                             const TL& t, bool proposed = false, PslTrack* ps = nullptr)
{
    const int lane = t.lane;
    if (proposed) {
        // learned mode: the restart state chosen by the proposal pass replaces the draw
        w.word = lane < kBitWords ? env.slot[lane] : 0u;
        if (env.rdump != nullptr) {
            const int k = *env.rdump_count;
            if (k < env.dump_cap) {
                if (lane < kBitWords) env.rdump[(int64_t)k * kBitWords + lane] = w.word;
                if (lane == 0) env.rdump_idx[k] = w.restart_idx;
            }
            t.sync();
            if (lane == 0) *env.rdump_count = k + 1;
        }
        t.sync();
        if (lane == 0) *env.slot_valid = 0;
    } else {
        w.word = lane < kBitWords ? start_word(env.p->seed, env.g, w.restart_idx, lane, env.n) : 0u;
    }
    w.isl = load_rows(base, SL, V, w.word, env.L, env.n, t);
    w.fp = fingerprint_all(w.word, env.zk, env.n, t);
    if (lane == 0) env.T[w.fp & env.tmask] = (w.fp & ~kGenMask) | w.gen;
    t.sync();
    w.since = w.isl;
    w.stag = 0;
    if (ps) {
        ps->psl = table_psl(V, env.n, t);
        ps->since_psl = ps->psl;
    }
    note_best(env, w, t, ps);
}

template <class TL>
__device__ void restart_walker(const WalkEnv& env, Walker& w, int* base, const WarpSmem& SL, const View& V,
                               const TL& t, PslTrack* ps = nullptr)
{
    w.restart_idx += 1;
    w.restarts += 1;
    w.gen += 1;
    if (w.gen > kGenMask) {
        const int64_t slots = (int64_t)env.tmask + 1;
        for (int64_t i = t.lane; i < slots; i += TL::kSize) env.T[i] = 0ull;
        t.sync();
        w.gen = 1;
    }
    int prop = 0;
    if (t.lane == 0 && env.slot_valid != nullptr) prop = *env.slot_valid != 0;
    const bool proposed = t.shfl(prop, 0) != 0;
    start_walker(env, w, base, SL, V, t, proposed, ps);
}

// Stop requests from the host-written control block (mapped host memory, slow to
// read).  One lane (`reader`) reads the deadline and the cancel flag when a walk call
// starts; after that it re-reads the cancel flag at every poll without waiting for it:
// the value lands while the steps run and is acted on at the next poll, kCheckEvery
// steps later.  The deadline is compared with %globaltimer at every poll.
struct StopCheck {
    uint64_t deadline = ~0ull;
    int next = 0;
    __device__ __forceinline__ void start(const KParams& p, bool reader)
    {
        if (reader && p.ctrl != nullptr) {
            deadline = p.ctrl->deadline_ns;
            next = p.ctrl->stop;
        }
    }
    // LABS_ECANCELLED, LABS_ETIMEOUT or 0, in the reader lane (0 elsewhere)
    __device__ __forceinline__ int poll(const KParams& p, bool reader)
    {
        int why = 0;
        if (reader && p.ctrl != nullptr) {
            if (next) why = LABS_ECANCELLED;
            else if (global_ns() >= deadline) why = LABS_ETIMEOUT;
            next = p.ctrl->stop;
        }
        return why;
    }
};

// Result of probing HT for one candidate.
struct Probe {
    bool visited;
    int64_t slot;  // insertion slot when not visited, -1 when no free slot within the cap
};

// Full linear probe of f: up to `cap` slots, TILE at a time.
template <class TL>
__device__ __forceinline__ Probe probe_full(const WalkEnv& env, uint64_t f, uint32_t gen, int cap, const TL& t)
{
    const uint64_t tag = (f & ~kGenMask) | gen;
    Probe pr{false, -1};
    for (int s0 = 0; s0 < cap; s0 += TL::kSize) {
        const int s = s0 + t.lane;
        uint64_t e = 0;
        if (s < cap) e = env.T[(f + (uint64_t)s) & env.tmask];
        const bool match = e == tag;
        const unsigned bal = t.ballot(s < cap && (((e & kGenMask) != gen) || match));
        if (bal) {
            const int fl = __ffs(bal) - 1;
            pr.visited = t.shfl(match ? 1 : 0, fl) != 0;
            pr.slot = (int64_t)((f + (uint64_t)(s0 + fl)) & env.tmask);
            break;
        }
    }
    return pr;
}

// Lowest (dl, i) among the lane outputs not in `excl` (every lane of the tile gets the
// result; bi = -1 when none is left).
template <class TL, int R>
__device__ __forceinline__ void tile_argmin(const int (&dl)[R], uint32_t excl, const Outs<TL, R>& o,
                                            const TL& t, int& bd, int& bi)
{
    int lm = INT_MAX, li = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (!((excl >> r) & 1u) && dl[r] < lm) {
            lm = dl[r];
            li = 2 * (o.v0 + r) + o.p;
        }
    bd = t.rmin(lm);
    bi = bd == INT_MAX ? -1 : t.rmin(lm == bd ? li : INT_MAX);
}

template <class TL, int R>
__device__ __forceinline__ void exclude(uint32_t& excl, int bi, const TL& t)
{
    const int vb = bi >> 1, pb = bi & 1;
    if (t.lane == pb * TL::kHalf + vb / R) excl |= 1u << (vb % R);
}

// Order-preserving map of a float score to int32 (the learned ordering compares these).
__device__ __forceinline__ int score_key(float f)
{
    const int k = __float_as_int(f);
    return k >= 0 ? k : (k ^ 0x7FFFFFFF);
}

// S <- S_f for free variable bi: the table E (C_{2m} += -4 s_i (s_{i-2m} + s_{i+2m}),
// the mirror's own term left out, -2 s_c (..) at the centre), P and the two row
// entries, all from the values before the flip.  Ends without a tile barrier.
template <class TL, int R>
__device__ __forceinline__ void flip_rows_table(const View& V, int n, const Outs<TL, R>& o, float (&P)[R], int bi,
                                                const TL& t)
{
    const int lane = t.lane, c = n - 1;
    const int pb = bi & 1, vb = bi >> 1;
    float* Ab = pb ? V.A1 : V.A0;
    const float as = Ab[vb];
    const bool centre = bi == c;
    const int vq = n - 1 - vb - pb;
    float dd[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {  // lags 2m, m = lane+1+TILE k < n (n <= TILE R)
        const int m = lane + 1 + TL::kSize * k;
        dd[k] = 0.f;
        if (m < n) {
            float up = Ab[vb + m];
            if (!centre && vb + m == vq) up = 0.f;
            const float dn = Ab[vb - m];
            dd[k] = ((centre ? -2.f : -4.f) * as) * (up + dn);
        }
    }
    p_update(V, n, o, P, pb, vb, centre ? -1 : vq);
    t.sync();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int m = lane + 1 + TL::kSize * k;
        if (m < n) set_E(V, m, V.G[m].x + dd[k]);
    }
    if (lane == 0) {
        set_row(V, pb, vb, -as);
        if (!centre) set_row(V, pb, vq, -Ab[vq]);
    }
}

// What a walk call records besides the trajectory.
struct StepExtras {
    const float* scores;  // learned flip scores for the first step of this call, or null
    int tau;              // learned candidates: dISL <= min dISL + tau
    float* sdump;         // replay dump of the scores used (traced walker), or null
    int64_t* sdump_step;
    int32_t* sdump_count;
    int dump_cap, n_max;
    labs_log_record* rec; // log record of this chunk, or null
};

template <class TL, int R>
__device__ void walk_steps(const WalkEnv& env, Walker& w, int64_t until, int* base, const WarpSmem& SL,
                           const View& V, int trace_slot, int64_t trace_start, const StepExtras& ex,
                           const TL& t)
{
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<TL, R> o(t);
    const int cap = p.probe_cap;
    constexpr int S = TL::kSize / 2;  // probe slots per candidate in the two-candidate round
    float P[R];
    p_direct(V, n, o, P);
    const int64_t first_step = w.steps;
    int log_first = 0, log_min = w.isl;
    bool log_live = true;
    StopCheck stop;
    stop.start(p, lane == 0);
    if (ex.rec != nullptr) {
        if (lane < kBitWords) ex.rec->bits[lane] = w.word;
        if (lane == 0) {
            ex.rec->isl = w.isl;
            ex.rec->L = env.L;
            ex.rec->walker = env.g;
            ex.rec->step = w.steps;
        }
    }
    while (w.steps < until) {
        if ((w.steps & (kCheckEvery - 1)) == 0) {
            const int why = t.shfl(stop.poll(p, lane == 0), 0);
            if (why) {
                if (lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        int dl[R];
        {
            float X[R];
            toeplitz_one(V, SL, n, o, t, X);
            assemble(V, n, o, X, P, dl);
        }

        // Best admissible flip: lowest (dISL, i) whose result is not in HT.  Two
        // candidates are probed per round, TILE/2 slots each (half the tile per
        // candidate); a longer chain falls back to a full probe.  The chosen flip is
        // the best one in about 40% of the steps and one of the best two in about 86%
        // (L = 201).
        uint32_t excl = 0;
        int best_i = -1, best_d = 0;
        int64_t slot = -1;
        uint64_t fnew = 0;
        if (ex.scores != nullptr && w.steps == first_step) {
            // Learned step: among the flips with dISL <= min dISL + tau, try them by
            // (score descending, i ascending) first; the plain order follows.
            int lm = INT_MAX;
#pragma unroll
            for (int r = 0; r < R; ++r) lm = min(lm, dl[r]);
            const int dmin = t.rmin(lm);
            const int thr = dmin > INT_MAX - ex.tau ? INT_MAX - 1 : dmin + ex.tau;
            int keys[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = 2 * (o.v0 + r) + o.p;
                keys[r] = dl[r] <= thr ? score_key(ex.scores[i]) : INT_MIN;
            }
            if (ex.sdump != nullptr) {
                const int k = *ex.sdump_count;
                if (k < ex.dump_cap) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int i = 2 * (o.v0 + r) + o.p;
                        if (dl[r] != INT_MAX) ex.sdump[(int64_t)k * ex.n_max + i] = ex.scores[i];
                    }
                    if (lane == 0) ex.sdump_step[k] = w.steps;
                }
                t.sync();
                if (lane == 0) *ex.sdump_count = k + 1;
                t.sync();
            }
            for (;;) {
                int lk = INT_MIN, li = INT_MAX, ld = INT_MAX;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (!((excl >> r) & 1u) && keys[r] > lk && dl[r] != INT_MAX) {
                        lk = keys[r];
                        li = 2 * (o.v0 + r) + o.p;
                        ld = dl[r];
                    }
                const int km = t.rmax(lk);
                if (km == INT_MIN) break;
                const int bi = t.rmin(lk == km ? li : INT_MAX);
                const int bd = t.rmin(li == bi ? ld : INT_MAX);
                const uint64_t f = w.fp ^ __ldg(env.zk + bi);
                const Probe pr = probe_full(env, f, w.gen, cap, t);
                if (!pr.visited) {
                    best_i = bi;
                    best_d = bd;
                    slot = pr.slot;
                    fnew = f;
                    break;
                }
                exclude<TL, R>(excl, bi, t);
            }
        }
        for (; best_i < 0;) {
            int d0, i0, d1, i1;
            tile_argmin(dl, excl, o, t, d0, i0);
            if (i0 < 0) break;
            uint32_t ex1 = excl;
            exclude<TL, R>(ex1, i0, t);
            tile_argmin(dl, ex1, o, t, d1, i1);
            const int hs = lane % S;
            const int mine = lane < S ? i0 : i1;
            bool hit = false, match = false;
            if (mine >= 0 && hs < cap) {
                const uint64_t f = w.fp ^ __ldg(env.zk + mine);
                const uint64_t e = env.T[(f + (uint64_t)hs) & env.tmask];
                match = e == ((f & ~kGenMask) | w.gen);
                hit = ((e & kGenMask) != w.gen) || match;
            }
            const unsigned bal = t.ballot(hit);
            const int cand[2] = {i0, i1};
            const int cdl[2] = {d0, d1};
            bool chosen = false;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (cand[g] < 0) break;
                const uint64_t fg = w.fp ^ __ldg(env.zk + cand[g]);
                const unsigned b = (bal >> (S * g)) & ((1u << S) - 1u);
                Probe pr;
                if (b) {
                    const int fl = __ffs(b) - 1;
                    pr.visited = t.shfl(match ? 1 : 0, S * g + fl) != 0;
                    pr.slot = (int64_t)((fg + (uint64_t)fl) & env.tmask);
                } else if (cap > S) {
                    pr = probe_full(env, fg, w.gen, cap, t);
                } else {
                    pr.visited = false;
                    pr.slot = -1;
                }
                if (!pr.visited) {
                    best_i = cand[g];
                    best_d = cdl[g];
                    slot = pr.slot;
                    fnew = fg;
                    chosen = true;
                    break;
                }
                exclude<TL, R>(excl, cand[g], t);
            }
            if (chosen) break;
        }

        w.steps += 1;
        int code;
        if (best_i < 0) {
            // Every neighbour is in HT: restart without a move.
            w.blocked += 1;
            restart_walker(env, w, base, SL, V, t);
            p_direct(V, n, o, P);
            code = LABS_TRACE_BLOCKED;
        } else {
            flip_rows_table(V, n, o, P, best_i, t);
            const bool stored = slot >= 0;
            if (lane == 0 && stored) env.T[slot] = (fnew & ~kGenMask) | w.gen;
            if (lane == (best_i >> 5)) w.word ^= 1u << (best_i & 31);
            t.sync();
            w.fp = fnew;
            w.isl += best_d;
            if (!stored) w.overflows += 1;
            note_best(env, w, t);
            if (w.isl < w.since) {
                w.since = w.isl;
                w.stag = 0;
            } else {
                w.stag += 1;
            }
            code = best_i;
            if (w.stag >= env.patience || !stored) {
                restart_walker(env, w, base, SL, V, t);
                p_direct(V, n, o, P);
                code |= LABS_TRACE_RESTART;
            }
        }
        if (trace_slot >= 0 && lane == 0) {
            const int64_t s = w.steps - 1 - trace_start;
            if (s >= 0 && s < p.status->trace_capacity) {
                p.status->trace_code[trace_slot * p.status->trace_capacity + s] = code;
                p.status->trace_isl[trace_slot * p.status->trace_capacity + s] = w.isl;
            }
        }
        if (ex.rec != nullptr && log_live) {
            // lowest ISL at the end of the chunk's steps before its first restart step
            if (w.steps == first_step + 1) log_first = code;
            if (code == LABS_TRACE_BLOCKED || (code & LABS_TRACE_RESTART)) log_live = false;
            else log_min = min(log_min, w.isl);
        }
    }
    if (ex.rec != nullptr && lane == 0) {
        ex.rec->first = log_first;
        ex.rec->min_isl = log_min;
    }
}

__device__ void load_walker(const WalkerState* st, Walker& w, int lane)
{
    w.word = lane < kBitWords ? st->cur[lane] : 0u;
    w.fp = st->fp;
    w.isl = st->isl;
    w.best_isl = st->best_isl;
    w.since = st->since_best;
    w.stag = st->stagnation;
    w.restart_idx = st->restart_idx;
    w.gen = st->gen;
    w.restarts = st->restarts;
    w.overflows = st->overflows;
    w.blocked = st->blocked;
    w.steps = st->steps_done;
    w.best_step = st->best_step;
    w.target_step = st->target_step;
}

__device__ void save_scalars(WalkerState* st, const Walker& w);

__device__ void save_walker(WalkerState* st, const Walker& w, int lane)
{
    if (lane < kBitWords) st->cur[lane] = w.word;
    if (lane == 0) save_scalars(st, w);
}

// Everything of the walker state but the bits (one thread).
__device__ void save_scalars(WalkerState* st, const Walker& w)
{
    {
        st->fp = w.fp;
        st->isl = w.isl;
        st->best_isl = w.best_isl;
        st->since_best = w.since;
        st->stagnation = w.stag;
        st->restart_idx = w.restart_idx;
        st->gen = w.gen;
        st->restarts = w.restarts;
        st->overflows = w.overflows;
        st->blocked = w.blocked;
        st->steps_done = w.steps;
        st->best_step = w.best_step;
        st->target_step = w.target_step;
    }
}

// ------------------------------------------------------------------ lockstep step
//
// The step of walk_steps without the learned extras, written for a warp that runs
// either one walker (lane group Tile<32>) or two walkers of the same length in
// lockstep (Pair: lanes 16h..16h+15 run walker h).  With two walkers both halves stay
// converged through the hot part of every step, so each full-warp collective serves
// both walkers and what differs between them is carried by predicates; restarts,
// which are rare, run divergently per half with tile-masked primitives (Tile<16>).
// The trajectory of each walker is exactly that of walk_steps.

// dISL of the lane's R outputs (returns how many exist): the assembly of `assemble`
// without bounds tests or branches, for the lockstep layouts (warp_smem pads the rows
// and the table for every lane output, existing or not), s_{3i-L+1} reading as 0 below
// index 0, and the centre's formula selected per output.  The results are exact
// integers below 2^22 in magnitude (|dISL| < 8 L^2 + 48 n for L <= 511), returned as
// dISL + 1.5 * 2^23 in fp32, whose bit pattern is 0x4B400000 + dISL: the integer sits in
// the low bits without a float-to-int conversion.  lane_keys packs them as
// (dISL + 2^22) << 8 | i, ascending in (dISL, i), or 0xFFFFFFFF where the output does
// not exist (keys are unique, below 2^31 and above 0).
constexpr float kIntBias = 12582912.f;  // 1.5 * 2^23
constexpr int kIntBiasBits = 0x4B400000;
constexpr int kKeyBias = 1 << 22;       // dISL = (key >> 8) - kKeyBias

__device__ __forceinline__ float row_value(float a)
{
    return a;
}
__device__ __forceinline__ float row_value(__half a)
{
    return __half2float(a);
}

// A: the lane's class row (FP32, or FP16 in the row kernels' tensor-core layout).
template <class LG, int R, class E>
__device__ __forceinline__ int lane_dlb_rows(const E* A, const View& V, int n, const Outs<LG, R>& o,
                                             const float (&X)[R], const float (&P)[R], uint32_t (&db)[R])
{
    // four walkers per warp: the rows are not padded for the missing outputs' reads
    constexpr bool kGuard = LG::kSize == 8;
    const int p = o.p, c = n - 1;
    const int rv = (p ? (n >> 1) : ((n + 1) >> 1)) - o.v0;
    const int rc = (c & 1) == p ? ((c - p) >> 1) - o.v0 : -1;  // the centre's r, if this lane has it
    const float base = (float)(16 * ((p ? n - 2 : n - 1) - 1)) + kIntBias, cbase = (float)(16 * (c >> 1)) + kIntBias;
    const E* Av = A + o.v0;                        // s_i          = Av[r]
    const E* Aq = A + (n - 1 - p - o.v0);          // s_q          = Aq[-r]
    const E* At = A + (3 * o.v0 + p - n + 1);      // s_{3i-L+1}   = At[3r]
    const float2* Gc = V.G + (c - p - 2 * o.v0);   // C_{q-i}      = Gc[-2r].x
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool ok = !kGuard || r < rv;
        const float av = row_value(Av[r]), sq = row_value(Aq[-r]);
        const float ck0 = ok ? Gc[-2 * r].x : 0.f, st = ok ? row_value(At[3 * r]) : 0.f;
        const bool ctr = r == rc;
        // every partial sum is an integer of magnitude below 2^24: exact
        const float add = ctr ? cbase : fmaf(32.f, fmaf(-sq, st, P[r]), base);
        const float mul = (ctr ? -4.f : -8.f) * av;
        db[r] = __float_as_uint(fmaf(mul, fmaf(-sq, ck0, X[r]), add));
    }
    return rv;  // outputs r below this exist
}

template <class LG, int R>
__device__ __forceinline__ int lane_dlb(const View& V, int n, const Outs<LG, R>& o, const float (&X)[R],
                                        const float (&P)[R], uint32_t (&db)[R])
{
    return lane_dlb_rows(o.p ? V.A1 : V.A0, V, n, o, X, P, db);
}

template <class LG, int R, class E>
__device__ __forceinline__ int lane_dl_rows(const E* A, const View& V, int n, const Outs<LG, R>& o,
                                            const float (&X)[R], const float (&P)[R], int (&dl)[R])
{
    uint32_t db[R];
    const int rv = lane_dlb_rows(A, V, n, o, X, P, db);
#pragma unroll
    for (int r = 0; r < R; ++r) dl[r] = (int)db[r] - kIntBiasBits;
    return rv;
}

template <class LG, int R>
__device__ __forceinline__ int lane_dl(const View& V, int n, const Outs<LG, R>& o, const float (&X)[R],
                                       const float (&P)[R], int (&dl)[R])
{
    return lane_dl_rows(o.p ? V.A1 : V.A0, V, n, o, X, P, dl);
}

template <class LG, int R>
__device__ __forceinline__ void lane_keys(const View& V, int n, const Outs<LG, R>& o, const float (&X)[R],
                                          const float (&P)[R], unsigned (&key)[R])
{
    uint32_t db[R];
    const int rv = lane_dlb(V, n, o, X, P, db);
    const unsigned i0 = (unsigned)(2 * o.v0 + o.p);
    // (0x4B400000 + dISL) << 8 drops the exponent: (2^22 + dISL) << 8
#pragma unroll
    for (int r = 0; r < R; ++r) key[r] = r < rv ? (db[r] << 8) + i0 + 2u * r : 0xFFFFFFFFu;
}

// The lane's two lowest keys above `floor` (0xFFFFFFFF where there are fewer).
template <int R>
__device__ __forceinline__ void top2_above(const unsigned (&key)[R], unsigned floor, unsigned& b1, unsigned& b2)
{
    b1 = 0xFFFFFFFFu;
    b2 = 0xFFFFFFFFu;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const unsigned k = key[r] > floor ? key[r] : 0xFFFFFFFFu;
        b2 = min(b2, max(b1, k));
        b1 = min(b1, k);
    }
}

// Removes free variable j from the lane's candidates (key `none`) when it is one of the
// lane's outputs; j < 0: none.  The lockstep steps drop the move back to the previous
// state this way: that state is in HT (every state of the walk since the last start
// was inserted, and a failed insertion restarts the walker), so the probe would find
// it visited, and leaving it out changes no choice while it saves most second rounds.
template <class LG, int R, class K>
__device__ __forceinline__ void drop_candidate(K (&key)[R], int j, const Outs<LG, R>& o, K none)
{
    const int d = (j >> 1) - o.v0;
    const bool mine = j >= 0 && (j & 1) == o.p;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (mine && d == r) key[r] = none;
}

// Full probe of f for the walkers (halves) with need set: every lane runs the same rounds.
template <class LG>
__device__ __forceinline__ Probe lockstep_probe_full(const WalkEnv& env, uint64_t f, uint32_t gen, int cap, bool need,
                                                     const LG& t)
{
    const uint64_t tag = (f & ~kGenMask) | gen;
    Probe pr{false, -1};
    bool found = false;
    for (int s0 = 0; s0 < cap; s0 += LG::kSize) {
        const int s = s0 + t.lane;
        uint64_t e = 0;
        const bool live = need && !found && s < cap;
        if (live) e = env.T[(f + (uint64_t)s) & env.tmask];
        const bool match = e == tag;
        const unsigned bal = t.ballot(live && (((e & kGenMask) != gen) || match));
        const int fl = bal ? __ffs(bal) - 1 : 0;
        const bool vis = t.shfl(match ? 1 : 0, fl) != 0;
        if (bal && !found) {
            found = true;
            pr.visited = vis;
            pr.slot = (int64_t)((f + (uint64_t)(s0 + fl)) & env.tmask);
        }
    }
    return pr;
}

// Flips free variable best_i (and its mirror) in the walker's rows, even-lag table and
// P, all from the values before the flip, when `moves` (the lanes of a walker without a
// move rewrite unchanged values).  The rows are padded so that no read or write needs a
// bounds test (four walkers per warp: reads of s_{i+2m} stay inside the class and the
// mirror half of the table is kept only as deep as the Toeplitz window reads).
template <class LG, int R>
__device__ __forceinline__ void apply_flip(const View& V, int n, const Outs<LG, R>& o, int lane, bool moves,
                                           int best_i, float (&P)[R])
{
    constexpr bool kQuad = LG::kSize == 8;
    const int c = n - 1;
    const int m0 = 1 + lane * R;  // this lane's lags 2m of the update, m = m0 .. m0+R-1
    const int pb = best_i & 1, vb = best_i >> 1;
    float* Ab = pb ? V.A1 : V.A0;
    const bool centre = best_i == c;
    const int vq = centre ? vb : n - 1 - vb - pb;
    const float as = Ab[vb], aq = centre ? 0.f : Ab[vq];
    __syncwarp();
    // The flipped entries read as 0 while the changes are taken: that drops the pairs
    // whose two ends both flip (unchanged) and the lag-0 terms from every sum below.
    if (moves && lane == 0) {
        Ab[vb] = 0.f;
        Ab[vq] = 0.f;
    }
    __syncwarp();
    // dC_{2m} = -4 s_i (s_{i+2m} + s_{i-2m}) (centre: -2 s_c (..)) for this lane's m
    const float coef = moves ? (centre ? -2.f : -4.f) * as : 0.f;
    float dd[R];
    {
        const float* up = Ab + vb + m0;
        const float* dn = Ab + vb - m0;
        const int ku = kQuad ? (pb ? n - 1 : n) - vb - m0 : R;  // s_{i+2m} inside the class for k < ku
#pragma unroll
        for (int k = 0; k < R; ++k) dd[k] = coef * ((k < ku ? up[k] : 0.f) + dn[-k]);
    }
    // P_v of the moved class: each pair (v+m, v-m) with exactly one flipped end
    // changes by -2 x its old product; the partner of w is 2v - w
    {
        const float g = (moves && o.p == pb) ? -2.f : 0.f;
        const float* B1 = Ab + 2 * o.v0 - vb;
        const float* B2 = Ab + 2 * o.v0 - vq;
#pragma unroll
        for (int r = 0; r < R; ++r) P[r] = fmaf(g, fmaf(aq, B2[2 * r], as * B1[2 * r]), P[r]);
    }
    {
        // E[m] += dd for this lane's m, in the pairs G[y] = (E[y], E[y+1]) and their
        // mirrors at -y (pairs shared with a neighbour lane are written field by field)
        float e[R + 1];
        e[R] = 0.f;
#pragma unroll
        for (int k = 0; k < R; k += 2) {
            const float2 g = V.G[m0 + k];
            e[k] = g.x + dd[k];
            if (k + 1 < R) e[k + 1] = g.y + dd[k + 1];
        }
        V.G[m0 - 1].y = e[0];
#pragma unroll
        for (int k = 0; k + 1 < R; ++k) V.G[m0 + k] = make_float2(e[k], e[k + 1]);
        V.G[m0 + R - 1].x = e[R - 1];
        if (!kQuad || m0 + R <= V.gpad) {
            V.G[-m0].x = e[0];
#pragma unroll
            for (int k = 0; k + 1 < R; ++k) V.G[-m0 - k - 1] = make_float2(e[k + 1], e[k]);
            V.G[-m0 - R].y = e[R - 1];
        }
    }
    __syncwarp();
    if (moves && lane == 0) {
        set_row(V, pb, vb, -as);
        if (!centre) set_row(V, pb, vq, -aq);
    }
}

// ISL at or below which the target merit factor is met (-1: no target).
__device__ __forceinline__ int target_isl(const KParams& p, int L)
{
    if (p.target_num <= 0 || p.target_den <= 0) return -1;
    return (int)min((int64_t)INT_MAX, (int64_t)p.target_den * L * L / (2 * (int64_t)p.target_num));
}

// Outcome of probing HT for a candidate.
enum : int { kProbeFree = 0, kProbeVisited = 1, kProbeUnknown = 2, kProbeNone = 3 };

// TC: the Toeplitz product on the tensor cores (two walkers per warp): 0 never, 1 always,
// 2 when the layout holds the FP16 rows (n_max <= 128).
template <class LG, class RT, int R, int TC = 0>
__device__ void walk_lockstep(const WalkEnv& env, Walker& w, int64_t until, bool real, int* base, const WarpSmem& SL,
                              const View& V, int trace_slot, int64_t trace_start, labs_log_record* rec, const LG& t,
                              const RT& tt)
{
    constexpr int S = LG::kSize / 2;            // HT slots probed per candidate in a round
    constexpr unsigned SM = (1u << S) - 1u;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<LG, R> o(t);
    const int cap = p.probe_cap;
    const uint32_t tmask = (uint32_t)env.tmask;  // HT slots <= 2^20
    // ISL at or below which the target merit factor is met (-1: no target)
    const int tisl = target_isl(p, env.L);
    float P[R];
    p_direct(V, n, o, P);
    const int64_t first_step = w.steps;
    int log_first = 0, log_min = w.isl;
    bool log_live = true;
    int prev = -1;  // the last flip since the walker's (re)start in this call, or -1
    StopCheck stop;
    stop.start(p, (threadIdx.x & 31) == 0);
    if (real && rec != nullptr) {
        if (lane < kBitWords) rec->bits[lane] = w.word;
        if (lane == 0) {
            rec->isl = w.isl;
            rec->L = env.L;
            rec->walker = env.g;
            rec->step = w.steps;
        }
    }
    for (;;) {
        const bool act = real && w.steps < until;
        if (!__any_sync(kFull, act)) break;
        if (__any_sync(kFull, act && (w.steps & (kCheckEvery - 1)) == 0)) {
            const int why = __shfl_sync(kFull, stop.poll(p, (threadIdx.x & 31) == 0), 0);
            if (why) {
                if (act && lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        unsigned key[R];
        {
            float X[R];
            if constexpr (TC == 1) {
                toeplitz_tc(V, SL, n, o, t.h, X);
            } else if constexpr (TC == 2) {
                if (SL.xp)
                    toeplitz_tc(V, SL, n, o, t.h, X);
                else
                    toeplitz_one(V, SL, n, o, t, X);
            } else {
                toeplitz_one(V, SL, n, o, t, X);
            }
            lane_keys(V, n, o, X, P, key);
            drop_candidate(key, prev, o, 0xFFFFFFFFu);
        }

        // Best admissible flip, as in walk_steps: candidates in ascending key order, two
        // per round, the first S HT slots of each probed by one half of the walker's
        // lanes; keys <= floor are known to lead to visited states.
        unsigned floor = 0u, kc = 0xFFFFFFFFu;
        int slot = -1;
        uint64_t fnew = 0;
        bool done = !act;
        do {
            unsigned b1, b2;
            top2_above(key, floor, b1, b2);
            const unsigned k0 = t.rminu(done ? 0xFFFFFFFFu : b1);
            const unsigned k1 = t.rminu(done ? 0xFFFFFFFFu : (b1 == k0 ? b2 : b1));
            const bool has0 = k0 != 0xFFFFFFFFu, has1 = k1 != 0xFFFFFFFFu;
            const uint64_t f0 = w.fp ^ (has0 ? __ldg(env.zk + (k0 & 0xFFu)) : 0ull);
            const uint64_t f1 = w.fp ^ (has1 ? __ldg(env.zk + (k1 & 0xFFu)) : 0ull);
            const int hs = lane & (S - 1);
            const bool second = lane >= S;
            const uint64_t f = second ? f1 : f0;
            const bool live = !done && (second ? has1 : has0) && hs < cap;
            uint64_t e = 0;
            if (live) e = env.T[((uint32_t)f + (uint32_t)hs) & tmask];
            const bool match = live && e == ((f & ~kGenMask) | w.gen);
            const bool hit = live && ((((uint32_t)e & (uint32_t)kGenMask) != w.gen) || match);
            const unsigned hb = t.ballot(hit), mb = t.ballot(match);
            const unsigned h0 = hb & SM, h1 = (hb >> S) & SM;
            int st0 = !has0 ? kProbeNone
                            : h0 ? ((mb & h0 & (0u - h0)) ? kProbeVisited : kProbeFree)
                                 : (cap > S ? kProbeUnknown : kProbeFree);
            int st1 = !has1 ? kProbeNone
                            : h1 ? (((mb >> S) & h1 & (0u - h1)) ? kProbeVisited : kProbeFree)
                                 : (cap > S ? kProbeUnknown : kProbeFree);
            // the slot of a candidate's first hit (its insertion slot when it is free) is
            // taken below for the candidate chosen; a full probe supplies its own
            int s0 = -2, s1 = -2;
            // chains longer than S slots (rare): full probes, of the second candidate only
            // when the first leads to a visited state
            const bool need0 = !done && st0 == kProbeUnknown;
            if (__any_sync(kFull, need0)) {
                const Probe pf = lockstep_probe_full(env, f0, w.gen, cap, need0, t);
                if (need0) {
                    st0 = pf.visited ? kProbeVisited : kProbeFree;
                    s0 = (int)pf.slot;
                }
            }
            const bool need1 = !done && st0 == kProbeVisited && st1 == kProbeUnknown;
            if (__any_sync(kFull, need1)) {
                const Probe pf = lockstep_probe_full(env, f1, w.gen, cap, need1, t);
                if (need1) {
                    st1 = pf.visited ? kProbeVisited : kProbeFree;
                    s1 = (int)pf.slot;
                }
            }
            if (!done) {
                if (st0 == kProbeFree) {
                    kc = k0, fnew = f0, done = true;
                    slot = s0 != -2 ? s0 : (h0 ? (int)(((uint32_t)f0 + (uint32_t)(__ffs(h0) - 1)) & tmask) : -1);
                } else if (st0 == kProbeNone || st1 == kProbeNone) {
                    done = true;  // every neighbour is in HT
                } else if (st1 == kProbeFree) {
                    kc = k1, fnew = f1, done = true;
                    slot = s1 != -2 ? s1 : (h1 ? (int)(((uint32_t)f1 + (uint32_t)(__ffs(h1) - 1)) & tmask) : -1);
                } else {
                    floor = k1;
                }
            }
        } while (__any_sync(kFull, !done));

        // Apply the move (walkers that have one), from the values before the flip.
        const bool moves = act && kc != 0xFFFFFFFFu;
        const int best_i = moves ? (int)(kc & 0xFFu) : 0, best_d = (int)(kc >> 8) - kKeyBias;
        apply_flip<LG, R>(V, n, o, lane, moves, best_i, P);
        const bool stored = slot >= 0;
        if (moves && lane == 0 && stored) env.T[slot] = (fnew & ~kGenMask) | w.gen;
        if (moves && lane == (best_i >> 5)) w.word ^= 1u << (best_i & 31);
        __syncwarp();
        int code = 0;
        bool again = false;
        if (act) {
            w.steps += 1;
            if (!moves) {
                w.blocked += 1;
                again = true;
                code = LABS_TRACE_BLOCKED;
            } else {
                w.fp = fnew;
                w.isl += best_d;
                if (!stored) w.overflows += 1;
                if (w.isl < w.best_isl) {
                    w.best_isl = w.isl;
                    w.best_step = w.steps;
                    if (lane < kBitWords) env.st->best[lane] = w.word;
                }
                if (w.target_step < 0 && w.isl <= tisl) w.target_step = w.steps;
                if (w.isl < w.since) {
                    w.since = w.isl;
                    w.stag = 0;
                } else {
                    w.stag += 1;
                }
                code = best_i;
                if (w.stag >= env.patience || !stored) {
                    again = true;
                    code |= LABS_TRACE_RESTART;
                }
            }
        }
        if (moves) prev = best_i;
        if (again) {  // two walkers per warp: divergent, only this half restarts
            restart_walker(env, w, base, SL, V, tt);
            p_direct(V, n, o, P);
            prev = -1;
        }
        __syncwarp();
        if (act) {
            if (trace_slot >= 0 && lane == 0) {
                const int64_t s = w.steps - 1 - trace_start;
                if (s >= 0 && s < p.status->trace_capacity) {
                    p.status->trace_code[trace_slot * p.status->trace_capacity + s] = code;
                    p.status->trace_isl[trace_slot * p.status->trace_capacity + s] = w.isl;
                }
            }
            if (rec != nullptr && log_live) {
                if (w.steps == first_step + 1) log_first = code;
                if (code == LABS_TRACE_BLOCKED || (code & LABS_TRACE_RESTART)) log_live = false;
                else log_min = min(log_min, w.isl);
            }
        }
    }
    if (real && rec != nullptr && lane == 0) {
        rec->first = log_first;
        rec->min_isl = log_min;
    }
}

// ------------------------------------------------------------- best-first search
//
// Algorithm 1 as printed (impxLast, Section 3): the neighbourhood of S fills a queue
// of LABS_QUEUE_SIZE evaluated neighbours ordered by merit factor and the next S is the
// queue's first entry (the readings are stated with labs_walk in labs.h).  One walker
// per warp; lane l holds queue entry l as a 64-bit key
//   ISL << 36 | (steps done before the step that produced it) << 8 | i
// (ascending = the queue order; ~0 = empty) and the entry's free variables live in
// global memory.  An entry produced by the current step is a neighbour of S and is
// applied incrementally; an older one rebuilds the rows and the table from its bits.

__device__ __forceinline__ uint64_t warp_min64(uint64_t v)
{
    const unsigned hi = __reduce_min_sync(kFull, (unsigned)(v >> 32));
    const unsigned lo = __reduce_min_sync(kFull, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xFFFFFFFFu);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_max64(uint64_t v)
{
    const unsigned hi = __reduce_max_sync(kFull, (unsigned)(v >> 32));
    const unsigned lo = __reduce_max_sync(kFull, (unsigned)(v >> 32) == hi ? (unsigned)v : 0u);
    return ((uint64_t)hi << 32) | lo;
}

// A new S that differs from S in at most this many free variables is reached by that
// many incremental flips (a neighbour of S, about half the steps, by one) rather than
// a rebuild from its bits; about four of five steps at L = 101..151 (measured with the
// Python statement), each flip costing about a sixth of a rebuild.
constexpr int kBestFirstMaxFlips = 5;

template <int R>
__device__ void walk_bestfirst(const WalkEnv& env, Walker& w, int64_t until, int* base, const WarpSmem& SL,
                               const View& V, int trace_slot, int64_t trace_start, const Tile<32>& t, uint64_t* qkey,
                               uint32_t* qbits)
{
    static_assert(LABS_QUEUE_SIZE == 32, "one queue entry per lane");
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<Tile<32>, R> o(t);
    const int cap = p.probe_cap;
    const int tisl = target_isl(p, env.L);
    uint64_t qk = qkey[lane];
    // xLastovka's second table (null when off): slot f mod size holds
    // (generation << 40) | (~f mod 2^40) of an evaluated neighbour f
    uint64_t* T2 = p.tabu2 != nullptr ? p.tabu2 + (env.T - p.tabu) : nullptr;
    constexpr uint64_t kLow40 = 0xFFFFFFFFFFull;
    int64_t hits = 0;
    float P[R];
    p_direct(V, n, o, P);
    StopCheck stop;
    stop.start(p, lane == 0);
    while (w.steps < until) {
        if ((w.steps & (kCheckEvery - 1)) == 0) {
            const int why = t.shfl(stop.poll(p, lane == 0), 0);
            if (why) {
                if (lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        const int64_t e = w.steps;
        unsigned key[R];
        {
            float X[R];
            toeplitz_one(V, SL, n, o, t, X);
            lane_keys(V, n, o, X, P, key);
        }
        if (T2 != nullptr) {
            // neighbours the table holds are skipped (their keys dropped); every other
            // one is inserted once all lanes have looked (larger word kept: the table
            // does not depend on the order of the insertions)
            uint64_t ins[R];
            int h = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ins[r] = 0ull;
                if (key[r] == 0xFFFFFFFFu) continue;
                const uint64_t f = w.fp ^ __ldg(env.zk + (key[r] & 0xFFu));
                const uint64_t tag = ((uint64_t)w.gen << 40) | (~f & kLow40);
                if (T2[f & env.tmask] == tag) {
                    key[r] = 0xFFFFFFFFu;
                    ++h;
                } else {
                    ins[r] = f;
                }
            }
            hits += t.radd(h);
            t.sync();
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (key[r] != 0xFFFFFFFFu)
                    atomicMax(reinterpret_cast<unsigned long long*>(T2 + (ins[r] & env.tmask)),
                              (unsigned long long)(((uint64_t)w.gen << 40) | (~ins[r] & kLow40)));
            t.sync();
        }
        // Neighbours in queue order (ISL, then i: the packed keys' order) while they
        // come before the queue's last entry or the queue has a free place.  The queue's
        // last entry only moves forward during the step, so the neighbours after its
        // value at the start cannot enter; the others are looked up in HT one by one as
        // the insertion reaches them (HT does not change during the insertion, so this
        // equals looking them all up first, at a few probes per step instead of one per
        // neighbour).
        const bool full0 = t.ballot(qk == ~0ull) == 0u;
        const uint64_t last0 = full0 ? warp_max64(qk) : ~0ull;
        bool fresh[R];  // candidate r: before last0
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const unsigned k = key[r];
            const uint64_t ck = ((uint64_t)(w.isl + (int)(k >> 8) - kKeyBias) << 36) | ((uint64_t)e << 8) |
                                (uint64_t)(k & 0xFFu);
            fresh[r] = k != 0xFFFFFFFFu && ck < last0;
        }
        unsigned floor = 0u;
        for (;;) {
            unsigned b = 0xFFFFFFFFu;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (fresh[r] && key[r] > floor) b = min(b, key[r]);
            const unsigned k = t.rminu(b);
            if (k == 0xFFFFFFFFu) break;
            floor = k;
            const int i = (int)(k & 0xFFu);
            const int isl_f = w.isl + (int)(k >> 8) - kKeyBias;
            const uint64_t ck = ((uint64_t)isl_f << 36) | ((uint64_t)e << 8) | (uint64_t)i;
            const unsigned empty = t.ballot(qk == ~0ull);
            int dst;
            if (empty) {
                dst = __ffs(empty) - 1;
            } else {
                const uint64_t last = warp_max64(qk);
                if (ck > last) break;  // every later neighbour comes after it too
                dst = __ffs(t.ballot(qk == last)) - 1;
            }
            {
                // HT lookup of this neighbour: up to probe_cap slots, four per round
                const uint64_t f = w.fp ^ __ldg(env.zk + i);
                const uint64_t tag = (f & ~kGenMask) | w.gen;
                bool visited = false;
                for (int s0 = 0; s0 < cap; s0 += 4) {
                    const bool mine = lane < 4 && s0 + lane < cap;
                    const uint64_t x = mine ? env.T[(f + (uint64_t)(s0 + lane)) & env.tmask] : 0ull;
                    const unsigned bal = t.ballot(mine && (((x & kGenMask) != w.gen) || x == tag));
                    if (bal) {
                        visited = t.shfl(x == tag ? 1 : 0, __ffs(bal) - 1) != 0;
                        break;
                    }
                }
                if (visited) continue;
            }
            if (lane == dst) qk = ck;
            const uint32_t word = w.word ^ (lane == (i >> 5) ? 1u << (i & 31) : 0u);
            if (lane < kBitWords) qbits[dst * kBitWords + lane] = word;
            if (isl_f < w.best_isl) {
                w.best_isl = isl_f;
                w.best_step = e + 1;
                if (lane < kBitWords) env.st->best[lane] = word;
            }
            if (w.target_step < 0 && isl_f <= tisl) w.target_step = e + 1;
        }
        t.sync();
        // S <- the queue's first entry not in HT (entries that are get dropped)
        int code = LABS_TRACE_BLOCKED;
        bool again = true;
        for (;;) {
            if (!t.ballot(qk != ~0ull)) {
                w.blocked += 1;  // empty queue: restart
                break;
            }
            const uint64_t first = warp_min64(qk);
            const int src = __ffs(t.ballot(qk == first)) - 1;
            const uint32_t word = lane < kBitWords ? qbits[src * kBitWords + lane] : 0u;
            if (lane == src) qk = ~0ull;
            const int i = (int)(first & 0xFFu);
            const bool nb = ((first >> 8) & 0xFFFFFFFull) == (uint64_t)e;  // a neighbour of S
            const uint64_t f = nb ? (w.fp ^ __ldg(env.zk + i)) : fingerprint_all(word, env.zk, n, t);
            const Probe pr = probe_full(env, f, w.gen, cap, t);
            if (pr.visited) continue;
            // free variables in which the new S differs from S (1 for a neighbour)
            uint32_t diff = lane < kBitWords ? (word ^ w.word) : 0u;
            const int k = nb ? 1 : t.radd(__popc(diff));
            if (k <= kBestFirstMaxFlips) {
                // flip them one by one (lowest first) with the walk's incremental update
                for (int j = 0; j < k; ++j) {
                    const unsigned bl = t.ballot(diff != 0u);
                    const int src_lane = __ffs(bl) - 1;
                    const int fi = nb ? i : 32 * src_lane + t.shfl(__ffs(diff) - 1, src_lane);
                    apply_flip<Tile<32>, R>(V, n, o, lane, true, fi, P);
                    t.sync();
                    if (lane == src_lane) diff &= diff - 1u;
                }
            } else {
                // rebuild from the bits; the walker's padding is still zero, so no clear
                rows_from_bits(V, word, env.L, n, t);
                build_table(V, n, t);
                p_direct(V, n, o, P);
            }
            w.word = word;
            w.isl = (int)(first >> 36);
            w.fp = f;
            code = (int)(f & 0xFFFFu);
            if (pr.slot >= 0) {
                if (lane == 0) env.T[pr.slot] = (f & ~kGenMask) | w.gen;
                again = false;
            } else {
                w.overflows += 1;  // no free HT slot for the new S: restart
                code |= LABS_TRACE_RESTART;
            }
            break;
        }
        w.steps += 1;
        if (again) {
            qk = ~0ull;
            const uint32_t gen0 = w.gen;
            restart_walker(env, w, base, SL, V, t);
            if (T2 != nullptr && w.gen < gen0) {  // generations wrapped: HT was zeroed, so is T2
                for (int64_t i = lane; i <= (int64_t)env.tmask; i += 32) T2[i] = 0ull;
                t.sync();
            }
            p_direct(V, n, o, P);
        }
        t.sync();
        if (trace_slot >= 0 && lane == 0) {
            const int64_t s = w.steps - 1 - trace_start;
            if (s >= 0 && s < p.status->trace_capacity) {
                p.status->trace_code[trace_slot * p.status->trace_capacity + s] = code;
                p.status->trace_isl[trace_slot * p.status->trace_capacity + s] = w.isl;
            }
        }
    }
    qkey[lane] = qk;
    if (lane == 0) env.st->cache_hits += hits;
}

// One launch advances every walker by up to chunk_steps steps toward the target.  The
// kernel is compiled for a tile of TILE lanes per walker and a largest lane block RMAX
// = block_R(n_max, TILE) (register allocation follows it; odd for TILE = 32); walkers
// whose n needs a smaller block run with RMAX-2, which covers them (any R >=
// block_R(n) computes the same values).  MODE picks the step: 0 the plain walk, 1 the
// learned mode, 2 the best-first search (one variant per kernel keeps the code small).
// ------------------------------------------------------------ PSL objective walk

// Order key of a flip under the PSL objective: PSL' << 43 | ISL' << 13 | i (PSL' < 2^21,
// ISL' < 2^30, i < 2^13 for every length served).
__device__ __forceinline__ uint64_t psl_key(int psl, int isl, int i)
{
    return ((uint64_t)psl << 43) | ((uint64_t)(uint32_t)isl << 13) | (uint64_t)i;
}
__device__ __forceinline__ int psl_key_i(uint64_t k) { return (int)(k & 0x1FFFu); }
__device__ __forceinline__ int psl_key_isl(uint64_t k) { return (int)((k >> 13) & 0x3FFFFFFFull); }
__device__ __forceinline__ int psl_key_psl(uint64_t k) { return (int)(k >> 43); }

// The same PSL values for the lane block R = 7 in one pass: s_{i-2m} and s_{i+2m} of the
// R outputs in two windows of R values that slide one class entry per lag (three shared
// loads per lag), and the mirror's term dropped by a compare and select per lag term.
template <class TL, int R>
__device__ __forceinline__ void psl_eval_select(const View& V, int n, const Outs<TL, R>& o, int (&pl)[R])
{
    const float* A = (o.p ? V.A1 : V.A0) + o.v0;
    const int c = n - 1;
    float cs[R], mx[R], lo[R], hi[R];
    int q0[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = 2 * (o.v0 + r) + o.p;
        cs[r] = (i == c ? -2.f : -4.f) * A[r];
        q0[r] = c - i;
        mx[r] = 0.f;
    }
    // lo[e mod R] = A[-e] for e = m-R+1 .. m, hi[e mod R] = A[e] for e = m .. m+R-1
#pragma unroll
    for (int k = 1; k < R; ++k) lo[k] = A[R - k];
#pragma unroll
    for (int e = 0; e + 1 < R; ++e) hi[e] = A[e];
    for (int m0 = 0; m0 < n; m0 += R) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int m = m0 + j;
            if (m >= n) break;
            lo[j] = A[-m];
            hi[(j + R - 1) % R] = A[m + R - 1];
            if (m == 0) continue;
            const float C = V.G[m].x;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float a = lo[(j - r + R) % R];
                const float b = m == q0[r] ? 0.f : hi[(j + r) % R];
                mx[r] = fmaxf(mx[r], fabsf(fmaf(cs[r], a + b, C)));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) pl[r] = (int)mx[r];
}

// PSL of every neighbour S_i for the lane's outputs i = 2(v0+r)+p: flipping s_i and its
// mirror s_{L-1-i} changes C_{2m} by -4 s_i (s_{i-2m} + s_{i+2m}) with the mirror's own
// term (i+2m = L-1-i, i.e. m = c-i) left out, or by -2 s_c (s_{c-2m} + s_{c+2m}) at the
// centre; the odd-lag C_k stay zero.  pl[r] = max_m |C_{2m} + dC_{2m}(i)| over
// m = 1..n-1 (Section 1's PSL).
// psl_ring takes the outputs C0 .. C0+RC-1 of the lane (block start w0 = v0 + C0).
// Output r takes lag m = t - 2r at iteration t, so that every output of the pass meets
// its mirror at the same iteration t* = c - p - 2 w0 (where m = c - i): there one
// multiplier z = 0 drops the mirror term of all of them, and a lag term costs three
// instructions (FMA, FMA, max of the absolute value).  s_{i-2m} = A_p[w0 + 3r - t],
// C_{2m} = E[t - 2r] and s_{i+2m} = A_p[w0 + t - r] come from three register rings of
// P = 3 RC - 2 entries indexed by t mod P (one new shared load each per iteration, the
// loop unrolled by P so that the ring indices are constants).  Lags outside 1..n-1 (the
// first 2 RC - 2 and the last iterations) are masked in the blocks that hold them.
// Exact in fp32: every value is an integer of magnitude below 2^10.
template <class TL, int R, int C0, int RC>
__device__ __forceinline__ void psl_ring(const View& V, int n, const Outs<TL, R>& o, int (&pl)[R])
{
    constexpr int P = 3 * RC - 2;
    const int w0 = o.v0 + C0;
    const float* A = (o.p ? V.A1 : V.A0) + w0;
    const int c = n - 1;
    const int tstar = c - o.p - 2 * w0;
    const int tend = n - 1 + 2 * (RC - 1);
    float cs[RC], mx[RC], ra[P], rc[P], rb[P];
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        const int i = 2 * (w0 + r) + o.p;
        cs[r] = (i == c ? -2.f : -4.f) * A[r];
        mx[r] = 0.f;
    }
    // entries e = -P+1 .. -1 (read only by masked lags)
#pragma unroll
    for (int k = 1; k < P; ++k) {
        ra[k] = A[P - k];
        rc[k] = V.G[k - P].x;
        rb[k] = A[k - P];
    }
    for (int t0 = 0; t0 <= tend; t0 += P) {
        if (t0 >= 2 * RC - 1 && t0 + P - 1 <= c) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int t = t0 + j;
                ra[j] = A[-t];
                rc[j] = V.G[t].x;
                rb[j] = A[t];
                const float z = t == tstar ? 0.f : 1.f;
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    const float cp = fmaf(cs[r], fmaf(rb[(j - r + P) % P], z, ra[(j - 3 * r + 3 * P) % P]),
                                          rc[(j - 2 * r + 2 * P) % P]);
                    mx[r] = fmaxf(mx[r], fabsf(cp));
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int t = t0 + j;
                if (t > tend) break;
                ra[j] = A[-t];
                rc[j] = V.G[t].x;
                rb[j] = A[t];
                const float z = t == tstar ? 0.f : 1.f;
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    const float cp = fmaf(cs[r], fmaf(rb[(j - r + P) % P], z, ra[(j - 3 * r + 3 * P) % P]),
                                          rc[(j - 2 * r + 2 * P) % P]);
                    const int m = t - 2 * r;
                    if (m >= 1 && m <= c) mx[r] = fmaxf(mx[r], fabsf(cp));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) pl[C0 + r] = (int)mx[r];
}

// All R outputs of the lane: one ring pass up to R = 6; wider lane blocks, whose three
// rings of 3R - 2 entries would not fit the registers, take the compare-and-select form
// at R = 7 (measured 2% faster there, two walkers per warp at L = 201) and two ring
// passes of (R+1)/2 and R - (R+1)/2 outputs from R = 9 (each pass reloads its rings:
// about twice the shared loads of one pass, but three instructions per lag term instead
// of a compare and select per term; 21-40% faster for the long lane blocks 9 and 11).
template <class TL, int R>
__device__ __forceinline__ void psl_eval(const View& V, int n, const Outs<TL, R>& o, int (&pl)[R])
{
    if constexpr (R == 7) {
        psl_eval_select<TL, R>(V, n, o, pl);
    } else if constexpr (R >= 8) {
        constexpr int H = (R + 1) / 2;
        psl_ring<TL, R, 0, H>(V, n, o, pl);
        psl_ring<TL, R, H, R - H>(V, n, o, pl);
    } else {
        psl_ring<TL, R, 0, R>(V, n, o, pl);
    }
}

// The walk under the PSL objective, one walker per warp: evaluate all n flips (dISL by
// the Toeplitz step of the plain walk, PSL by psl_eval), move to the lowest
// (PSL, ISL, i) whose result is not in HT, and keep the best sequence, the stagnation
// count and the restarts on (PSL, ISL) pairs; HT and the restart rules are the walk's.
template <int R>
__device__ void walk_psl(const WalkEnv& env, Walker& w, PslTrack& ps, int64_t until, int* base, const WarpSmem& SL,
                         const View& V, int trace_slot, int64_t trace_start, const Tile<32>& t)
{
    using TL = Tile<32>;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<TL, R> o(t);
    const int cap = p.probe_cap;
    float P[R];
    p_direct(V, n, o, P);
    StopCheck stop;
    stop.start(p, lane == 0);
    while (w.steps < until) {
        if ((w.steps & (kCheckEvery - 1)) == 0) {
            const int why = t.shfl(stop.poll(p, lane == 0), 0);
            if (why) {
                if (lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        int dl[R], pl[R];
        {
            float X[R];
            toeplitz_one(V, SL, n, o, t, X);
            assemble(V, n, o, X, P, dl);
        }
        psl_eval(V, n, o, pl);
        uint64_t key[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            key[r] = dl[r] == INT_MAX ? ~0ull : psl_key(pl[r], w.isl + dl[r], 2 * (o.v0 + r) + o.p);
        uint32_t excl = 0;
        int best_i = -1;
        uint64_t best_key = 0, fnew = 0;
        int64_t slot = -1;
        for (;;) {
            uint64_t lm = ~0ull;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (!((excl >> r) & 1u) && key[r] < lm) lm = key[r];
            const uint64_t km = warp_min64(lm);
            if (km == ~0ull) break;
            const int bi = psl_key_i(km);
            const uint64_t f = w.fp ^ __ldg(env.zk + bi);
            const Probe pr = probe_full(env, f, w.gen, cap, t);
            if (!pr.visited) {
                best_i = bi;
                best_key = km;
                slot = pr.slot;
                fnew = f;
                break;
            }
            exclude<TL, R>(excl, bi, t);
        }

        w.steps += 1;
        int code;
        if (best_i < 0) {
            w.blocked += 1;
            restart_walker(env, w, base, SL, V, t, &ps);
            p_direct(V, n, o, P);
            code = LABS_TRACE_BLOCKED;
        } else {
            flip_rows_table(V, n, o, P, best_i, t);
            const bool stored = slot >= 0;
            if (lane == 0 && stored) env.T[slot] = (fnew & ~kGenMask) | w.gen;
            if (lane == (best_i >> 5)) w.word ^= 1u << (best_i & 31);
            t.sync();
            w.fp = fnew;
            w.isl = psl_key_isl(best_key);
            ps.psl = psl_key_psl(best_key);
            if (!stored) w.overflows += 1;
            note_best(env, w, t, &ps);
            if (psl_better(ps.psl, w.isl, ps.since_psl, w.since)) {
                w.since = w.isl;
                ps.since_psl = ps.psl;
                w.stag = 0;
            } else {
                w.stag += 1;
            }
            code = best_i;
            if (w.stag >= env.patience || !stored) {
                restart_walker(env, w, base, SL, V, t, &ps);
                p_direct(V, n, o, P);
                code |= LABS_TRACE_RESTART;
            }
        }
        if (trace_slot >= 0 && lane == 0) {
            const int64_t s = w.steps - 1 - trace_start;
            if (s >= 0 && s < p.status->trace_capacity) {
                p.status->trace_code[trace_slot * p.status->trace_capacity + s] = code;
                p.status->trace_isl[trace_slot * p.status->trace_capacity + s] = w.isl;
            }
        }
    }
}

// The lane's two lowest 64-bit keys above `floor` (~0 where there are fewer).
template <int R>
__device__ __forceinline__ void top2_above64(const uint64_t (&key)[R], uint64_t floor, uint64_t& b1, uint64_t& b2)
{
    b1 = ~0ull;
    b2 = ~0ull;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t k = key[r] > floor ? key[r] : ~0ull;
        b2 = min(b2, max(b1, k));
        b1 = min(b1, k);
    }
}

// Lowest 64-bit value of the lane group: the lowest high word, then the lowest low word
// among the lanes that hold it.
template <class LG>
__device__ __forceinline__ uint64_t group_min64(uint64_t v, const LG& t)
{
    const uint32_t hi = t.rminu((uint32_t)(v >> 32));
    const uint32_t lo = t.rminu((uint32_t)(v >> 32) == hi ? (uint32_t)v : 0xFFFFFFFFu);
    return ((uint64_t)hi << 32) | lo;
}

// The walk under the PSL objective with two walkers per warp in lockstep (Pair): the
// dISL of every flip from the lockstep Toeplitz step (on the tensor cores when TC says
// so, as in walk_lockstep), the PSL of every neighbour from psl_eval, and the candidate
// rounds of walk_lockstep on the (PSL', ISL', i) keys: two candidates per round, the
// first S HT slots of each probed by half of the walker's lanes, full probes for longer
// chains.  The trajectory of each walker is exactly that of walk_psl: the lowest key
// whose state is not in HT is taken, and the best, stagnation and restart rules are the
// same.  Restarts run divergently per half (RT = Tile<16>).
template <class LG, class RT, int R, int TC>
__device__ void walk_psl_lockstep(const WalkEnv& env, Walker& w, PslTrack& ps, int64_t until, bool real, int* base,
                                  const WarpSmem& SL, const View& V, int trace_slot, int64_t trace_start,
                                  const LG& t, const RT& tt)
{
    constexpr int S = LG::kSize / 2;  // HT slots probed per candidate in a round
    constexpr unsigned SM = (1u << S) - 1u;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<LG, R> o(t);
    const int cap = p.probe_cap;
    const uint32_t tmask = (uint32_t)env.tmask;  // HT slots <= 2^20
    float P[R];
    p_direct(V, n, o, P);
    int prev = -1;  // the last flip since the walker's (re)start in this call, or -1
    StopCheck stop;
    stop.start(p, (threadIdx.x & 31) == 0);
    for (;;) {
        const bool act = real && w.steps < until;
        if (!__any_sync(kFull, act)) break;
        if (__any_sync(kFull, act && (w.steps & (kCheckEvery - 1)) == 0)) {
            const int why = __shfl_sync(kFull, stop.poll(p, (threadIdx.x & 31) == 0), 0);
            if (why) {
                if (act && lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        uint64_t key[R];
        {
            int dl[R], pl[R];
            int rv;
            {
                float X[R];
                if constexpr (TC == 1) {
                    toeplitz_tc(V, SL, n, o, t.h, X);
                } else if constexpr (TC == 2) {
                    if (SL.xp)
                        toeplitz_tc(V, SL, n, o, t.h, X);
                    else
                        toeplitz(V, n, o, X);
                } else {
                    toeplitz(V, n, o, X);
                }
                rv = lane_dl(V, n, o, X, P, dl);
            }
            psl_eval<LG, R>(V, n, o, pl);
#pragma unroll
            for (int r = 0; r < R; ++r)
                key[r] = r < rv ? psl_key(pl[r], w.isl + dl[r], 2 * (o.v0 + r) + o.p) : ~0ull;
            drop_candidate(key, prev, o, ~(uint64_t)0);
        }

        // Best admissible flip: candidates in ascending key order, two per round; keys
        // <= floor are known to lead to visited states.
        uint64_t floor = 0ull, kc = ~0ull;
        int slot = -1;
        uint64_t fnew = 0;
        bool done = !act;
        do {
            uint64_t b1, b2;
            top2_above64(key, floor, b1, b2);
            const uint64_t k0 = group_min64(done ? ~0ull : b1, t);
            const uint64_t k1 = group_min64(done ? ~0ull : (b1 == k0 ? b2 : b1), t);
            const bool has0 = k0 != ~0ull, has1 = k1 != ~0ull;
            const uint64_t f0 = w.fp ^ (has0 ? __ldg(env.zk + psl_key_i(k0)) : 0ull);
            const uint64_t f1 = w.fp ^ (has1 ? __ldg(env.zk + psl_key_i(k1)) : 0ull);
            const int hs = lane & (S - 1);
            const bool second = lane >= S;
            const uint64_t f = second ? f1 : f0;
            const bool live = !done && (second ? has1 : has0) && hs < cap;
            uint64_t e = 0;
            if (live) e = env.T[((uint32_t)f + (uint32_t)hs) & tmask];
            const bool match = live && e == ((f & ~kGenMask) | w.gen);
            const bool hit = live && ((((uint32_t)e & (uint32_t)kGenMask) != w.gen) || match);
            const unsigned hb = t.ballot(hit), mb = t.ballot(match);
            const unsigned h0 = hb & SM, h1 = (hb >> S) & SM;
            int st0 = !has0 ? kProbeNone
                            : h0 ? ((mb & h0 & (0u - h0)) ? kProbeVisited : kProbeFree)
                                 : (cap > S ? kProbeUnknown : kProbeFree);
            int st1 = !has1 ? kProbeNone
                            : h1 ? (((mb >> S) & h1 & (0u - h1)) ? kProbeVisited : kProbeFree)
                                 : (cap > S ? kProbeUnknown : kProbeFree);
            int s0 = -2, s1 = -2;
            const bool need0 = !done && st0 == kProbeUnknown;
            if (__any_sync(kFull, need0)) {
                const Probe pf = lockstep_probe_full(env, f0, w.gen, cap, need0, t);
                if (need0) {
                    st0 = pf.visited ? kProbeVisited : kProbeFree;
                    s0 = (int)pf.slot;
                }
            }
            const bool need1 = !done && st0 == kProbeVisited && st1 == kProbeUnknown;
            if (__any_sync(kFull, need1)) {
                const Probe pf = lockstep_probe_full(env, f1, w.gen, cap, need1, t);
                if (need1) {
                    st1 = pf.visited ? kProbeVisited : kProbeFree;
                    s1 = (int)pf.slot;
                }
            }
            if (!done) {
                if (st0 == kProbeFree) {
                    kc = k0, fnew = f0, done = true;
                    slot = s0 != -2 ? s0 : (h0 ? (int)(((uint32_t)f0 + (uint32_t)(__ffs(h0) - 1)) & tmask) : -1);
                } else if (st0 == kProbeNone || st1 == kProbeNone) {
                    done = true;  // every neighbour is in HT
                } else if (st1 == kProbeFree) {
                    kc = k1, fnew = f1, done = true;
                    slot = s1 != -2 ? s1 : (h1 ? (int)(((uint32_t)f1 + (uint32_t)(__ffs(h1) - 1)) & tmask) : -1);
                } else {
                    floor = k1;
                }
            }
        } while (__any_sync(kFull, !done));

        // Apply the move (walkers that have one), from the values before the flip.
        const bool moves = act && kc != ~0ull;
        const int best_i = moves ? psl_key_i(kc) : 0;
        apply_flip<LG, R>(V, n, o, lane, moves, best_i, P);
        const bool stored = slot >= 0;
        if (moves && lane == 0 && stored) env.T[slot] = (fnew & ~kGenMask) | w.gen;
        if (moves && lane == (best_i >> 5)) w.word ^= 1u << (best_i & 31);
        __syncwarp();
        int code = 0;
        bool again = false;
        if (act) {
            w.steps += 1;
            if (!moves) {
                w.blocked += 1;
                again = true;
                code = LABS_TRACE_BLOCKED;
            } else {
                w.fp = fnew;
                w.isl = psl_key_isl(kc);
                ps.psl = psl_key_psl(kc);
                if (!stored) w.overflows += 1;
                note_best(env, w, t, &ps);
                if (psl_better(ps.psl, w.isl, ps.since_psl, w.since)) {
                    w.since = w.isl;
                    ps.since_psl = ps.psl;
                    w.stag = 0;
                } else {
                    w.stag += 1;
                }
                code = best_i;
                if (w.stag >= env.patience || !stored) {
                    again = true;
                    code |= LABS_TRACE_RESTART;
                }
            }
        }
        if (moves) prev = best_i;
        if (again) {  // divergent: only this half restarts
            restart_walker(env, w, base, SL, V, tt, &ps);
            p_direct(V, n, o, P);
            prev = -1;
        }
        __syncwarp();
        if (act && trace_slot >= 0 && lane == 0) {
            const int64_t s = w.steps - 1 - trace_start;
            if (s >= 0 && s < p.status->trace_capacity) {
                p.status->trace_code[trace_slot * p.status->trace_capacity + s] = code;
                p.status->trace_isl[trace_slot * p.status->trace_capacity + s] = w.isl;
            }
        }
    }
}

template <int TILE, int RMAX, int MODE>
__global__ void __launch_bounds__(256, LABS_WALK_MIN_BLOCKS) walk_chunk_kernel(KParams p, int chunk_index)
{
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = warp_smem(p.n_max, TILE);
    const Tile<TILE> t(threadIdx.x & 31);
    const int slot_id = threadIdx.x / TILE;  // walker slot of this tile in the CTA
    int* base = smem + slot_id * SL.words;
    const View V = make_view(base, SL);
    const int64_t target = p.status->target_steps;
    for (;;) {
        uint32_t q = 0;
        if (t.lane == 0) q = atomicAdd(&p.queue[chunk_index], 1u);
        const int64_t wi = (int64_t)t.shfl(q, 0);
        if (wi >= p.W) break;
        WalkerState* st = p.states + wi;
        const int64_t steps_done = st->steps_done;
        const int64_t until = min(target, steps_done + (int64_t)p.chunk_steps);
        if (steps_done >= until) continue;
        const DevGroup G = p.groups[st->group];
        WalkEnv env;
        env.p = &p;
        env.tmask = (1ull << p.tabu_log2) - 1ull;
        env.T = p.tabu + ((uint64_t)wi << p.tabu_log2);
        env.zk = p.zkeys + G.zkey_off;
        env.st = st;
        env.L = G.L;
        env.n = G.n;
        env.patience = p.patience > 0 ? p.patience : 2 * G.n;
        env.g = (uint32_t)wi;
        Walker w;
        load_walker(st, w, t.lane);
        const int trace_slot = st->trace_slot;
        const int64_t trace_start = trace_slot >= 0 ? p.trace_start[trace_slot] : 0;
        const int isl = load_rows(base, SL, V, w.word, G.L, G.n, t);
        if (isl != w.isl) {
            if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)wi);
            continue;
        }
        StepExtras ex;
        ex.scores = nullptr;
        ex.sdump = nullptr;
        ex.rec = nullptr;
        ex.tau = 0;
        ex.dump_cap = 0;
        ex.n_max = p.n_max;
        env.slot = nullptr;
        env.slot_valid = nullptr;
        env.rdump = nullptr;
        env.rdump_idx = nullptr;
        env.rdump_count = nullptr;
        env.dump_cap = 0;
        DevStatus* S = p.status;
        if (MODE == 0 && S->learned) {
            // restart-only learned mode: the proposed restart state, and its record for
            // a traced walker
            env.slot = S->l_slot + wi * kBitWords;
            env.slot_valid = S->l_slot_valid + wi;
            if (trace_slot >= 0 && S->d_restart != nullptr) {
                env.rdump = S->d_restart + (int64_t)trace_slot * S->d_cap * kBitWords;
                env.rdump_idx = S->d_restart_idx + (int64_t)trace_slot * S->d_cap;
                env.rdump_count = S->d_restart_count + trace_slot;
                env.dump_cap = S->d_cap;
            }
        }
        if (MODE == 1 && S->learned) {
            env.slot = S->l_slot + wi * kBitWords;
            env.slot_valid = S->l_slot_valid + wi;
            if (S->l_score_step[wi] == steps_done) {
                ex.scores = S->l_scores + wi * p.n_max;
                ex.tau = S->l_tau;
            }
            if (trace_slot >= 0 && S->d_scores != nullptr) {
                ex.sdump = S->d_scores + (int64_t)trace_slot * S->d_cap * p.n_max;
                ex.sdump_step = S->d_score_step + (int64_t)trace_slot * S->d_cap;
                ex.sdump_count = S->d_score_count + trace_slot;
                ex.dump_cap = S->d_cap;
                env.rdump = S->d_restart + (int64_t)trace_slot * S->d_cap * kBitWords;
                env.rdump_idx = S->d_restart_idx + (int64_t)trace_slot * S->d_cap;
                env.rdump_count = S->d_restart_count + trace_slot;
                env.dump_cap = S->d_cap;
            }
        }
        if (S->log != nullptr && p.chunk_steps > 0) {
            const int64_t since = steps_done - S->log_start;
            if (since >= 0 && since % p.chunk_steps == 0) {
                const int64_t idx = (since / p.chunk_steps) * p.W + wi;
                if (idx < S->log_capacity) ex.rec = S->log + idx;
            }
        }
        // the learned mode's step (walk_steps), the best-first search, or the lockstep
        // step of the plain walk
        constexpr int R2 = RMAX > 2 ? RMAX - 2 : 1;
        const bool full = RMAX <= 2 || block_R(G.n, TILE) >= RMAX;
        if constexpr (MODE == 3) {
            PslTrack ps;
            ps.psl = table_psl(V, G.n, t);
            ps.best_psl = st->best_psl;
            ps.since_psl = st->since_psl;
            if (ps.psl != st->psl) {
                if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)wi);
                continue;
            }
            if (full)
                walk_psl<RMAX>(env, w, ps, until, base, SL, V, trace_slot, trace_start, t);
            else
                walk_psl<R2>(env, w, ps, until, base, SL, V, trace_slot, trace_start, t);
            if (t.lane == 0) {
                st->psl = ps.psl;
                st->best_psl = ps.best_psl;
                st->since_psl = ps.since_psl;
            }
        } else if constexpr (MODE == 2) {
            uint64_t* qk = p.pq_key + wi * LABS_QUEUE_SIZE;
            uint32_t* qb = p.pq_bits + wi * LABS_QUEUE_SIZE * kBitWords;
            if (full)
                walk_bestfirst<RMAX>(env, w, until, base, SL, V, trace_slot, trace_start, t, qk, qb);
            else
                walk_bestfirst<R2>(env, w, until, base, SL, V, trace_slot, trace_start, t, qk, qb);
        } else if constexpr (MODE == 1) {
            if (full)
                walk_steps<Tile<TILE>, RMAX>(env, w, until, base, SL, V, trace_slot, trace_start, ex, t);
            else
                walk_steps<Tile<TILE>, R2>(env, w, until, base, SL, V, trace_slot, trace_start, ex, t);
        } else {
            if (full)
                walk_lockstep<Tile<TILE>, Tile<TILE>, RMAX>(env, w, until, true, base, SL, V, trace_slot, trace_start,
                                                            ex.rec, t, t);
            else
                walk_lockstep<Tile<TILE>, Tile<TILE>, R2>(env, w, until, true, base, SL, V, trace_slot, trace_start,
                                                          ex.rec, t, t);
        }
        save_walker(st, w, t.lane);
        t.sync();
    }
}


// Walk launch with WPW = 32 / LG::kSize walkers per warp (two for n <= 160, four for
// short sequences): the warp takes WPW consecutive walkers; when their lengths differ
// (a group boundary) or fewer are left, it runs them one after the other with the other
// lane groups idle.  RT is the tile type a lane group restarts with (divergently).
// MODE 0: the plain walk; 3: the walk under the PSL objective (two walkers per warp).
template <class LG, class RT, int RMAX, int MODE = 0>
__device__ __forceinline__ void walk_group(const KParams& p, int chunk_index)
{
    constexpr int WPW = 32 / LG::kSize;
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = warp_smem(p.n_max, LG::kSize, MODE == 3);
    const LG t(threadIdx.x & 31);
    const RT tt(threadIdx.x & 31);
    int* base = smem + (threadIdx.x / LG::kSize) * SL.words;
    const View V = make_view(base, SL);
    const int64_t target = p.status->target_steps;
    DevStatus* S = p.status;
    for (;;) {
        uint32_t q = 0;
        if ((threadIdx.x & 31) == 0) q = atomicAdd(&p.queue[chunk_index], (uint32_t)WPW);
        q = __shfl_sync(kFull, q, 0);
        if ((int64_t)q >= p.W) break;
        const int64_t mine_w = (int64_t)q + t.h;
        const bool exists = mine_w < p.W;
        const int my_n = exists ? p.groups[p.states[mine_w].group].n : -1;
        const int n0 = __shfl_sync(kFull, my_n, 0);
        const bool together = __all_sync(kFull, exists && my_n == n0);
        const int passes = together ? 1 : (int)min((int64_t)WPW, p.W - (int64_t)q);
        for (int pass = 0; pass < passes; ++pass) {
            // together: every group runs its walker; else pass k runs group k alone
            const bool real0 = exists && (together || pass == t.h);
            // the idle groups mirror the running group's length so that loops match
            const int64_t lead_w = together ? mine_w : (int64_t)q + pass;
            const DevGroup G = p.groups[p.states[lead_w].group];
            WalkEnv env;
            env.p = &p;
            env.tmask = (1ull << p.tabu_log2) - 1ull;
            env.T = p.tabu + ((uint64_t)mine_w << p.tabu_log2);
            env.L = G.L;
            env.n = G.n;
            env.patience = p.patience > 0 ? p.patience : 2 * G.n;
            env.g = (uint32_t)mine_w;
            env.st = p.states + (exists ? mine_w : lead_w);
            env.slot = nullptr;
            env.slot_valid = nullptr;
            env.rdump = nullptr;
            env.rdump_idx = nullptr;
            env.rdump_count = nullptr;
            env.dump_cap = 0;
            env.zk = p.zkeys + G.zkey_off;
            Walker w;
            load_walker(env.st, w, t.lane);
            int64_t steps_done = w.steps;
            int64_t until = min(target, steps_done + (int64_t)p.chunk_steps);
            bool real = real0 && steps_done < until;
            const int trace_slot = real ? env.st->trace_slot : -1;
            if (MODE == 0 && real && S->learned) {
                // restart-only learned mode: the proposed restart state (and its record
                // for a traced walker)
                env.slot = S->l_slot + mine_w * kBitWords;
                env.slot_valid = S->l_slot_valid + mine_w;
                if (trace_slot >= 0 && S->d_restart != nullptr) {
                    env.rdump = S->d_restart + (int64_t)trace_slot * S->d_cap * kBitWords;
                    env.rdump_idx = S->d_restart_idx + (int64_t)trace_slot * S->d_cap;
                    env.rdump_count = S->d_restart_count + trace_slot;
                    env.dump_cap = S->d_cap;
                }
            }
            const int64_t trace_start = trace_slot >= 0 ? p.trace_start[trace_slot] : 0;
            const int isl = load_rows(base, SL, V, w.word, G.L, G.n, t);
            if (real && isl != w.isl) {
                if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)mine_w);
                real = false;
            }
            PslTrack ps;
            if constexpr (MODE == 3) {
                ps.psl = table_psl(V, G.n, t);
                ps.best_psl = env.st->best_psl;
                ps.since_psl = env.st->since_psl;
                if (real && ps.psl != env.st->psl) {
                    if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)mine_w);
                    real = false;
                }
            }
            labs_log_record* rec = nullptr;
            if (MODE == 0 && real && S->log != nullptr && p.chunk_steps > 0) {
                const int64_t since = steps_done - S->log_start;
                if (since >= 0 && since % p.chunk_steps == 0) {
                    const int64_t idx = (since / p.chunk_steps) * p.W + mine_w;
                    if (idx < S->log_capacity) rec = S->log + idx;
                }
            }
            // lane block: block_R(n) when it is one of RMAX .. RMAX-3, else the smallest
            // bank-conflict-free one of those.  Two walkers per warp take the Toeplitz
            // product to the tensor cores while n_max <= 128 (lane blocks up to 9; the
            // second product for n > 128 would be mostly padding)
            constexpr int TC = LG::kSize != 16 ? 0 : RMAX <= 8 ? 1 : RMAX == 9 ? 2 : 0;
            int R = block_R(G.n, LG::kSize);
            if (R < RMAX - 3) R = conflict_free_R(RMAX - 3, LG::kSize);
            if constexpr (MODE == 3) {
                if (R >= RMAX)
                    walk_psl_lockstep<LG, RT, RMAX, TC>(env, w, ps, until, real, base, SL, V, trace_slot, trace_start,
                                                        t, tt);
                else if (R == RMAX - 1)
                    walk_psl_lockstep<LG, RT, (RMAX > 1 ? RMAX - 1 : 1), TC>(env, w, ps, until, real, base, SL, V,
                                                                         trace_slot, trace_start, t, tt);
                else if (R == RMAX - 2)
                    walk_psl_lockstep<LG, RT, (RMAX > 2 ? RMAX - 2 : 1), TC>(env, w, ps, until, real, base, SL, V,
                                                                         trace_slot, trace_start, t, tt);
                else
                    walk_psl_lockstep<LG, RT, (RMAX > 3 ? RMAX - 3 : 1), TC>(env, w, ps, until, real, base, SL, V,
                                                                         trace_slot, trace_start, t, tt);
            } else {
                if (R >= RMAX)
                    walk_lockstep<LG, RT, RMAX, TC>(env, w, until, real, base, SL, V, trace_slot, trace_start, rec, t,
                                                    tt);
                else if (R == RMAX - 1)
                    walk_lockstep<LG, RT, (RMAX > 1 ? RMAX - 1 : 1), TC>(env, w, until, real, base, SL, V, trace_slot,
                                                                     trace_start, rec, t, tt);
                else if (R == RMAX - 2)
                    walk_lockstep<LG, RT, (RMAX > 2 ? RMAX - 2 : 1), TC>(env, w, until, real, base, SL, V, trace_slot,
                                                                     trace_start, rec, t, tt);
                else
                    walk_lockstep<LG, RT, (RMAX > 3 ? RMAX - 3 : 1), TC>(env, w, until, real, base, SL, V, trace_slot,
                                                                     trace_start, rec, t, tt);
            }
            if (real) {
                save_walker(env.st, w, t.lane);
                if constexpr (MODE == 3) {
                    if (t.lane == 0) {
                        env.st->psl = ps.psl;
                        env.st->best_psl = ps.best_psl;
                        env.st->since_psl = ps.since_psl;
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <int RMAX>
__global__ void __launch_bounds__(256, LABS_WALK_MIN_BLOCKS) walk_pair_kernel(KParams p, int chunk_index)
{
    walk_group<Pair, Tile<16>, RMAX>(p, chunk_index);
}

template <int RMAX>
__global__ void __launch_bounds__(256, LABS_WALK_MIN_BLOCKS) walk_psl_pair_kernel(KParams p, int chunk_index)
{
    walk_group<Pair, Tile<16>, RMAX, 3>(p, chunk_index);
}

template <int RMAX>
__global__ void __launch_bounds__(256, LABS_WALK_MIN_BLOCKS) walk_quad_kernel(KParams p, int chunk_index)
{
    walk_group<Quad, Tile<8>, RMAX>(p, chunk_index);
}

}  // namespace
}  // namespace labsgpu
