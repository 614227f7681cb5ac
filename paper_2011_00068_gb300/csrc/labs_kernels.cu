// labs_kernels.cu -- sm_103a kernels of the skew-symmetric LABS search
// (Brest & Boskovic, arXiv 2011.00068).
//
// One warp owns one walker (or one input row).  A walker's sequence is kept in shared
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
// loop.  Lanes 0-15 hold the even class, lanes 16-31 the odd class; each lane owns R
// consecutive outputs v0..v0+R-1 and slides a window of R values of E along u.
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

// Per-warp views of the shared-memory layout.
struct View {
    int* A0;      // A0[-apad .. n_max+apad)
    int* A1;
    int* E;       // E[-kEPad .. n_max+8)
    uint32_t* B;  // bit-packed classes and reversals, 4 x kBitVec words
};

__device__ __forceinline__ View make_view(int* base, const WarpSmem& L)
{
    View v;
    v.A0 = base + L.apad;
    v.A1 = base + L.alen + L.apad;
    v.E = base + 2 * L.alen + kEPad;
    v.B = reinterpret_cast<uint32_t*>(base + L.boff);
    return v;
}

// Zeroes the rows, the table and the bit vectors (not the fingerprint keys Z, which
// stay for the chunk).
__device__ __forceinline__ void clear_warp(int* base, const WarpSmem& L, int lane)
{
    int4* b4 = reinterpret_cast<int4*>(base);
    for (int t = lane; t < L.zoff / 4; t += kWarp) b4[t] = make_int4(0, 0, 0, 0);
    __syncwarp();
}

// Fills A0/A1 from the free-variable bits (word j of the bits lives in lane j's
// `word`), by Eq. 4: s_j = x_j for j <= c, s_{c+t} = (-1)^t x_{c-t}.
__device__ __forceinline__ void rows_from_bits(const View& V, uint32_t word, int L, int n, int lane)
{
    const int c = n - 1;
    for (int j0 = 0; j0 < L; j0 += kWarp) {
        int j = j0 + lane;
        int f = j <= c ? j : 2 * c - j;
        if (j >= L) f = 0;
        uint32_t w = __shfl_sync(kFull, word, f >> 5);
        if (j < L) {
            int x = ((w >> (f & 31)) & 1u) ? -1 : 1;
            int s = (j > c && ((j - c) & 1)) ? -x : x;
            if (j & 1) V.A1[j >> 1] = s;
            else V.A0[j >> 1] = s;
        }
    }
    __syncwarp();
}

// Bit-packed classes: B[p*kBitVec + k] holds bits 32k..32k+31 of class p (bit u set
// <=> A_p[u] = -1); B[(2+p)*kBitVec + k] the same for the reversed class (bit t is
// class entry n_p-1-t).  One ballot per word; zero beyond the class length.
__device__ __forceinline__ void bits_from_rows(const View& V, int n, int lane)
{
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int* A = p ? V.A1 : V.A0;
        const int np = p ? n - 1 : n;
        for (int k = 0; k < kBitVec; ++k) {
            const int u = 32 * k + lane;
            const uint32_t w = __ballot_sync(kFull, u < np && A[u] < 0);
            const int t = np - 1 - u;
            const uint32_t r = __ballot_sync(kFull, u < np && A[t] < 0);
            if (lane == 0) {
                V.B[p * kBitVec + k] = w;
                V.B[(2 + p) * kBitVec + k] = r;
            }
        }
    }
    __syncwarp();
}

// Number of differing bits between x and x >> sh over bits [0, len) (x = B vector).
__device__ __forceinline__ int shifted_mismatch(const uint32_t* x, const uint32_t* y, int sh, int len)
{
    const int q = sh >> 5, r = sh & 31;
    int cnt = 0;
    for (int k = 0; 32 * k < len; ++k) {
        const uint32_t s = __funnelshift_r(y[k + q], y[k + q + 1], r);
        uint32_t v = x[k] ^ s;
        const int valid = len - 32 * k;
        if (valid < 32) v &= (1u << valid) - 1u;
        cnt += __popc(v);
    }
    return cnt;
}

// Even-lag autocorrelations (Eq. 1) into E and the ISL (Eq. 2) from the bit-packed
// classes: for each class, sum_u a_u a_{u+m} = (n_p - m) - 2 #{u : a_u != a_{u+m}}.
__device__ __forceinline__ int build_table(const View& V, int n, int lane)
{
    bits_from_rows(V, n, lane);
    int part = 0;
    for (int m = 1 + lane; m < n; m += kWarp) {
        int d = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int len = (p ? n - 1 : n) - m;
            if (len <= 0) continue;
            const uint32_t* x = V.B + p * kBitVec;
            d += len - 2 * shifted_mismatch(x, x, m, len);
        }
        V.E[m] = d;
        if (m <= kEPad) V.E[-m] = d;
        part += d * d;
    }
    __syncwarp();
    return __reduce_add_sync(kFull, part);
}

// X_v = sum_u A_p[u] E[u-v] for the lane's R outputs v = v0..v0+R-1 (the Toeplitz
// product).  The window of E slides one position per u.  When R is a multiple of 4
// the lane's block starts on a 16-byte boundary and E is read four values at a time
// (the 16 distinct blocks of a half-warp are then contiguous: no bank conflicts);
// for other R the scalar reads have an odd or conflict-free stride.
template <int R>
__device__ __forceinline__ void toeplitz(const View& V, int n, int lane, int (&acc)[R])
{
    const int p = lane >> 4;
    const int v0 = (lane & 15) * R;
    const int* A = p ? V.A1 : V.A0;
    const int* E = V.E;
    const int nu = (n + 3) & ~3;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    if constexpr (R % 4 == 0) {
        // win[j] = E[u - v0 - R + j], j = 0 .. R+3
        int win[R + 4];
#pragma unroll
        for (int c = 0; c < R / 4; ++c) {
            const int4 q = *reinterpret_cast<const int4*>(E - v0 - R + 4 * c);
            win[4 * c] = q.x;
            win[4 * c + 1] = q.y;
            win[4 * c + 2] = q.z;
            win[4 * c + 3] = q.w;
        }
#pragma unroll kToeplitzUnroll
        for (int u = 0; u < nu; u += 4) {
            const int4 q = *reinterpret_cast<const int4*>(E + u - v0);
            win[R] = q.x;
            win[R + 1] = q.y;
            win[R + 2] = q.z;
            win[R + 3] = q.w;
            const int4 a4 = *reinterpret_cast<const int4*>(A + u);
            const int a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += a[t] * win[R + t - r];
#pragma unroll
            for (int j = 0; j < R; ++j) win[j] = win[j + 4];
        }
    } else {
        // win[r] = E[u - v0 - r]
        int win[R];
#pragma unroll
        for (int r = 0; r < R; ++r) win[r] = E[-1 - v0 - r];
        for (int u = 0; u < nu; u += 4) {
            const int4 a4 = *reinterpret_cast<const int4*>(A + u);
            const int a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
#pragma unroll
                for (int r = R - 1; r > 0; --r) win[r] = win[r - 1];
                win[0] = E[u + t - v0];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += a[t] * win[r];
            }
        }
    }
}

// P_v = sum_{m=1}^{v} A_p[v+m] A_p[v-m] from scratch for the lane's outputs, from the
// bit-packed classes (built by build_table): the pairs compare bits v+1.. of the
// class with bits n_p-v.. of the reversed class, P_v = v - 2 #{mismatches}.
template <int R>
__device__ __forceinline__ void p_direct(const View& V, int n, int lane, int (&P)[R])
{
    const int p = lane >> 4;
    const int v0 = (lane & 15) * R;
    const int np = p ? n - 1 : n;
    const int nv = p ? (n >> 1) : ((n + 1) >> 1);
    const uint32_t* x = V.B + p * kBitVec;
    const uint32_t* xr = V.B + (2 + p) * kBitVec;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        P[r] = 0;
        if (v >= nv || v == 0) continue;
        const int q1 = (v + 1) >> 5, r1 = (v + 1) & 31;
        const int q2 = (np - v) >> 5, r2 = (np - v) & 31;
        int cnt = 0;
        for (int k = 0; 32 * k < v; ++k) {
            const uint32_t a = __funnelshift_r(x[k + q1], x[k + q1 + 1], r1);
            const uint32_t b = __funnelshift_r(xr[k + q2], xr[k + q2 + 1], r2);
            uint32_t d = a ^ b;
            const int valid = v - 32 * k;
            if (valid < 32) d &= (1u << valid) - 1u;
            cnt += __popc(d);
        }
        P[r] = v - 2 * cnt;
    }
}

// Change of P for a move that negates class-pb entries w1 and w2 (w2 < 0: centre, one
// entry).  A pair (v+m, v-m) with exactly one negated end changes by -2 x its old
// product; pairs with both ends negated are unchanged.  Reads A before the flip.
template <int R>
__device__ __forceinline__ void p_update(const View& V, int n, int lane, int (&P)[R], int pb, int w1, int w2)
{
    const int p = lane >> 4;
    if (p != pb) return;
    const int v0 = (lane & 15) * R;
    const int* A = pb ? V.A1 : V.A0;
    const int nv = pb ? (n >> 1) : ((n + 1) >> 1);
    const int a1 = A[w1];
    const int a2 = w2 >= 0 ? A[w2] : 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        if (v >= nv) continue;
        int d = 0;
        const int t1 = 2 * v - w1;
        if (v != w1 && t1 != w2) d += a1 * A[t1];
        if (w2 >= 0) {
            const int t2 = 2 * v - w2;
            if (v != w2 && t2 != w1) d += a2 * A[t2];
        }
        P[r] -= 2 * d;
    }
}

// dl[r] = dISL of free variable i = 2(v0+r)+p, or INT_MAX where that output does not
// exist.  Formula in the header comment.
template <int R>
__device__ __forceinline__ void assemble(const View& V, int n, int lane, const int (&X)[R], const int (&P)[R],
                                         int (&dl)[R])
{
    const int p = lane >> 4;
    const int v0 = (lane & 15) * R;
    const int* A = p ? V.A1 : V.A0;
    const int nv = p ? (n >> 1) : ((n + 1) >> 1);
    const int c = n - 1;
    const int N = p ? n - 2 : n - 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        if (v >= nv) {
            dl[r] = INT_MAX;
            continue;
        }
        const int i = 2 * v + p;
        const int av = A[v];
        if (i == c) {
            dl[r] = -4 * av * X[r] + 16 * (c >> 1);
            continue;
        }
        const int sq = A[n - 1 - v - p];
        const int ck0 = V.E[c - i];
        const int t = 3 * v + p - n + 1;
        const int corr = t >= 0 ? sq * A[t] : 0;
        dl[r] = -8 * av * (X[r] - sq * ck0) + 16 * (N - 1) + 32 * (P[r] - corr);
    }
}

// Rebuilds the walker's rows and table from its bits; returns the ISL.
__device__ __forceinline__ int load_rows(int* base, const WarpSmem& SL, const View& V, uint32_t word,
                                         int L, int n, int lane)
{
    clear_warp(base, SL, lane);
    rows_from_bits(V, word, L, n, lane);
    return build_table(V, n, lane);
}

// HT fingerprint (Zobrist): XOR of the keys of the free variables equal to -1.
__device__ __forceinline__ uint64_t fingerprint_all(uint32_t word, const uint64_t* zk, int n, int lane)
{
    uint64_t f = 0;
    const int nr = (n + kWarp - 1) & ~(kWarp - 1);
    for (int i0 = 0; i0 < nr; i0 += kWarp) {
        const int i = i0 + lane;
        uint32_t w = __shfl_sync(kFull, word, i0 >> 5);
        if (i < n && ((w >> (i & 31)) & 1u)) f ^= zk[i];
    }
    uint32_t lo = __reduce_xor_sync(kFull, (uint32_t)f);
    uint32_t hi = __reduce_xor_sync(kFull, (uint32_t)(f >> 32));
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Registers of one walker while its warp runs it.
struct Walker {
    uint32_t word;   // lane j < 8: bits word j
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
    int L, n, patience, lane;
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

__device__ __forceinline__ void note_best(const WalkEnv& env, Walker& w)
{
    if (w.isl < w.best_isl) {
        w.best_isl = w.isl;
        w.best_step = w.steps;
        if (env.lane < kBitWords) env.st->best[env.lane] = w.word;
    }
    if (w.target_step < 0 && target_met(*env.p, env.L, w.isl)) w.target_step = w.steps;
}

// Algorithm 1 start: random skew-symmetric S (restart index w.restart_idx), its ISL,
// insert it into HT (a fresh generation: its home slot is free), best update.
__device__ void start_walker(const WalkEnv& env, Walker& w, int* base, const WarpSmem& SL, const View& V,
                             bool proposed = false)
{
    const int lane = env.lane;
    if (proposed) {
        // learned mode: the restart state chosen by the proposal pass replaces the draw
        w.word = lane < kBitWords ? env.slot[lane] : 0u;
        if (env.rdump != nullptr) {
            const int k = *env.rdump_count;
            if (k < env.dump_cap) {
                if (lane < kBitWords) env.rdump[(int64_t)k * kBitWords + lane] = w.word;
                if (lane == 0) env.rdump_idx[k] = w.restart_idx;
            }
            __syncwarp();
            if (lane == 0) *env.rdump_count = k + 1;
        }
        __syncwarp();
        if (lane == 0) *env.slot_valid = 0;
    } else {
        w.word = lane < kBitWords ? start_word(env.p->seed, env.g, w.restart_idx, lane, env.n) : 0u;
    }
    w.isl = load_rows(base, SL, V, w.word, env.L, env.n, lane);
    w.fp = fingerprint_all(w.word, env.zk, env.n, lane);
    if (lane == 0) env.T[w.fp & env.tmask] = (w.fp & ~kGenMask) | w.gen;
    __syncwarp();
    w.since = w.isl;
    w.stag = 0;
    note_best(env, w);
}

__device__ void restart_walker(const WalkEnv& env, Walker& w, int* base, const WarpSmem& SL,
                               const View& V)
{
    w.restart_idx += 1;
    w.restarts += 1;
    w.gen += 1;
    if (w.gen > kGenMask) {
        const int64_t slots = (int64_t)env.tmask + 1;
        for (int64_t t = env.lane; t < slots; t += kWarp) env.T[t] = 0ull;
        __syncwarp();
        w.gen = 1;
    }
    const bool proposed = env.slot_valid != nullptr && *env.slot_valid != 0;
    start_walker(env, w, base, SL, V, proposed);
}

// Warp-uniform: lane 0 reads the host-written control block and broadcasts.
__device__ __forceinline__ int stop_requested(const KParams& p, int lane)
{
    int why = 0;
    if (lane == 0 && p.ctrl != nullptr) {
        if (p.ctrl->stop) why = LABS_ECANCELLED;
        else if (global_ns() >= p.ctrl->deadline_ns) why = LABS_ETIMEOUT;
    }
    return __shfl_sync(kFull, why, 0);
}

// Result of probing HT for one candidate.
struct Probe {
    bool visited;
    int64_t slot;  // insertion slot when not visited, -1 when no free slot within the cap
};

// Full linear probe of f (all `cap` slots at once, one per lane).
__device__ __forceinline__ Probe probe_full(const WalkEnv& env, uint64_t f, uint32_t gen, int cap)
{
    const int lane = env.lane;
    const uint64_t tag = (f & ~kGenMask) | gen;
    uint64_t e = 0;
    if (lane < cap) e = env.T[(f + (uint64_t)lane) & env.tmask];
    const bool match = e == tag;
    const unsigned bal = __ballot_sync(kFull, lane < cap && (((e & kGenMask) != gen) || match));
    Probe pr{false, -1};
    if (bal) {
        const int fl = __ffs(bal) - 1;
        pr.visited = __shfl_sync(kFull, match ? 1 : 0, fl) != 0;
        pr.slot = (int64_t)((f + (uint64_t)fl) & env.tmask);
    }
    return pr;
}

// Lowest (dl, i) among the lane outputs not in `excl` (all lanes get the result;
// bi = -1 when none is left).
template <int R>
__device__ __forceinline__ void warp_argmin(const int (&dl)[R], uint32_t excl, int v0, int pcls, int& bd, int& bi)
{
    int lm = INT_MAX, li = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (!((excl >> r) & 1u) && dl[r] < lm) {
            lm = dl[r];
            li = 2 * (v0 + r) + pcls;
        }
    bd = __reduce_min_sync(kFull, lm);
    bi = bd == INT_MAX ? -1 : __reduce_min_sync(kFull, lm == bd ? li : INT_MAX);
}

template <int R>
__device__ __forceinline__ void exclude(uint32_t& excl, int bi, int lane)
{
    const int vb = bi >> 1, pb = bi & 1;
    if (lane == pb * 16 + vb / R) excl |= 1u << (vb % R);
}

// Order-preserving map of a float score to int32 (the learned ordering compares these).
__device__ __forceinline__ int score_key(float f)
{
    const int k = __float_as_int(f);
    return k >= 0 ? k : (k ^ 0x7FFFFFFF);
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

template <int R>
__device__ void walk_steps(const WalkEnv& env, Walker& w, int64_t until, int* base, const WarpSmem& SL,
                           const View& V, int trace_slot, int64_t trace_start, const StepExtras& ex)
{
    const KParams& p = *env.p;
    const int lane = env.lane, n = env.n, c = n - 1;
    const int pcls = lane >> 4, v0 = (lane & 15) * R;
    const int cap = p.probe_cap;
    int P[R];
    p_direct<R>(V, n, lane, P);
    const int64_t first_step = w.steps;
    int log_first = 0, log_min = w.isl;
    bool log_live = true;
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
            const int why = stop_requested(p, lane);
            if (why) {
                if (lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        int dl[R];
        {
            int X[R];
            toeplitz<R>(V, n, lane, X);
            assemble<R>(V, n, lane, X, P, dl);
        }

        // Best admissible flip: lowest (dISL, i) whose result is not in HT.  Two
        // candidates are probed per round, 16 slots each (half a warp per candidate);
        // a longer chain falls back to a full probe.  The chosen flip is the best one
        // in about 40% of the steps and one of the best two in about 86% (L = 201).
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
            const int dmin = __reduce_min_sync(kFull, lm);
            const int thr = dmin > INT_MAX - ex.tau ? INT_MAX - 1 : dmin + ex.tau;
            int keys[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = 2 * (v0 + r) + pcls;
                keys[r] = dl[r] <= thr ? score_key(ex.scores[i]) : INT_MIN;
            }
            if (ex.sdump != nullptr) {
                const int k = *ex.sdump_count;
                if (k < ex.dump_cap) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int i = 2 * (v0 + r) + pcls;
                        if (dl[r] != INT_MAX) ex.sdump[(int64_t)k * ex.n_max + i] = ex.scores[i];
                    }
                    if (lane == 0) ex.sdump_step[k] = w.steps;
                }
                __syncwarp();
                if (lane == 0) *ex.sdump_count = k + 1;
                __syncwarp();
            }
            for (;;) {
                int lk = INT_MIN, li = INT_MAX, ld = INT_MAX;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (!((excl >> r) & 1u) && keys[r] > lk && dl[r] != INT_MAX) {
                        lk = keys[r];
                        li = 2 * (v0 + r) + pcls;
                        ld = dl[r];
                    }
                const int km = __reduce_max_sync(kFull, lk);
                if (km == INT_MIN) break;
                const int bi = __reduce_min_sync(kFull, lk == km ? li : INT_MAX);
                const int bd = __reduce_min_sync(kFull, li == bi ? ld : INT_MAX);
                const uint64_t f = w.fp ^ env.zk[bi];
                const Probe pr = probe_full(env, f, w.gen, cap);
                if (!pr.visited) {
                    best_i = bi;
                    best_d = bd;
                    slot = pr.slot;
                    fnew = f;
                    break;
                }
                exclude<R>(excl, bi, lane);
            }
        }
        for (; best_i < 0;) {
            int d0, i0, d1, i1;
            warp_argmin<R>(dl, excl, v0, pcls, d0, i0);
            if (i0 < 0) break;
            uint32_t ex1 = excl;
            exclude<R>(ex1, i0, lane);
            warp_argmin<R>(dl, ex1, v0, pcls, d1, i1);
            const int half = lane & 15;
            const int mine = lane < 16 ? i0 : i1;
            bool hit = false, match = false;
            if (mine >= 0 && half < cap) {
                const uint64_t f = w.fp ^ env.zk[mine];
                const uint64_t e = env.T[(f + (uint64_t)half) & env.tmask];
                match = e == ((f & ~kGenMask) | w.gen);
                hit = ((e & kGenMask) != w.gen) || match;
            }
            const unsigned bal = __ballot_sync(kFull, hit);
            const int cand[2] = {i0, i1};
            const int cdl[2] = {d0, d1};
            bool chosen = false;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (cand[g] < 0) break;
                const uint64_t fg = w.fp ^ env.zk[cand[g]];
                const unsigned b = (bal >> (16 * g)) & 0xFFFFu;
                Probe pr;
                if (b) {
                    const int fl = __ffs(b) - 1;
                    pr.visited = __shfl_sync(kFull, match ? 1 : 0, 16 * g + fl) != 0;
                    pr.slot = (int64_t)((fg + (uint64_t)fl) & env.tmask);
                } else if (cap > 16) {
                    pr = probe_full(env, fg, w.gen, cap);
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
                exclude<R>(excl, cand[g], lane);
            }
            if (chosen) break;
        }

        w.steps += 1;
        int code;
        if (best_i < 0) {
            // Every neighbour is in HT: restart without a move.
            w.blocked += 1;
            restart_walker(env, w, base, SL, V);
            p_direct<R>(V, n, lane, P);
            code = LABS_TRACE_BLOCKED;
        } else {
            // S <- S_f: table, P and rows (all from the values before the flip).
            const int pb = best_i & 1, vb = best_i >> 1;
            int* Ab = pb ? V.A1 : V.A0;
            const int as = Ab[vb];
            const bool centre = best_i == c;
            const int vq = n - 1 - vb - pb;
            int dd[R];
#pragma unroll
            for (int t = 0; t < R; ++t) {  // lags 2m, m = lane+1+32t < n (n <= 32 R)
                const int m = lane + 1 + kWarp * t;
                dd[t] = 0;
                if (m < n) {
                    int up = Ab[vb + m];
                    if (!centre && vb + m == vq) up = 0;
                    const int dn = Ab[vb - m];
                    dd[t] = (centre ? -2 : -4) * as * (up + dn);
                }
            }
            p_update<R>(V, n, lane, P, pb, vb, centre ? -1 : vq);
            __syncwarp();
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int m = lane + 1 + kWarp * t;
                if (m < n) {
                    V.E[m] += dd[t];
                    if (m <= kEPad) V.E[-m] += dd[t];
                }
            }
            if (lane == 0) {
                Ab[vb] = -as;
                if (!centre) Ab[vq] = -Ab[vq];
            }
            const bool stored = slot >= 0;
            if (lane == 0 && stored) env.T[slot] = (fnew & ~kGenMask) | w.gen;
            if (lane == (best_i >> 5)) w.word ^= 1u << (best_i & 31);
            __syncwarp();
            w.fp = fnew;
            w.isl += best_d;
            if (!stored) w.overflows += 1;
            note_best(env, w);
            if (w.isl < w.since) {
                w.since = w.isl;
                w.stag = 0;
            } else {
                w.stag += 1;
            }
            code = best_i;
            if (w.stag >= env.patience || !stored) {
                restart_walker(env, w, base, SL, V);
                p_direct<R>(V, n, lane, P);
                code |= LABS_TRACE_RESTART;
            }
        }
        if (trace_slot >= 0 && lane == 0) {
            const int64_t t = w.steps - 1 - trace_start;
            if (t >= 0 && t < p.status->trace_capacity) {
                p.status->trace_code[trace_slot * p.status->trace_capacity + t] = code;
                p.status->trace_isl[trace_slot * p.status->trace_capacity + t] = w.isl;
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

__device__ void save_walker(WalkerState* st, const Walker& w, int lane)
{
    if (lane < kBitWords) st->cur[lane] = w.word;
    if (lane == 0) {
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

__device__ __forceinline__ int lanes_R(int n)
{
    return (((n + 1) >> 1) + 15) >> 4;
}

template <int R>
__device__ void run_chunk(const WalkEnv& env, Walker& w, int64_t until, int* base, const WarpSmem& SL,
                          const View& V, int trace_slot, int64_t trace_start, const StepExtras& ex)
{
    walk_steps<R>(env, w, until, base, SL, V, trace_slot, trace_start, ex);
}

// One launch advances every walker by up to chunk_steps steps toward the target.  The
// kernel is compiled for a largest lane block RMAX (register allocation follows it);
// walkers whose n needs RMAX-1 or fewer outputs per lane run with RMAX-1, which covers
// them (any R >= lanes_R(n) computes the same values).
template <int RMAX>
__global__ void __launch_bounds__(256, LABS_WALK_MIN_BLOCKS) walk_chunk_kernel(KParams p, int chunk_index)
{
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = warp_smem(p.n_max);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const int64_t target = p.status->target_steps;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&p.queue[chunk_index], 1u);
        const int64_t wi = (int64_t)__shfl_sync(kFull, t, 0);
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
        {
            uint64_t* zs = reinterpret_cast<uint64_t*>(base + SL.zoff);
            const uint64_t* zg = p.zkeys + G.zkey_off;
            for (int i = lane; i < G.n; i += kWarp) zs[i] = zg[i];
            env.zk = zs;
            __syncwarp();
        }
        env.st = st;
        env.L = G.L;
        env.n = G.n;
        env.patience = p.patience > 0 ? p.patience : 2 * G.n;
        env.lane = lane;
        env.g = (uint32_t)wi;
        Walker w;
        load_walker(st, w, lane);
        const int trace_slot = st->trace_slot;
        const int64_t trace_start = trace_slot >= 0 ? p.trace_start[trace_slot] : 0;
        const int isl = load_rows(base, SL, V, w.word, G.L, G.n, lane);
        if (isl != w.isl) {
            if (lane == 0) raise_error(p.status, LABS_ESTATE, (int)wi);
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
        if (S->learned) {
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
        if (RMAX == 1 || lanes_R(G.n) == RMAX)
            run_chunk<RMAX>(env, w, until, base, SL, V, trace_slot, trace_start, ex);
        else
            run_chunk<(RMAX > 1 ? RMAX - 1 : 1)>(env, w, until, base, SL, V, trace_slot, trace_start, ex);
        save_walker(st, w, lane);
        __syncwarp();
    }
}

// Start of every walker (restart index 0, HT generation 1; HT zeroed by the caller).
__global__ void __launch_bounds__(512) reset_kernel(KParams p)
{
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = warp_smem(p.n_max);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; wi < p.W; wi += nwarps) {
        int gidx = 0;
        for (int g = 0; g < p.nG; ++g)
            if (wi >= p.groups[g].first && wi < p.groups[g].first + p.groups[g].count) gidx = g;
        const DevGroup G = p.groups[gidx];
        WalkerState* st = p.states + wi;
        WalkEnv env;
        env.p = &p;
        env.tmask = (1ull << p.tabu_log2) - 1ull;
        env.T = p.tabu + ((uint64_t)wi << p.tabu_log2);
        env.zk = p.zkeys + G.zkey_off;
        env.st = st;
        env.L = G.L;
        env.n = G.n;
        env.patience = p.patience > 0 ? p.patience : 2 * G.n;
        env.lane = lane;
        env.g = (uint32_t)wi;
        env.slot = nullptr;
        env.slot_valid = nullptr;
        env.rdump = nullptr;
        env.rdump_idx = nullptr;
        env.rdump_count = nullptr;
        env.dump_cap = 0;
        Walker w;
        w.restart_idx = 0;
        w.gen = 1;
        w.restarts = w.overflows = w.blocked = 0;
        w.steps = 0;
        w.best_isl = INT_MAX;
        w.best_step = 0;
        w.target_step = -1;
        start_walker(env, w, base, SL, V);
        save_walker(st, w, lane);
        if (lane == 0) {
            st->group = gidx;
            st->trace_slot = -1;
        }
        __syncwarp();
    }
}

__global__ void prep_walk_kernel(DevStatus* st, uint32_t* queue, int64_t steps, int nchunks)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->target_steps += steps;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nchunks; j += gridDim.x * blockDim.x)
        queue[j] = 0u;
}

__global__ void zobrist_kernel(uint64_t* zkeys, int64_t off, int L, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c0 = (uint32_t)i, c1 = (uint32_t)L, c2 = 0u, c3 = 2u;
    philox(c0, c1, c2, c3, kZobristKey0, kZobristKey1);
    zkeys[off + i] = (uint64_t)c0 | ((uint64_t)c1 << 32);
}

// --------------------------------------------------------- batch kernels (rows)

// Eq. 2 for arbitrary +-1 rows, one warp per row.
__global__ void __launch_bounds__(256) isl_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                  int32_t* __restrict__ out, DevStatus* status)
{
    extern __shared__ __align__(16) int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int stride = (L + 3) & ~3;
    int* s = smem + warp * stride;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; row < batch; row += nwarps) {
        const int8_t* src = seqs + row * (int64_t)L;
        bool ok = true;
        for (int j = lane; j < L; j += kWarp) {
            const int v = src[j];
            ok = ok && (v == 1 || v == -1);
            s[j] = v;
        }
        __syncwarp();
        const bool all_ok = __all_sync(kFull, ok);
        int part = 0;
        if (all_ok) {
            for (int k = 1 + lane; k < L; k += kWarp) {
                int ck = 0;
                for (int j = 0; j + k < L; ++j) ck += s[j] * s[j + k];
                part += ck * ck;
            }
        }
        const int e = __reduce_add_sync(kFull, part);
        if (lane == 0) {
            out[row] = all_ok ? e : -1;
            if (!all_ok && status) atomicAdd(&status->invalid_rows, 1);
        }
        __syncwarp();
    }
}

template <int R>
__device__ void delta_row(const View& V, int n, int lane, int32_t* dst)
{
    int dl[R];
    {
        int X[R], P[R];
        toeplitz<R>(V, n, lane, X);
        p_direct<R>(V, n, lane, P);
        assemble<R>(V, n, lane, X, P, dl);
    }
    const int p = lane >> 4, v0 = (lane & 15) * R;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (dl[r] != INT_MAX) dst[2 * (v0 + r) + p] = dl[r];
}

// The neighbourhood of Algorithm 1 for skew-symmetric rows, one warp per row, R
// outputs per lane (R = lanes_R(n), chosen by the host).
template <int R>
__global__ void __launch_bounds__(256) delta_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                    int32_t* __restrict__ out, DevStatus* status)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = warp_smem(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; row < batch; row += nwarps) {
        clear_warp(base, SL, lane);
        const int8_t* src = seqs + row * (int64_t)L;
        bool ok = true;
        for (int j = lane; j < L; j += kWarp) {
            const int v = src[j];
            ok = ok && (v == 1 || v == -1);
            if (j & 1) V.A1[j >> 1] = v;
            else V.A0[j >> 1] = v;
        }
        __syncwarp();
        for (int j = 1 + lane; j <= c; j += kWarp) {  // Eq. 4
            const int hi = c + j, lo = c - j;
            const int shi = (hi & 1) ? V.A1[hi >> 1] : V.A0[hi >> 1];
            const int slo = (lo & 1) ? V.A1[lo >> 1] : V.A0[lo >> 1];
            ok = ok && (shi == ((j & 1) ? -slo : slo));
        }
        int32_t* dst = out + row * (int64_t)n;
        if (!__all_sync(kFull, ok)) {
            for (int i = lane; i < n; i += kWarp) dst[i] = INT_MIN;
            if (lane == 0 && status) atomicAdd(&status->invalid_rows, 1);
            __syncwarp();
            continue;
        }
        build_table(V, n, lane);
        delta_row<R>(V, n, lane, dst);
        __syncwarp();
    }
}

// --------------------------------------------------- learned proposal support

// Network inputs of states given by their free-variable bits (8 words each, `stride`
// words apart): x[b][0][i] = s_i, x[b][1][i] = C_{2(i+1)}/sqrt(L) (0 for i = n-1),
// x[b][2][i] = dISL_i/(8L).  One warp per state.
template <int R>
__device__ void features_row(const View& V, int n, int L, int lane, float* xb)
{
    int dl[R];
    {
        int X[R], P[R];
        toeplitz<R>(V, n, lane, X);
        p_direct<R>(V, n, lane, P);
        assemble<R>(V, n, lane, X, P, dl);
    }
    const int p = lane >> 4, v0 = (lane & 15) * R;
    const float inv8L = (float)(8 * L);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (dl[r] != INT_MAX) xb[2 * n + 2 * (v0 + r) + p] = (float)dl[r] / inv8L;
}

__global__ void __launch_bounds__(256) features_kernel(const uint32_t* __restrict__ bits, int64_t stride,
                                                       int64_t count, int L, float* __restrict__ x)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2;
    const WarpSmem SL = warp_smem(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const float sq = sqrtf((float)L);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; b < count; b += nwarps) {
        const uint32_t word = lane < kBitWords ? bits[b * stride + lane] : 0u;
        load_rows(base, SL, V, word, L, n, lane);
        float* xb = x + b * 3 * n;
        for (int i = lane; i < n; i += kWarp) {
            xb[i] = (float)((i & 1) ? V.A1[i >> 1] : V.A0[i >> 1]);
            xb[n + i] = i < n - 1 ? (float)V.E[i + 1] / sq : 0.f;
        }
        switch (lanes_R(n)) {
            case 1: features_row<1>(V, n, L, lane, xb); break;
            case 2: features_row<2>(V, n, L, lane, xb); break;
            case 3: features_row<3>(V, n, L, lane, xb); break;
            case 4: features_row<4>(V, n, L, lane, xb); break;
            case 5: features_row<5>(V, n, L, lane, xb); break;
            case 6: features_row<6>(V, n, L, lane, xb); break;
            case 7: features_row<7>(V, n, L, lane, xb); break;
            default: features_row<8>(V, n, L, lane, xb); break;
        }
        __syncwarp();
    }
}

// Restart candidates of walkers [first, first+count) of one length: candidate 0 is the
// walker's own next random start (what the plain walk would use); candidates c >= 1
// perturb the walker's best state by flipping r = 1 + (u mod max(1, n/8)) free
// variables drawn by Philox (key = seed, counter = (walker, next restart index,
// c << 16 | t, 1)).  Output bits [count][P][8].
__global__ void candidates_kernel(KParams p, int64_t first, int64_t count, int n, int P, uint32_t* __restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count * P;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = first + t / P;
        const int c = (int)(t % P);
        const WalkerState& st = p.states[w];
        const uint32_t ridx = st.restart_idx + 1;
        uint32_t bits[kBitWords];
        if (c == 0) {
#pragma unroll
            for (int j = 0; j < kBitWords; ++j) bits[j] = start_word(p.seed, (uint32_t)w, ridx, j, n);
        } else {
#pragma unroll
            for (int j = 0; j < kBitWords; ++j) bits[j] = st.best[j];
            uint32_t c0 = (uint32_t)w, c1 = ridx, c2 = (uint32_t)c << 16, c3 = 1u;
            philox(c0, c1, c2, c3, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
            const int r = 1 + (int)(c0 % (uint32_t)max(1, n / 8));
            for (int k = 0; k < r; ++k) {
                uint32_t d0 = (uint32_t)w, d1 = ridx, d2 = ((uint32_t)c << 16) | (uint32_t)(k + 1), d3 = 1u;
                philox(d0, d1, d2, d3, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
                const int i = (int)(d0 % (uint32_t)n);
#pragma unroll
                for (int j = 0; j < kBitWords; ++j)
                    if (j == (i >> 5)) bits[j] ^= 1u << (i & 31);
            }
        }
#pragma unroll
        for (int j = 0; j < kBitWords; ++j) out[t * kBitWords + j] = bits[j];
    }
}

// Per walker: the candidate with the highest restart score (ties: lowest c) becomes the
// walker's proposed restart state.
__global__ void select_kernel(KParams p, int64_t first, int64_t count, int P, const float* __restrict__ score,
                              const uint32_t* __restrict__ cand)
{
    DevStatus* S = p.status;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        int best = 0;
        for (int c = 1; c < P; ++c)
            if (score[t * P + c] > score[t * P + best]) best = c;
        const int64_t w = first + t;
#pragma unroll
        for (int j = 0; j < kBitWords; ++j) S->l_slot[w * kBitWords + j] = cand[(t * P + best) * kBitWords + j];
        S->l_slot_valid[w] = 1;
    }
}

// Flip scores of walkers [first, first+count) for their current step.
__global__ void scores_kernel(KParams p, int64_t first, int64_t count, int n, const float* __restrict__ score)
{
    DevStatus* S = p.status;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = first + t / n;
        const int i = (int)(t % n);
        S->l_scores[w * p.n_max + i] = score[t];
        if (i == 0) S->l_score_step[w] = p.states[w].steps_done;
    }
}

// Training labels of log records: target = the flip of the first step (0 when the step
// moved nowhere), wf = 1 when the ISL fell below the start ISL later in the chunk,
// y = L^2 / (2 min_isl) / 8 (the merit factor reached, scaled).
__global__ void labels_kernel(const labs_log_record* __restrict__ rec, int64_t count, int32_t* __restrict__ target,
                              float* __restrict__ y, float* __restrict__ wf)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const labs_log_record r = rec[t];
        const bool moved = r.first >= 0;
        target[t] = moved ? (r.first & 0xFFFF) : 0;
        wf[t] = (moved && r.min_isl < r.isl) ? 1.f : 0.f;
        y[t] = (float)r.L * (float)r.L / (2.f * (float)r.min_isl) / 8.f;
    }
}

// ------------------------------------------------------------ reductions, tracing

__global__ void best_kernel(KParams p, int L)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < p.W;
         wi += (int64_t)gridDim.x * blockDim.x) {
        const WalkerState& st = p.states[wi];
        if (L != 0 && p.groups[st.group].L != L) continue;
        const unsigned long long key = ((unsigned long long)(uint32_t)st.best_isl << 32) |
                                       (unsigned long long)(uint32_t)wi;
        atomicMin(&p.status->best_key, key);
    }
}

__global__ void stats_kernel(KParams p, int L)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < p.W;
         wi += (int64_t)gridDim.x * blockDim.x) {
        const WalkerState& st = p.states[wi];
        const DevGroup& G = p.groups[st.group];
        if (L != 0 && G.L != L) continue;
        DevStatus* s = p.status;
        atomicAdd(&s->st_steps, (unsigned long long)st.steps_done);
        atomicAdd(&s->st_evals, (unsigned long long)st.steps_done * (unsigned long long)G.n);
        atomicAdd(&s->st_restarts, (unsigned long long)st.restarts);
        atomicAdd(&s->st_overflows, (unsigned long long)st.overflows);
        atomicAdd(&s->st_blocked, (unsigned long long)st.blocked);
        if (st.target_step >= 0) {
            atomicAdd(&s->st_at_target, 1ull);
            atomicMin(&s->st_target_step, (long long)st.target_step);
        }
        const unsigned long long key = ((unsigned long long)(uint32_t)st.best_isl << 32) |
                                       (unsigned long long)(uint32_t)wi;
        atomicMin(&s->best_key, key);
    }
}

__global__ void trace_clear_kernel(KParams p)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < p.W;
         wi += (int64_t)gridDim.x * blockDim.x)
        p.states[wi].trace_slot = -1;
}

__global__ void trace_set_kernel(KParams p, const int64_t* ids, int k, int32_t* code, int32_t* isl,
                                 int64_t capacity)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        p.status->trace_code = code;
        p.status->trace_isl = isl;
        p.status->trace_capacity = capacity;
    }
    if (j < k) {
        const int64_t wi = ids[j];
        p.states[wi].trace_slot = j;
        p.trace_start[j] = p.states[wi].steps_done;
    }
}

__global__ void time_probe_kernel(unsigned long long* out)
{
    *out = global_ns();
}

int status_of(cudaError_t e)
{
    return e == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

}  // namespace

// ------------------------------------------------------------------- launchers

int launch_zobrist(const KParams&, uint64_t* zkeys, const DevGroup* host_groups, int nG, void* stream)
{
    for (int g = 0; g < nG; ++g) {
        const DevGroup& G = host_groups[g];
        zobrist_kernel<<<(G.n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(zkeys, G.zkey_off, G.L, G.n);
    }
    return status_of(cudaGetLastError());
}

int launch_reset(const KParams& p, int grid, int block, void* stream)
{
    const size_t smem = (size_t)(block / kWarp) * warp_smem(p.n_max).words * sizeof(int);
    cudaFuncSetAttribute(reset_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    reset_kernel<<<grid, block, smem, (cudaStream_t)stream>>>(p);
    return status_of(cudaGetLastError());
}

int launch_prep_walk(const KParams& p, int64_t steps, int nchunks, void* stream)
{
    prep_walk_kernel<<<(nchunks + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p.status, p.queue, steps,
                                                                              nchunks);
    return status_of(cudaGetLastError());
}

using WalkFn = void (*)(KParams, int);
static WalkFn walk_fn(int rmax)
{
    switch (rmax) {
        case 1: return walk_chunk_kernel<1>;
        case 2: return walk_chunk_kernel<2>;
        case 3: return walk_chunk_kernel<3>;
        case 4: return walk_chunk_kernel<4>;
        case 5: return walk_chunk_kernel<5>;
        case 6: return walk_chunk_kernel<6>;
        case 7: return walk_chunk_kernel<7>;
        default: return walk_chunk_kernel<8>;
    }
}

int lanes_for(int n)
{
    return (((n + 1) >> 1) + 15) >> 4;
}

int walk_kernel_config(int rmax, int warps_per_cta, size_t smem_bytes, int* ctas_per_sm, int* regs)
{
    const WalkFn fn = walk_fn(rmax);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return LABS_ECUDA;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return LABS_ECUDA;
    if (regs) *regs = fa.numRegs;
    if (warps_per_cta * kWarp > fa.maxThreadsPerBlock) {
        *ctas_per_sm = 0;
        return LABS_EINVAL;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, warps_per_cta * kWarp, smem_bytes);
    return status_of(e);
}

int launch_walk_chunk(const KParams& p, int chunk_index, int grid, int warps_per_cta, size_t smem_bytes,
                      void* stream)
{
    const WalkFn fn = walk_fn(p.rmax);
    fn<<<grid, warps_per_cta * kWarp, smem_bytes, (cudaStream_t)stream>>>(p, chunk_index);
    return status_of(cudaGetLastError());
}

static int row_grid(int64_t batch, int warps)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t need = (batch + warps - 1) / warps;
    int64_t cap = (int64_t)sms * 8;
    return (int)(need < cap ? need : cap);
}

int launch_isl(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status, void* stream)
{
    if (batch == 0) return LABS_OK;
    const int warps = 8;
    const size_t smem = (size_t)warps * ((L + 3) & ~3) * sizeof(int);
    isl_kernel<<<row_grid(batch, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out,
                                                                                       status);
    return status_of(cudaGetLastError());
}

int launch_delta(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status, void* stream)
{
    if (batch == 0) return LABS_OK;
    const int warps = 8;
    const size_t smem = (size_t)warps * warp_smem((L + 1) / 2).words * sizeof(int);
    using DeltaFn = void (*)(const int8_t*, int64_t, int, int32_t*, DevStatus*);
    DeltaFn fn;
    switch (lanes_for((L + 1) / 2)) {
        case 1: fn = delta_kernel<1>; break;
        case 2: fn = delta_kernel<2>; break;
        case 3: fn = delta_kernel<3>; break;
        case 4: fn = delta_kernel<4>; break;
        case 5: fn = delta_kernel<5>; break;
        case 6: fn = delta_kernel<6>; break;
        case 7: fn = delta_kernel<7>; break;
        default: fn = delta_kernel<8>; break;
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<row_grid(batch, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out, status);
    return status_of(cudaGetLastError());
}

int launch_best(const KParams& p, int32_t L, void* stream)
{
    best_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
    return status_of(cudaGetLastError());
}

int launch_stats(const KParams& p, int32_t L, void* stream)
{
    stats_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
    return status_of(cudaGetLastError());
}

int launch_trace_arm(const KParams& p, const int64_t* dev_ids, int32_t k, int32_t* code, int32_t* isl,
                     int64_t capacity, void* stream)
{
    trace_clear_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p);
    trace_set_kernel<<<(k + 255) / 256 + 1, 256, 0, (cudaStream_t)stream>>>(p, dev_ids, k, code, isl, capacity);
    return status_of(cudaGetLastError());
}

int launch_features(const uint32_t* bits, int64_t stride, int64_t count, int32_t L, float* x, void* stream)
{
    if (count == 0) return LABS_OK;
    const int warps = 8;
    const size_t smem = (size_t)warps * warp_smem((L + 1) / 2).words * sizeof(int);
    cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    features_kernel<<<row_grid(count, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(bits, stride, count, L, x);
    return status_of(cudaGetLastError());
}

int launch_candidates(const KParams& p, int64_t first, int64_t count, int n, int P, uint32_t* out, void* stream)
{
    candidates_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, first, count, n, P, out);
    return status_of(cudaGetLastError());
}

int launch_select(const KParams& p, int64_t first, int64_t count, int P, const float* score, const uint32_t* cand,
                  void* stream)
{
    select_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, first, count, P, score, cand);
    return status_of(cudaGetLastError());
}

int launch_scores(const KParams& p, int64_t first, int64_t count, int n, const float* score, void* stream)
{
    scores_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, first, count, n, score);
    return status_of(cudaGetLastError());
}

int launch_labels(const labs_log_record* rec, int64_t count, int32_t* target, float* y, float* wf, void* stream)
{
    labels_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(rec, count, target, y, wf);
    return status_of(cudaGetLastError());
}

int launch_time_probe(unsigned long long* dev_out, void* stream)
{
    time_probe_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(dev_out);
    return status_of(cudaGetLastError());
}

}  // namespace labsgpu
