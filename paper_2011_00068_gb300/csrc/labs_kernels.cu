// labs_kernels.cu -- sm_103a kernels of the skew-symmetric LABS search
// (Brest & Boskovic, arXiv 2011.00068): walker starts, the stateless row kernels
// (ISL, neighbourhood), learned-proposal support, reductions and the launchers.
// The walk itself is in labs_device.cuh, instantiated by the labs_walk*.cu units.
#include <algorithm>

#include "labs_async.cuh"
#include "labs_device.cuh"

namespace labsgpu {

namespace {

// Start of every walker (restart index 0, HT generation 1; HT zeroed by the caller).
__global__ void __launch_bounds__(512) reset_kernel(KParams p)
{
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = warp_smem(p.n_max, 32);
    const Tile<32> t(threadIdx.x & 31);
    const int warp = threadIdx.x >> 5;
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
        PslTrack ps;
        ps.best_psl = INT_MAX;
        start_walker(env, w, base, SL, V, t, false, p.mode == 3 ? &ps : nullptr);
        save_walker(st, w, t.lane);
        if (p.best_first) p.pq_key[wi * LABS_QUEUE_SIZE + t.lane] = ~0ull;  // empty queue
        if (t.lane == 0) {
            st->group = gidx;
            st->trace_slot = -1;
            st->psl = p.mode == 3 ? ps.psl : -1;
            st->best_psl = p.mode == 3 ? ps.best_psl : -1;
            st->since_psl = p.mode == 3 ? ps.since_psl : -1;
        }
        t.sync();
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
        long long part = 0;
        if (all_ok) {
            for (int k = 1 + lane; k < L; k += kWarp) {
                int ck = 0;
                for (int j = 0; j + k < L; ++j) ck += s[j] * s[j + k];
                part += (long long)ck * ck;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        if (lane == 0) {
            // an ISL above INT32_MAX (long rows only) is reported as -2 with LABS_ERANGE
            out[row] = !all_ok ? -1 : part > INT_MAX ? -2 : (int32_t)part;
            if (!all_ok && status) atomicAdd(&status->invalid_rows, 1);
            if (all_ok && part > INT_MAX && status) raise_error(status, LABS_ERANGE, (int)row);
        }
        __syncwarp();
    }
}

// ------------------------------------------ stateless rows (labs_neighbor_delta)
//
// A row kernel sees each input row once, so it builds everything from the row itself:
//   - the two parity classes as bit vectors held in registers (NW words each, bit u of
//     class p set <=> A_p[u] = -1), from warp ballots of the row's bytes, while the
//     bytes also go to the float rows A0/A1 that the Toeplitz product reads;
//   - the Eq. 4 check on those words: class p of a skew-symmetric row is a palindrome
//     when c + p is even and an antipalindrome when it is odd (entries u and n_p-1-u are
//     positions c-j and c+j of the sequence), so its bit vector reversed over its n_p
//     bits equals itself, or itself with every bit inverted;
//   - the even-lag table C_{2m} = C0_m + C1_m, C^{(p)}_m = (n_p - m) - 2 #{u : a_u !=
//     a_{u+m}}, from popcounts of class words against the class shifted by m;
//   - P without a pass of its own: with a_{n_p-1-u} = s_p a_u (s_p = +-1 as above), the
//     pairs (v+m, v-m), m = 1..v, of P_v are the upper half of the pairs of the class's
//     lag d = n_p-1-2v, whose lower half repeats them term by term and whose middle pair
//     (v, n_p-1-v) has product s_p; so C^{(p)}_d = 2 s_p P_v + s_p, i.e.
//     P_v = (s_p C^{(p)}_d - 1) / 2.  Lag m serves the class with n_p - 1 = m (mod 2),
//     p = (c - m) & 1, whose sign is then s_p = (-1)^m; the lane that counts lag m
//     stores that class's P value in Q[m], and the lane of output v reads Q[n_p-1-2v].
// Then the Toeplitz product and the assembly as in the walk.

// Row `src` (has = false: no row for this lane group) into A_p[u] (floats) and the
// class words x0/x1.  TILE lanes per row (16: two rows per warp; 32: one); lane l reads
// class l / (TILE/2), entries u = (TILE/2) it + l % (TILE/2).  With STAGED, bytes j <
// lim of the row are read from its staged copy stg (shared memory), the rest from src.
// Returns true when a byte of this lane is not +-1.
// HALF: the rows are FP16 (hrow: class 0's entry 0; class 1 lies hstride halves further).
template <int TILE, int NW, bool STAGED, bool HALF = false>
__device__ __forceinline__ bool row_load(const View& V, const int8_t* __restrict__ src, const int8_t* stg,
                                         int64_t lim, bool has, int L, int lane, int h, uint32_t (&x0)[NW],
                                         uint32_t (&x1)[NW], __half* hrow = nullptr, int hstride = 0)
{
    constexpr int G = TILE / 2;               // lanes per class
    constexpr int IT = 32 / G;                // ballots per class word
    const int p = lane / G, e = lane % G;
    float* A = p ? V.A1 : V.A0;
    __half* H = hrow + p * hstride;
    uint32_t bad = 0u;  // v in {1, -1} <=> (v + 1) & ~2 == 0
    // rows held whole by the staging buffer (all but the input's last few bytes) read
    // shared memory only; the choice is the same for the whole warp
    const bool whole = STAGED && __all_sync(kFull, has && lim >= L);
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        uint32_t bl[IT];
#pragma unroll
        for (int tt = 0; tt < IT; ++tt) {
            bl[tt] = 0u;
            // only the last word's rounds can lie wholly past the row (n > 32 (NW - 1))
            if (k == NW - 1 && 2 * G * (IT * k + tt) >= L) continue;  // uniform
            const int u = G * (IT * k + tt) + e, j = 2 * u + p;
            int v = 1;
            if (whole) {
                // every row exists, and rounds below the last word lie inside the row
                if (k < NW - 1 || j < L) {
                    v = stg[j];
                    if constexpr (HALF)
                        H[u] = __int2half_rn(v);
                    else
                        A[u] = (float)v;
                }
            } else if (has && j < L) {
                v = (STAGED && j < lim) ? stg[j] : src[j];
                if constexpr (HALF)
                    H[u] = __int2half_rn(v);
                else
                    A[u] = (float)v;
            }
            bad |= (uint32_t)(v + 1) & ~2u;
            bl[tt] = __ballot_sync(kFull, v < 0);
        }
        if constexpr (TILE == 16) {
            // ballot bit 16h + 8p + e: byte 2h + p of the four ballots, in order
            const uint32_t s0 = (uint32_t)(((4 + 2 * h) << 4) | (2 * h)), s1 = s0 + 0x11u;
            x0[k] = __byte_perm(__byte_perm(bl[0], bl[1], s0), __byte_perm(bl[2], bl[3], s0), 0x5410);
            x1[k] = __byte_perm(__byte_perm(bl[0], bl[1], s1), __byte_perm(bl[2], bl[3], s1), 0x5410);
        } else {
            // ballot bit 16p + e: half p of the two ballots
            x0[k] = __byte_perm(bl[0], bl[1], 0x5410);
            x1[k] = __byte_perm(bl[0], bl[1], 0x7632);
        }
    }
    return bad != 0u;
}

// Bits of class entries below np in word k.
__device__ __forceinline__ uint32_t class_mask(int np, int k)
{
    const int w = np - 32 * k;
    return w >= 32 ? ~0u : (w <= 0 ? 0u : (1u << w) - 1u);
}

// xr = x reversed over its np bits (bit t of xr = bit np-1-t of x), np >= 32 (NW-1).
template <int NW>
__device__ __forceinline__ void reverse_class(const uint32_t (&x)[NW], int np, uint32_t (&xr)[NW])
{
    uint32_t rv[NW + 1];
#pragma unroll
    for (int k = 0; k < NW; ++k) rv[k] = __brev(x[NW - 1 - k]);
    rv[NW] = 0u;
    const int sh = 32 * NW - np;  // 0 .. 32
#pragma unroll
    for (int k = 0; k < NW; ++k) xr[k] = __funnelshift_rc(rv[k], rv[k + 1], sh);
}

// The table E (set_E) and Q from the class words; lane `lane` of TILE counts the lags
// m = 32q + lane + TILE j (q < NW, j < 32/TILE) of both classes.  Mismatches of lag m
// over the valid pairs u < n_p - m: over the first NW - q words against the class
// shifted by m, plus the set bits of the words beyond (positions whose partner lies
// past the vector), minus the set bits of the top m entries (partners past the class,
// counted as mismatches by the shifted words) = the reversed class's first m bits.
template <int TILE, int NW>
__device__ __forceinline__ void row_table(const View& V, float* __restrict__ Q, int n, int lane,
                                          const uint32_t (&x0)[NW], const uint32_t (&x1)[NW],
                                          const uint32_t (&xr0)[NW], const uint32_t (&xr1)[NW])
{
    const int n1 = n - 1;
    int pre0[NW], pre1[NW], suf0[NW + 1], suf1[NW + 1];
    pre0[0] = pre1[0] = 0;
#pragma unroll
    for (int k = 1; k < NW; ++k) {
        pre0[k] = pre0[k - 1] + __popc(xr0[k - 1]);
        pre1[k] = pre1[k - 1] + __popc(xr1[k - 1]);
    }
    suf0[NW] = suf1[NW] = 0;
#pragma unroll
    for (int k = NW - 1; k >= 0; --k) {
        suf0[k] = suf0[k + 1] + __popc(x0[k]);
        suf1[k] = suf1[k + 1] + __popc(x1[k]);
    }
    // mismatch counts of lag 32q + r start from the words beyond the shift and the
    // top-entry correction; those parts not depending on r are shared by both j
    int base0[NW], base1[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        base0[q] = suf0[NW - q] - pre0[q];
        base1[q] = suf1[NW - q] - pre1[q];
    }
#pragma unroll
    for (int j = 0; j < 32 / TILE; ++j) {
        const int r = lane + TILE * j;  // < 32
        const uint32_t low = (1u << r) - 1u;
        // lag m = 32q + r has the parity of r: Q[m] belongs to class (n1 - r) & 1, sign (-1)^r
        const bool use1 = ((n1 - r) & 1) != 0;
        const float half = (r & 1) ? -0.5f : 0.5f;
        uint32_t s0[NW], s1[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            s0[k] = __funnelshift_r(x0[k], k + 1 < NW ? x0[k + 1] : 0u, r);
            s1[k] = __funnelshift_r(x1[k], k + 1 < NW ? x1[k + 1] : 0u, r);
        }
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int m = 32 * q + r;
            int t0 = base0[q] - __popc(xr0[q] & low);
            int t1 = base1[q] - __popc(xr1[q] & low);
#pragma unroll
            for (int k = 0; k + q < NW; ++k) {
                t0 += __popc(x0[k] ^ s0[k + q]);
                t1 += __popc(x1[k] ^ s1[k + q]);
            }
            // lags below the last word group exist in both classes (n1 >= 32 (NW - 1))
            if (q < NW - 1 || m < n) {
                const int c0 = (n - m) - 2 * t0;
                // class 1 has n1 = n - 1 entries: no pair at lag n - 1
                const int c1 = (q < NW - 1 || m < n1) ? (n1 - m) - 2 * t1 : 0;
                if (q > 0 || m > 0) {
                    // E[m] in both pairs that hold it and in the mirror half (the row
                    // layouts keep gpad >= n, so every mirror entry exists)
                    const float e = (float)(c0 + c1);
                    V.G[m].x = e;
                    V.G[m - 1].y = e;
                    V.G[-m].x = e;
                    V.G[-m - 1].y = e;
                }
                // Q[0] belongs to the centre, whose dISL has no P term
                Q[m] = fmaf(half, (float)(use1 ? c1 : c0), -0.5f);
            }
        }
    }
}

// P of the lane's R outputs from Q.
template <class TL, int R>
__device__ __forceinline__ void row_p(const float* __restrict__ Q, int n, const Outs<TL, R>& o, float (&P)[R])
{
    const int top = (o.p ? n - 2 : n - 1) - 2 * o.v0;  // n_p - 1 - 2 v0
#pragma unroll
    for (int r = 0; r < R; ++r) P[r] = Q[max(top - 2 * r, 0)];
}

// Staging of input rows: each warp copies the bytes of its next rows (rows r0 .. r0+k-1,
// global bytes [r0 L, (r0+k) L)) into one of two shared-memory buffers with one bulk
// copy while it evaluates the current rows from the other buffer.  A bulk copy moves
// 16-byte aligned blocks, so the copy covers [floor16(r0 L), ceil16((r0+k) L)), cut at
// the last 16-byte boundary of the input (the few bytes past it, and every byte when the
// input is not 16-byte aligned, are read from global memory directly).
__host__ __device__ inline int stage_bytes(int L, int rows)
{
    return (rows * L + 32 + 15) & ~15;
}

struct StageRange {
    int64_t a0, a1;  // staged global bytes [a0, a1); a1 <= a0: none
};

__device__ __forceinline__ StageRange stage_range(int64_t r0, int rows, int L, int64_t total)
{
    const int64_t e = min((r0 + rows) * (int64_t)L, total);
    StageRange g;
    g.a0 = (r0 * L) & ~(int64_t)15;
    g.a1 = min((e + 15) & ~(int64_t)15, total & ~(int64_t)15);
    return g;
}

// Issued by one lane: the copy of rows r0 .. r0+rows-1 into the buffer at shared address
// dst, counted on barrier bar (an arrival without bytes when nothing is staged).
__device__ __forceinline__ void stage_rows(const int8_t* seqs, int64_t r0, int rows, int L, int64_t total,
                                           uint32_t dst, uint32_t bar)
{
    const StageRange g = stage_range(r0, rows, L, total);
    fence_async_shared();  // earlier reads of the buffer come before the copy's writes
    if (g.a1 > g.a0) {
        const uint32_t bytes = (uint32_t)(g.a1 - g.a0);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(dst, seqs + g.a0, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

// The neighbourhood of Algorithm 1 for skew-symmetric rows, one warp per row (n > 160),
// R outputs per lane (R = block_R(n, 32)), NW = ceil(n/32) words per class; with
// STAGED, rows come through the staging buffers after the rows' shared memory.
template <int R, int NW, bool STAGED>
__global__ void __launch_bounds__(256) delta_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                    int32_t* __restrict__ out, DevStatus* status)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = row_smem(n, 32);
    const Tile<32> t(threadIdx.x & 31);
    const int lane = t.lane, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    float* Q = reinterpret_cast<float*>(base + SL.poff);
    const Outs<Tile<32>, R> o(t);
    // every row writes the same entries of the rows and the table: clear them once
    clear_rows(base, SL, t);
    const int SB = stage_bytes(L, 1);
    const int8_t* stg = reinterpret_cast<const int8_t*>(smem + (blockDim.x >> 5) * SL.words) + warp * (2 * SB + 16);
    const uint32_t sdst = smem_addr(stg), bar = sdst + 2 * SB;  // two buffers, then two barriers
    const int64_t total = batch * (int64_t)L;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t first = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (STAGED) {
        if (lane == 0) {
            mbar_init(bar, 1);
            mbar_init(bar + 8, 1);
            mbar_init_fence();
        }
        __syncwarp();
        if (lane == 0 && first < batch) stage_rows(seqs, first, 1, L, total, sdst, bar);
    }
    int it = 0;
    for (int64_t row = first; row < batch; row += nwarps, ++it) {
        const int b = it & 1;
        StageRange g{0, 0};
        if (STAGED) {
            const int64_t next = row + nwarps;
            const bool more = next < batch;
            if (lane == 0 && more) stage_rows(seqs, next, 1, L, total, sdst + (b ^ 1) * SB, bar + 8 * (b ^ 1));
            if (!__all_sync(kFull, mbar_wait(bar + 8 * b, (it >> 1) & 1))) {
                if (lane == 0 && status) raise_error(status, LABS_ECUDA, (int)row);
                if (more) mbar_wait(bar + 8 * (b ^ 1), ((it + 1) >> 1) & 1);  // the copy in flight
                return;
            }
            g = stage_range(row, 1, L, total);
        }
        const int64_t rs = row * (int64_t)L;
        uint32_t x0[NW], x1[NW], xr0[NW], xr1[NW];
        bool bad = row_load<32, NW, STAGED>(V, seqs + rs, stg + b * SB + (rs - g.a0), g.a1 - rs, true, L, lane, 0,
                                            x0, x1);
        reverse_class(x0, n, xr0);
        reverse_class(x1, n - 1, xr1);
        const uint32_t f0 = (c & 1) ? ~0u : 0u, f1 = ~f0;  // antipalindromic class: all bits inverted
        uint32_t diff = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            diff |= (xr0[k] ^ x0[k] ^ (f0 & class_mask(n, k))) | (xr1[k] ^ x1[k] ^ (f1 & class_mask(n - 1, k)));
        bad |= diff != 0;
        int32_t* dst = out + row * (int64_t)n;
        if (__any_sync(kFull, bad)) {
            for (int i = lane; i < n; i += kWarp) dst[i] = INT_MIN;
            if (lane == 0 && status) atomicAdd(&status->invalid_rows, 1);
            t.sync();
            continue;
        }
        row_table<32, NW>(V, Q, n, lane, x0, x1, xr0, xr1);
        t.sync();  // rows, table and Q written
        int dl[R];
        {
            float X[R], P[R];
            row_p(Q, n, o, P);
            toeplitz(V, n, o, X);
            assemble(V, n, o, X, P, dl);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (dl[r] != INT_MAX) dst[2 * (o.v0 + r) + o.p] = dl[r];
        t.sync();  // the next row overwrites the rows, the table, Q and this staging buffer
    }
}

// The same for two rows per warp (n <= 160), 16 lanes per row in lockstep: rows r0, r0+1
// of each warp; R = block_R(n, 16).  The rows' shared memory is cleared once, each row
// overwrites every entry the previous one set.
template <int R, int NW, bool STAGED>
__global__ void __launch_bounds__(256, R <= 7 ? 3 : 2) delta_pair_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                         int32_t* __restrict__ out, DevStatus* status)
{
    // n <= 128 (at most four class words): the Toeplitz product on the tensor cores over
    // FP16 rows (row_smem's tensor-core layout); above, the FP32 product
    constexpr bool TC = NW <= 4;
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = row_smem(n, 16);
    const Pair t(threadIdx.x & 31);
    const int lane = t.lane, wl = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = smem + (threadIdx.x / 16) * SL.words;
    const View V = make_view(base, SL);
    float* Q = reinterpret_cast<float*>(base + SL.poff);
    const Outs<Pair, R> o(t);
    clear_rows(base, SL, t);
    const int SB = stage_bytes(L, 2);
    const int8_t* stg = reinterpret_cast<const int8_t*>(smem + (blockDim.x >> 4) * SL.words) + warp * (2 * SB + 16);
    const uint32_t sdst = smem_addr(stg), bar = sdst + 2 * SB;
    const int64_t total = batch * (int64_t)L;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t first = 2 * ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp);
    if (STAGED) {
        if (wl == 0) {
            mbar_init(bar, 1);
            mbar_init(bar + 8, 1);
            mbar_init_fence();
        }
        __syncwarp();
        if (wl == 0 && first < batch) stage_rows(seqs, first, 2, L, total, sdst, bar);
    }
    int it = 0;
    for (int64_t r0 = first; r0 < batch; r0 += 2 * nwarps, ++it) {
        const int b = it & 1;
        StageRange g{0, 0};
        if (STAGED) {
            const int64_t next = r0 + 2 * nwarps;
            const bool more = next < batch;
            if (wl == 0 && more) stage_rows(seqs, next, 2, L, total, sdst + (b ^ 1) * SB, bar + 8 * (b ^ 1));
            if (!__all_sync(kFull, mbar_wait(bar + 8 * b, (it >> 1) & 1))) {
                if (wl == 0 && status) raise_error(status, LABS_ECUDA, (int)r0);
                if (more) mbar_wait(bar + 8 * (b ^ 1), ((it + 1) >> 1) & 1);  // the copy in flight
                return;
            }
            g = stage_range(r0, 2, L, total);
        }
        const int64_t row = r0 + t.h;
        const bool has = row < batch;
        const int64_t rs = row * (int64_t)L;
        uint32_t x0[NW], x1[NW], xr0[NW], xr1[NW];
        bool bad = row_load<16, NW, STAGED, TC>(V, seqs + rs, stg + b * SB + (rs - g.a0), g.a1 - rs, has, L, lane,
                                                t.h, x0, x1, reinterpret_cast<__half*>(base + SL.hoff) + SL.hpad,
                                                2 * SL.hlen);
        reverse_class(x0, n, xr0);
        reverse_class(x1, n - 1, xr1);
        const uint32_t f0 = (c & 1) ? ~0u : 0u, f1 = ~f0;
        uint32_t diff = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            diff |= (xr0[k] ^ x0[k] ^ (f0 & class_mask(n, k))) | (xr1[k] ^ x1[k] ^ (f1 & class_mask(n - 1, k)));
        bad |= diff != 0;
        // the ballot is a full-warp collective: both halves take it, with or without a row
        const unsigned any_bad = t.ballot(bad);
        const bool valid = has && any_bad == 0u;
        int32_t* dst = out + row * (int64_t)n;
        if (has && !valid) {
            for (int i = lane; i < n; i += 16) dst[i] = INT_MIN;
            if (lane == 0 && status) atomicAdd(&status->invalid_rows, 1);
        }
        row_table<16, NW>(V, Q, n, lane, x0, x1, xr0, xr1);
        t.sync();  // rows, table and Q written
        int dl[R];
        int rv;
        {
            float X[R], P[R];
            row_p(Q, n, o, P);
            if constexpr (TC) {
                __syncwarp();  // the product's results overwrite Q
                toeplitz_tc(V, SL, n, o, t.h, X);
                const __half* H = reinterpret_cast<const __half*>(base + SL.hoff + o.p * SL.hlen) + SL.hpad;
                rv = lane_dl_rows(H, V, n, o, X, P, dl);
            } else {
                toeplitz(V, n, o, X);
                rv = lane_dl(V, n, o, X, P, dl);
            }
        }
        if (valid) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r < rv) dst[2 * (o.v0 + r) + o.p] = dl[r];
        }
        t.sync();  // the next rows overwrite the rows, the table, Q and this staging buffer
    }
}

// --------------------------------------------------- learned proposal support

// Network inputs of states given by their free-variable bits (8 words each, `stride`
// words apart): x[b][0][i] = s_i, x[b][1][i] = C_{2(i+1)}/sqrt(L) (0 for i = n-1),
// x[b][2][i] = dISL_i/(8L).  One warp per state.
template <int R>
__device__ void features_row(const View& V, int n, int L, const Tile<32>& t, float* xb)
{
    const Outs<Tile<32>, R> o(t);
    int dl[R];
    {
        float X[R], P[R];
        toeplitz(V, n, o, X);
        p_direct(V, n, o, P);
        assemble(V, n, o, X, P, dl);
    }
    const float inv8L = (float)(8 * L);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (dl[r] != INT_MAX) xb[2 * n + 2 * (o.v0 + r) + o.p] = (float)dl[r] / inv8L;
}

__global__ void __launch_bounds__(256) features_kernel(const uint32_t* __restrict__ bits, int64_t stride,
                                                       int64_t count, int L, float* __restrict__ x)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2;
    const WarpSmem SL = warp_smem(n, 32);
    const Tile<32> t(threadIdx.x & 31);
    const int lane = t.lane, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const float sq = sqrtf((float)L);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; b < count; b += nwarps) {
        const uint32_t word = lane < kBitWords ? bits[b * stride + lane] : 0u;
        load_rows(base, SL, V, word, L, n, t);
        float* xb = x + b * 3 * n;
        for (int i = lane; i < n; i += kWarp) {
            xb[i] = (i & 1) ? V.A1[i >> 1] : V.A0[i >> 1];
            xb[n + i] = i < n - 1 ? V.G[i + 1].x / sq : 0.f;
        }
        switch (block_R(n, 32)) {
            case 1: features_row<1>(V, n, L, t, xb); break;
            case 3: features_row<3>(V, n, L, t, xb); break;
            case 5: features_row<5>(V, n, L, t, xb); break;
            case 7: features_row<7>(V, n, L, t, xb); break;
            default: features_row<9>(V, n, L, t, xb); break;
        }
        t.sync();
    }
}

// Restart candidates of walkers [first, first+count) of one length: candidate 0 is the
// walker's own next random start (what the plain walk would use); candidates c >= 1 are
// further random starts, Philox with key = seed and counter = (walker, next restart
// index, block, c) laid out as start_word's.  (Perturbations of the walker's best state
// were tried as candidates instead: the walkers then crowd around their old optima and
// found worse sequences, best F 6.81 against 7.23 at L = 255.)  Output bits [count][P][8].
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
            for (int j = 0; j < kBitWords; ++j) {
                uint32_t c0 = (uint32_t)w, c1 = ridx, c2 = (uint32_t)(j >> 2), c3 = (uint32_t)c;
                philox(c0, c1, c2, c3, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
                const uint32_t v = (j & 3) == 0 ? c0 : (j & 3) == 1 ? c1 : (j & 3) == 2 ? c2 : c3;
                const int lo = 32 * j;
                bits[j] = n <= lo ? 0u : (n - lo >= 32 ? v : v & ((1u << (n - lo)) - 1u));
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

// Objective of a walker's best sequence: its ISL, or (PSL << 32) | ISL under the PSL
// objective.
__device__ __forceinline__ unsigned long long best_objective(const KParams& p, const WalkerState& st)
{
    const unsigned long long isl = (uint32_t)st.best_isl;
    return p.mode == 3 ? ((unsigned long long)(uint32_t)st.best_psl << 32) | isl : isl;
}

// Lowest objective over the walkers of length L (0: all), into status->best_obj.
__global__ void best_obj_kernel(KParams p, int L)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < p.W;
         wi += (int64_t)gridDim.x * blockDim.x) {
        const WalkerState& st = p.states[wi];
        if (L != 0 && p.groups[st.group].L != L) continue;
        atomicMin(&p.status->best_obj, best_objective(p, st));
    }
}

// Lowest (best ISL, walker); under the PSL objective only among the walkers whose
// objective equals status->best_obj (best_obj_kernel ran first).
__global__ void best_kernel(KParams p, int L)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < p.W;
         wi += (int64_t)gridDim.x * blockDim.x) {
        const WalkerState& st = p.states[wi];
        if (L != 0 && p.groups[st.group].L != L) continue;
        if (p.mode == 3 && best_objective(p, st) != p.status->best_obj) continue;
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
        atomicAdd(&s->st_cache_hits, (unsigned long long)st.cache_hits);
        if (st.target_step >= 0) {
            atomicAdd(&s->st_at_target, 1ull);
            atomicMin(&s->st_target_step, (long long)st.target_step);
        }
        if (p.mode == 3) {
            atomicMin(&s->best_obj, best_objective(p, st));
            continue;
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
    const size_t smem = (size_t)(block / kWarp) * warp_smem(p.n_max, 32).words * sizeof(int);
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

static WalkFn walk_fn(int tile, int rmax, int mode)
{
    if (tile == 8) return rmax <= 6 ? walk_fn8a(rmax) : walk_fn8b(rmax);
    if (tile == 16 && mode == 3) return rmax <= 5 ? walk_fn16p(rmax) : walk_fn16q(rmax);
    if (tile == 16) return rmax <= 5 ? walk_fn16a(rmax) : walk_fn16b(rmax);
    switch (mode) {
        case 1: return walk_fn32l(rmax);
        case 2: return walk_fn32b(rmax);
        case 3: return walk_fn32p(rmax);
        default: return walk_fn32(rmax);
    }
}

int lanes_for(int n, int tile)
{
    return block_R(n, tile);
}

int walk_kernel_config(int tile, int rmax, int mode, int warps_per_cta, size_t smem_bytes, int* ctas_per_sm,
                       int* regs)
{
    const WalkFn fn = walk_fn(tile, rmax, mode);
    // every variant a context of this shape may launch (the learned mode is switched on
    // and off at run time) gets the shared-memory size
    for (int m = 0; m < (tile == 32 ? 3 : 1); ++m) {
        const cudaError_t e = cudaFuncSetAttribute(walk_fn(tile, rmax, m), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem_bytes);
        if (e != cudaSuccess) return LABS_ECUDA;
    }
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
    const WalkFn fn = walk_fn(p.tile, p.rmax, p.mode);
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
    // one row of ints per warp; long rows take fewer warps per CTA (48 KB of shared memory)
    const size_t row_bytes = (size_t)((L + 3) & ~3) * sizeof(int);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / row_bytes));
    const size_t smem = (size_t)warps * row_bytes;
    isl_kernel<<<row_grid(batch, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out,
                                                                                       status);
    return status_of(cudaGetLastError());
}

int launch_delta(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status, void* stream)
{
    if (batch == 0) return LABS_OK;
    const int warps = 8, n = (L + 1) / 2, nw = (n + 31) / 32;
    using DeltaFn = void (*)(const int8_t*, int64_t, int, int32_t*, DevStatus*);
    const bool pair = n <= 160;
    const int rows = pair ? 2 : 1;
    const size_t rows_bytes = (size_t)rows * warps * row_smem(n, pair ? 16 : 32).words * sizeof(int);
    const size_t stage = (size_t)warps * (2 * stage_bytes(L, rows) + 16);
    // staged rows need a 16-byte aligned input, and are used where they keep as many CTAs
    // on an SM as the rows alone (three two-row CTAs of 8 warps, two one-row CTAs)
    const size_t sm_bytes = 226 * 1024;
    const size_t cap = pair && block_R(n, 16) <= 7 ? 3 : 2;  // the kernels' launch bounds
    const size_t ctas_plain = std::min(cap, sm_bytes / rows_bytes);
    const size_t ctas_staged = std::min(cap, sm_bytes / (rows_bytes + stage));
    const bool staged = ((uintptr_t)seqs & 15) == 0 && ctas_staged >= ctas_plain;
    // (lane block, words per class) of every length: block_R(n, 16) and ceil(n/32)
    // for n <= 160 (two rows per warp), block_R(n, 32) above
    const int key = 16 * (pair ? block_R(n, 16) : block_R(n, 32)) + nw;
#define LABS_DELTA_CASE(KIND, R, W)                                         \
    case 16 * R + W:                                                        \
        fn = staged ? KIND<R, W, true> : KIND<R, W, false>;                 \
        break;
    DeltaFn fn = nullptr;
    if (pair) {
        switch (key) {
            LABS_DELTA_CASE(delta_pair_kernel, 1, 1)
            LABS_DELTA_CASE(delta_pair_kernel, 2, 1)
            LABS_DELTA_CASE(delta_pair_kernel, 3, 2)
            LABS_DELTA_CASE(delta_pair_kernel, 5, 2)
            LABS_DELTA_CASE(delta_pair_kernel, 5, 3)
            LABS_DELTA_CASE(delta_pair_kernel, 6, 3)
            LABS_DELTA_CASE(delta_pair_kernel, 7, 4)
            LABS_DELTA_CASE(delta_pair_kernel, 9, 4)
            LABS_DELTA_CASE(delta_pair_kernel, 9, 5)
            LABS_DELTA_CASE(delta_pair_kernel, 10, 5)
            default: return LABS_EINVAL;
        }
    } else {
        switch (key) {
            LABS_DELTA_CASE(delta_kernel, 7, 6)
            LABS_DELTA_CASE(delta_kernel, 7, 7)
            LABS_DELTA_CASE(delta_kernel, 9, 8)
            default: return LABS_EINVAL;
        }
    }
#undef LABS_DELTA_CASE
    const size_t smem = rows_bytes + (staged ? stage : 0);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // more CTAs than fit at once (up to 8 per SM): measured faster than one resident wave
    const int64_t units = pair ? (batch + 1) / 2 : batch;
    const int grid = row_grid(units, warps);
    fn<<<grid, warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out, status);
    return status_of(cudaGetLastError());
}

int launch_best(const KParams& p, int32_t L, void* stream)
{
    if (p.mode == 3) best_obj_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
    best_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
    return status_of(cudaGetLastError());
}

int launch_stats(const KParams& p, int32_t L, void* stream)
{
    stats_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
    if (p.mode == 3) best_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(p, L);
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
    const size_t smem = (size_t)warps * warp_smem((L + 1) / 2, 32).words * sizeof(int);
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
