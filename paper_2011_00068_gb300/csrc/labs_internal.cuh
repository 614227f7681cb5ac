// labs_internal.cuh -- device-memory layout shared by the host API (labs_api.cu) and
// the kernels (labs_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "labs.h"

namespace labsgpu {

constexpr int kWarp = 32;
constexpr int kMaxN = (LABS_MAX_L + 1) / 2;  // 256 free variables
constexpr int kBitWords = kMaxN / 32;        // 8 words of free-variable bits
// Long sequences (LABS_MAX_L < L <= LABS_MAX_L_LONG) run one walker per CTA of
// kLongThreads threads; their free-variable bits live beside the walker states.
constexpr int kMaxNLong = (LABS_MAX_L_LONG + 1) / 2;  // 5632 free variables
constexpr int kBitWordsLong = kMaxNLong / 32;          // 176 words
constexpr int kLongThreads = 512;       // threads of a long walker's CTA, n > kLongMidMaxN
constexpr int kLongThreadsMid = 256;    // ... for kLongSmallMaxN < n <= kLongMidMaxN (two CTAs per SM)
constexpr int kLongThreadsSmall = 128;  // ... for n <= kLongSmallMaxN (four CTAs per SM)
constexpr int kLongSmallMaxN = 1152;    // lane block <= 9 with 128 threads
constexpr int kLongMidMaxN = 2304;      // lane block <= 9 with 256 threads
constexpr int kQuadMaxR = 10;                // largest lane block of four walkers per warp (n <= 80)
constexpr int kMaxChunksPerCall = 4096;      // chunk launches per labs_walk call
constexpr int kMaxTrace = 4096;              // traced walkers
constexpr int kCheckEvery = 64;              // steps between stop checks
constexpr uint64_t kGenMask = 0xFFFFFull;    // HT generation field (low 20 bits)
constexpr uint32_t kZobristKey0 = 0x1BADB002u;  // Philox key of the HT fingerprint keys
constexpr uint32_t kZobristKey1 = 0x2011A068u;

// Either learned mode (full: flip scores and restart proposals; restarts only).
constexpr int kLearnedAny = LABS_FLAG_LEARNED | LABS_FLAG_LEARNED_RESTARTS;

// One length group: walkers [first, first+count) of length L, n = (L+1)/2 free vars.
struct DevGroup {
    int32_t L;
    int32_t n;
    int64_t first;
    int64_t count;
    int64_t zkey_off;  // offset of this group's n fingerprint keys in the zkey array
};

// Persistent state of one walker between chunk launches (the rest -- the +-1 rows,
// the C_k table, the ISL -- is rebuilt from `cur` at the start of every chunk).
struct alignas(32) WalkerState {
    uint32_t cur[kBitWords];   // free variables of the current sequence: bit i set <=> s_i = -1
    uint32_t best[kBitWords];  // free variables of the best sequence
    int64_t steps_done;
    int64_t best_step;         // steps_done when best_isl was first reached
    int64_t target_step;       // steps_done when the F target first held, -1 never
    uint64_t fp;               // HT fingerprint of `cur`
    int32_t isl;
    int32_t best_isl;
    int32_t since_best;        // best ISL since the last (re)start
    int32_t stagnation;        // steps since since_best last improved
    uint32_t restart_idx;      // Philox counter word of the current start
    uint32_t gen;              // HT generation
    int32_t restarts;
    int32_t overflows;
    int32_t blocked;
    int32_t group;
    int32_t trace_slot;        // -1: not traced
    int32_t psl;               // PSL objective only: PSL of `cur`, of `best`, and the
    int32_t best_psl;          // PSL of the best (PSL, ISL) pair since the last (re)start
    int32_t since_psl;         // (whose ISL is since_best)
    int64_t cache_hits;        // best-first search with the second table: skipped neighbours
};
static_assert(sizeof(WalkerState) == 160, "WalkerState layout");

// Status block at the start of the workspace.
struct alignas(256) DevStatus {
    int32_t error;          // first LABS_E* raised on the device (0 = none)
    int32_t error_detail;   // walker id / row index of that error
    int32_t invalid_rows;   // rows rejected by labs_isl / labs_neighbor_delta
    int32_t pad0;
    int64_t target_steps;   // every walker advances to this step count
    int32_t* trace_code;    // trace logs (labs_trace)
    int32_t* trace_isl;
    int64_t trace_capacity;
    unsigned long long best_key;  // (best_isl << 32) | walker, reduction target
    unsigned long long best_obj;  // PSL objective: lowest (best_psl << 32) | best_isl
    // stats accumulators (labs_stats)
    unsigned long long st_steps, st_evals, st_restarts, st_overflows, st_blocked, st_at_target, st_cache_hits;
    long long st_target_step;     // min over walkers, LLONG_MAX = none
    unsigned long long probe_ns;  // %globaltimer sample (clock alignment for deadlines)
    // walk log (labs_log): record k*W + w is walker w's chunk k since arming
    labs_log_record* log;
    int64_t log_capacity;
    int64_t log_start;            // step count at arming
    // learned mode (labs_learned)
    float* l_scores;              // [W][n_max] flip scores for the step l_score_step[w]
    int64_t* l_score_step;        // [W], -1 = none
    uint32_t* l_slot;             // [W][8] proposed restart state
    int32_t* l_slot_valid;        // [W]
    int32_t l_tau;
    int32_t learned;
    // replay dumps of traced walkers in learned mode
    float* d_scores;              // [trace slot][cap][n_max]
    int64_t* d_score_step;        // [trace slot][cap]
    int32_t* d_score_count;       // [trace slot]
    uint32_t* d_restart;          // [trace slot][cap][8]
    int64_t* d_restart_idx;       // [trace slot][cap]
    int32_t* d_restart_count;     // [trace slot]
    int32_t d_cap;
    int32_t pad1[1];
};

// Host-written control block in mapped pinned host memory (read by running kernels).
struct Control {
    volatile int32_t stop;           // 1 = cancel requested
    int32_t pad;
    volatile uint64_t deadline_ns;   // GPU %globaltimer deadline, UINT64_MAX = none
};

struct KParams {
    DevStatus* status;
    const DevGroup* groups;
    const uint64_t* zkeys;
    WalkerState* states;
    uint64_t* tabu;
    int64_t* trace_start;
    uint32_t* queue;          // one work counter per chunk of a labs_walk call
    const Control* ctrl;
    int64_t W;
    int32_t nG;
    int32_t n_max;            // largest n among the groups (sizes shared memory)
    int32_t tabu_log2;
    int32_t probe_cap;
    int32_t patience;         // 0 = 2n
    int32_t target_num, target_den;
    int32_t chunk_steps;
    int32_t rmax;             // lane block of the walk kernel instantiation (block_R(n_max, tile))
    int32_t tile;             // lanes per walker: 32, 16 (two walkers per warp) or 8 (four)
    int32_t best_first;       // 1: best-first search (one walker per warp, queue below)
    int32_t mode;             // walk kernel variant: 0 plain walk, 1 learned mode, 2 best-first,
                              // 3 walk under the PSL objective
    int32_t long_mode;        // 1: lengths above LABS_MAX_L, one walker per CTA
    uint32_t* cur_bits;       // long mode: [W][kBitWordsLong] free variables of the current
    uint32_t* best_bits;      // and of the best sequence (WalkerState.cur / best unused)
    uint64_t* pq_key;         // [W][LABS_QUEUE_SIZE] queue keys, ~0 = empty
    uint32_t* pq_bits;        // [W][LABS_QUEUE_SIZE][kBitWords] queue entries' free variables
    uint64_t* tabu2;          // best-first search: xLastovka's second table, as many slots per
                              // walker as HT (null when off)
    uint64_t seed;
};

// Shared-memory layout of one walker, in 32-bit words.  Rows and table hold small
// integers as floats (exact: every value and every partial sum of the neighbourhood
// stays below 2^24 in magnitude for L <= 511), so that the Toeplitz product runs on
// the FP32 pipes (or, two walkers per warp, on the tensor cores from FP16 copies of the
// same integers, |C_k| < 2^11).
//   A0: even positions s_0, s_2, .. (n values) as +-1.0f; zero from -apad up to the
//       row end (indices [-apad, alen - apad)); the padding covers every index the
//       walk reads without a bounds test
//   A1: odd positions s_1, s_3, .. (n-1 values), laid out the same way
//   G : pairs G[y] = (E[y], E[y+1]) for y in [-gpad, glen - gpad), where
//       E[d] = C_{2|d|} for 0 < |d| < n and E[d] = 0 otherwise (E[0] = 0)
//   B : bit-packed classes (bit u set <=> A_p[u] = -1) and their reversals,
//       4 vectors x bvec words (kBitVec in the warp layouts), zero beyond the class
//       length
constexpr int kTcPad = 48;  // FP16 row entries the tensor-core product reads below u = 0
constexpr int kBitVec = 9;  // 256 bits per class plus one zero word read by the shifts
struct WarpSmem {
    int apad;   // zero words below index 0 of each row (multiple of 4)
    int alen;   // words per row (multiple of 4)
    int gpad;   // pairs of G below y = 0 (>= the deepest read or write)
    int glen;   // pairs of G
    int goff;   // word offset of G[-gpad] (even)
    int boff;   // word offset of B
    int bvec;   // words per bit vector of B
    int xoff;   // long layout: word offset of the CTA scratch (kLongThreads words) and the
                // free-variable bits (kBitWordsLong words)
    int poff;   // row layout: word offset of the per-lag P values Q[0 .. n_max) (0: none)
    int roff;   // tensor-core layouts: word offset of the Toeplitz results X[2][xp]
    int xp;     // floats per class of the Toeplitz results (0: no tensor-core product)
    int hoff;   // tensor-core layouts: word offset of FP16 rows (copies of the rows in the
                // walk, the only rows in the row kernels), class p at hoff + p hlen, entry
                // u at half index hpad + u, zero around the class
    int hlen;   // words per FP16 row (4 mod 8: the two classes' operand loads use
                // different banks; 0: no FP16 rows)
    int hpad;   // FP16 entries below u = 0 (even)
    int words;  // total words per walker (multiple of 4: walkers stay 16-byte aligned)
};
// Outputs per lane (the lane block R) for n free variables and `tile` lanes per walker
// (tile/2 lanes per parity class): at least ceil(ceil(n/2) / (tile/2)), raised until
// the lanes of a class, whose table windows lie 8R bytes apart, read 16 distinct pairs
// of banks, i.e. until 16 / gcd(R, 16) >= tile/2.
__host__ __device__ inline int conflict_free_R(int R, int tile)  // smallest such R' >= R
{
    for (;;) {
        const int low = R & -R;  // gcd(R, 16) for R < 32
        if (16 / (low < 16 ? low : 16) >= tile / 2) return R;
        ++R;
    }
}
__host__ __device__ inline int block_R(int n, int tile)
{
    const int h = tile / 2;
    return conflict_free_R((((n + 1) >> 1) + h - 1) / h, tile);
}

// Shared memory of one SM that the walk layouts may fill (of 228 KB, 1 KB per CTA kept).
constexpr int kSmemBudget = 226 * 1024;

// n_max: largest number of free variables served; tile: lanes per walker (32, 16 or 8);
// tc: with the regions of the tensor-core Toeplitz product (FP16 rows, results); psl:
// two walkers per warp under the PSL objective (the rows and the table padded for the
// PSL neighbourhood's reads, as every one-walker-per-warp layout is).
__host__ __device__ inline WarpSmem warp_layout(int n_max, int tile, bool tc, bool psl = false)
{
    WarpSmem w;
    const int R = block_R(n_max, tile);
    const int top = ((n_max + 7) & ~7) + 2;  // G above 0: the Toeplitz window reaches round8(n)
    if (tile == 8) {
        // four walkers per warp (tight on shared memory): the lag update of lane l covers
        // m = 1+lR .. (l+1)R (up to 8R) and reads s_{i+2m} only inside the class, the
        // keys read s_{3i-L+1} and C_{q-i} only for existing outputs, and the mirror half
        // of G is kept down to E[-(4R+1)], what the Toeplitz window reads
        const int lo = n_max > 8 * R + 1 ? n_max : 8 * R + 1;
        const int hi = n_max + 8 > 8 * R + 2 ? n_max + 8 : 8 * R + 2;
        w.apad = (lo + 3) & ~3;
        w.alen = w.apad + ((hi + 7) & ~7);
        w.gpad = 4 * R + 1;
        w.glen = w.gpad + (top > 8 * R + 2 ? top : 8 * R + 2);
    } else {
        // the lockstep walk step: the lag update of lane l covers m = 1+lR .. (l+1)R of
        // its walker (up to tile R) without bounds tests, in the rows and in G, and the
        // keys read s_{3i-L+1} for every lane output (index below 3 (tile/2) R)
        const int span = tile * R + 2;
        int hi = (3 * n_max) / 2 + 2 > n_max + 8 ? (3 * n_max) / 2 + 2 : n_max + 8;
        if ((n_max + 1) / 2 + span > hi) hi = (n_max + 1) / 2 + span;
        if (3 * (tile / 2) * R > hi) hi = 3 * (tile / 2) * R;
        int lo = n_max > span ? n_max : span;
        int gtop = top > span ? top : span;
        int gdeep = 0;
        if (tc) {
            // the Toeplitz product on the tensor cores reads the table from
            // y = -(16 T - 1) up to 16 S, with S = ceil(n/16) row blocks and
            // T = ceil(ceil(n/2) / 16) output blocks
            const int S = (n_max + 15) >> 4, T = (((n_max + 1) >> 1) + 15) >> 4;
            if (gtop < 16 * S) gtop = 16 * S;
            gdeep = 16 * T - 1;
        }
        if (tile == 32 || (psl && tile == 16)) {
            // the PSL neighbourhood runs its lags 2R - 2 past n - 1: class entries from
            // v0 - n - 2R up to v0 + n + 2R (v0 <= (tile/2 - 1) R) and the table up to n + 2R
            if (n_max + (tile / 2 + 2) * R > hi) hi = n_max + (tile / 2 + 2) * R;
            if (n_max + 2 * R > lo) lo = n_max + 2 * R;
            if (n_max + 2 * R > gtop) gtop = n_max + 2 * R;
        }
        w.apad = (lo + 3) & ~3;
        w.alen = w.apad + ((hi + 7) & ~7);
        // one walker per warp: lanes 0-15 read row A0 and lanes 16-31 row A1 at the same
        // offsets v0 + d, v0 = hR with R odd, i.e. banks {hR + d} and {hR + d + alen}:
        // the two sets are disjoint (no conflicts) when alen = 16 (mod 32)
        if (tile == 32) w.alen += (48 - (w.alen & 31)) & 31;
        w.gpad = (tile / 2) * R > span ? (tile / 2) * R : span;
        if (w.gpad < gdeep) w.gpad = gdeep;
        w.glen = w.gpad + gtop;
    }
    w.goff = 2 * w.alen;
    w.boff = w.goff + 2 * w.glen;
    w.bvec = kBitVec;
    w.xoff = 0;
    w.poff = 0;
    w.xp = 0;
    w.roff = 0;
    w.hoff = 0;
    w.hlen = 0;
    w.hpad = 0;
    w.words = (w.boff + 4 * kBitVec + 3) & ~3;
    if (tc) {
        // the tensor-core Toeplitz product.  Its results: 16 T outputs per class written,
        // (tile/2) R read; xp = 16 (mod 32) puts the two classes' entries in different
        // banks
        const int T = (((n_max + 1) >> 1) + 15) >> 4, S = (n_max + 15) >> 4;
        const int need = 16 * T > (tile / 2) * R ? 16 * T : (tile / 2) * R;
        w.roff = w.words;
        w.xp = ((need + 15) & ~31) + 16;
        // FP16 rows: u from -kTcPad up to 16 S + kTcPad (16 S + 96 halves)
        w.hoff = w.roff + 2 * w.xp;
        w.hpad = kTcPad;
        w.hlen = ((8 * S + kTcPad + 3) & ~7) + 4;
        w.words = w.hoff + 2 * w.hlen;
    }
    return w;
}

// The walk layout of n_max free variables with `tile` lanes per walker.  Two walkers per
// warp take the tensor-core Toeplitz product up to n_max = 128 (one product per block
// diagonal covers the outputs); one walker per warp takes it when its regions keep the
// 16 walkers of two 8-warp CTAs within an SM's shared memory; four walkers per warp keep
// the FP32 product.  psl: the layout of the PSL walk with two walkers per warp (tile 16).
__host__ __device__ inline WarpSmem warp_smem(int n_max, int tile, bool psl = false)
{
    if (tile == 16) return warp_layout(n_max, tile, n_max <= 128, psl);
    if (tile == 32) {
        const WarpSmem w = warp_layout(n_max, tile, true);
        if (w.words * 4 * 16 <= kSmemBudget) return w;
    }
    return warp_layout(n_max, tile, false);
}

// Layout of one row of the stateless row kernels (labs_neighbor_delta), `tile` lanes per
// row with lane block R = block_R(n_max, tile) (v0 <= (tile/2 - 1) R):
//   A rows: the Toeplitz loop reads A_p[0 .. round8(n)) (zero beyond the class), the
//     assembly A_p[v], A_p[n-1-p-v] and A_p[3v+p-n+1] for every lane output v (down to
//     -(n-1), below 3 (tile/2) R - n);
//   G: the table writes E[m] and its mirror for 1 <= m < n (pairs -n .. n-1), the
//     window reads pairs -(tile/2) R .. round8(n), the assembly C_{q-i} at pairs above
//     c - 2 (tile/2) R;
//   Q[0 .. n_max): the per-lag P values (see the row kernels); no bit vectors (the
//     classes stay in registers).
__host__ __device__ inline WarpSmem row_smem(int n_max, int tile)
{
    WarpSmem w;
    const int R = block_R(n_max, tile);
    const int vtop = (tile / 2) * R;             // one past the largest lane output
    if (tile == 16 && n_max <= 128) {
        // two rows per warp with the Toeplitz product on the tensor cores: FP16 rows only
        // (the product's operand blocks u = -kTcPad .. 16 S + kTcPad and the assembly's
        // reads, down to -(n-1)), the table for the product (pairs -(16 T - 1) .. 16 S)
        // and the assembly, then Q, which the product's results X[2][xp] overwrite
        const int S = (n_max + 15) >> 4, T = (((n_max + 1) >> 1) + 15) >> 4;
        int hlo = kTcPad > n_max - 1 ? kTcPad : n_max - 1;
        if (vtop - n_max + 1 > hlo) hlo = vtop - n_max + 1;
        int hhi = 16 * S + kTcPad;               // A_p[v] (v < vtop), A_p[3v+p-n+1], A_p[n-1]
        if (vtop > hhi) hhi = vtop;
        if (3 * vtop - n_max > hhi) hhi = 3 * vtop - n_max;
        if (n_max > hhi) hhi = n_max;
        w.apad = 0;
        w.alen = 0;
        w.hoff = 0;
        w.hpad = (hlo + 1) & ~1;
        w.hlen = (((w.hpad + hhi + 1) / 2 + 3) & ~7) + 4;
        int gl = n_max + 1;                      // mirror of E down to pair -n
        if (16 * T - 1 > gl) gl = 16 * T - 1;    // the product's first pairs
        if (2 * vtop - n_max + 2 > gl) gl = 2 * vtop - n_max + 2;  // C_{q-i} below 0
        w.gpad = gl;
        w.glen = w.gpad + (16 * S > n_max + 2 ? 16 * S : n_max + 2);
        w.goff = 2 * w.hlen;
        w.boff = w.goff + 2 * w.glen;
        w.bvec = 0;
        const int need = 16 * T > vtop ? 16 * T : vtop;
        w.xp = ((need + 15) & ~31) + 16;
        w.poff = (w.boff + 3) & ~3;
        w.xoff = 0;
        w.roff = w.poff;
        const int q = 2 * w.xp > n_max ? 2 * w.xp : n_max;
        w.words = w.poff + ((q + 3) & ~3);
        return w;
    }
    const int nu = (n_max + 7) & ~7;
    int lo = n_max, hi = nu;
    if (vtop > hi) hi = vtop;                    // A_p[v] with v < vtop
    if (3 * vtop - n_max > hi) hi = 3 * vtop - n_max;  // A_p[3v+p-n+1] <= 3 vtop - n - 1
    if (n_max + 2 > lo) lo = n_max + 2;          // A_p[n-1-p-v] down to n - 1 - vtop
    if (vtop - n_max + 2 > lo) lo = vtop - n_max + 2;
    w.apad = (lo + 3) & ~3;
    w.alen = w.apad + ((hi + 7) & ~7);
    // one row per warp: the halves read A0 and A1 at equal offsets, on disjoint banks
    // when alen = 16 (mod 32)
    if (tile == 32) w.alen += (48 - (w.alen & 31)) & 31;
    int gl = n_max + 1;                          // mirror of E down to pair -n
    if (vtop + R > gl) gl = vtop + R;            // the window's first pairs
    if (2 * vtop - n_max + 2 > gl) gl = 2 * vtop - n_max + 2;  // C_{q-i} below 0
    w.gpad = gl;
    w.glen = w.gpad + nu + 2;
    w.goff = 2 * w.alen;
    w.boff = w.goff + 2 * w.glen;
    w.bvec = 0;
    w.xoff = 0;
    w.xp = 0;
    w.roff = 0;
    w.hoff = 0;
    w.hlen = 0;
    w.hpad = 0;
    w.poff = (w.boff + 3) & ~3;
    w.words = w.poff + ((n_max + 3) & ~3);
    return w;
}

// Threads of a long walker's CTA for n_max free variables: 128 (four walkers per SM) up
// to n = 1152, 256 (two) up to 2304, else 512.  The walk under the PSL objective keeps
// 256 threads below n = 1152, where its lane block stays at most 5 and psl_eval uses
// its ring form (faster there than lane block 9 with 128 threads).
__host__ __device__ inline int long_threads(int n_max, bool psl = false)
{
    if (n_max <= kLongSmallMaxN && !psl) return kLongThreadsSmall;
    return n_max <= kLongMidMaxN ? kLongThreadsMid : kLongThreads;
}

// Lane block of the long layout: ceil(ceil(n/2) / (threads/2)) raised to odd, so that the
// lanes of a warp (all in one parity class, R entries apart) hit distinct banks.
__host__ __device__ inline int long_R(int n, int threads)
{
    const int h = threads / 2;
    const int R = (((n + 1) >> 1) + h - 1) / h;
    return R | 1;
}

// Shared-memory layout of one long walker (one CTA): the rows and the table as in the
// warp layout (bounds from the tile code with tile = the CTA width), bit vectors sized
// for n_max, then the CTA scratch, the bits and the best-first queue's keys.
__host__ __device__ inline WarpSmem long_layout(int n_max, int tile, bool tc)
{
    WarpSmem w;
    const int R = long_R(n_max, tile);
    const int top = ((n_max + 7) & ~7) + 2;
    const int span = tile * R + 2;
    int hi = (3 * n_max) / 2 + 2 > n_max + 8 ? (3 * n_max) / 2 + 2 : n_max + 8;
    if ((n_max + 1) / 2 + span > hi) hi = (n_max + 1) / 2 + span;
    int lo = n_max > span ? n_max : span;
    int gtop = top > span ? top : span;
    // the PSL neighbourhood runs its lags 2R - 2 past n - 1 (as in the warp layout)
    if (n_max + (tile / 2 + 2) * R > hi) hi = n_max + (tile / 2 + 2) * R;
    if (n_max + 2 * R > lo) lo = n_max + 2 * R;
    if (n_max + 2 * R > gtop) gtop = n_max + 2 * R;
    const int S = (n_max + 15) >> 4, T = (((n_max + 1) >> 1) + 15) >> 4;
    if (tc && gtop < 16 * S) gtop = 16 * S;  // the tensor-core product's table reads
    w.apad = (lo + 3) & ~3;
    w.alen = w.apad + ((hi + 7) & ~7);
    w.gpad = (tile / 2) * R > span ? (tile / 2) * R : span;
    if (tc && w.gpad < 16 * T - 1) w.gpad = 16 * T - 1;
    w.glen = w.gpad + gtop;
    w.goff = 2 * w.alen;
    w.boff = w.goff + 2 * w.glen;
    w.bvec = (n_max + 31) / 32 + 2;
    w.poff = 0;
    w.xp = 0;
    w.roff = 0;
    w.hoff = 0;
    w.hlen = 0;
    w.hpad = 0;
    w.xoff = (w.boff + 4 * w.bvec + 3) & ~3;
    if (tc) {
        // FP16 rows (cleared with the rows, below xoff): u from -kTcPad up to 16 S + kTcPad
        w.hoff = w.xoff;
        w.hpad = kTcPad;
        w.hlen = ((8 * S + kTcPad + 3) & ~7) + 4;
        w.xoff = w.hoff + 2 * w.hlen;
    }
    // scratch, bits, then the best-first search's queue keys (LABS_QUEUE_SIZE 64-bit
    // words), each warp's lowest candidate keys (32 per warp), the keys entered in a
    // round, two words of round state and the entered keys' places (LABS_QUEUE_SIZE ints)
    w.words = w.xoff + tile + kBitWordsLong + 2 * LABS_QUEUE_SIZE + 2 * tile + 2 * LABS_QUEUE_SIZE + 4 +
              LABS_QUEUE_SIZE;
    if (tc) {
        // the tensor-core product's results X[2][xp] (16 T written, (tile/2) R read per class)
        const int need = 16 * T > (tile / 2) * R ? 16 * T : (tile / 2) * R;
        w.xp = ((need + 15) & ~31) + 16;
        w.roff = (w.words + 3) & ~3;
        w.words = w.roff + 2 * w.xp;
    }
    return w;
}

// The long layout (one walker per CTA of `tile` threads) takes the tensor-core Toeplitz
// product when its regions keep the kLongThreads / tile CTAs of an SM within its shared
// memory.
__host__ __device__ inline WarpSmem long_smem(int n_max, int tile)
{
    const WarpSmem w = long_layout(n_max, tile, true);
    if ((int64_t)w.words * 4 * (kLongThreads / tile) <= kSmemBudget) return w;
    return long_layout(n_max, tile, false);
}

// Largest ISL for which the long walk's fp32 neighbourhood stays exact.  Every value in
// the dISL assembly is bounded by 16 sum_m |C_{2m}| + 8L + 32n + 32, and by
// Cauchy-Schwarz sum_m |C_{2m}| <= sqrt((n-1) ISL); the limit keeps the bound below
// 2^24, and caps ISL at 2^29 so that a neighbour's ISL (at most 2^24 more) fits the 30
// bits the PSL objective's order key gives it.
__host__ __device__ inline int long_isl_limit(int L, int n)
{
    const double room = ((double)(1 << 24) - 8.0 * L - 32.0 * n - 32.0) / 16.0;
    double lim = room * room / (double)(n > 1 ? n - 1 : 1);
    if (lim > (double)(1 << 29)) lim = (double)(1 << 29);
    return (int)lim - 1;
}

// Walk kernel instantiations (labs_walk8a.cu, labs_walk8b.cu: four walkers per warp,
// lane blocks 1-6 and 7-10; labs_walk16a.cu, labs_walk16b.cu: two walkers per warp,
// lane blocks 1-5 and 6-10; labs_walk32.cu: one walker per warp).
using WalkFn = void (*)(KParams, int);
WalkFn walk_fn8a(int rmax);
WalkFn walk_fn8b(int rmax);
WalkFn walk_fn16a(int rmax);
WalkFn walk_fn16b(int rmax);
WalkFn walk_fn16p(int rmax);  // two walkers per warp, PSL objective, lane blocks 1-5 (labs_walk16p.cu)
WalkFn walk_fn16q(int rmax);  // the same, lane blocks 6-9 (labs_walk16q.cu)
WalkFn walk_fn32(int rmax);   // one walker per warp: plain walk
WalkFn walk_fn32l(int rmax);  // learned mode (labs_walk32l.cu)
WalkFn walk_fn32b(int rmax);  // best-first search (labs_walk32b.cu)
WalkFn walk_fn32p(int rmax);  // walk under the PSL objective (labs_walk32p.cu)

// Long-L walk (labs_long.cu).
int long_kernel_config(int n_max, int mode, size_t smem_bytes, int* ctas_per_sm, int* regs);
int launch_long_reset(const KParams& p, size_t smem_bytes, void* stream);
int launch_long_walk_chunk(const KParams& p, int chunk_index, int grid, size_t smem_bytes, void* stream);
int launch_long_delta(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status, void* stream);

// Launchers (labs_kernels.cu).
int launch_zobrist(const KParams& p, uint64_t* zkeys, const DevGroup* host_groups, int nG,
                   void* stream);
int launch_reset(const KParams& p, int grid, int block, void* stream);
int launch_prep_walk(const KParams& p, int64_t steps, int nchunks, void* stream);
int launch_walk_chunk(const KParams& p, int chunk_index, int grid, int warps_per_cta,
                      size_t smem_bytes, void* stream);
int walk_kernel_config(int tile, int rmax, int mode, int warps_per_cta, size_t smem_bytes, int* ctas_per_sm,
                       int* regs);
int lanes_for(int n, int tile);  // block_R(n, tile)
int launch_isl(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status,
               void* stream);
int launch_delta(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status,
                 void* stream);
int launch_best(const KParams& p, int32_t L, void* stream);
int launch_stats(const KParams& p, int32_t L, void* stream);
int launch_trace_arm(const KParams& p, const int64_t* dev_ids, int32_t k, int32_t* code,
                     int32_t* isl, int64_t capacity, void* stream);
int launch_time_probe(unsigned long long* dev_out, void* stream);
int launch_features(const uint32_t* bits, int64_t stride, int64_t count, int32_t L, float* x, void* stream);
int launch_candidates(const KParams& p, int64_t first, int64_t count, int n, int P, uint32_t* out, void* stream);
int launch_select(const KParams& p, int64_t first, int64_t count, int P, const float* score, const uint32_t* cand,
                  void* stream);
int launch_scores(const KParams& p, int64_t first, int64_t count, int n, const float* score, void* stream);
int launch_labels(const labs_log_record* rec, int64_t count, int32_t* target, float* y, float* wf, void* stream);

// Learned network (labs_net.cu): forward of a batch of float inputs [B][3][n] into the
// caller's workspace; scores [B][n] and restart [B] are returned as device pointers
// inside that workspace.
size_t net_workspace_bytes(int64_t B, int n);
int net_forward_ws(const float* params, const float* x, int64_t B, int n, void* ws, const float** scores,
                   const float** restart, void* stream);

// Partial / final result of the exhaustive skew search (labs_enum.cu).
struct EnumPart {
    long long min_isl;
    unsigned long long count;
    unsigned long long first;
    unsigned long long pad;
};
int enum_blocks(int L);
size_t enum_scratch_bytes(int L);
int enum_run(int L, EnumPart* scratch, void* stream, EnumPart* host_out);

}  // namespace labsgpu
