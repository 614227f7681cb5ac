// labs_long.cu -- long sequences (LABS_MAX_L < L <= LABS_MAX_L_LONG): one CTA of 256 or
// 512 threads runs one walker (long_threads).  The walk's step (Algorithm 1 in its
// self-avoiding form): all n flips evaluated by the Toeplitz form of dISL, the lowest
// (dISL, i) whose result is not in HT taken, C_k and P updated in O(n) per move; the same
// under the PSL objective, and the best-first search (Algorithm 1 as printed).
// The per-lane arithmetic is the warp kernels' (labs_device.cuh), run by a lane group
// that spans the CTA; the collectives go through shared memory.
#include "labs_device.cuh"

namespace labsgpu {

namespace {

// The CTA as one lane group (the interface of Tile<>; every call must be reached by all
// threads).  x: NT words of shared scratch.
template <int NT>
struct Blk {
    static constexpr int kSize = NT;
    static constexpr int kHalf = NT / 2;
    static constexpr int kWarps = NT / 32;
    int lane;
    int* x;
    __device__ Blk(int tid, int* scratch) : lane(tid), x(scratch) {}
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int shfl(int v, int src) const
    {
        x[lane] = v;
        __syncthreads();
        const int r = x[src];
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ uint32_t shfl(uint32_t v, int src) const { return (uint32_t)shfl((int)v, src); }
    // warp partials in x[0 .. kWarps), combined by every thread
    __device__ __forceinline__ int rmin(int v) const
    {
        v = __reduce_min_sync(kFull, v);
        if ((lane & 31) == 0) x[lane >> 5] = v;
        __syncthreads();
        int r = x[0];
#pragma unroll
        for (int k = 1; k < kWarps; ++k) r = min(r, x[k]);
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ int rmax(int v) const { return -rmin(-v); }
    __device__ __forceinline__ unsigned rminu(unsigned v) const
    {
        v = __reduce_min_sync(kFull, v);
        if ((lane & 31) == 0) x[lane >> 5] = (int)v;
        __syncthreads();
        unsigned r = (unsigned)x[0];
#pragma unroll
        for (int k = 1; k < kWarps; ++k) r = min(r, (unsigned)x[k]);
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ uint32_t rxor(uint32_t v) const
    {
        v = __reduce_xor_sync(kFull, v);
        if ((lane & 31) == 0) x[lane >> 5] = (int)v;
        __syncthreads();
        uint32_t r = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) r ^= (uint32_t)x[k];
        __syncthreads();
        return r;
    }
    // 64-bit minimum (order keys of the PSL objective)
    __device__ __forceinline__ uint64_t rmin64(uint64_t v) const
    {
        v = warp_min64(v);
        unsigned long long* y = reinterpret_cast<unsigned long long*>(x);
        if ((lane & 31) == 0) y[lane >> 5] = v;
        __syncthreads();
        uint64_t r = y[0];
#pragma unroll
        for (int k = 1; k < kWarps; ++k) r = min(r, (uint64_t)y[k]);
        __syncthreads();
        return r;
    }
    // sum in 64 bits, saturated to INT_MAX (a saturated ISL fails the range check)
    __device__ __forceinline__ int radd(int v) const
    {
        long long a = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
        long long* y = reinterpret_cast<long long*>(x);
        if ((lane & 31) == 0) y[lane >> 5] = a;
        __syncthreads();
        long long r = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) r += y[k];
        __syncthreads();
        return r > INT_MAX ? INT_MAX : (int)r;
    }
};

// One long walker: the walk's environment plus its bit rows in global memory and the
// CTA's shared copy of the current bits.
struct LongWalk {
    WalkEnv e;
    uint32_t* cur;    // [kBitWordsLong] in global memory
    uint32_t* best;
    uint32_t* bits;   // shared copy of the current bits (kBitWordsLong words)
    int nw;           // words of free-variable bits, ceil(n / 32)
    int isl_limit;    // exact-range bound of the ISL (long_isl_limit)
};

// Zeroes rows, table and bit vectors (everything below the scratch and the bits).
template <class LB>
__device__ __forceinline__ void long_clear(int* base, const WarpSmem& SL, const LB& t)
{
    int4* b4 = reinterpret_cast<int4*>(base);
    for (int i = t.lane; i < SL.xoff / 4; i += LB::kSize) b4[i] = make_int4(0, 0, 0, 0);
    t.sync();
}

// Rows from the shared bits (Eq. 4: s_j = x_j for j <= c, s_{c+t} = (-1)^t x_{c-t}),
// then the table; returns the ISL.
template <class LB>
__device__ int long_load_rows(const LongWalk& lw, const WarpSmem& SL, int* base, const View& V, uint32_t word,
                              const LB& t)
{
    const int L = lw.e.L, n = lw.e.n, c = n - 1;
    if (t.lane < lw.nw) lw.bits[t.lane] = word;
    long_clear(base, SL, t);  // ends with a barrier
    for (int j = t.lane; j < L; j += LB::kSize) {
        const int f = j <= c ? j : 2 * c - j;
        const int x = ((lw.bits[f >> 5] >> (f & 31)) & 1u) ? -1 : 1;
        const int s = (j > c && ((j - c) & 1)) ? -x : x;
        set_row(V, j & 1, j >> 1, (float)s);
    }
    t.sync();
    return build_table(V, n, t);
}

// HT fingerprint of the shared bits (long_load_rows ran first).
template <class LB>
__device__ uint64_t long_fingerprint(const LongWalk& lw, const LB& t)
{
    uint64_t f = 0;
    for (int i = t.lane; i < lw.e.n; i += LB::kSize)
        if ((lw.bits[i >> 5] >> (i & 31)) & 1u) f ^= __ldg(lw.e.zk + i);
    const uint32_t lo = t.rxor((uint32_t)f);
    const uint32_t hi = t.rxor((uint32_t)(f >> 32));
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

template <class LB>
__device__ __forceinline__ void long_note_best(const LongWalk& lw, Walker& w, const LB& t, PslTrack* ps = nullptr)
{
    const bool better = ps ? psl_better(ps->psl, w.isl, ps->best_psl, w.best_isl) : w.isl < w.best_isl;
    if (better) {
        w.best_isl = w.isl;
        if (ps) ps->best_psl = ps->psl;
        w.best_step = w.steps;
        if (t.lane < lw.nw) lw.best[t.lane] = w.word;
    }
    if (w.target_step < 0 && target_met(*lw.e.p, lw.e.L, w.isl)) w.target_step = w.steps;
}

// Algorithm 1 start: random S (restart index w.restart_idx), rows, table, ISL, HT
// insertion, best update.
template <class LB>
__device__ void long_start(const LongWalk& lw, Walker& w, const WarpSmem& SL, int* base, const View& V,
                           const LB& t, PslTrack* ps = nullptr)
{
    const WalkEnv& env = lw.e;
    w.word = t.lane < lw.nw ? start_word(env.p->seed, env.g, w.restart_idx, t.lane, env.n) : 0u;
    w.isl = long_load_rows(lw, SL, base, V, w.word, t);
    w.fp = long_fingerprint(lw, t);
    if (t.lane == 0) env.T[w.fp & env.tmask] = (w.fp & ~kGenMask) | w.gen;
    t.sync();
    w.since = w.isl;
    w.stag = 0;
    if (ps) {
        ps->psl = table_psl(V, env.n, t);
        ps->since_psl = ps->psl;
    }
    long_note_best(lw, w, t, ps);
}

template <class LB>
__device__ void long_restart(const LongWalk& lw, Walker& w, const WarpSmem& SL, int* base, const View& V,
                             const LB& t, PslTrack* ps = nullptr)
{
    w.restart_idx += 1;
    w.restarts += 1;
    w.gen += 1;
    if (w.gen > kGenMask) {
        const int64_t slots = (int64_t)lw.e.tmask + 1;
        for (int64_t i = t.lane; i < slots; i += LB::kSize) lw.e.T[i] = 0ull;
        t.sync();
        w.gen = 1;
    }
    long_start(lw, w, SL, base, V, t, ps);
}

// HT probe of f by the first warp (the walk's linear probe of up to probe_cap <= 32
// slots), result shared with the CTA.
template <class LB>
__device__ Probe long_probe(const LongWalk& lw, uint64_t f, uint32_t gen, const LB& t)
{
    long long* y = reinterpret_cast<long long*>(t.x);
    if (t.lane < 32) {
        const Tile<32> tw(t.lane);
        const Probe pr = probe_full(lw.e, f, gen, lw.e.p->probe_cap, tw);
        if (t.lane == 0) {
            y[0] = pr.visited ? 1 : 0;
            y[1] = pr.slot;
        }
    }
    __syncthreads();
    Probe pr;
    pr.visited = y[0] != 0;
    pr.slot = y[1];
    __syncthreads();
    return pr;
}

// Steps of one long walker until `until` (or a stop request, or the exact-range check).
template <class LB, int R>
__device__ void long_walk(const LongWalk& lw, Walker& w, int64_t until, const WarpSmem& SL, int* base,
                          const View& V, int trace_slot, int64_t trace_start, const LB& t)
{
    const WalkEnv& env = lw.e;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<LB, R> o(t);
    float P[R];
    p_direct(V, n, o, P);
    StopCheck stop;
    stop.start(p, lane == 0);
    while (w.steps < until) {
        if (w.isl > lw.isl_limit) {
            if (lane == 0) raise_error(p.status, LABS_ERANGE, (int)env.g);
            break;
        }
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
        // lowest (dISL, i) whose result is not in HT
        uint32_t excl = 0;
        int best_i = -1, best_d = 0;
        int64_t slot = -1;
        uint64_t fnew = 0;
        for (;;) {
            int bd, bi;
            tile_argmin(dl, excl, o, t, bd, bi);
            if (bi < 0) break;
            const uint64_t f = w.fp ^ __ldg(env.zk + bi);
            const Probe pr = long_probe(lw, f, w.gen, t);
            if (!pr.visited) {
                best_i = bi;
                best_d = bd;
                slot = pr.slot;
                fnew = f;
                break;
            }
            exclude<LB, R>(excl, bi, t);
        }
        w.steps += 1;
        int code;
        if (best_i < 0) {
            w.blocked += 1;
            long_restart(lw, w, SL, base, V, t);
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
            long_note_best(lw, w, t);
            if (w.isl < w.since) {
                w.since = w.isl;
                w.stag = 0;
            } else {
                w.stag += 1;
            }
            code = best_i;
            if (w.stag >= env.patience || !stored) {
                long_restart(lw, w, SL, base, V, t);
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

// The walk under the PSL objective for a long walker (the rules of walk_psl): the
// Toeplitz dISL and the PSL of every neighbour, the lowest (PSL, ISL, i) not in HT, best
// and stagnation on (PSL, ISL) pairs.
template <class LB, int R>
__device__ void long_walk_psl(const LongWalk& lw, Walker& w, PslTrack& ps, int64_t until, const WarpSmem& SL,
                              int* base, const View& V, int trace_slot, int64_t trace_start, const LB& t)
{
    const WalkEnv& env = lw.e;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<LB, R> o(t);
    float P[R];
    p_direct(V, n, o, P);
    StopCheck stop;
    stop.start(p, lane == 0);
    while (w.steps < until) {
        if (w.isl > lw.isl_limit) {
            if (lane == 0) raise_error(p.status, LABS_ERANGE, (int)env.g);
            break;
        }
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
            const uint64_t km = t.rmin64(lm);
            if (km == ~0ull) break;
            const int bi = psl_key_i(km);
            const uint64_t f = w.fp ^ __ldg(env.zk + bi);
            const Probe pr = long_probe(lw, f, w.gen, t);
            if (!pr.visited) {
                best_i = bi;
                best_key = km;
                slot = pr.slot;
                fnew = f;
                break;
            }
            exclude<LB, R>(excl, bi, t);
        }
        w.steps += 1;
        int code;
        if (best_i < 0) {
            w.blocked += 1;
            long_restart(lw, w, SL, base, V, t, &ps);
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
            long_note_best(lw, w, t, &ps);
            if (psl_better(ps.psl, w.isl, ps.since_psl, w.since)) {
                w.since = w.isl;
                ps.since_psl = ps.psl;
                w.stag = 0;
            } else {
                w.stag += 1;
            }
            code = best_i;
            if (w.stag >= env.patience || !stored) {
                long_restart(lw, w, SL, base, V, t, &ps);
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

// Best-first search for a long walker (the rules of walk_bestfirst, Algorithm 1 as
// printed): the queue's 32 keys ISL << 34 | (steps before the producing step) << 13 | i
// (ISL < 2^30 under the exact-range bound, at most LABS_BEST_FIRST_MAX_STEPS_LONG steps)
// sit in shared memory: the first warp updates them during the insertion, and every
// thread reads them when S moves, so each decision is taken identically by the whole
// CTA; the entries' bits (kBitWordsLong words each) are in global memory, each word
// written and read by the same thread.  An entry that differs from S in at most
// kBestFirstMaxFlips free variables is reached by that many incremental flips, any other
// by a rebuild.
constexpr uint64_t kLongEmpty = ~0ull;

__device__ __forceinline__ int long_queue_min(const uint64_t* Q, uint64_t& v)
{
    int k = -1;
    v = kLongEmpty;
#pragma unroll
    for (int j = 0; j < LABS_QUEUE_SIZE; ++j)
        if (Q[j] < v) {
            v = Q[j];
            k = j;
        }
    return k;
}

template <class LB, int R>
__device__ void long_walk_bestfirst(const LongWalk& lw, Walker& w, int64_t until, const WarpSmem& SL, int* base,
                                    const View& V, int trace_slot, int64_t trace_start, const LB& t, uint64_t* Q,
                                    uint32_t* qbits)
{
    const WalkEnv& env = lw.e;
    const KParams& p = *env.p;
    const int lane = t.lane, n = env.n;
    const Outs<LB, R> o(t);
    const int tisl = target_isl(p, env.L);
    uint64_t* WL = Q + LABS_QUEUE_SIZE;                  // [warps][32] each warp's lowest keys
    uint64_t* IK = WL + LB::kSize;                       // [32] keys entered in a round
    uint64_t* meta = IK + LABS_QUEUE_SIZE;               // entered | another round << 8; last key
    int* ID = reinterpret_cast<int*>(meta + 2);          // [32] their places in the queue
    float P[R];
    p_direct(V, n, o, P);
    StopCheck stop;
    stop.start(p, lane == 0);
    while (w.steps < until) {
        if (w.isl > lw.isl_limit) {
            if (lane == 0) raise_error(p.status, LABS_ERANGE, (int)env.g);
            break;
        }
        if ((w.steps & (kCheckEvery - 1)) == 0) {
            const int why = t.shfl(stop.poll(p, lane == 0), 0);
            if (why) {
                if (lane == 0) raise_error(p.status, why, (int)env.g);
                break;
            }
        }
        const uint64_t e = (uint64_t)w.steps;
        int dl[R];
        {
            float X[R];
            toeplitz_one(V, SL, n, o, t, X);
            assemble(V, n, o, X, P, dl);
        }
        // the queue's last entry at the start of the step (empty place: no bound)
        uint64_t last0 = 0;
        bool full0 = true;
#pragma unroll
        for (int j = 0; j < LABS_QUEUE_SIZE; ++j) {
            if (Q[j] == kLongEmpty) full0 = false;
            else last0 = max(last0, Q[j]);
        }
        if (!full0) last0 = kLongEmpty;
        uint64_t key[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            key[r] = kLongEmpty;
            if (dl[r] != INT_MAX) {
                const uint64_t ck = ((uint64_t)(uint32_t)(w.isl + dl[r]) << 34) | (e << 13) |
                                    (uint64_t)(2 * (o.v0 + r) + o.p);
                if (ck < last0) key[r] = ck;
            }
        }
        // Neighbours in queue order while they come before the queue's last entry or the
        // queue has a free place, in rounds of LABS_QUEUE_SIZE candidates: each warp sorts
        // out its lowest keys, the first warp merges them into the CTA's lowest, looks
        // them all up in HT at once (one per lane; HT does not change during the
        // insertion, so this equals looking each up when the insertion reaches it) and
        // runs the insertion on its registers; the other threads then write the entered
        // entries' bits.  An entry entered during the step is never replaced in the same
        // step (every later neighbour comes after it), so the places written are distinct.
        // A further round runs only when all LABS_QUEUE_SIZE candidates were taken or
        // skipped without reaching the queue's last entry.
        uint64_t floor = 0;
        for (;;) {
            {
                const int wl = lane & 31, wid = lane >> 5;
                uint64_t fl = floor;
                for (int k = 0; k < 32; ++k) {
                    uint64_t b = kLongEmpty;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (key[r] > fl) b = min(b, key[r]);
                    b = warp_min64(b);
                    if (wl == 0) WL[wid * 32 + k] = b;
                    if (b == kLongEmpty) break;
                    fl = b;
                }
            }
            t.sync();
            if (lane < 32) {
                int h = 0, cnt = 0;
                uint64_t v = lane < LB::kWarps ? WL[lane * 32] : kLongEmpty, mine = kLongEmpty;
                for (; cnt < LABS_QUEUE_SIZE; ++cnt) {
                    const uint64_t m = warp_min64(v);
                    if (m == kLongEmpty) break;
                    if (lane == cnt) mine = m;
                    if (v == m) {
                        ++h;
                        v = h < 32 ? WL[lane * 32 + h] : kLongEmpty;
                    }
                }
                bool vis = false;
                if (lane < cnt) {
                    const uint64_t f = w.fp ^ __ldg(env.zk + (int)(mine & 0x1FFFu));
                    const uint64_t tag = (f & ~kGenMask) | w.gen;
                    for (int s = 0; s < p.probe_cap; ++s) {
                        const uint64_t x = env.T[(f + (uint64_t)s) & env.tmask];
                        if (x == tag) {
                            vis = true;
                            break;
                        }
                        if ((x & kGenMask) != w.gen) break;
                    }
                }
                const unsigned visited = __ballot_sync(kFull, vis);
                uint64_t qk = Q[lane];
                int nins = 0;
                bool stopped = false;
                for (int k = 0; k < cnt; ++k) {
                    if ((visited >> k) & 1u) continue;
                    const uint64_t ck = __shfl_sync(kFull, mine, k);
                    const unsigned empty = __ballot_sync(kFull, qk == kLongEmpty);
                    int dst;
                    if (empty) {
                        dst = __ffs(empty) - 1;
                    } else {
                        const uint64_t last = warp_max64(qk);
                        if (ck > last) {
                            stopped = true;  // every later neighbour comes after it too
                            break;
                        }
                        dst = __ffs(__ballot_sync(kFull, qk == last)) - 1;
                    }
                    if (lane == dst) qk = ck;
                    if (lane == 0) {
                        IK[nins] = ck;
                        ID[nins] = dst;
                    }
                    ++nins;
                }
                Q[lane] = qk;
                const uint64_t lastc = __shfl_sync(kFull, mine, cnt > 0 ? cnt - 1 : 0);
                if (lane == 0) {
                    meta[0] = (uint64_t)nins | (!stopped && cnt == LABS_QUEUE_SIZE ? 256u : 0u);
                    meta[1] = lastc;
                }
            }
            t.sync();
            const int m0 = (int)meta[0], nins = m0 & 0xFF;
            for (int j = 0; j < nins; ++j) {
                const int i = (int)(IK[j] & 0x1FFFu);
                if (lane < lw.nw)
                    qbits[ID[j] * kBitWordsLong + lane] = w.word ^ (lane == (i >> 5) ? 1u << (i & 31) : 0u);
            }
            if (nins > 0) {  // the round's first entry has the lowest ISL entered so far
                const uint64_t ck = IK[0];
                const int i = (int)(ck & 0x1FFFu), isl_f = (int)(ck >> 34);
                if (isl_f < w.best_isl) {
                    w.best_isl = isl_f;
                    w.best_step = (int64_t)e + 1;
                    if (lane < lw.nw) lw.best[lane] = w.word ^ (lane == (i >> 5) ? 1u << (i & 31) : 0u);
                }
                if (w.target_step < 0 && isl_f <= tisl) w.target_step = (int64_t)e + 1;
            }
            if (!(m0 & 256)) break;
            floor = meta[1];
            t.sync();  // this round's lists are read before the next round writes them
        }
        // S <- the queue's first entry not in HT (entries that are get dropped)
        int code = LABS_TRACE_BLOCKED;
        bool again = true;
        for (;;) {
            uint64_t first;
            const int src = long_queue_min(Q, first);
            if (src < 0) {
                w.blocked += 1;  // empty queue: restart
                break;
            }
            const uint32_t word = lane < lw.nw ? qbits[src * kBitWordsLong + lane] : 0u;
            t.sync();  // every thread has read Q
            if (lane == 0) Q[src] = kLongEmpty;
            if (lane < lw.nw) lw.bits[lane] = word;
            t.sync();
            const int i = (int)(first & 0x1FFFu);
            const bool nb = ((first >> 13) & 0x1FFFFFull) == e;  // a neighbour of S
            const uint64_t f = nb ? (w.fp ^ __ldg(env.zk + i)) : long_fingerprint(lw, t);
            const Probe pr = long_probe(lw, f, w.gen, t);
            if (pr.visited) continue;
            // free variables in which the new S differs from S (1 for a neighbour)
            uint32_t diff = lane < lw.nw ? (word ^ w.word) : 0u;
            const int k = nb ? 1 : t.radd(__popc(diff));
            if (k <= kBestFirstMaxFlips) {
                for (int j = 0; j < k; ++j) {
                    const int lo = diff ? 32 * lane + __ffs(diff) - 1 : INT_MAX;
                    const int fi = nb ? i : t.rmin(lo);
                    flip_rows_table(V, n, o, P, fi, t);
                    t.sync();
                    if (lane == (fi >> 5)) diff &= ~(1u << (fi & 31));
                }
            } else {
                long_load_rows(lw, SL, base, V, word, t);
                p_direct(V, n, o, P);
            }
            w.word = word;
            w.isl = (int)(first >> 34);
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
            t.sync();
            if (lane < LABS_QUEUE_SIZE) Q[lane] = kLongEmpty;
            long_restart(lw, w, SL, base, V, t);
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
}

__device__ LongWalk long_env(const KParams& p, int64_t wi, const DevGroup& G, uint32_t* bits)
{
    LongWalk lw;
    lw.e.p = &p;
    lw.e.tmask = (1ull << p.tabu_log2) - 1ull;
    lw.e.T = p.tabu + ((uint64_t)wi << p.tabu_log2);
    lw.e.zk = p.zkeys + G.zkey_off;
    lw.e.st = p.states + wi;
    lw.e.L = G.L;
    lw.e.n = G.n;
    lw.e.patience = p.patience > 0 ? p.patience : 2 * G.n;
    lw.e.g = (uint32_t)wi;
    lw.e.slot = nullptr;
    lw.e.slot_valid = nullptr;
    lw.e.rdump = nullptr;
    lw.e.rdump_idx = nullptr;
    lw.e.rdump_count = nullptr;
    lw.e.dump_cap = 0;
    lw.cur = p.cur_bits + wi * kBitWordsLong;
    lw.best = p.best_bits + wi * kBitWordsLong;
    lw.bits = bits;
    lw.nw = (G.n + 31) / 32;
    lw.isl_limit = long_isl_limit(G.L, G.n);
    return lw;
}

// First start of every long walker (restart index 0, HT generation 1; HT zeroed by the
// caller), one walker per CTA at a time.
template <int NT>
__global__ void __launch_bounds__(NT, kLongThreads / NT) long_reset_kernel(KParams p)
{
    using LB = Blk<NT>;
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = long_smem(p.n_max, NT);
    const LB t(threadIdx.x, smem + SL.xoff);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem + SL.xoff + NT);
    const View V = make_view(smem, SL);
    for (int64_t wi = blockIdx.x; wi < p.W; wi += gridDim.x) {
        int gidx = 0;
        for (int g = 0; g < p.nG; ++g)
            if (wi >= p.groups[g].first && wi < p.groups[g].first + p.groups[g].count) gidx = g;
        const DevGroup G = p.groups[gidx];
        const LongWalk lw = long_env(p, wi, G, bits);
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
        const bool psl = p.mode == 3;
        long_start(lw, w, SL, smem, V, t, psl ? &ps : nullptr);
        if (t.lane < lw.nw) lw.cur[t.lane] = w.word;
        if (p.best_first && t.lane < LABS_QUEUE_SIZE) p.pq_key[wi * LABS_QUEUE_SIZE + t.lane] = ~0ull;
        if (t.lane == 0) {
            WalkerState* st = lw.e.st;
            save_scalars(st, w);
            st->group = gidx;
            st->trace_slot = -1;
            st->psl = psl ? ps.psl : -1;
            st->best_psl = psl ? ps.best_psl : -1;
            st->since_psl = psl ? ps.since_psl : -1;
        }
        t.sync();
    }
}

// One chunk of steps for every long walker; walkers are taken from a counter.  MODE: 0
// the walk, 1 the walk under the PSL objective, 2 the best-first search (its queue keys
// are copied into shared memory for the chunk and back at its end).
template <int NT, int R, int MODE>
__global__ void __launch_bounds__(NT, kLongThreads / NT) long_walk_kernel(KParams p, int chunk_index)
{
    using LB = Blk<NT>;
    extern __shared__ __align__(16) int smem[];
    const WarpSmem SL = long_smem(p.n_max, NT);
    const LB t(threadIdx.x, smem + SL.xoff);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem + SL.xoff + NT);
    const View V = make_view(smem, SL);
    const int64_t target = p.status->target_steps;
    for (;;) {
        int q = 0;
        if (t.lane == 0) q = (int)atomicAdd(&p.queue[chunk_index], 1u);
        const int64_t wi = (int64_t)(uint32_t)t.shfl(q, 0);
        if (wi >= p.W) break;
        WalkerState* st = p.states + wi;
        const int64_t steps_done = st->steps_done;
        const int64_t until = min(target, steps_done + (int64_t)p.chunk_steps);
        if (steps_done >= until) continue;
        const DevGroup G = p.groups[st->group];
        const LongWalk lw = long_env(p, wi, G, bits);
        Walker w;
        load_walker(st, w, 32);  // scalars only (lane 32 reads no bits)
        w.word = t.lane < lw.nw ? lw.cur[t.lane] : 0u;
        const int trace_slot = st->trace_slot;
        const int64_t trace_start = trace_slot >= 0 ? p.trace_start[trace_slot] : 0;
        const int isl = long_load_rows(lw, SL, smem, V, w.word, t);
        if (isl != w.isl) {
            if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)wi);
            continue;
        }
        if constexpr (MODE == 1) {
            PslTrack ps;
            ps.psl = table_psl(V, G.n, t);
            ps.best_psl = st->best_psl;
            ps.since_psl = st->since_psl;
            if (ps.psl != st->psl) {
                if (t.lane == 0) raise_error(p.status, LABS_ESTATE, (int)wi);
                continue;
            }
            long_walk_psl<LB, R>(lw, w, ps, until, SL, smem, V, trace_slot, trace_start, t);
            if (t.lane == 0) {
                st->psl = ps.psl;
                st->best_psl = ps.best_psl;
                st->since_psl = ps.since_psl;
            }
        } else if constexpr (MODE == 2) {
            uint64_t* Q = reinterpret_cast<uint64_t*>(smem + SL.xoff + NT + kBitWordsLong);
            uint64_t* qk = p.pq_key + wi * LABS_QUEUE_SIZE;
            if (t.lane < LABS_QUEUE_SIZE) Q[t.lane] = qk[t.lane];
            t.sync();
            long_walk_bestfirst<LB, R>(lw, w, until, SL, smem, V, trace_slot, trace_start, t, Q,
                                       p.pq_bits + wi * LABS_QUEUE_SIZE * kBitWordsLong);
            t.sync();
            if (t.lane < LABS_QUEUE_SIZE) qk[t.lane] = Q[t.lane];
        } else {
            long_walk<LB, R>(lw, w, until, SL, smem, V, trace_slot, trace_start, t);
        }
        if (t.lane < lw.nw) lw.cur[t.lane] = w.word;
        if (t.lane == 0) save_scalars(st, w);
        t.sync();
    }
}

// The neighbourhood of Algorithm 1 for long skew-symmetric rows, one row per CTA.
// Rows that are not +-1 or break Eq. 4 get INT32_MIN (LABS_EINVAL); rows whose ISL is
// above the exact-range bound get INT32_MIN too (LABS_ERANGE).
template <int NT, int R>
__global__ void __launch_bounds__(NT, kLongThreads / NT) long_delta_kernel(const int8_t* __restrict__ seqs,
                                                                          int64_t batch, int L,
                                                                          int32_t* __restrict__ out, DevStatus* status)
{
    using LB = Blk<NT>;
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = long_smem(n, NT);
    const LB t(threadIdx.x, smem + SL.xoff);
    const View V = make_view(smem, SL);
    const Outs<LB, R> o(t);
    for (int64_t row = blockIdx.x; row < batch; row += gridDim.x) {
        const int8_t* src = seqs + row * (int64_t)L;
        long_clear(smem, SL, t);
        bool ok = true;
        for (int j = t.lane; j < L; j += LB::kSize) {
            const int v = src[j];
            ok = ok && (v == 1 || v == -1);
            if (j > c) {
                const int m = src[2 * c - j];
                ok = ok && (v == ((((j - c) & 1) ? -m : m)));
            }
            set_row(V, j & 1, j >> 1, (float)v);
        }
        const bool all_ok = t.rmin(ok ? 1 : 0) != 0;
        int32_t* dst = out + row * (int64_t)n;
        if (!all_ok) {
            for (int i = t.lane; i < n; i += LB::kSize) dst[i] = INT32_MIN;
            if (t.lane == 0 && status) {
                atomicAdd(&status->invalid_rows, 1);
                raise_error(status, LABS_EINVAL, (int)row);
            }
            t.sync();
            continue;
        }
        const int isl = build_table(V, n, t);
        if (isl > long_isl_limit(L, n)) {
            for (int i = t.lane; i < n; i += LB::kSize) dst[i] = INT32_MIN;
            if (t.lane == 0 && status) raise_error(status, LABS_ERANGE, (int)row);
            t.sync();
            continue;
        }
        int dl[R];
        {
            float X[R], P[R];
            toeplitz_one(V, SL, n, o, t, X);
            p_direct(V, n, o, P);
            assemble(V, n, o, X, P, dl);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (dl[r] != INT_MAX) dst[2 * (o.v0 + r) + o.p] = dl[r];
        t.sync();
    }
}

using LongFn = void (*)(KParams, int);
using LongDeltaFn = void (*)(const int8_t*, int64_t, int, int32_t*, DevStatus*);

// Lane blocks in use (long_R): 3..9 with 128 or 256 threads (257 <= n <= 2304), 5..11
// with 512 (2304 < n <= 5632).
template <int NT, int MODE>
LongFn long_fn_nt(int R)
{
    if constexpr (NT != kLongThreads) {
        switch (R) {
            case 3: return long_walk_kernel<NT, 3, MODE>;
            case 5: return long_walk_kernel<NT, 5, MODE>;
            case 7: return long_walk_kernel<NT, 7, MODE>;
            default: return long_walk_kernel<NT, 9, MODE>;
        }
    } else {
        switch (R) {
            case 5: return long_walk_kernel<NT, 5, MODE>;
            case 7: return long_walk_kernel<NT, 7, MODE>;
            case 9: return long_walk_kernel<NT, 9, MODE>;
            default: return long_walk_kernel<NT, 11, MODE>;
        }
    }
}

template <int MODE>
LongFn long_fn_mode(int NT, int R)
{
    return NT == kLongThreadsSmall ? long_fn_nt<kLongThreadsSmall, MODE>(R)
           : NT == kLongThreadsMid ? long_fn_nt<kLongThreadsMid, MODE>(R)
                                   : long_fn_nt<kLongThreads, MODE>(R);
}

template <int NT>
LongDeltaFn long_delta_fn_nt(int R)
{
    if constexpr (NT != kLongThreads) {
        switch (R) {
            case 3: return long_delta_kernel<NT, 3>;
            case 5: return long_delta_kernel<NT, 5>;
            case 7: return long_delta_kernel<NT, 7>;
            default: return long_delta_kernel<NT, 9>;
        }
    } else {
        switch (R) {
            case 5: return long_delta_kernel<NT, 5>;
            case 7: return long_delta_kernel<NT, 7>;
            case 9: return long_delta_kernel<NT, 9>;
            default: return long_delta_kernel<NT, 11>;
        }
    }
}

// kernels for n_max free variables: CTA width long_threads(n_max), lane block long_R;
// mode 0 the walk, 1 the walk under the PSL objective, 2 the best-first search
LongFn long_fn(int n_max, int mode)
{
    const int NT = long_threads(n_max, mode == 1), R = long_R(n_max, NT);
    return mode == 1 ? long_fn_mode<1>(NT, R) : mode == 2 ? long_fn_mode<2>(NT, R) : long_fn_mode<0>(NT, R);
}

LongDeltaFn long_delta_fn(int n)
{
    const int NT = long_threads(n), R = long_R(n, NT);
    return NT == kLongThreadsSmall ? long_delta_fn_nt<kLongThreadsSmall>(R)
           : NT == kLongThreadsMid ? long_delta_fn_nt<kLongThreadsMid>(R)
                                   : long_delta_fn_nt<kLongThreads>(R);
}

using ResetFn = void (*)(KParams);
ResetFn long_reset_fn(int n_max, bool psl)
{
    const int NT = long_threads(n_max, psl);
    return NT == kLongThreadsSmall ? long_reset_kernel<kLongThreadsSmall>
           : NT == kLongThreadsMid ? long_reset_kernel<kLongThreadsMid>
                                   : long_reset_kernel<kLongThreads>;
}

}  // namespace

int long_kernel_config(int n_max, int mode, size_t smem_bytes, int* ctas_per_sm, int* regs)
{
    const LongFn fn = long_fn(n_max, mode);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return LABS_ECUDA;
    e = cudaFuncSetAttribute(long_reset_fn(n_max, mode == 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return LABS_ECUDA;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return LABS_ECUDA;
    if (regs) *regs = fa.numRegs;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, long_threads(n_max, mode == 1), smem_bytes);
    return e == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int launch_long_reset(const KParams& p, size_t smem_bytes, void* stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = p.W < sms ? (p.W > 0 ? p.W : 1) : sms;
    const bool psl = p.mode == 3;
    long_reset_fn(p.n_max, psl)<<<(int)grid, long_threads(p.n_max, psl), smem_bytes, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int launch_long_walk_chunk(const KParams& p, int chunk_index, int grid, size_t smem_bytes, void* stream)
{
    const int mode = p.mode == 3 ? 1 : p.mode == 2 ? 2 : 0;
    long_fn(p.n_max, mode)<<<grid, long_threads(p.n_max, mode == 1), smem_bytes, (cudaStream_t)stream>>>(p,
                                                                                                    chunk_index);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

int launch_long_delta(const int8_t* seqs, int64_t batch, int32_t L, int32_t* out, DevStatus* status, void* stream)
{
    if (batch == 0) return LABS_OK;
    const int n = (L + 1) / 2;
    const size_t smem = (size_t)long_smem(n, long_threads(n)).words * sizeof(int);
    const LongDeltaFn fn = long_delta_fn(n);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LABS_ECUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // as many resident CTAs as fit (four per SM with 128 threads, two with 256, one with 512)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, long_threads(n), smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t slots = (int64_t)per_sm * sms;
    const int grid = (int)(batch < slots ? batch : slots);
    fn<<<grid, long_threads(n), smem, (cudaStream_t)stream>>>(seqs, batch, L, out, status);
    return cudaGetLastError() == cudaSuccess ? LABS_OK : LABS_ECUDA;
}

}  // namespace labsgpu
