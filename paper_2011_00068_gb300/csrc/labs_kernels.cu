// labs_kernels.cu -- sm_103a kernels of the skew-symmetric LABS search
// (Brest & Boskovic, arXiv 2011.00068): walker starts, the stateless row kernels
// (ISL, neighbourhood), learned-proposal support, reductions and the launchers.
// The walk itself is in labs_device.cuh, instantiated by the labs_walk*.cu units.
#include <algorithm>

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

template <int R>
__device__ void delta_row(const View& V, int n, const Tile<32>& t, int32_t* dst)
{
    const Outs<Tile<32>, R> o(t);
    int dl[R];
    {
        float X[R], P[R];
        toeplitz(V, n, o, X);
        p_direct(V, n, o, P);
        assemble(V, n, o, X, P, dl);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (dl[r] != INT_MAX) dst[2 * (o.v0 + r) + o.p] = dl[r];
}

// The neighbourhood of Algorithm 1 for skew-symmetric rows, one warp per row, R
// outputs per lane (R = block_R(n, 32), odd, chosen by the host).
template <int R>
__global__ void __launch_bounds__(256) delta_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                    int32_t* __restrict__ out, DevStatus* status)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = warp_smem(n, 32);
    const Tile<32> t(threadIdx.x & 31);
    const int lane = t.lane, warp = threadIdx.x >> 5;
    int* base = smem + warp * SL.words;
    const View V = make_view(base, SL);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; row < batch; row += nwarps) {
        clear_rows(base, SL, t);
        const int8_t* src = seqs + row * (int64_t)L;
        bool ok = true;
        for (int j = lane; j < L; j += kWarp) {
            const int v = src[j];
            ok = ok && (v == 1 || v == -1);
            if (j & 1) V.A1[j >> 1] = (float)v;
            else V.A0[j >> 1] = (float)v;
        }
        t.sync();
        for (int j = 1 + lane; j <= c; j += kWarp) {  // Eq. 4
            const int hi = c + j, lo = c - j;
            const float shi = (hi & 1) ? V.A1[hi >> 1] : V.A0[hi >> 1];
            const float slo = (lo & 1) ? V.A1[lo >> 1] : V.A0[lo >> 1];
            ok = ok && (shi == ((j & 1) ? -slo : slo));
        }
        int32_t* dst = out + row * (int64_t)n;
        if (!__all_sync(kFull, ok)) {
            for (int i = lane; i < n; i += kWarp) dst[i] = INT_MIN;
            if (lane == 0 && status) atomicAdd(&status->invalid_rows, 1);
            t.sync();
            continue;
        }
        build_table(V, n, t);
        delta_row<R>(V, n, t, dst);
        t.sync();
    }
}

// The same for two rows per warp (n <= 160), 16 lanes per row in lockstep: rows r0, r0+1
// of each warp; R = block_R(n, 16).  The rows' shared memory is cleared once, each row
// overwrites every entry the previous one set.
template <int R>
__global__ void __launch_bounds__(256) delta_pair_kernel(const int8_t* __restrict__ seqs, int64_t batch, int L,
                                                         int32_t* __restrict__ out, DevStatus* status)
{
    extern __shared__ __align__(16) int smem[];
    const int n = (L + 1) / 2, c = n - 1;
    const WarpSmem SL = warp_smem(n, 16);
    const Pair t(threadIdx.x & 31);
    const int lane = t.lane;
    int* base = smem + (threadIdx.x / 16) * SL.words;
    const View V = make_view(base, SL);
    const Outs<Pair, R> o(t);
    clear_rows(base, SL, t);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r0 = 2 * ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); r0 < batch;
         r0 += 2 * nwarps) {
        const int64_t row = r0 + t.h;
        const bool has = row < batch;
        const int8_t* src = seqs + row * (int64_t)L;
        bool ok = true;
        if (has) {
            for (int j = lane; j < L; j += 16) {
                const int v = src[j];
                ok = ok && (v == 1 || v == -1);
                ((j & 1) ? V.A1 : V.A0)[j >> 1] = (float)v;
            }
        }
        t.sync();
        if (has) {
            for (int j = 1 + lane; j <= c; j += 16) {  // Eq. 4
                const int hi = c + j, lo = c - j;
                const float shi = (hi & 1) ? V.A1[hi >> 1] : V.A0[hi >> 1];
                const float slo = (lo & 1) ? V.A1[lo >> 1] : V.A0[lo >> 1];
                ok = ok && (shi == ((j & 1) ? -slo : slo));
            }
        }
        const bool valid = has && t.ballot(!ok) == 0u;
        int32_t* dst = out + row * (int64_t)n;
        if (has && !valid) {
            for (int i = lane; i < n; i += 16) dst[i] = INT_MIN;
            if (lane == 0 && status) atomicAdd(&status->invalid_rows, 1);
        }
        build_table(V, n, t);
        int dl[R];
        int rv;
        {
            float X[R], P[R];
            toeplitz(V, n, o, X);
            p_direct(V, n, o, P);
            rv = lane_dl(V, n, o, X, P, dl);
        }
        if (valid) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r < rv) dst[2 * (o.v0 + r) + o.p] = dl[r];
        }
        t.sync();
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
    const int warps = 8, n = (L + 1) / 2;
    using DeltaFn = void (*)(const int8_t*, int64_t, int, int32_t*, DevStatus*);
    DeltaFn fn;
    if (block_R(n, 16) <= 10) {  // two rows per warp
        const size_t smem = (size_t)2 * warps * warp_smem(n, 16).words * sizeof(int);
        switch (block_R(n, 16)) {
            case 1: fn = delta_pair_kernel<1>; break;
            case 2: fn = delta_pair_kernel<2>; break;
            case 3: fn = delta_pair_kernel<3>; break;
            case 5: fn = delta_pair_kernel<5>; break;
            case 6: fn = delta_pair_kernel<6>; break;
            case 7: fn = delta_pair_kernel<7>; break;
            case 9: fn = delta_pair_kernel<9>; break;
            default: fn = delta_pair_kernel<10>; break;
        }
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fn<<<row_grid((batch + 1) / 2, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out,
                                                                                           status);
        return status_of(cudaGetLastError());
    }
    const size_t smem = (size_t)warps * warp_smem(n, 32).words * sizeof(int);
    switch (lanes_for(n, 32)) {
        case 1: fn = delta_kernel<1>; break;
        case 3: fn = delta_kernel<3>; break;
        case 5: fn = delta_kernel<5>; break;
        case 7: fn = delta_kernel<7>; break;
        default: fn = delta_kernel<9>; break;
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<row_grid(batch, warps), warps * kWarp, smem, (cudaStream_t)stream>>>(seqs, batch, L, out, status);
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
