// labs_api.cu -- host side of the liblabs C ABI (include/labs.h): contexts, workspace
// layout, chunked and graph-captured walk launches, reductions, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "labs_internal.cuh"
#include "labs_nvtx.h"

using namespace labsgpu;

struct labs_ctx {
    labs_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;  // private stream used only to record CUDA graphs
    uint64_t seed = 0;
    int device = 0;
    int sms = 0;
    int nG = 0;
    DevGroup groups[LABS_MAX_GROUPS];
    int64_t W = 0;
    int n_max = 0;
    // workspace layout (byte offsets)
    size_t off_status = 0, off_groups = 0, off_zkeys = 0, off_states = 0, off_trace_start = 0,
           off_trace_ids = 0, off_queue = 0, off_l_scores = 0, off_l_step = 0, off_l_slot = 0, off_l_valid = 0,
           off_pq_key = 0, off_pq_bits = 0, off_cur_bits = 0, off_best_bits = 0, off_tabu = 0, off_tabu2 = 0,
           total = 0;
    bool long_mode = false;  // lengths above LABS_MAX_L: one walker per CTA, bits beside the states
    // device pointers kept in the status block (restored after every reset)
    labs_log_record* log = nullptr;
    int64_t log_capacity = 0, log_start = 0;
    float* d_scores = nullptr;
    int64_t* d_score_step = nullptr;
    int32_t* d_score_count = nullptr;
    uint32_t* d_restart = nullptr;
    int64_t* d_restart_idx = nullptr;
    int32_t* d_restart_count = nullptr;
    int32_t d_cap = 0;
    // learned mode
    const float* l_params = nullptr;
    int32_t l_tau = 0, l_cands = 0;
    char* l_ws = nullptr;
    size_t l_ws_bytes = 0;
    char* ws = nullptr;
    Control* ctrl_host = nullptr;
    Control* ctrl_dev = nullptr;
    long long gpu_minus_host_ns = 0;
    int warps_per_cta = 0, ctas_per_sm = 0, grid = 0, chunk = 0, regs = 0, tile = 32;
    size_t smem_bytes = 0;
    bool catch_up = false;
    int64_t planned = 0;
    std::map<int, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

constexpr uint64_t kCkptMagic = 0x4C41425343503031ull;  // "LABSCP01"

int fail(labs_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(labs_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, LABS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a)
{
    return (x + a - 1) / a * a;
}

long long host_ns()
{
    timespec ts;
    clock_gettime(CLOCK_REALTIME, &ts);
    return (long long)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

template <class T>
T* at(labs_ctx* c, size_t off)
{
    return reinterpret_cast<T*>(c->ws + off);
}

KParams params(labs_ctx* c)
{
    KParams p;
    p.status = at<DevStatus>(c, c->off_status);
    p.groups = at<DevGroup>(c, c->off_groups);
    p.zkeys = at<uint64_t>(c, c->off_zkeys);
    p.states = at<WalkerState>(c, c->off_states);
    p.tabu = at<uint64_t>(c, c->off_tabu);
    p.trace_start = at<int64_t>(c, c->off_trace_start);
    p.queue = at<uint32_t>(c, c->off_queue);
    p.ctrl = c->ctrl_dev;
    p.W = c->W;
    p.nG = c->nG;
    p.n_max = c->n_max;
    p.tabu_log2 = c->cfg.tabu_log2;
    p.probe_cap = c->cfg.probe_cap;
    p.patience = c->cfg.patience;
    p.target_num = c->cfg.target_num;
    p.target_den = c->cfg.target_den;
    p.chunk_steps = c->chunk;
    p.rmax = c->long_mode ? long_R(c->n_max, c->tile) : lanes_for(c->n_max, c->tile);
    p.tile = c->tile;
    p.long_mode = c->long_mode ? 1 : 0;
    p.cur_bits = c->long_mode ? at<uint32_t>(c, c->off_cur_bits) : nullptr;
    p.best_bits = c->long_mode ? at<uint32_t>(c, c->off_best_bits) : nullptr;
    p.seed = c->seed;
    p.best_first = (c->cfg.flags & LABS_FLAG_BEST_FIRST) ? 1 : 0;
    p.pq_key = p.best_first ? at<uint64_t>(c, c->off_pq_key) : nullptr;
    p.pq_bits = p.best_first ? at<uint32_t>(c, c->off_pq_bits) : nullptr;
    p.tabu2 = (c->cfg.flags & LABS_FLAG_SECOND_HASH) ? at<uint64_t>(c, c->off_tabu2) : nullptr;
    p.mode = (c->cfg.flags & LABS_FLAG_PSL) ? 3 : p.best_first ? 2 : (c->l_params ? 1 : 0);
    return p;
}

bool valid_L(int32_t L)
{
    return L >= 3 && L <= LABS_MAX_L && (L & 1) == 1;
}

bool valid_long_L(int32_t L)
{
    return L > LABS_MAX_L && L <= LABS_MAX_L_LONG && (L & 1) == 1;
}

// Free-variable bits of walker w's current (best = false) or best sequence.
int walker_bits(labs_ctx* c, int64_t w, const WalkerState& ws, bool best, uint32_t* out)
{
    if (!c->long_mode) {
        memcpy(out, best ? ws.best : ws.cur, sizeof(uint32_t) * kBitWords);
        return LABS_OK;
    }
    const size_t off = (best ? c->off_best_bits : c->off_cur_bits) + sizeof(uint32_t) * kBitWordsLong * (size_t)w;
    const cudaError_t e = cudaMemcpy(out, c->ws + off, sizeof(uint32_t) * kBitWordsLong, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LABS_OK : cuda_fail(c, e, "walker bits read");
}

// One chunk launch of the walk kernel of this context.
int launch_chunk(labs_ctx* c, const KParams& p, int j, cudaStream_t stream)
{
    if (c->long_mode) return launch_long_walk_chunk(p, j, c->grid, c->smem_bytes, stream);
    return launch_walk_chunk(p, j, c->grid, c->warps_per_cta, c->smem_bytes, stream);
}

int need_ws(labs_ctx* c)
{
    if (!c) return LABS_EINVAL;
    if (!c->ws) return fail(c, LABS_ENOMEM, "no workspace bound (labs_bind_workspace)");
    return LABS_OK;
}

// Sequence (+-1) of free-variable bits by Eq. 4.
void expand_bits(const uint32_t* bits, int L, int8_t* out)
{
    const int n = (L + 1) / 2, c = n - 1;
    for (int j = 0; j < L; ++j) {
        const int f = j <= c ? j : 2 * c - j;
        int x = ((bits[f >> 5] >> (f & 31)) & 1u) ? -1 : 1;
        if (j > c && ((j - c) & 1)) x = -x;
        out[j] = (int8_t)x;
    }
}

// Encoding described below Table 1: first symbol most significant, 0 <-> +1,
// 1 <-> -1, leading zero bits up to whole hex digits.
void hex_of(const int8_t* s, int L, char* out)
{
    static const char digits[] = "0123456789ABCDEF";
    const int nd = (L + 3) / 4, pad = 4 * nd - L;
    for (int d = 0; d < nd; ++d) {
        int v = 0;
        for (int t = 0; t < 4; ++t) {
            const int b = 4 * d + t - pad;
            v = (v << 1) | (b >= 0 && s[b] < 0 ? 1 : 0);
        }
        out[d] = digits[v];
    }
    out[nd] = 0;
}

int setup(labs_ctx* c, const int32_t* Ls, const int64_t* counts, int32_t nL, uint64_t seed,
          const labs_config* cfg, void* stream)
{
    labs_default_config(&c->cfg);
    if (cfg) c->cfg = *cfg;
    labs_config& k = c->cfg;
    if (k.tabu_log2 < 1 || k.tabu_log2 > 20) return fail(c, LABS_EINVAL, "tabu_log2 must be 1..20");
    if (k.probe_cap < 1 || k.probe_cap > 32) return fail(c, LABS_EINVAL, "probe_cap must be 1..32");
    if (k.patience < 0 || k.chunk_steps < 0 || k.warps_per_cta < 0 || k.warps_per_cta > 8)
        return fail(c, LABS_EINVAL, "bad patience / chunk_steps / warps_per_cta (0..8)");
    if (nL < 1 || nL > LABS_MAX_GROUPS) return fail(c, LABS_EINVAL, "need 1..%d lengths", LABS_MAX_GROUPS);
    if ((k.flags & LABS_FLAG_LEARNED) && (k.flags & LABS_FLAG_LEARNED_RESTARTS))
        return fail(c, LABS_EINVAL, "LABS_FLAG_LEARNED and LABS_FLAG_LEARNED_RESTARTS do not combine");
    if ((k.flags & LABS_FLAG_BEST_FIRST) && (k.flags & kLearnedAny))
        return fail(c, LABS_EINVAL, "LABS_FLAG_BEST_FIRST and the learned modes do not combine");
    if ((k.flags & LABS_FLAG_SECOND_HASH) && !(k.flags & LABS_FLAG_BEST_FIRST))
        return fail(c, LABS_EINVAL, "LABS_FLAG_SECOND_HASH needs LABS_FLAG_BEST_FIRST");
    if ((k.flags & LABS_FLAG_PSL) && (k.flags & (LABS_FLAG_BEST_FIRST | kLearnedAny)))
        return fail(c, LABS_EINVAL, "LABS_FLAG_PSL combines with neither LABS_FLAG_BEST_FIRST nor the learned modes");
    if (nL >= 1 && Ls && valid_long_L(Ls[0])) {
        c->long_mode = true;
        if (k.flags & (kLearnedAny | LABS_FLAG_SECOND_HASH))
            return fail(c, LABS_EINVAL, "lengths above %d run the walk (plain or PSL objective) or the best-first "
                        "search without the second table", LABS_MAX_L);
    }
    c->seed = seed;
    c->stream = (cudaStream_t)stream;
    c->nG = nL;
    int64_t first = 0, zoff = 0;
    for (int g = 0; g < nL; ++g) {
        if (c->long_mode ? !valid_long_L(Ls[g]) : !valid_L(Ls[g]))
            return fail(c, LABS_EINVAL, "L=%d: need odd 3 <= L <= %d, or odd %d < L <= %d (every length of a context "
                        "on the same side)", Ls[g], LABS_MAX_L, LABS_MAX_L, LABS_MAX_L_LONG);
        if (counts[g] < 0) return fail(c, LABS_EINVAL, "negative walker count");
        DevGroup& G = c->groups[g];
        G.L = Ls[g];
        G.n = (Ls[g] + 1) / 2;
        G.first = first;
        G.count = counts[g];
        G.zkey_off = zoff;
        first += counts[g];
        zoff += G.n;
        c->n_max = std::max(c->n_max, G.n);
    }
    c->W = first;
    if (c->W > (int64_t)UINT32_MAX - 1) return fail(c, LABS_EINVAL, "too many walkers");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceGetAttribute");
    // workspace layout
    size_t off = 0;
    c->off_status = off;
    off = align_up(off + sizeof(DevStatus), 256);
    c->off_groups = off;
    off = align_up(off + sizeof(DevGroup) * LABS_MAX_GROUPS, 256);
    c->off_zkeys = off;
    off = align_up(off + sizeof(uint64_t) * (size_t)zoff, 256);
    c->off_states = off;
    off = align_up(off + sizeof(WalkerState) * (size_t)c->W, 256);
    if (c->long_mode) {
        c->off_cur_bits = off;
        off = align_up(off + sizeof(uint32_t) * kBitWordsLong * (size_t)c->W, 256);
        c->off_best_bits = off;
        off = align_up(off + sizeof(uint32_t) * kBitWordsLong * (size_t)c->W, 256);
    }
    c->off_trace_start = off;
    off = align_up(off + sizeof(int64_t) * kMaxTrace, 256);
    c->off_trace_ids = off;
    off = align_up(off + sizeof(int64_t) * kMaxTrace, 256);
    c->off_queue = off;
    off = align_up(off + sizeof(uint32_t) * kMaxChunksPerCall, 256);
    if (k.flags & kLearnedAny) {
        c->off_l_scores = off;
        off = align_up(off + sizeof(float) * (size_t)c->W * c->n_max, 256);
        c->off_l_step = off;
        off = align_up(off + sizeof(int64_t) * (size_t)c->W, 256);
        c->off_l_slot = off;
        off = align_up(off + sizeof(uint32_t) * kBitWords * (size_t)c->W, 256);
        c->off_l_valid = off;
        off = align_up(off + sizeof(int32_t) * (size_t)c->W, 256);
    }
    if (k.flags & LABS_FLAG_BEST_FIRST) {
        c->off_pq_key = off;
        off = align_up(off + sizeof(uint64_t) * LABS_QUEUE_SIZE * (size_t)c->W, 256);
        c->off_pq_bits = off;
        const size_t qwords = c->long_mode ? kBitWordsLong : kBitWords;
        off = align_up(off + sizeof(uint32_t) * qwords * LABS_QUEUE_SIZE * (size_t)c->W, 256);
    }
    c->off_tabu = off;
    off = align_up(off + sizeof(uint64_t) * ((size_t)c->W << k.tabu_log2), 256);
    if (k.flags & LABS_FLAG_SECOND_HASH) {  // zeroed with HT by labs_reset (it follows HT)
        c->off_tabu2 = off;
        off = align_up(off + sizeof(uint64_t) * ((size_t)c->W << k.tabu_log2), 256);
    }
    c->total = off;
    // launch shape of the walk kernel: four walkers per warp (8 lanes each) while 8
    // lanes cover n with at most kQuadMaxR outputs per lane (n <= 80; measured faster
    // than two per warp there, equal from n = 88 to 104), two walkers per warp (16 lanes
    // each, the Toeplitz product on the tensor cores) up to n = 128, else one walker per
    // warp (tensor-core product; measured 7-12% faster than two walkers per warp with the
    // FP32 product from n = 129 to 160, which LABS_FLAG_TWO_PER_WARP keeps; the learned
    // mode and the best-first search run one walker per warp).  The PSL objective runs
    // two walkers per warp up to n = 128 (LABS_FLAG_WARP_PER_WALKER: one per warp), one
    // above.
    if (c->long_mode) {
        // one walker per CTA of 256 or 512 threads
        c->tile = long_threads(c->n_max, (k.flags & LABS_FLAG_PSL) != 0);
        c->smem_bytes = (size_t)long_smem(c->n_max, c->tile).words * sizeof(int);
        int occ = 0;
        const int mode = (k.flags & LABS_FLAG_PSL) ? 1 : (k.flags & LABS_FLAG_BEST_FIRST) ? 2 : 0;
        if (long_kernel_config(c->n_max, mode, c->smem_bytes, &occ, &c->regs) != LABS_OK ||
            occ < 1)
            return fail(c, LABS_ECUDA, "long walk kernel does not fit on an SM (%zu bytes of shared memory)",
                        c->smem_bytes);
        c->ctas_per_sm = occ;
        c->warps_per_cta = c->tile / kWarp;
        c->grid = c->sms * c->ctas_per_sm;
        c->chunk = k.chunk_steps ? k.chunk_steps : 64;
    } else {
        const bool psl = (k.flags & LABS_FLAG_PSL) != 0;
        if (psl)
            c->tile = c->n_max <= 128 && !(k.flags & LABS_FLAG_WARP_PER_WALKER) ? 16 : 32;
        else if ((k.flags & (LABS_FLAG_WARP_PER_WALKER | LABS_FLAG_LEARNED | LABS_FLAG_BEST_FIRST)) ||
                 lanes_for(c->n_max, 16) > 10 || (c->n_max > 128 && !(k.flags & LABS_FLAG_TWO_PER_WARP)))
            c->tile = 32;
        else if (!(k.flags & LABS_FLAG_TWO_PER_WARP) && lanes_for(c->n_max, 8) <= kQuadMaxR)
            c->tile = 8;
        else
            c->tile = 16;
        const size_t per_warp = (size_t)warp_smem(c->n_max, c->tile, psl).words * sizeof(int) * (kWarp / c->tile);
        int warps = k.warps_per_cta ? k.warps_per_cta : 8;
        for (;;) {
            c->smem_bytes = per_warp * (size_t)warps;
            int occ = 0;
            const int mode = (k.flags & LABS_FLAG_PSL) ? 3 : (k.flags & LABS_FLAG_BEST_FIRST) ? 2 : 0;
            if (walk_kernel_config(c->tile, lanes_for(c->n_max, c->tile), mode, warps, c->smem_bytes, &occ,
                                   &c->regs) == LABS_OK &&
                occ > 0) {
                c->ctas_per_sm = occ;
                break;
            }
            if (warps == 1) return fail(c, LABS_ECUDA, "walk kernel does not fit on an SM");
            warps /= 2;
        }
        c->warps_per_cta = warps;
        c->grid = c->sms * c->ctas_per_sm;
        c->chunk = k.chunk_steps ? k.chunk_steps : 1024;
    }
    e = cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreate");
    e = cudaHostAlloc((void**)&c->ctrl_host, sizeof(Control), cudaHostAllocMapped);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaHostAlloc");
    c->ctrl_host->stop = 0;
    c->ctrl_host->deadline_ns = UINT64_MAX;
    e = cudaHostGetDevicePointer((void**)&c->ctrl_dev, c->ctrl_host, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaHostGetDevicePointer");
    return LABS_OK;
}

int create(labs_ctx** out, const int32_t* Ls, const int64_t* counts, int32_t nL, uint64_t seed,
           const labs_config* cfg, void* stream)
{
    if (!out || !Ls || !counts) return LABS_EINVAL;
    *out = nullptr;
    labs_ctx* c = new (std::nothrow) labs_ctx();
    if (!c) return LABS_ENOMEM;
    const int rc = setup(c, Ls, counts, nL, seed, cfg, stream);
    *out = c;  // returned even on failure so that labs_last_error can explain; caller destroys
    return rc;
}

int sync_status(labs_ctx* c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
    DevStatus st;
    e = cudaMemcpy(&st, at<DevStatus>(c, c->off_status), sizeof(DevStatus), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    if (st.error) {
        const char* what = st.error == LABS_ETIMEOUT     ? "deadline passed"
                           : st.error == LABS_ECANCELLED ? "cancelled"
                           : st.error == LABS_ESTATE     ? "walker state failed its consistency check"
                           : st.error == LABS_ERANGE     ? "sequence outside the exact range of the long walk"
                                                         : "device error";
        return fail(c, st.error, "%s (walker %d)", what, st.error_detail);
    }
    if (st.invalid_rows) {
        const int32_t zero = 0;
        cudaMemcpy(&at<DevStatus>(c, c->off_status)->invalid_rows, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        return fail(c, LABS_EINVAL, "%d input rows were not +-1 / not skew-symmetric", st.invalid_rows);
    }
    return LABS_OK;
}

// Writes the log / learned / dump pointers into the device status block.
int push_status(labs_ctx* c)
{
    DevStatus h;
    memset(&h, 0, sizeof(h));
    h.log = c->log;
    h.log_capacity = c->log_capacity;
    h.log_start = c->log_start;
    const bool lw = (c->cfg.flags & kLearnedAny) != 0;
    h.l_scores = lw ? at<float>(c, c->off_l_scores) : nullptr;
    h.l_score_step = lw ? at<int64_t>(c, c->off_l_step) : nullptr;
    h.l_slot = lw ? at<uint32_t>(c, c->off_l_slot) : nullptr;
    h.l_slot_valid = lw ? at<int32_t>(c, c->off_l_valid) : nullptr;
    h.l_tau = c->l_tau;
    h.learned = (lw && c->l_params) ? 1 : 0;
    h.d_scores = c->d_scores;
    h.d_score_step = c->d_score_step;
    h.d_score_count = c->d_score_count;
    h.d_restart = c->d_restart;
    h.d_restart_idx = c->d_restart_idx;
    h.d_restart_count = c->d_restart_count;
    h.d_cap = c->d_cap;
    const size_t a = offsetof(DevStatus, log), b = offsetof(DevStatus, pad1);
    cudaError_t e = cudaMemcpyAsync(c->ws + c->off_status + a, reinterpret_cast<char*>(&h) + a, b - a,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LABS_OK : cuda_fail(c, e, "status pointers");
}

constexpr int64_t kProposalBatch = 8192;  // states per network call in a proposal pass

size_t learned_ws_bytes(const labs_ctx* c, int cands)
{
    const size_t x = align_up(sizeof(float) * 3 * (size_t)c->n_max * kProposalBatch, 256);
    const size_t cand = align_up(sizeof(uint32_t) * kBitWords * (size_t)kProposalBatch, 256);
    (void)cands;
    return x + cand + net_workspace_bytes(kProposalBatch, c->n_max);
}

// Flip scores and restart proposals for every walker (learned mode), before a chunk.
int proposal_pass(labs_ctx* c)
{
    const KParams p = params(c);
    const int P = c->l_cands;
    float* x = reinterpret_cast<float*>(c->l_ws);
    uint32_t* cand =
        reinterpret_cast<uint32_t*>(c->l_ws + align_up(sizeof(float) * 3 * (size_t)c->n_max * kProposalBatch, 256));
    void* nws = c->l_ws + (learned_ws_bytes(c, P) - net_workspace_bytes(kProposalBatch, c->n_max));
    const int64_t S = std::max<int64_t>(1, kProposalBatch / P);
    const WalkerState* states = at<WalkerState>(c, c->off_states);
    for (int g = 0; g < c->nG; ++g) {
        const DevGroup& G = c->groups[g];
        for (int64_t s0 = G.first; s0 < G.first + G.count; s0 += S) {
            const int64_t cnt = std::min<int64_t>(S, G.first + G.count - s0);
            const float *sc = nullptr, *rs = nullptr;
            int rc = LABS_OK;
            if (!(c->cfg.flags & LABS_FLAG_LEARNED_RESTARTS)) {  // flip scores: the full learned mode
                rc = launch_features(reinterpret_cast<const uint32_t*>(states + s0), sizeof(WalkerState) / 4, cnt,
                                     G.L, x, c->stream);
                if (!rc) rc = net_forward_ws(c->l_params, x, cnt, G.n, nws, &sc, &rs, c->stream);
                if (!rc) rc = launch_scores(p, s0, cnt, G.n, sc, c->stream);
            }
            if (!rc) rc = launch_candidates(p, s0, cnt, G.n, P, cand, c->stream);
            if (!rc) rc = launch_features(cand, kBitWords, cnt * P, G.L, x, c->stream);
            if (!rc) rc = net_forward_ws(c->l_params, x, cnt * P, G.n, nws, &sc, &rs, c->stream);
            if (!rc) rc = launch_select(p, s0, cnt, P, rs, cand, c->stream);
            if (rc) return fail(c, rc, "proposal pass: %s", cudaGetErrorString(cudaGetLastError()));
        }
    }
    return LABS_OK;
}

int graph_for(labs_ctx* c, int nchunks, cudaGraphExec_t* exec)
{
    auto it = c->graphs.find(nchunks);
    if (it != c->graphs.end()) {
        *exec = it->second;
        return LABS_OK;
    }
    const KParams p = params(c);
    cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    int rc = LABS_OK;
    for (int j = 0; j < nchunks && rc == LABS_OK; ++j) rc = launch_chunk(c, p, j, c->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->capture, &g);
    if (rc != LABS_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e != cudaSuccess ? e : cudaGetLastError(), "graph capture");
    }
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graphs[nchunks] = *exec;
    return LABS_OK;
}

void drop_graphs(labs_ctx* c)
{
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

}  // namespace

extern "C" {

void labs_default_config(labs_config* cfg)
{
    if (!cfg) return;
    cfg->tabu_log2 = 16;
    cfg->probe_cap = 32;
    cfg->patience = 0;
    cfg->target_num = 17;
    cfg->target_den = 2;
    cfg->chunk_steps = 0;
    cfg->warps_per_cta = 0;
    cfg->flags = 0;
}

int labs_init(labs_ctx** ctx, int32_t L, int64_t walkers, uint64_t seed, const labs_config* cfg,
              void* cuda_stream)
{
    LABS_API_RANGE();
    return create(ctx, &L, &walkers, 1, seed, cfg, cuda_stream);
}

int labs_init_multi(labs_ctx** ctx, const int32_t* Ls, const int64_t* walkers_per_L, int32_t nL,
                    uint64_t seed, const labs_config* cfg, void* cuda_stream)
{
    LABS_API_RANGE();
    return create(ctx, Ls, walkers_per_L, nL, seed, cfg, cuda_stream);
}

int labs_workspace_bytes(const labs_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return LABS_EINVAL;
    *bytes = ctx->total;
    return LABS_OK;
}

int labs_reset(labs_ctx* c)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemsetAsync(c->ws + c->off_status, 0, sizeof(DevStatus), c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->ws + c->off_states, 0, sizeof(WalkerState) * (size_t)c->W, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->ws + c->off_tabu, 0, c->total - c->off_tabu, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "workspace clear");
    const KParams p = params(c);
    if (c->W > 0 && c->long_mode) {
        rc = launch_long_reset(p, c->smem_bytes, c->stream);
        if (rc) return fail(c, rc, "reset launch: %s", cudaGetErrorString(cudaGetLastError()));
    } else if (c->W > 0) {
        const int block = 8 * kWarp;
        const int64_t need = (c->W + 7) / 8;
        const int grid = (int)std::min<int64_t>(need, (int64_t)c->sms * 4);
        rc = launch_reset(p, grid, block, c->stream);
        if (rc) return fail(c, rc, "reset launch: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (c->cfg.flags & kLearnedAny) {
        e = cudaMemsetAsync(c->ws + c->off_l_step, 0xFF, sizeof(int64_t) * (size_t)c->W, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + c->off_l_valid, 0, sizeof(int32_t) * (size_t)c->W, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "learned state clear");
    }
    c->planned = 0;
    c->catch_up = false;
    c->log_start = 0;
    return push_status(c);
}

int labs_bind_workspace(labs_ctx* c, void* dev_workspace, size_t bytes)
{
    LABS_API_RANGE();
    if (!c || !dev_workspace) return LABS_EINVAL;
    if (bytes < c->total) return fail(c, LABS_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, c->total);
    if (((uintptr_t)dev_workspace & 255) != 0) return fail(c, LABS_EINVAL, "workspace must be 256-byte aligned");
    cudaSetDevice(c->device);
    c->ws = (char*)dev_workspace;
    cudaError_t e = cudaMemcpy(c->ws + c->off_groups, c->groups, sizeof(DevGroup) * c->nG, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "group table upload");
    const KParams p = params(c);
    int rc = launch_zobrist(p, at<uint64_t>(c, c->off_zkeys), c->groups, c->nG, c->stream);
    if (rc) return fail(c, rc, "fingerprint keys");
    // align the host clock with the GPU global timer for deadlines
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    unsigned long long* probe = &at<DevStatus>(c, c->off_status)->probe_ns;
    const long long t0 = host_ns();
    launch_time_probe(probe, c->stream);
    e = cudaStreamSynchronize(c->stream);
    const long long t1 = host_ns();
    if (e != cudaSuccess) return cuda_fail(c, e, "clock probe");
    uint64_t g = 0;
    cudaMemcpy(&g, probe, sizeof(g), cudaMemcpyDeviceToHost);
    c->gpu_minus_host_ns = (long long)g - (t0 + (t1 - t0) / 2);
    return labs_reset(c);
}

int labs_isl(labs_ctx* c, const int8_t* dev_seqs, int64_t batch, int32_t* dev_isl_out)
{
    LABS_API_RANGE();
    if (!c) return LABS_EINVAL;
    if (c->nG != 1) return fail(c, LABS_EINVAL, "labs_isl needs a single-length context");
    if (batch < 0 || (batch > 0 && (!dev_seqs || !dev_isl_out))) return fail(c, LABS_EINVAL, "bad batch");
    cudaSetDevice(c->device);
    DevStatus* st = c->ws ? at<DevStatus>(c, c->off_status) : nullptr;
    const int rc = launch_isl(dev_seqs, batch, c->groups[0].L, dev_isl_out, st, c->stream);
    return rc ? fail(c, rc, "labs_isl launch: %s", cudaGetErrorString(cudaGetLastError())) : LABS_OK;
}

int labs_neighbor_delta(labs_ctx* c, const int8_t* dev_seqs, int64_t batch, int32_t* dev_delta_out)
{
    LABS_API_RANGE();
    if (!c) return LABS_EINVAL;
    if (c->nG != 1) return fail(c, LABS_EINVAL, "labs_neighbor_delta needs a single-length context");
    if (batch < 0 || (batch > 0 && (!dev_seqs || !dev_delta_out))) return fail(c, LABS_EINVAL, "bad batch");
    cudaSetDevice(c->device);
    DevStatus* st = c->ws ? at<DevStatus>(c, c->off_status) : nullptr;
    const int rc = c->long_mode ? launch_long_delta(dev_seqs, batch, c->groups[0].L, dev_delta_out, st, c->stream)
                                : launch_delta(dev_seqs, batch, c->groups[0].L, dev_delta_out, st, c->stream);
    return rc ? fail(c, rc, "labs_neighbor_delta launch: %s", cudaGetErrorString(cudaGetLastError())) : LABS_OK;
}

int labs_walk(labs_ctx* c, int64_t steps)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (steps < 0) return fail(c, LABS_EINVAL, "negative steps");
    const long long bf_max = c->long_mode ? LABS_BEST_FIRST_MAX_STEPS_LONG : LABS_BEST_FIRST_MAX_STEPS;
    if ((c->cfg.flags & LABS_FLAG_BEST_FIRST) && c->planned + steps > bf_max)
        return fail(c, LABS_EINVAL, "best-first search: at most %lld steps per walker", bf_max);
    if ((steps == 0 && !c->catch_up) || c->W == 0) return LABS_OK;
    cudaSetDevice(c->device);
    const KParams p = params(c);
    while (steps > 0 || c->catch_up) {
        int64_t take = std::min<int64_t>(steps, (int64_t)c->chunk * (kMaxChunksPerCall - 1));
        int64_t span = take;
        if (c->catch_up) {
            span = c->planned + take;  // walkers stopped early may be anywhere behind
            c->catch_up = false;
        }
        const int nchunks = (int)std::min<int64_t>((span + c->chunk - 1) / c->chunk, kMaxChunksPerCall);
        rc = launch_prep_walk(p, take, nchunks, c->stream);
        if (rc) return fail(c, rc, "walk preparation launch");
        if ((c->cfg.flags & LABS_FLAG_NO_GRAPH) || c->l_params) {
            for (int j = 0; j < nchunks; ++j) {
                if (c->l_params) {
                    rc = proposal_pass(c);
                    if (rc) return rc;
                }
                rc = launch_chunk(c, p, j, c->stream);
                if (rc) return fail(c, rc, "walk launch: %s", cudaGetErrorString(cudaGetLastError()));
            }
        } else {
            cudaGraphExec_t exec = nullptr;
            rc = graph_for(c, nchunks, &exec);
            if (rc) return rc;
            cudaError_t e = cudaGraphLaunch(exec, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
        }
        c->planned += take;
        steps -= take;
    }
    return LABS_OK;
}

int labs_sync(labs_ctx* c)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) {
        if (!c) return rc;
        cudaError_t e = cudaStreamSynchronize(c->stream);
        return e == cudaSuccess ? LABS_OK : cuda_fail(c, e, "stream synchronise");
    }
    cudaSetDevice(c->device);
    rc = sync_status(c);
    if (rc || !(c->cfg.flags & LABS_FLAG_STRICT_HT)) return rc;
    labs_counters cnt;
    rc = labs_stats(c, 0, &cnt);
    if (rc) return rc;
    if (cnt.overflows > 0)
        return fail(c, LABS_ETABU_FULL, "%lld HT insertions found no free slot within probe_cap = %d",
                    (long long)cnt.overflows, c->cfg.probe_cap);
    return LABS_OK;
}

// The walker with the best sequence among walkers of length L (0: all): lowest best
// ISL, or under the PSL objective lowest (best PSL, best ISL); ties to the lowest id.
static int best_state(labs_ctx* c, int32_t L, WalkerState* out, int64_t* walker)
{
    int rc = need_ws(c);
    if (rc) return rc;
    cudaSetDevice(c->device);
    DevStatus* st = at<DevStatus>(c, c->off_status);
    cudaError_t e = cudaMemsetAsync(&st->best_key, 0xFF, sizeof(st->best_key) + sizeof(st->best_obj), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "best reset");
    rc = launch_best(params(c), L, c->stream);
    if (rc) return fail(c, rc, "best launch");
    rc = sync_status(c);
    if (rc) return rc;
    unsigned long long key = 0;
    e = cudaMemcpy(&key, &st->best_key, sizeof(key), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "best read");
    if (key == ~0ull) return fail(c, LABS_EINVAL, "no walker of length %d", L);
    const int64_t w = (int64_t)(key & 0xFFFFFFFFull);
    e = cudaMemcpy(out, at<WalkerState>(c, c->off_states) + w, sizeof(*out), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "best state read");
    *walker = w;
    return LABS_OK;
}

static int best_outputs(labs_ctx* c, int64_t w, const WalkerState& ws, int8_t* host_seq_out, int32_t* L_out,
                        char* hex_out)
{
    const int Lw = c->groups[ws.group].L;
    std::vector<uint32_t> bits(kBitWordsLong);
    const int rc = walker_bits(c, w, ws, true, bits.data());
    if (rc) return rc;
    std::vector<int8_t> seq((size_t)Lw);
    expand_bits(bits.data(), Lw, seq.data());
    if (host_seq_out) memcpy(host_seq_out, seq.data(), (size_t)Lw);
    if (L_out) *L_out = Lw;
    if (hex_out) hex_of(seq.data(), Lw, hex_out);
    return LABS_OK;
}

int labs_best(labs_ctx* c, int32_t L, int8_t* host_seq_out, int32_t* isl, double* F, int32_t* L_out,
              char* hex_out)
{
    LABS_API_RANGE();
    WalkerState ws;
    int64_t w = 0;
    int rc = best_state(c, L, &ws, &w);
    if (rc) return rc;
    const int Lw = c->groups[ws.group].L;
    rc = best_outputs(c, w, ws, host_seq_out, L_out, hex_out);
    if (rc) return rc;
    if (isl) *isl = ws.best_isl;
    if (F) *F = (double)Lw * Lw / (2.0 * ws.best_isl);
    return LABS_OK;
}

int labs_best_psl(labs_ctx* c, int32_t L, int8_t* host_seq_out, int32_t* psl, int32_t* isl, int32_t* L_out,
                  char* hex_out)
{
    LABS_API_RANGE();
    if (c && !(c->cfg.flags & LABS_FLAG_PSL)) return fail(c, LABS_EINVAL, "context created without LABS_FLAG_PSL");
    WalkerState ws;
    int64_t w = 0;
    int rc = best_state(c, L, &ws, &w);
    if (rc) return rc;
    rc = best_outputs(c, w, ws, host_seq_out, L_out, hex_out);
    if (rc) return rc;
    if (psl) *psl = ws.best_psl;
    if (isl) *isl = ws.best_isl;
    return LABS_OK;
}

int labs_walker_psl(labs_ctx* c, int64_t first, int64_t count, int32_t* host_psl, int32_t* host_best_psl)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (!(c->cfg.flags & LABS_FLAG_PSL)) return fail(c, LABS_EINVAL, "context created without LABS_FLAG_PSL");
    if (first < 0 || count < 0 || first + count > c->W) return fail(c, LABS_EINVAL, "walker range out of bounds");
    cudaSetDevice(c->device);
    rc = sync_status(c);
    if (rc) return rc;
    std::vector<WalkerState> v((size_t)count);
    if (count) {
        cudaError_t e = cudaMemcpy(v.data(), at<WalkerState>(c, c->off_states) + first, sizeof(WalkerState) * count,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "walker state read");
    }
    for (int64_t j = 0; j < count; ++j) {
        if (host_psl) host_psl[j] = v[j].psl;
        if (host_best_psl) host_best_psl[j] = v[j].best_psl;
    }
    return LABS_OK;
}

int labs_walker_results(labs_ctx* c, int64_t first, int64_t count, int32_t* host_isl, int32_t* host_best_isl,
                        int8_t* host_seq, int8_t* host_best_seq, int64_t* host_target_step)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (first < 0 || count < 0 || first + count > c->W) return fail(c, LABS_EINVAL, "walker range out of bounds");
    cudaSetDevice(c->device);
    rc = sync_status(c);
    if (rc) return rc;
    std::vector<WalkerState> v((size_t)count);
    if (count) {
        cudaError_t e = cudaMemcpy(v.data(), at<WalkerState>(c, c->off_states) + first, sizeof(WalkerState) * count,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "walker state read");
    }
    int Lw = count ? c->groups[v[0].group].L : 0;
    if ((host_seq || host_best_seq))
        for (auto& s : v)
            if (c->groups[s.group].L != Lw) return fail(c, LABS_EINVAL, "walkers in the range differ in length");
    std::vector<uint32_t> cur, best;
    if (c->long_mode && count && (host_seq || host_best_seq)) {
        cur.resize((size_t)count * kBitWordsLong);
        best.resize((size_t)count * kBitWordsLong);
        const size_t row = sizeof(uint32_t) * kBitWordsLong;
        cudaError_t e = cudaMemcpy(cur.data(), c->ws + c->off_cur_bits + row * (size_t)first, row * count,
                                   cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(best.data(), c->ws + c->off_best_bits + row * (size_t)first, row * count,
                           cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "walker bits read");
    }
    for (int64_t j = 0; j < count; ++j) {
        if (host_isl) host_isl[j] = v[j].isl;
        if (host_best_isl) host_best_isl[j] = v[j].best_isl;
        if (host_target_step) host_target_step[j] = v[j].target_step;
        const uint32_t* cb = c->long_mode ? cur.data() + j * kBitWordsLong : v[j].cur;
        const uint32_t* bb = c->long_mode ? best.data() + j * kBitWordsLong : v[j].best;
        if (host_seq) expand_bits(cb, Lw, host_seq + j * Lw);
        if (host_best_seq) expand_bits(bb, Lw, host_best_seq + j * Lw);
    }
    return LABS_OK;
}

int labs_stats(labs_ctx* c, int32_t L, labs_counters* out)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (!out) return fail(c, LABS_EINVAL, "null output");
    cudaSetDevice(c->device);
    DevStatus* st = at<DevStatus>(c, c->off_status);
    rc = sync_status(c);
    if (rc) return rc;
    DevStatus h;
    cudaError_t e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    h.best_key = ~0ull;
    h.best_obj = ~0ull;
    h.st_steps = h.st_evals = h.st_restarts = h.st_overflows = h.st_blocked = h.st_at_target = h.st_cache_hits = 0;
    h.st_target_step = LLONG_MAX;
    e = cudaMemcpy(st, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "status write");
    rc = launch_stats(params(c), L, c->stream);
    if (rc) return fail(c, rc, "stats launch");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    out->steps = (int64_t)h.st_steps;
    out->flip_evaluations = (int64_t)h.st_evals;
    out->restarts = (int64_t)h.st_restarts;
    out->overflows = (int64_t)h.st_overflows;
    out->blocked = (int64_t)h.st_blocked;
    out->cache_hits = (int64_t)h.st_cache_hits;
    out->walkers_at_target = (int64_t)h.st_at_target;
    out->walkers_per_warp = kWarp / c->tile;  // 0 for long sequences: one walker per CTA
    out->lane_block = c->long_mode ? long_R(c->n_max, c->tile) : lanes_for(c->n_max, c->tile);
    out->tensor_cores = (c->long_mode ? long_smem(c->n_max, c->tile).xp
                                      : warp_smem(c->n_max, c->tile, (c->cfg.flags & LABS_FLAG_PSL) != 0).xp) != 0;
    out->target_step = h.st_target_step == LLONG_MAX ? -1 : (int64_t)h.st_target_step;
    out->best_psl = -1;
    if (h.best_key == ~0ull) {
        out->best_isl = -1;
        out->best_L = 0;
        out->best_walker = -1;
    } else {
        out->best_isl = (int32_t)(h.best_key >> 32);
        out->best_walker = (int64_t)(h.best_key & 0xFFFFFFFFull);
        WalkerState ws;
        cudaMemcpy(&ws, at<WalkerState>(c, c->off_states) + out->best_walker, sizeof(ws), cudaMemcpyDeviceToHost);
        out->best_L = c->groups[ws.group].L;
        if (c->cfg.flags & LABS_FLAG_PSL) out->best_psl = ws.best_psl;
    }
    return LABS_OK;
}

int labs_trace(labs_ctx* c, const int64_t* host_walker_ids, int32_t k, int64_t capacity, int32_t* dev_code_log,
               int32_t* dev_isl_log)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (k < 0 || k > kMaxTrace) return fail(c, LABS_EINVAL, "0 <= k <= %d", kMaxTrace);
    if (k > 0 && (!host_walker_ids || !dev_code_log || !dev_isl_log || capacity < 0))
        return fail(c, LABS_EINVAL, "bad trace buffers");
    for (int j = 0; j < k; ++j)
        if (host_walker_ids[j] < 0 || host_walker_ids[j] >= c->W)
            return fail(c, LABS_EINVAL, "walker id %lld out of range", (long long)host_walker_ids[j]);
    cudaSetDevice(c->device);
    int64_t* ids = at<int64_t>(c, c->off_trace_ids);
    if (k > 0) {
        cudaError_t e = cudaMemcpyAsync(ids, host_walker_ids, sizeof(int64_t) * k, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "trace ids upload");
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    }
    rc = launch_trace_arm(params(c), ids, k, dev_code_log, dev_isl_log, capacity, c->stream);
    return rc ? fail(c, rc, "trace launch") : LABS_OK;
}

int labs_log(labs_ctx* c, labs_log_record* dev_records, int64_t capacity)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (capacity < 0 || (capacity > 0 && !dev_records)) return fail(c, LABS_EINVAL, "bad log buffer");
    if (capacity > 0 && ((c->cfg.flags & (LABS_FLAG_BEST_FIRST | LABS_FLAG_PSL)) || c->long_mode))
        return fail(c, LABS_EINVAL, "the walk log records the plain walk of lengths up to %d only", LABS_MAX_L);
    cudaSetDevice(c->device);
    c->log = capacity > 0 ? dev_records : nullptr;
    c->log_capacity = capacity;
    c->log_start = c->planned;
    return push_status(c);
}

int labs_log_labels(const labs_log_record* dev_records, int64_t count, int32_t* dev_target, float* dev_y,
                    float* dev_wf, void* cuda_stream)
{
    LABS_API_RANGE();
    if (count < 0 || (count > 0 && (!dev_records || !dev_target || !dev_y || !dev_wf))) return LABS_EINVAL;
    if (count == 0) return LABS_OK;
    return launch_labels(dev_records, count, dev_target, dev_y, dev_wf, cuda_stream);
}

int labs_features(int32_t L, const uint32_t* dev_bits, int64_t stride_words, int64_t count, float* dev_x,
                  void* cuda_stream)
{
    LABS_API_RANGE();
    if (!valid_L(L) || count < 0 || stride_words < kBitWords || (count > 0 && (!dev_bits || !dev_x)))
        return LABS_EINVAL;
    return launch_features(dev_bits, stride_words, count, L, dev_x, cuda_stream);
}

int labs_learned_workspace_bytes(const labs_ctx* c, int32_t candidates, size_t* bytes)
{
    if (!c || !bytes || candidates < 1 || candidates > 64) return LABS_EINVAL;
    *bytes = learned_ws_bytes(c, candidates);
    return LABS_OK;
}

int labs_learned(labs_ctx* c, const float* dev_params, int32_t tau, int32_t candidates, void* dev_ws, size_t ws_bytes)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (dev_params) {
        if (!(c->cfg.flags & kLearnedAny))
            return fail(c, LABS_EINVAL, "context created without LABS_FLAG_LEARNED or LABS_FLAG_LEARNED_RESTARTS");
        if (tau < 0 || candidates < 1 || candidates > 64) return fail(c, LABS_EINVAL, "bad tau / candidates");
        if (!dev_ws || ws_bytes < learned_ws_bytes(c, candidates))
            return fail(c, LABS_ENOMEM, "learned workspace needs %zu bytes", learned_ws_bytes(c, candidates));
    }
    cudaSetDevice(c->device);
    c->l_params = dev_params;
    c->l_tau = tau;
    c->l_cands = candidates;
    c->l_ws = static_cast<char*>(dev_ws);
    c->l_ws_bytes = ws_bytes;
    return push_status(c);
}

int labs_trace_learned(labs_ctx* c, int32_t capacity, float* dev_scores, int64_t* dev_score_step,
                       int32_t* dev_score_count, uint32_t* dev_restart, int64_t* dev_restart_idx,
                       int32_t* dev_restart_count)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (capacity < 0 || (capacity > 0 && (!dev_scores || !dev_score_step || !dev_score_count || !dev_restart ||
                                          !dev_restart_idx || !dev_restart_count)))
        return fail(c, LABS_EINVAL, "bad dump buffers");
    cudaSetDevice(c->device);
    const bool on = capacity > 0;
    c->d_scores = on ? dev_scores : nullptr;
    c->d_score_step = on ? dev_score_step : nullptr;
    c->d_score_count = on ? dev_score_count : nullptr;
    c->d_restart = on ? dev_restart : nullptr;
    c->d_restart_idx = on ? dev_restart_idx : nullptr;
    c->d_restart_count = on ? dev_restart_count : nullptr;
    c->d_cap = capacity;
    return push_status(c);
}

int labs_enumerate_scratch_bytes(int32_t L, size_t* bytes)
{
    if (!bytes || L < 3 || L > 63 || (L & 1) == 0) return LABS_EINVAL;
    *bytes = enum_scratch_bytes(L);
    return LABS_OK;
}

int labs_enumerate(int32_t L, void* dev_scratch, size_t scratch_bytes, int64_t* min_isl, uint64_t* count,
                   uint64_t* first_assignment, void* cuda_stream)
{
    LABS_API_RANGE();
    if (L < 3 || L > 63 || (L & 1) == 0 || !dev_scratch) return LABS_EINVAL;
    if (scratch_bytes < enum_scratch_bytes(L)) return LABS_ENOMEM;
    if (((uintptr_t)dev_scratch & 15) != 0) return LABS_EINVAL;
    EnumPart r;
    const int rc = enum_run(L, (EnumPart*)dev_scratch, cuda_stream, &r);
    if (rc) return rc;
    if (min_isl) *min_isl = r.min_isl;
    if (count) *count = r.count;
    if (first_assignment) *first_assignment = r.first;
    return LABS_OK;
}

// Header word 7 of a checkpoint: the objective, and for long sequences the long flag and
// the words per bit row (the rows' stride in the checkpoint).
static uint64_t ckpt_kind(const labs_ctx* c)
{
    return (uint64_t)(c->cfg.flags & LABS_FLAG_PSL) | (c->long_mode ? 0x100u | ((uint64_t)kBitWordsLong << 16) : 0u);
}

int labs_checkpoint(labs_ctx* c, int with_tabu, void* host_buf, size_t* bytes)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (c->cfg.flags & LABS_FLAG_BEST_FIRST) return fail(c, LABS_EINVAL, "no checkpoints of a best-first search");
    if (!bytes) return fail(c, LABS_EINVAL, "null size");
    const size_t hdr = 64;
    // walker states, and for long sequences the two bit rows of every walker (they follow
    // the states in the workspace)
    const size_t sbytes = c->long_mode ? c->off_best_bits + sizeof(uint32_t) * kBitWordsLong * (size_t)c->W -
                                             c->off_states
                                       : sizeof(WalkerState) * (size_t)c->W;
    const size_t tbytes = with_tabu ? sizeof(uint64_t) * ((size_t)c->W << c->cfg.tabu_log2) : 0;
    const size_t need = hdr + sbytes + tbytes;
    if (!host_buf) {
        *bytes = need;
        return LABS_OK;
    }
    if (*bytes < need) return fail(c, LABS_ENOMEM, "checkpoint buffer has %zu bytes, needs %zu", *bytes, need);
    cudaSetDevice(c->device);
    rc = sync_status(c);
    if (rc) return rc;
    uint64_t h[8] = {kCkptMagic, (uint64_t)c->W, (uint64_t)c->nG, (uint64_t)c->cfg.tabu_log2,
                     (uint64_t)(with_tabu ? 1 : 0), (uint64_t)c->planned, c->seed, ckpt_kind(c)};
    memcpy(host_buf, h, sizeof(h));
    char* dst = (char*)host_buf + hdr;
    cudaError_t e = cudaMemcpy(dst, c->ws + c->off_states, sbytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && tbytes) e = cudaMemcpy(dst + sbytes, c->ws + c->off_tabu, tbytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    *bytes = need;
    return LABS_OK;
}

int labs_restore(labs_ctx* c, const void* host_buf, size_t bytes)
{
    LABS_API_RANGE();
    int rc = need_ws(c);
    if (rc) return rc;
    if (c->cfg.flags & LABS_FLAG_BEST_FIRST) return fail(c, LABS_EINVAL, "no checkpoints of a best-first search");
    if (!host_buf || bytes < 64) return fail(c, LABS_EINVAL, "bad checkpoint");
    uint64_t h[8];
    memcpy(h, host_buf, sizeof(h));
    if (h[0] != kCkptMagic || h[1] != (uint64_t)c->W || h[2] != (uint64_t)c->nG ||
        h[3] != (uint64_t)c->cfg.tabu_log2 || h[6] != c->seed || h[7] != ckpt_kind(c))
        return fail(c, LABS_EINVAL, "checkpoint does not match this context");
    const size_t sbytes = c->long_mode ? c->off_best_bits + sizeof(uint32_t) * kBitWordsLong * (size_t)c->W -
                                             c->off_states
                                       : sizeof(WalkerState) * (size_t)c->W;
    const size_t tbytes = h[4] ? sizeof(uint64_t) * ((size_t)c->W << c->cfg.tabu_log2) : 0;
    if (bytes < 64 + sbytes + tbytes) return fail(c, LABS_EINVAL, "checkpoint truncated");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    const char* src = (const char*)host_buf + 64;
    e = cudaMemcpy(c->ws + c->off_states, src, sbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "restore copy");
    if (tbytes) {
        e = cudaMemcpy(c->ws + c->off_tabu, src + sbytes, tbytes, cudaMemcpyHostToDevice);
    } else {
        // Without the HT every walker continues with an empty table (zeroed slots hold
        // generation 0, which no walker uses).
        e = cudaMemset(c->ws + c->off_tabu, 0, c->total - c->off_tabu);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "restore copy");
    const int64_t planned = (int64_t)h[5];
    DevStatus* st = at<DevStatus>(c, c->off_status);
    e = cudaMemcpy(&st->target_steps, &planned, sizeof(planned), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "restore copy");
    c->planned = planned;
    c->catch_up = true;
    return LABS_OK;
}

int labs_set_deadline(labs_ctx* c, uint64_t ns_from_now)
{
    if (!c || !c->ctrl_host) return LABS_EINVAL;
    if (ns_from_now == UINT64_MAX) {
        c->ctrl_host->deadline_ns = UINT64_MAX;
    } else {
        const long long now = host_ns() + c->gpu_minus_host_ns;
        const unsigned long long base = now < 0 ? 0ull : (unsigned long long)now;
        c->ctrl_host->deadline_ns =
            ns_from_now == 0 ? 0ull : (UINT64_MAX - base < ns_from_now ? UINT64_MAX : base + ns_from_now);
    }
    return LABS_OK;
}

int labs_cancel(labs_ctx* c)
{
    if (!c || !c->ctrl_host) return LABS_EINVAL;
    c->ctrl_host->stop = 1;
    return LABS_OK;
}

int labs_clear_stop(labs_ctx* c)
{
    int rc = need_ws(c);
    if (rc) return rc;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    c->ctrl_host->stop = 0;
    c->ctrl_host->deadline_ns = UINT64_MAX;
    const int32_t zero[2] = {0, 0};
    e = cudaMemcpy(at<DevStatus>(c, c->off_status), zero, sizeof(zero), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "status clear");
    c->catch_up = true;
    return LABS_OK;
}

const char* labs_last_error(const labs_ctx* c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

void labs_destroy(labs_ctx* c)
{
    if (!c) return;
    if (c->ws) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->ctrl_host) cudaFreeHost(c->ctrl_host);
    delete c;
}

}  // extern "C"
