/*
 * labs.h -- C ABI of liblabs, a single-GPU (GB300, sm_103a) search for skew-symmetric
 * binary sequences with a high merit factor, after Brest & Boskovic, "Computational
 * Search of Long Skew-symmetric Binary Sequences with High Merit Factors"
 * (arXiv 2011.00068).
 *
 * Terms (Section 1 of the paper):
 *   S = (s_0 .. s_{L-1}), s_i in {+1, -1}, stored as int8 rows of length L.
 *   C_k = sum_i s_i s_{i+k}                                   (Eq. 1)
 *   ISL = sum_{k=1}^{L-1} C_k^2                               (Eq. 2)
 *   F   = L^2 / (2 ISL)                                       (Eq. 3)
 *   skew symmetry, L = 2n-1, centre c = n-1:
 *         s_{c+j} = (-1)^j s_{c-j}, j = 1..n-1                 (Eq. 4, 0-based)
 *   The n free variables are s_0 .. s_c; flipping free variable i negates s_i and
 *   its mirror s_{L-1-i} (only s_c for i = c), which keeps Eq. 4 (Algorithm 1,
 *   neighbourhood loop).
 *
 * Conventions for every call:
 *   - Returns LABS_OK (0) or a negative LABS_E* code; labs_last_error() gives text.
 *   - "dev" pointers are device memory owned by the caller; "host" pointers are
 *     host memory owned by the caller.  The library allocates no device memory for
 *     its searches: a context's state lives in one caller-allocated workspace
 *     (labs_workspace_bytes / labs_bind_workspace).
 *   - Calls that launch work are asynchronous on the CUDA stream given to labs_init
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).  Errors
 *     detected on the device are reported by the next synchronising call
 *     (labs_sync, labs_best, labs_walker_results, labs_stats, labs_checkpoint).
 *   - Lengths: odd L with 3 <= L <= LABS_MAX_L (walkers run one, two or four per warp),
 *     or LABS_MAX_L < L <= LABS_MAX_L_LONG (long sequences: one walker per CTA of 128,
 *     256 or 512 threads, the same step rules: the walk under the ISL or the PSL
 *     objective, or the best-first search without the second table); a context holds
 *     lengths of one kind only.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef LABS_H
#define LABS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LABS_OK 0
#define LABS_EINVAL (-1)     /* bad argument, or invalid input rows seen on the device */
#define LABS_ENOMEM (-2)     /* workspace missing or too small, host allocation failed */
#define LABS_ECUDA (-3)      /* a CUDA runtime call failed */
#define LABS_ETIMEOUT (-4)   /* the deadline set by labs_set_deadline passed */
#define LABS_ECANCELLED (-5) /* labs_cancel was called */
#define LABS_ESTATE (-6)     /* a walker's stored state failed its consistency check */
#define LABS_ERANGE (-7)     /* a long sequence left the range in which the library's fp32
                                neighbourhood is exact (ISL above the bound stated at
                                labs_walk); random starts and walks stay far below it */
#define LABS_ETABU_FULL (-8) /* with LABS_FLAG_STRICT_HT: an HT insertion found no free
                                slot within probe_cap (that walker restarted) */

#define LABS_MAX_L 511       /* n = (L+1)/2 <= 256 free variables */
#define LABS_MAX_L_LONG 11263 /* long sequences: n <= 5632 free variables */
#define LABS_MAX_GROUPS 64   /* distinct lengths in one context */

/* Step trace codes written by labs_trace (one int32 per walker step).  The walk writes
 * the flipped free variable i; the best-first search the low 16 bits of the new S's
 * fingerprint (the XOR of its Zobrist keys). */
#define LABS_TRACE_RESTART 0x10000 /* OR-ed into the code: the step ended in a restart */
#define LABS_TRACE_BLOCKED (-1)    /* no admissible next state (every neighbour visited, or
                                      an empty best-first queue): restart */

typedef struct labs_ctx labs_ctx;

/* Walk parameters.  The paper fixes none of these (Algorithm 1 names a visited-set
 * hash table HT and a stopping rule only); the defaults are the library's reading. */
typedef struct labs_config {
    int32_t tabu_log2;       /* HT slots per walker = 2^tabu_log2, 1..20; default 16 */
    int32_t probe_cap;       /* linear-probe limit of HT, 1..32; default 32 */
    int32_t patience;        /* restart after this many steps without a new best since
                                the last restart; 0 (default) = 2n */
    int32_t target_num;      /* time-to-target threshold F >= target_num/target_den; */
    int32_t target_den;      /* default 17/2 (F >= 8.5); 0/0 disables it */
    int32_t chunk_steps;     /* steps per kernel launch inside labs_walk; 0 = auto */
    int32_t warps_per_cta;   /* walkers resident per CTA (one warp each), 1..8; 0 = 8 */
    int32_t flags;           /* LABS_FLAG_* */
} labs_config;

#define LABS_FLAG_NO_GRAPH 1     /* launch chunks one by one instead of a CUDA graph */
#define LABS_FLAG_CHECK_STATE 2  /* accepted, no further effect: the check is always on.
                                    Every chunk start rebuilds a walker's rows and C_k table
                                    from its stored bits and compares the ISL (and, under the
                                    PSL objective, the PSL) with the stored value; a mismatch
                                    stops that walker and labs_sync returns LABS_ESTATE */
#define LABS_FLAG_LEARNED 4      /* reserve workspace for the learned mode (labs_learned) */
#define LABS_FLAG_WARP_PER_WALKER 8 /* one walker per warp even where two per warp fit */
#define LABS_FLAG_TWO_PER_WARP 16   /* at most two walkers per warp even where four fit,
                                       and two (FP32 Toeplitz product) where one per warp
                                       would run (n = 129..160) */
#define LABS_FLAG_BEST_FIRST 32     /* labs_walk runs Algorithm 1 as printed: best-first
                                       search with a queue of LABS_QUEUE_SIZE evaluated
                                       neighbours per walker (see labs_walk); one walker per
                                       warp (per CTA for long sequences); not with
                                       LABS_FLAG_LEARNED, no checkpoints */
#define LABS_FLAG_STRICT_HT 256     /* labs_sync returns LABS_ETABU_FULL once any HT insertion
                                       of the context found no free slot within probe_cap
                                       (the overflows counter of labs_stats is nonzero); the
                                       walk itself is unchanged (the walker restarts).  Each
                                       labs_sync then runs labs_stats (a reduction kernel and
                                       three blocking copies); labs_reset clears the count */
#define LABS_FLAG_SECOND_HASH 128   /* with LABS_FLAG_BEST_FIRST: xLastovka's second table of
                                       evaluated neighbours (Section 3), one per walker with
                                       as many slots as HT; neighbours it holds are skipped
                                       (see labs_walk); lengths up to LABS_MAX_L */
#define LABS_FLAG_PSL 64            /* labs_walk minimises PSL (Section 1) instead of ISL: the
                                       walk's rules with (PSL, ISL) pairs as the objective (see
                                       labs_walk); two walkers per warp up to L = 255 (one
                                       with LABS_FLAG_WARP_PER_WALKER, the same trajectories),
                                       one per warp above, one per CTA for long sequences;
                                       not with LABS_FLAG_BEST_FIRST or LABS_FLAG_LEARNED */
#define LABS_FLAG_LEARNED_RESTARTS 512 /* reserve workspace for the restart-only learned mode:
                                       labs_learned then runs only the restart half of the
                                       proposal pass (see labs_learned) and the walk keeps its
                                       plain kernels (two or four walkers per warp); lengths
                                       up to LABS_MAX_L; not with LABS_FLAG_LEARNED,
                                       LABS_FLAG_BEST_FIRST or LABS_FLAG_PSL */
#define LABS_QUEUE_SIZE 32           /* entries of a walker's best-first queue */
#define LABS_BEST_FIRST_MAX_STEPS (1ll << 28) /* steps per walker the queue order can number */
#define LABS_BEST_FIRST_MAX_STEPS_LONG (1ll << 21) /* the same for lengths above LABS_MAX_L */

/* Counters of a context, summed over its walkers (labs_stats). */
typedef struct labs_counters {
    int64_t steps;             /* walker steps taken */
    int64_t flip_evaluations;  /* n per step: every free-variable flip is evaluated */
    int64_t restarts;          /* restarts after the first start */
    int64_t overflows;         /* HT insertions that found no free slot within probe_cap */
    int64_t blocked;           /* steps whose whole neighbourhood was in HT */
    int32_t best_isl;          /* lowest ISL seen by any walker of the selected length */
    int32_t best_L;            /* its length */
    int64_t best_walker;       /* lowest walker id reaching it */
    int64_t target_step;       /* fewest steps after which some walker met the target,
                                  -1 if none did */
    int64_t walkers_at_target; /* walkers that met the target */
    int32_t walkers_per_warp;  /* launch shape of the walk kernel: 4, 2 or 1; 0 for long
                                  sequences (one walker per CTA) */
    int32_t lane_block;        /* outputs per lane of the widest walker (R) */
    int32_t best_psl;          /* LABS_FLAG_PSL: PSL of the best sequence (whose ISL is
                                  best_isl; best in the (PSL, ISL) order); else -1 */
    int32_t tensor_cores;      /* 1: the walk's Toeplitz product (the neighbourhood's
                                  O(n^2) part) runs on the tensor cores as exact FP16 x FP16
                                  -> FP32 block products; 0: on the FP32 pipes */
    int64_t cache_hits;        /* LABS_FLAG_SECOND_HASH: neighbours skipped because the
                                  second table held them (flip_evaluations counts all n
                                  per step: the GPU evaluates them anyway) */
} labs_counters;

/* One record of the walk log (labs_log): the state of a walker at the start of a
 * chunk of steps and what followed it.  64 bytes. */
typedef struct labs_log_record {
    uint32_t bits[8];  /* free variables at the chunk start: bit i set <=> s_i = -1 */
    int32_t isl;       /* ISL at the chunk start */
    int32_t first;     /* trace code of the chunk's first step */
    int32_t min_isl;   /* lowest ISL reached in the chunk before its first restart */
    int32_t L;
    int64_t walker;
    int64_t step;      /* steps done at the chunk start */
} labs_log_record;

/* Fills *cfg with the defaults above. */
void labs_default_config(labs_config *cfg);

/* Creates a context for `walkers` independent walkers of one odd length L
 * (Algorithm 1: input L; every walker is one run of the search).  Walker w starts
 * from the random skew-symmetric sequence drawn by Philox4x32-10 under key `seed`
 * (Algorithm 1, start: a random skew-symmetric first sequence).  cfg may be NULL
 * (defaults).  No device work happens until a workspace is bound. */
int labs_init(labs_ctx **ctx, int32_t L, int64_t walkers, uint64_t seed,
              const labs_config *cfg, void *cuda_stream);

/* As labs_init for nL lengths at once (Table 1 covers L = 201..303): walkers_per_L[j]
 * walkers of length Ls[j].  Walker ids run group by group in the order given. */
int labs_init_multi(labs_ctx **ctx, const int32_t *Ls, const int64_t *walkers_per_L,
                    int32_t nL, uint64_t seed, const labs_config *cfg, void *cuda_stream);

/* Device bytes the caller must allocate for the context's workspace (state of all
 * walkers, their HT tables, counters).  Alignment 256 bytes. */
int labs_workspace_bytes(const labs_ctx *ctx, size_t *bytes);

/* Hands the workspace to the context (the caller keeps ownership and must keep it
 * alive until labs_destroy) and starts every walker at step 0 (see labs_reset). */
int labs_bind_workspace(labs_ctx *ctx, void *dev_workspace, size_t bytes);

/* Puts every walker back to its first random start, step 0, empty HT. */
int labs_reset(labs_ctx *ctx);

/* Eq. 2 for a batch of arbitrary +-1 rows: dev_seqs is int8 [batch][L] (row-major,
 * L = the context's single length), dev_isl_out is int32 [batch].  A row holding a
 * value other than +-1 gets ISL -1 (and labs_sync then reports LABS_EINVAL when a
 * workspace is bound); a long row whose ISL exceeds INT32_MAX gets -2 (LABS_ERANGE).
 * batch may be 0. */
int labs_isl(labs_ctx *ctx, const int8_t *dev_seqs, int64_t batch, int32_t *dev_isl_out);

/* The neighbourhood of Algorithm 1 (neighbourhood evaluation: the ISL of every
 * one-flip neighbour S_f, from the current C_k in O(L) per flip) for a
 * batch of skew-symmetric rows: dev_delta_out is int32 [batch][n], entry i = ISL after
 * flipping free variable i (and its mirror) minus ISL before, i = 0..n-1.  A row that
 * is not +-1 or breaks Eq. 4 gets INT32_MIN in every entry (and labs_sync reports
 * LABS_EINVAL when a workspace is bound).  For long rows (L > LABS_MAX_L) a row whose
 * ISL is above the exact-range bound stated at labs_walk gets INT32_MIN too
 * (LABS_ERANGE). */
int labs_neighbor_delta(labs_ctx *ctx, const int8_t *dev_seqs, int64_t batch,
                        int32_t *dev_delta_out);

/* Advances every walker by `steps` steps of the walk (Algorithm 1, self-avoiding
 * form; the step rule is stated here and implemented in csrc/labs_device.cuh):
 *   evaluate all n flips; take the flip with the lowest dISL whose result is not in
 *   the walker's HT (ties to the lowest i); move there and insert it into HT; keep
 *   the best sequence (strictly lower ISL); restart from a new random sequence with
 *   an empty HT after `patience` steps without a new best since the last restart,
 *   when every neighbour is in HT, or when HT has no free slot for the new state.
 * With LABS_FLAG_BEST_FIRST a step is Algorithm 1 as printed (impxLast, Section 3):
 *   evaluate all n flips of S; every neighbour not in HT enters the walker's queue,
 *   ordered by (ISL, step that produced it, i) ascending, while it comes before the
 *   queue's last entry or the queue has a free place (a full queue drops its last
 *   entry); then S becomes the queue's first entry that is not in HT by now (entries
 *   that are get dropped) and is inserted into HT.  The best sequence is kept as in
 *   the walk; the walker restarts (HT and queue emptied) when the queue runs empty or
 *   HT has no free slot for the new S; `patience` is not used.  At most
 *   LABS_BEST_FIRST_MAX_STEPS steps per walker, LABS_BEST_FIRST_MAX_STEPS_LONG for
 *   lengths above LABS_MAX_L (LABS_EINVAL beyond).
 *   LABS_FLAG_SECOND_HASH adds xLastovka's second table (the library's reading of
 *   Section 3): a slot (fingerprint mod size) holds (HT generation << 40) | (~f mod 2^40)
 *   of a neighbour f; at the start of a step every neighbour whose slot holds its word is
 *   skipped (not offered to the queue, counted in cache_hits), and after the queue
 *   update every other neighbour is inserted by keeping the larger of the slot's old and
 *   new word (so the table does not depend on the insertion order); a restart empties it
 *   with HT.
 * With LABS_FLAG_PSL the objective is the pair (PSL, ISL), compared lexicographically
 *   (PSL = max_k |C_k|, Section 1; the paper optimises F and reports PSL in Table 1,
 *   so this order is the library's reading of a PSL search): the step takes the flip
 *   with the lowest (PSL, ISL, i) whose result is not in HT, the best sequence and the
 *   stagnation count use "strictly lower pair", and HT and the restarts are as in the
 *   walk.  The trace's ISL log still holds ISL.
 * Long sequences (L > LABS_MAX_L) take the same steps with the neighbourhood in exact
 *   fp32 arithmetic, which holds while ISL < ((2^24 - 8L - 32n - 32) / 16)^2 / (n - 1)
 *   (capped at 2^29; 2.6e8 at L = 8191 and 1.9e8 at L = 11263, above random starts,
 *   whose ISL is near L^2/2, by a factor of 8 and 3): a walker whose ISL exceeds it
 *   stops and labs_sync reports LABS_ERANGE.
 * The trajectory of a walker depends only on (seed, walker id, L, cfg), never on
 * chunking, launch shape or the other walkers. */
int labs_walk(labs_ctx *ctx, int64_t steps);

/* Waits for the context's stream; returns the first device-side error, if any. */
int labs_sync(labs_ctx *ctx);

/* Best sequence found so far among walkers of length L (L = 0: all lengths):
 * lowest ISL (with LABS_FLAG_PSL: lowest (PSL, ISL) pair), ties to the lowest walker id.  Synchronising.  host_seq_out: int8 [L]
 * (nullable; sized for the winning length, which *L_out gives), isl/F/L_out nullable,
 * hex_out: ceil(L/4)+1 chars in the encoding described below Table 1 (nullable). */
int labs_best(labs_ctx *ctx, int32_t L, int8_t *host_seq_out, int32_t *isl, double *F,
              int32_t *L_out, char *hex_out);

/* LABS_FLAG_PSL contexts only (LABS_EINVAL otherwise): the best sequence in the
 * (PSL, ISL) order, as labs_best, with its PSL and ISL. */
int labs_best_psl(labs_ctx *ctx, int32_t L, int8_t *host_seq_out, int32_t *psl, int32_t *isl,
                  int32_t *L_out, char *hex_out);

/* LABS_FLAG_PSL contexts only: PSL of the current and of the best sequence of walkers
 * [first, first+count) (host int32 arrays, nullable).  Synchronising. */
int labs_walker_psl(labs_ctx *ctx, int64_t first, int64_t count, int32_t *host_psl,
                    int32_t *host_best_psl);

/* Per-walker results for walkers [first, first+count): current and best ISL (int32),
 * and optionally their sequences (int8 [count][Lw], all walkers in the range must have
 * the same length Lw).  Any pointer may be NULL.  Synchronising. */
int labs_walker_results(labs_ctx *ctx, int64_t first, int64_t count, int32_t *host_isl,
                        int32_t *host_best_isl, int8_t *host_seq, int8_t *host_best_seq,
                        int64_t *host_target_step);

/* Counters summed over the walkers of length L (0 = all).  Synchronising. */
int labs_stats(labs_ctx *ctx, int32_t L, labs_counters *out);

/* Arms per-step tracing of k walkers (host_walker_ids, host array) for the following
 * labs_walk calls: step t (counted from this call) of walker host_walker_ids[j] writes
 * its trace code to dev_code_log[j*capacity + t] and its ISL at the end of the step to
 * dev_isl_log[j*capacity + t], for t < capacity.  k = 0 disarms.  The logs are caller
 * device buffers of k*capacity int32 each. */
int labs_trace(labs_ctx *ctx, const int64_t *host_walker_ids, int32_t k, int64_t capacity,
               int32_t *dev_code_log, int32_t *dev_isl_log);

/* Exhaustive search over all skew-symmetric sequences of odd length L (3 <= L <= 63)
 * with the centre s_c = +1 (negation keeps Eq. 4 and ISL): returns the minimum ISL,
 * the number of minimising assignments, and the lowest minimising assignment a, where
 * bit i of a set means s_i = -1 (i < c).  Needs caller device scratch of
 * labs_enumerate_scratch_bytes(L) bytes.  Synchronises `cuda_stream`. */
int labs_enumerate_scratch_bytes(int32_t L, size_t *bytes);
int labs_enumerate(int32_t L, void *dev_scratch, size_t scratch_bytes, int64_t *min_isl,
                   uint64_t *count, uint64_t *first_assignment, void *cuda_stream);

/* Allocation-free form of labs_enumerate (the paper has no counterpart: it is a
 * library convenience).  It is for callers that cannot allocate device memory when
 * they call: for example a real-time signal chain that reserves all of its GPU memory
 * at start-up and must not call cudaMalloc later (it can synchronise the device and
 * has no latency bound), or a plugin whose host owns every device allocation.
 * Same arguments and results as labs_enumerate minus the scratch buffer: the scratch
 * lives in a fixed array inside the library, 33,280 bytes, which every GPU that loads
 * the library holds until the process exits.  It fits every L the call accepts
 * (odd 3 <= L <= 63, at most 1025 partial results); LABS_EINVAL for other L and
 * LABS_ENOMEM if a length ever needed more than the array holds.  The call allocates
 * nothing (no cudaMalloc / cudaFree / allocating library routine); it clears the part
 * of the array it uses, then runs on cuda_stream and synchronises it.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, so make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) invalidates the looked-up address: a call whose CUDA work fails
 * forgets it, and the next call on that device looks it up again.  All calls share
 * the one array: calls that overlap on the GPU (from several host threads or streams)
 * race and give wrong results. */
int labs_enumerate_noalloc(int32_t L, int64_t *min_isl, uint64_t *count,
                           uint64_t *first_assignment, void *cuda_stream);

/* ---- Learned proposal network (the library's addition: the paper has no learned
 * component).  A small BF16 network ranks flips and restart points; the exact int32
 * ISL still decides every move.  Per state of n free variables (2 <= n <= 256):
 *   input x: float32 [batch][3][n] -- s_i, C_{2(i+1)}/sqrt(L) (0 for i = n-1) and
 *            dISL_i/(8L) per free variable i (rounded to bfloat16 on entry);
 *   a1..a3 = relu(conv(a_{l-1}) + b_l), Conv1d with 64 channels, 7 taps, zero padding 3;
 *   h = relu(W4 a3 + b4) per position; score_i = w5 . h_i + b5 (flip score);
 *   restart = w6 . mean_i(a3_i) + b6 (restart score).
 * Parameters are one float32 array in the order W1[64][16][7] b1 W2[64][64][7] b2
 * W3[64][64][7] b3 W4[64][64] b4 w5[64] b5 w6[64] b6 (labs_net_sizes gives the count);
 * products use bfloat16 copies with float32 accumulation on the tensor cores.
 * Loss per sample: wf * CE(softmax(score), target) + 0.5 (restart - y)^2, batch mean.
 * All pointers are device memory; calls are asynchronous on cuda_stream. */
int labs_net_sizes(int32_t n, int64_t batch, size_t *param_count, size_t *workspace_bytes);
int labs_net_init(float *dev_params, uint64_t seed, void *cuda_stream);
int labs_net_forward(const float *dev_params, const float *dev_x, int64_t batch, int32_t n,
                     float *dev_scores /* [batch][n], nullable */, float *dev_restart /* [batch], nullable */,
                     void *dev_ws, size_t ws_bytes, void *cuda_stream);
/* Gradients of the batch-mean loss into dev_grads (overwritten; same layout as the
 * parameters) and the loss into dev_loss (nullable). */
int labs_net_gradients(const float *dev_params, const float *dev_x, const int32_t *dev_target,
                       const float *dev_y, const float *dev_wf, int64_t batch, int32_t n,
                       float *dev_grads, float *dev_loss, void *dev_ws, size_t ws_bytes,
                       void *cuda_stream);
/* One AdamW step (beta 0.9/0.999, eps 1e-8; weight decay on weights, not biases). */
int labs_net_adamw(float *dev_params, const float *dev_grads, float *dev_m, float *dev_v, int64_t t,
                   float lr, float weight_decay, void *cuda_stream);

/* ---- Learned proposal in the walk.
 *
 * labs_log arms the walk log (plain walk only: LABS_EINVAL with LABS_FLAG_BEST_FIRST or
 * LABS_FLAG_PSL): from the next labs_walk on, at the start of every chunk
 * of chunk_steps steps, walker w fills record k*walkers + w of dev_records (k = chunks
 * since this call) with its state and what followed it in the chunk, while the index
 * is below capacity.  capacity 0 disarms. */
int labs_log(labs_ctx *ctx, labs_log_record *dev_records, int64_t capacity);

/* Training inputs of log records: target = the free variable flipped by the first step,
 * wf = 1 when the ISL later fell below the record's start ISL (else 0; the flip term of
 * the loss is then off), y = L^2 / (2 min_isl) / 8 (the merit factor reached within
 * the chunk, scaled). */
int labs_log_labels(const labs_log_record *dev_records, int64_t count, int32_t *dev_target,
                    float *dev_y, float *dev_wf, void *cuda_stream);

/* Network inputs (float32 [count][3][n], the layout labs_net_forward takes) of states
 * given by their free-variable bits: 8 words each, stride_words apart (16 for a
 * labs_log_record array). */
int labs_features(int32_t L, const uint32_t *dev_bits, int64_t stride_words, int64_t count,
                  float *dev_x, void *cuda_stream);

/* Turns the learned mode on (dev_params != NULL) or off.  Needs LABS_FLAG_LEARNED (or
 * LABS_FLAG_LEARNED_RESTARTS) at init.  Before every chunk launch of labs_walk the
 * library then runs a proposal pass (with LABS_FLAG_LEARNED_RESTARTS only its restart
 * half, and tau is ignored):
 *   - flip scores of every walker's current state; at the chunk's first step the walker
 *     tries, among the flips with dISL <= (lowest dISL) + tau, the highest-scored
 *     (ties: lowest i) first, and continues in the plain order when none is admissible;
 *   - restart candidates: the walker's own next random start (the plain choice) and
 *     candidates-1 further random starts (Philox, counter (walker, next restart index,
 *     block, c) for candidate c); the one with the highest restart score (ties: lowest
 *     index) is used at the walker's next restart.
 * The exact ISL decides every move; the network only orders candidates.
 * dev_ws: labs_learned_workspace_bytes bytes.  Chunks run without a CUDA graph. */
int labs_learned_workspace_bytes(const labs_ctx *ctx, int32_t candidates, size_t *bytes);
int labs_learned(labs_ctx *ctx, const float *dev_params, int32_t tau, int32_t candidates,
                 void *dev_ws, size_t ws_bytes);

/* Replay dumps for the walkers armed by labs_trace, in learned mode: per traced walker
 * j, up to capacity learned steps (the scores it used, [j][capacity][n_max] floats, and
 * the step, [j][capacity]) and up to capacity proposed restarts (the state used,
 * [j][capacity][8] words, and the restart index, [j][capacity]).  The count arrays ([k]
 * int32, zeroed by the caller) receive how many entries each walker wrote. */
int labs_trace_learned(labs_ctx *ctx, int32_t capacity, float *dev_scores, int64_t *dev_score_step,
                       int32_t *dev_score_count, uint32_t *dev_restart, int64_t *dev_restart_idx,
                       int32_t *dev_restart_count);

/* Checkpoint of every walker's state (sequence, ISL, best, counters, random-stream
 * position) and, with with_tabu != 0, its HT.  With the HT included a restored run
 * continues bit-identically; without it the HT restarts empty (the walks with two or
 * four walkers per warp, and the plain walk with one, still never move straight back to
 * the state a walker has just left, which they leave out without probing: the same
 * choice as the probe's wherever HT holds the walker's states).  host_buf NULL queries
 * the size; a checkpoint restores only into a context with the same walker count,
 * lengths' kind (short or long; for long ones the same LABS_MAX_L_LONG), HT size,
 * seed and LABS_FLAG_PSL (LABS_EINVAL otherwise).  Synchronising.  LABS_EINVAL for a
 * context with LABS_FLAG_BEST_FIRST (its queues are not part of the checkpoint). */
int labs_checkpoint(labs_ctx *ctx, int with_tabu, void *host_buf, size_t *bytes);
int labs_restore(labs_ctx *ctx, const void *host_buf, size_t bytes);

/* Deadline, in nanoseconds of the GPU's global timer from now (0 = already passed,
 * UINT64_MAX = none): walkers stop at the next check and labs_sync reports
 * LABS_ETIMEOUT.  labs_cancel stops them the same way with LABS_ECANCELLED.  Walkers
 * stop between steps, with their state saved; labs_clear_stop resumes. */
int labs_set_deadline(labs_ctx *ctx, uint64_t ns_from_now);
int labs_cancel(labs_ctx *ctx);
int labs_clear_stop(labs_ctx *ctx);

/* Text of the last error on this context (never NULL). */
const char *labs_last_error(const labs_ctx *ctx);

void labs_destroy(labs_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LABS_H */
