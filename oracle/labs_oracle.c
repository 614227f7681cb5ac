/*
 * labs_oracle.c -- plain, slow CPU oracle for the skew-symmetric LABS search of
 * Brest & Boskovic, "Computational Search of Long Skew-symmetric Binary Sequences
 * with High Merit Factors" (arXiv 2011.00068).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the GPU
 * library is checked against.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA library, and it never calls it.
 *
 * Everything is written straight from the paper's definitions, in the paper's order:
 *   - C_k by Eq. 1, ISL by Eq. 2, F by Eq. 3, PSL as defined in Section 1.
 *   - the skew-symmetric map of Eq. 4 in 0-based form: with L = 2n-1 and centre
 *     c = n-1, s[c+j] = (-1)^j s[c-j] for j = 1..n-1 (the reading that decodes all
 *     rows of Table 1).
 *   - the hexadecimal encoding stated below Table 1.
 *   - the neighbourhood of Algorithm 1: flipping free variable i (i = 0..n-1) changes
 *     s_i and its mirror q = L-1-i.  The change of every C_k is taken from the
 *     general two-position formula over ALL k (odd k included, where it must vanish),
 *     and dISL_i = sum_k dC_k (2 C_k + dC_k).
 *   - the search loop of Algorithm 1 in the self-avoiding-walk form (move to the best
 *     neighbour that is not in the visited set HT, ties to the lowest i), with
 *     restarts from a fresh random sequence as in lssOrel (Section 2).
 *   - the same walk with PSL (Section 1) as the objective instead of ISL: every
 *     neighbour is built and its PSL and ISL recomputed from Eq. 1.  The paper only
 *     reports PSL (Table 1, Section 4); ordering by (PSL, ISL) is the library's reading.
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for every random draw.
 * Where the paper is silent (tie-break, restart rule, hash-table layout, random
 * stream layout) the reading is fixed in the comments below and mirrored by the
 * GPU library from its own code.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---------------------------------------------------------------- definitions */

/* Eq. 1: aperiodic autocorrelation at shift k (|k| < L). */
int64_t lo_ck(const int8_t *s, int32_t L, int32_t k)
{
    if (k < 0) k = -k;
    int64_t acc = 0;
    for (int32_t i = 0; i + k < L; ++i) acc += (int64_t)s[i] * (int64_t)s[i + k];
    return acc;
}

/* Eq. 2: integrated sidelobe level, sum of C_k^2 over k = 1..L-1. */
int64_t lo_isl(const int8_t *s, int32_t L)
{
    int64_t e = 0;
    for (int32_t k = 1; k < L; ++k) {
        int64_t c = lo_ck(s, L, k);
        e += c * c;
    }
    return e;
}

/* Section 1: peak sidelobe level, max |C_k| over k = 1..L-1. */
int64_t lo_psl(const int8_t *s, int32_t L)
{
    int64_t p = 0;
    for (int32_t k = 1; k < L; ++k) {
        int64_t c = lo_ck(s, L, k);
        if (c < 0) c = -c;
        if (c > p) p = c;
    }
    return p;
}

/* Eq. 3: merit factor. */
double lo_merit(int32_t L, int64_t isl)
{
    return (double)L * (double)L / (2.0 * (double)isl);
}

/* Eq. 4, 0-based: free variables x[0..n-1] are s[0..c]; s[c+j] = (-1)^j s[c-j]. */
int lo_skew_expand(const int8_t *x, int32_t L, int8_t *s)
{
    if (L < 1 || (L & 1) == 0) return -1;
    int32_t n = (L + 1) / 2, c = n - 1;
    for (int32_t i = 0; i < n; ++i) s[i] = x[i];
    for (int32_t j = 1; j < n; ++j) s[c + j] = (j & 1) ? (int8_t)(-s[c - j]) : s[c - j];
    return 0;
}

/* 1 when s is +-1 valued and satisfies Eq. 4, else 0. */
int lo_is_skew(const int8_t *s, int32_t L)
{
    if (L < 1 || (L & 1) == 0) return 0;
    int32_t c = (L + 1) / 2 - 1;
    for (int32_t i = 0; i < L; ++i)
        if (s[i] != 1 && s[i] != -1) return 0;
    for (int32_t j = 1; j <= c; ++j) {
        int8_t want = (j & 1) ? (int8_t)(-s[c - j]) : s[c - j];
        if (s[c + j] != want) return 0;
    }
    return 1;
}

/* Table 1 note: each hex digit -> 4 bits (first digit most significant), leading
 * bits dropped to keep the last L, then 0 -> +1 and 1 -> -1.  The dropped bits must
 * be zero.  Returns 0 or -1. */
int lo_hex_decode(const char *hex, int32_t L, int8_t *s)
{
    int32_t nd = (int32_t)strlen(hex);
    int32_t nbits = 4 * nd;
    if (nbits < L) return -1;
    int32_t drop = nbits - L;
    for (int32_t b = 0; b < nbits; ++b) {
        char ch = hex[b / 4];
        int v;
        if (ch >= '0' && ch <= '9') v = ch - '0';
        else if (ch >= 'A' && ch <= 'F') v = ch - 'A' + 10;
        else if (ch >= 'a' && ch <= 'f') v = ch - 'a' + 10;
        else return -1;
        int bit = (v >> (3 - (b % 4))) & 1;
        if (b < drop) {
            if (bit) return -1;
        } else {
            s[b - drop] = bit ? -1 : 1;
        }
    }
    return 0;
}

/* Inverse of lo_hex_decode with the fewest digits, ceil(L/4); out gets a NUL. */
int lo_hex_encode(const int8_t *s, int32_t L, char *out)
{
    int32_t nd = (L + 3) / 4;
    int32_t pad = 4 * nd - L;
    static const char digits[] = "0123456789ABCDEF";
    for (int32_t d = 0; d < nd; ++d) {
        int v = 0;
        for (int32_t t = 0; t < 4; ++t) {
            int32_t b = 4 * d + t - pad;
            int bit = 0;
            if (b >= 0) {
                if (s[b] != 1 && s[b] != -1) return -1;
                bit = s[b] < 0;
            }
            v = (v << 1) | bit;
        }
        out[d] = digits[v];
    }
    out[nd] = 0;
    return 0;
}

/* ----------------------------------------------------- neighbourhood (Alg. 1) */

static int64_t sat(const int8_t *s, int32_t L, int32_t j)
{
    return (j >= 0 && j < L) ? (int64_t)s[j] : 0;
}

/* Change of C_k when the positions {i, q} (q = L-1-i, possibly q == i) are negated.
 * A pair (j, j+k) with exactly one end flipped changes by -2 s_j s_{j+k}; the sum
 * below counts every pair that touches a flipped position, so the pair (i, q) with
 * both ends flipped (k = q - i) is counted twice and its true change is zero:
 * the + 4 s_i s_q term removes it. */
static int64_t delta_ck(const int8_t *s, int32_t L, int32_t i, int32_t k)
{
    int32_t q = L - 1 - i;
    int64_t d = -2 * (int64_t)s[i] * (sat(s, L, i + k) + sat(s, L, i - k));
    if (q != i) {
        d += -2 * (int64_t)s[q] * (sat(s, L, q + k) + sat(s, L, q - k));
        if (k == (q > i ? q - i : i - q)) d += 4 * (int64_t)s[i] * (int64_t)s[q];
    }
    return d;
}

/* dISL for every free-variable flip i = 0..n-1 of a skew-symmetric s (Alg. 1,
 * "fast calculate merit factor of S_f").  C is taken from Eq. 1 directly.
 * Returns 0, or -1 if s is not skew-symmetric, or -2 if an odd-k change is nonzero
 * (impossible for a skew-symmetric sequence, Eq. 4). */
int lo_neighbor_delta(const int8_t *s, int32_t L, int64_t *delta)
{
    if (!lo_is_skew(s, L)) return -1;
    int32_t n = (L + 1) / 2;
    int64_t *C = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    for (int32_t k = 0; k < L; ++k) C[k] = lo_ck(s, L, k);
    int rc = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t acc = 0;
        for (int32_t k = 1; k < L; ++k) {
            int64_t d = delta_ck(s, L, i, k);
            if ((k & 1) && d != 0) rc = -2;
            acc += d * (2 * C[k] + d);
        }
        delta[i] = acc;
    }
    free(C);
    return rc;
}

/* --------------------------------------------------------------- Philox4x32-10 */

/* Salmon et al., SC'11, Philox4x32 with 10 rounds: each round multiplies words 0
 * and 2 by the two round constants, swaps and xors with the key; the key advances
 * by the two Weyl constants between rounds. */
void lo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random stream layout (a reading: the paper only says "initialize a starting
 * sequence", Alg. 1).  Key = (seed low word, seed high word).  The start of restart
 * r of walker g draws counter blocks (g, r, b, 0), b = 0, 1, ...; free variable i
 * reads bit (i mod 32) of word (i/32 mod 4) of block i/128, and a set bit means -1. */
void lo_random_start(uint64_t seed, uint32_t g, uint32_t r, int32_t L, int8_t *x)
{
    int32_t n = (L + 1) / 2;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    for (int32_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {g, r, (uint32_t)(i / 128), 0u};
        lo_philox4x32_10(ctr, key, out);
        uint32_t w = out[(i / 32) % 4];
        x[i] = ((w >> (i % 32)) & 1u) ? -1 : 1;
    }
}

/* ------------------------------------------------------- visited set HT (Alg. 1) */

/* Fingerprint of a skew-symmetric state: the XOR, over the free variables equal
 * to -1, of a 64-bit key per (L, i) (Zobrist hashing).  Key (L, i) is words 0 and 1
 * of the Philox block with counter (i, L, 0, 2) under the fixed key below. */
#define LO_ZKEY0 0x1BADB002u
#define LO_ZKEY1 0x2011A068u
uint64_t lo_zobrist_key(int32_t L, int32_t i)
{
    uint32_t key[2] = {LO_ZKEY0, LO_ZKEY1};
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)L, 0u, 2u};
    uint32_t out[4];
    lo_philox4x32_10(ctr, key, out);
    return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

uint64_t lo_fingerprint(const int8_t *s, int32_t L)
{
    int32_t n = (L + 1) / 2;
    uint64_t fp = 0;
    for (int32_t i = 0; i < n; ++i)
        if (s[i] < 0) fp ^= lo_zobrist_key(L, i);
    return fp;
}

/* HT layout: 2^log2 slots of 64 bits, linear probing from slot fp mod 2^log2, at
 * most `cap` probes.  A slot holds (fp with its low 20 bits cleared) | generation;
 * a slot whose generation differs from the current one is empty, so a restart
 * empties HT by advancing the generation (1 .. 2^20-1; at wrap-around the slots are
 * zeroed and the generation restarts at 1). */
#define LO_GEN_MASK 0xFFFFFull

typedef struct {
    uint64_t *slot;
    uint64_t mask;
    int32_t cap;
    uint64_t gen;
} lo_ht;

static int ht_contains(const lo_ht *h, uint64_t fp)
{
    uint64_t tag = (fp & ~LO_GEN_MASK) | h->gen;
    for (int32_t p = 0; p < h->cap; ++p) {
        uint64_t e = h->slot[(fp + (uint64_t)p) & h->mask];
        if ((e & LO_GEN_MASK) != h->gen) return 0;
        if (e == tag) return 1;
    }
    return 0;
}

/* 1 = present or stored, 0 = no free slot within cap probes (overflow). */
static int ht_insert(lo_ht *h, uint64_t fp)
{
    uint64_t tag = (fp & ~LO_GEN_MASK) | h->gen;
    for (int32_t p = 0; p < h->cap; ++p) {
        uint64_t *e = &h->slot[(fp + (uint64_t)p) & h->mask];
        if ((*e & LO_GEN_MASK) != h->gen) {
            *e = tag;
            return 1;
        }
        if (*e == tag) return 1;
    }
    return 0;
}

static void ht_new_generation(lo_ht *h)
{
    h->gen += 1;
    if (h->gen > LO_GEN_MASK) {
        memset(h->slot, 0, sizeof(uint64_t) * (size_t)(h->mask + 1));
        h->gen = 1;
    }
}

/* ------------------------------------------------------------ the walk (Alg. 1) */

typedef struct {
    int32_t tabu_log2;  /* HT has 2^tabu_log2 slots per walker */
    int32_t probe_cap;  /* linear-probe limit */
    int32_t patience;   /* restart after this many steps without a new best since
                           the last restart; 0 means 2n */
    int32_t target_num; /* threshold F >= target_num / target_den for the */
    int32_t target_den; /* time-to-threshold record (0/0 disables it) */
} lo_walk_cfg;

typedef struct {
    int32_t final_isl;
    int32_t best_isl;
    int64_t best_step;    /* steps completed when best_isl was first reached */
    int64_t target_step;  /* steps completed when F >= target first held, or -1 */
    int32_t restarts;
    int32_t overflows;    /* HT insertions that found no free slot */
    int32_t final_psl;    /* PSL (Section 1) of the final and of the best sequence */
    int32_t best_psl;
    int64_t cache_hits;   /* best-first search with the second table: neighbours skipped
                             because the table held them (not evaluated) */
} lo_walk_result;

/* Trace codes, one per step: the flipped free variable i (0..n-1), with bit 16 set
 * when the step ended in a restart; or -1 when every neighbour was in HT (the step
 * only restarts).  The ISL trace holds the ISL at the end of the step. */
#define LO_TRACE_RESTART 0x10000

/* Learned-mode replay inputs (the network's choices recorded by the GPU run):
 * at step score_step[k] (steps done before it) the walker used scores[k][0..n) with the
 * threshold tau; at restart index restart_idx[k] it started from restart_bits[k][0..8). */
typedef struct {
    int32_t tau;
    int32_t n_score;
    const int64_t *score_step;
    const float *scores;
    int32_t score_stride;
    int32_t n_restart;
    const int64_t *restart_idx;
    const uint32_t *restart_bits;
} lo_replay;

typedef struct {
    int32_t L, n;
    uint64_t seed;
    uint32_t g;
    const lo_walk_cfg *cfg;
    const uint64_t *zkey;
    const lo_replay *replay;
    int32_t objective;  /* 0: ISL (Eq. 2); 1: PSL first, ties by ISL */
    uint64_t *cache;    /* best-first search: xLastovka's second table of evaluated
                           neighbours (NULL when off), as many slots as HT */
    int8_t *x, *s, *s_best, *sf, *tried;
    int64_t *delta, *cand_psl, *cand_isl;
    int32_t *order;
    lo_ht ht;
    uint32_t restart_index;
    int64_t isl, best_isl, since_restart_best;
    int64_t psl, best_psl, since_restart_best_psl;
    int32_t stagnation;
    uint64_t fp;
    lo_walk_result res;
} lo_walker;

static int target_met(const lo_walker *w, int64_t isl)
{
    if (w->cfg->target_num <= 0 || w->cfg->target_den <= 0) return 0;
    /* F = L^2 / (2 ISL) >= num/den  <=>  den * L^2 >= 2 * num * ISL */
    return (int64_t)w->cfg->target_den * w->L * w->L >= 2 * (int64_t)w->cfg->target_num * isl;
}

/* Is (psl, isl) better than (psl0, isl0) under the walker's objective?  The ISL
 * objective compares ISL alone; the PSL objective compares PSL and breaks ties by ISL
 * (the paper optimises F and only reports PSL; this order is the library's reading of
 * a PSL search that stays comparable with it). */
static int better(const lo_walker *w, int64_t psl, int64_t isl, int64_t psl0, int64_t isl0)
{
    if (w->objective) return psl < psl0 || (psl == psl0 && isl < isl0);
    return isl < isl0;
}

static void note_best(lo_walker *w, int64_t steps_done)
{
    if (better(w, w->psl, w->isl, w->best_psl, w->best_isl)) {
        w->best_isl = w->isl;
        w->best_psl = w->psl;
        memcpy(w->s_best, w->s, (size_t)w->L);
        w->res.best_step = steps_done;
    }
    if (w->res.target_step < 0 && target_met(w, w->isl)) w->res.target_step = steps_done;
}

/* Alg. 1 first steps: initialise a random skew-symmetric S, compute F (here ISL),
 * insert S into HT, and take it as the best so far. */
static void start(lo_walker *w, int64_t steps_done)
{
    const lo_replay *rp = w->replay;
    int32_t k = -1;
    if (rp)
        for (int32_t j = 0; j < rp->n_restart; ++j)
            if (rp->restart_idx[j] == (int64_t)w->restart_index) k = j;
    if (k >= 0) {
        for (int32_t i = 0; i < w->n; ++i)
            w->x[i] = ((rp->restart_bits[8 * k + i / 32] >> (i % 32)) & 1u) ? -1 : 1;
    } else {
        lo_random_start(w->seed, w->g, w->restart_index, w->L, w->x);
    }
    lo_skew_expand(w->x, w->L, w->s);
    w->isl = lo_isl(w->s, w->L);
    w->psl = lo_psl(w->s, w->L);
    w->fp = lo_fingerprint(w->s, w->L);
    ht_insert(&w->ht, w->fp);
    w->since_restart_best = w->isl;
    w->since_restart_best_psl = w->psl;
    w->stagnation = 0;
    note_best(w, steps_done);
}

static void restart(lo_walker *w, int64_t steps_done)
{
    w->restart_index += 1;
    w->res.restarts += 1;
    uint64_t gen0 = w->ht.gen;
    ht_new_generation(&w->ht);
    if (w->cache && w->ht.gen < gen0) memset(w->cache, 0, sizeof(uint64_t) * (size_t)(w->ht.mask + 1));
    start(w, steps_done);
}

static int cmp_pair(const int64_t *delta, int32_t a, int32_t b)
{
    if (delta[a] != delta[b]) return delta[a] < delta[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* Scores are compared through a monotone map of their bit pattern to int32. */
static int32_t score_key(float f)
{
    int32_t k;
    memcpy(&k, &f, sizeof(k));
    return k >= 0 ? k : (k ^ 0x7FFFFFFF);
}

/* One step of the walk; returns the trace code, or -99 on an internal mismatch. */
static int32_t walk_step(lo_walker *w, int64_t steps_done_after)
{
    int32_t L = w->L, n = w->n;
    if (lo_neighbor_delta(w->s, L, w->delta) != 0) return -99;
    /* candidates in the order (dISL ascending, i ascending): insertion sort */
    for (int32_t i = 0; i < n; ++i) {
        int32_t j = i;
        while (j > 0 && cmp_pair(w->delta, i, w->order[j - 1]) < 0) {
            w->order[j] = w->order[j - 1];
            --j;
        }
        w->order[j] = i;
    }
    int32_t chosen = -1;
    uint64_t fp_new = 0;
    /* learned step: flips with dISL <= min dISL + tau, by (score desc, i asc), first */
    const lo_replay *rp = w->replay;
    int32_t ks = -1;
    if (rp)
        for (int32_t j = 0; j < rp->n_score; ++j)
            if (rp->score_step[j] == steps_done_after - 1) ks = j;
    if (ks >= 0) {
        const float *sc = rp->scores + (int64_t)ks * rp->score_stride;
        int64_t thr = w->delta[w->order[0]] + rp->tau;
        for (;;) {
            int32_t pick = -1;
            for (int32_t i = 0; i < n; ++i) {
                if (w->delta[i] > thr || w->tried[i]) continue;
                if (pick < 0 || score_key(sc[i]) > score_key(sc[pick])) pick = i;
            }
            if (pick < 0) break;
            w->tried[pick] = 1;
            uint64_t f = w->fp ^ w->zkey[pick];
            if (!ht_contains(&w->ht, f)) {
                chosen = pick;
                fp_new = f;
                break;
            }
        }
        for (int32_t i = 0; i < n; ++i) w->tried[i] = 0;
    }
    for (int32_t t = 0; t < n && chosen < 0; ++t) {
        int32_t i = w->order[t];
        uint64_t f = w->fp ^ w->zkey[i];
        if (!ht_contains(&w->ht, f)) {
            chosen = i;
            fp_new = f;
            break;
        }
    }
    if (chosen < 0) {
        restart(w, steps_done_after);
        return -1;
    }
    /* S <- S_f: negate s_i and its mirror */
    int32_t q = L - 1 - chosen;
    w->s[chosen] = (int8_t)(-w->s[chosen]);
    if (q != chosen) w->s[q] = (int8_t)(-w->s[q]);
    int64_t expect = w->isl + w->delta[chosen];
    w->isl = lo_isl(w->s, L);
    if (w->isl != expect) return -99;
    w->fp = fp_new;
    int stored = ht_insert(&w->ht, fp_new);
    if (!stored) w->res.overflows += 1;
    note_best(w, steps_done_after);
    if (w->isl < w->since_restart_best) {
        w->since_restart_best = w->isl;
        w->stagnation = 0;
    } else {
        w->stagnation += 1;
    }
    int32_t patience = w->cfg->patience > 0 ? w->cfg->patience : 2 * n;
    if (w->stagnation >= patience || !stored) {
        restart(w, steps_done_after);
        return chosen | LO_TRACE_RESTART;
    }
    return chosen;
}

/* One step of the walk under the PSL objective.  Every neighbour S_i (free variable i
 * and its mirror negated) is built and measured from the definitions: PSL_i = max |C_k|
 * (Section 1) and ISL_i (Eq. 2), C_k by Eq. 1.  The walker moves to the first
 * neighbour not in HT in the order (PSL_i, ISL_i, i) ascending; HT, the best sequence,
 * the stagnation count and the restarts follow the same rules as the ISL walk, with
 * "better" meaning a lower (PSL, ISL) pair. */
static int32_t walk_step_psl(lo_walker *w, int64_t steps_done_after)
{
    int32_t L = w->L, n = w->n;
    for (int32_t i = 0; i < n; ++i) {
        memcpy(w->sf, w->s, (size_t)L);
        w->sf[i] = (int8_t)(-w->sf[i]);
        if (L - 1 - i != i) w->sf[L - 1 - i] = (int8_t)(-w->sf[L - 1 - i]);
        w->cand_psl[i] = lo_psl(w->sf, L);
        w->cand_isl[i] = lo_isl(w->sf, L);
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t j = i;
        while (j > 0) {
            int32_t o = w->order[j - 1];
            int before = w->cand_psl[i] < w->cand_psl[o] ||
                         (w->cand_psl[i] == w->cand_psl[o] && w->cand_isl[i] < w->cand_isl[o]);
            if (!before) break;
            w->order[j] = o;
            --j;
        }
        w->order[j] = i;
    }
    int32_t chosen = -1;
    uint64_t fp_new = 0;
    for (int32_t t = 0; t < n && chosen < 0; ++t) {
        int32_t i = w->order[t];
        uint64_t f = w->fp ^ w->zkey[i];
        if (!ht_contains(&w->ht, f)) {
            chosen = i;
            fp_new = f;
        }
    }
    if (chosen < 0) {
        restart(w, steps_done_after);
        return -1;
    }
    int32_t q = L - 1 - chosen;
    w->s[chosen] = (int8_t)(-w->s[chosen]);
    if (q != chosen) w->s[q] = (int8_t)(-w->s[q]);
    w->isl = w->cand_isl[chosen];
    w->psl = w->cand_psl[chosen];
    w->fp = fp_new;
    int stored = ht_insert(&w->ht, fp_new);
    if (!stored) w->res.overflows += 1;
    note_best(w, steps_done_after);
    if (better(w, w->psl, w->isl, w->since_restart_best_psl, w->since_restart_best)) {
        w->since_restart_best = w->isl;
        w->since_restart_best_psl = w->psl;
        w->stagnation = 0;
    } else {
        w->stagnation += 1;
    }
    int32_t patience = w->cfg->patience > 0 ? w->cfg->patience : 2 * n;
    if (w->stagnation >= patience || !stored) {
        restart(w, steps_done_after);
        return chosen | LO_TRACE_RESTART;
    }
    return chosen;
}

typedef struct {
    int32_t L;
    uint64_t seed;
    int64_t g0, count, steps;
    const lo_walk_cfg *cfg;
    const uint64_t *zkey;
    lo_walk_result *res;
    int8_t *best_seq;
    int8_t *final_seq;
    int32_t *trace_code, *trace_isl;
    int32_t pq_size;  /* 0: the walk; > 0: best-first search with this queue size */
    int32_t objective;  /* walk only: 0 ISL, 1 PSL then ISL */
    int32_t second_hash;  /* best-first only: xLastovka's second table of evaluated neighbours */
    int64_t next;
    pthread_mutex_t lock;
    int status;
} lo_walk_job;

static int run_bestfirst(lo_walk_job *job, int64_t w_idx);

static int run_walker(lo_walk_job *job, int64_t w_idx, const lo_replay *replay)
{
    int32_t L = job->L, n = (L + 1) / 2;
    lo_walker w;
    memset(&w, 0, sizeof(w));
    w.L = L;
    w.n = n;
    w.seed = job->seed;
    w.g = (uint32_t)(job->g0 + w_idx);
    w.cfg = job->cfg;
    w.zkey = job->zkey;
    w.replay = replay;
    w.objective = job->objective;
    w.tried = (int8_t *)calloc((size_t)n, 1);
    w.x = (int8_t *)malloc((size_t)L);
    w.s = (int8_t *)malloc((size_t)L);
    w.s_best = (int8_t *)malloc((size_t)L);
    w.delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    w.order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    w.sf = (int8_t *)malloc((size_t)L);
    w.cand_psl = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    w.cand_isl = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    w.ht.mask = (1ull << job->cfg->tabu_log2) - 1;
    w.ht.cap = job->cfg->probe_cap;
    if ((uint64_t)w.ht.cap > w.ht.mask + 1) w.ht.cap = (int32_t)(w.ht.mask + 1);
    w.ht.slot = (uint64_t *)calloc((size_t)(w.ht.mask + 1), sizeof(uint64_t));
    w.ht.gen = 1;
    w.best_isl = INT64_MAX;
    w.best_psl = INT64_MAX;
    w.res.target_step = -1;
    int rc = 0;
    if (!w.x || !w.s || !w.s_best || !w.delta || !w.order || !w.ht.slot || !w.tried || !w.sf || !w.cand_psl ||
        !w.cand_isl) {
        rc = -3;
        goto done;
    }
    start(&w, 0);
    for (int64_t t = 0; t < job->steps; ++t) {
        int32_t code = w.objective ? walk_step_psl(&w, t + 1) : walk_step(&w, t + 1);
        if (code == -99) {
            rc = -2;
            break;
        }
        if (job->trace_code) {
            job->trace_code[w_idx * job->steps + t] = code;
            job->trace_isl[w_idx * job->steps + t] = (int32_t)w.isl;
        }
    }
    w.res.final_isl = (int32_t)w.isl;
    w.res.best_isl = (int32_t)w.best_isl;
    w.res.final_psl = (int32_t)lo_psl(w.s, L);
    w.res.best_psl = (int32_t)lo_psl(w.s_best, L);
    job->res[w_idx] = w.res;
    if (job->best_seq) memcpy(job->best_seq + w_idx * L, w.s_best, (size_t)L);
    if (job->final_seq) memcpy(job->final_seq + w_idx * L, w.s, (size_t)L);
done:
    free(w.x); free(w.s); free(w.s_best); free(w.delta); free(w.order); free(w.ht.slot); free(w.tried);
    free(w.sf); free(w.cand_psl); free(w.cand_isl);
    return rc;
}

static void *walk_thread(void *arg)
{
    lo_walk_job *job = (lo_walk_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t w = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (w >= job->count) break;
        int rc = job->pq_size > 0 ? run_bestfirst(job, w) : run_walker(job, w, NULL);
        if (rc != 0) {
            pthread_mutex_lock(&job->lock);
            job->status = rc;
            pthread_mutex_unlock(&job->lock);
        }
    }
    return NULL;
}

/* Walkers g0 .. g0+count-1 of length L each take `steps` steps of the walk (pq_size 0)
 * or of the best-first search with a queue of pq_size entries (pq_size > 0, with
 * xLastovka's second table when second_hash is set).  Results per walker
 * go to res[], best_seq/final_seq ([count][L], nullable) and, when trace_code is not
 * NULL, per-step traces ([count][steps]).  nthreads <= 0 uses every online core.
 * Returns 0, -1 on bad arguments, -2 on an internal mismatch, -3 on allocation
 * failure. */
static int walk_many(int32_t L, uint64_t seed, int64_t g0, int64_t count, int64_t steps,
                     const lo_walk_cfg *cfg, int32_t pq_size, int32_t second_hash, int32_t objective,
                     lo_walk_result *res, int8_t *best_seq,
                     int8_t *final_seq, int32_t *trace_code, int32_t *trace_isl, int32_t nthreads)
{
    if (L < 3 || (L & 1) == 0 || count < 0 || steps < 0 || !cfg || !res) return -1;
    if (cfg->tabu_log2 < 1 || cfg->tabu_log2 > 20 || cfg->probe_cap < 1) return -1;
    if (g0 < 0 || g0 + count > 0x100000000ll) return -1;
    if ((trace_code == NULL) != (trace_isl == NULL)) return -1;
    int32_t n = (L + 1) / 2;
    uint64_t *zkey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    if (!zkey) return -3;
    for (int32_t i = 0; i < n; ++i) zkey[i] = lo_zobrist_key(L, i);
    lo_walk_job job;
    memset(&job, 0, sizeof(job));
    job.L = L; job.seed = seed; job.g0 = g0; job.count = count; job.steps = steps;
    job.cfg = cfg; job.zkey = zkey; job.res = res; job.best_seq = best_seq;
    job.final_seq = final_seq; job.trace_code = trace_code; job.trace_isl = trace_isl;
    job.pq_size = pq_size;
    job.second_hash = second_hash;
    job.objective = objective;
    pthread_mutex_init(&job.lock, NULL);
    if (nthreads <= 0) nthreads = (int32_t)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > count) nthreads = (int32_t)(count > 0 ? count : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int32_t t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, walk_thread, &job);
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    free(zkey);
    return job.status;
}

int lo_walk(int32_t L, uint64_t seed, int64_t g0, int64_t count, int64_t steps,
            const lo_walk_cfg *cfg, lo_walk_result *res, int8_t *best_seq, int8_t *final_seq,
            int32_t *trace_code, int32_t *trace_isl, int32_t nthreads)
{
    return walk_many(L, seed, g0, count, steps, cfg, 0, 0, 0, res, best_seq, final_seq, trace_code, trace_isl,
                     nthreads);
}

/* As lo_walk with the PSL objective (walk_step_psl): the ISL trace still holds the ISL
 * at the end of each step, and res[].best_psl / best_isl describe the best sequence in
 * the (PSL, ISL) order. */
int lo_walk_psl(int32_t L, uint64_t seed, int64_t g0, int64_t count, int64_t steps,
                const lo_walk_cfg *cfg, lo_walk_result *res, int8_t *best_seq, int8_t *final_seq,
                int32_t *trace_code, int32_t *trace_isl, int32_t nthreads)
{
    return walk_many(L, seed, g0, count, steps, cfg, 0, 0, 1, res, best_seq, final_seq, trace_code, trace_isl,
                     nthreads);
}

/* One walker (id g) replayed with the learned-mode choices of a GPU run (lo_replay);
 * outputs as lo_walk for a single walker (trace arrays of `steps` entries, nullable). */
int lo_walk_replay(int32_t L, uint64_t seed, int64_t g, int64_t steps, const lo_walk_cfg *cfg, int32_t tau,
                   int32_t n_score, const int64_t *score_step, const float *scores, int32_t score_stride,
                   int32_t n_restart, const int64_t *restart_idx, const uint32_t *restart_bits,
                   lo_walk_result *res, int8_t *best_seq, int8_t *final_seq, int32_t *trace_code,
                   int32_t *trace_isl)
{
    if (L < 3 || (L & 1) == 0 || steps < 0 || !cfg || !res || g < 0 || g >= 0x100000000ll) return -1;
    if (cfg->tabu_log2 < 1 || cfg->tabu_log2 > 20 || cfg->probe_cap < 1) return -1;
    int32_t n = (L + 1) / 2;
    uint64_t *zkey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    if (!zkey) return -3;
    for (int32_t i = 0; i < n; ++i) zkey[i] = lo_zobrist_key(L, i);
    lo_replay rp = {tau, n_score, score_step, scores, score_stride, n_restart, restart_idx, restart_bits};
    lo_walk_job job;
    memset(&job, 0, sizeof(job));
    job.L = L; job.seed = seed; job.g0 = g; job.count = 1; job.steps = steps;
    job.cfg = cfg; job.zkey = zkey; job.res = res; job.best_seq = best_seq;
    job.final_seq = final_seq; job.trace_code = trace_code; job.trace_isl = trace_isl;
    int rc = run_walker(&job, 0, &rp);
    free(zkey);
    return rc;
}

/* ------------------------------------------- best-first search (Algorithm 1) */

/* Algorithm 1 as printed (impxLast): every neighbour of the current S that is not in
 * HT is evaluated and goes into a priority queue of fixed size K ordered by merit
 * factor (the best is kept), and the next S is removed from the front of the queue.
 * Readings where the paper is silent:
 *   - HT holds the sequences that have been S, as in the walk; a neighbour in HT is
 *     skipped, and an entry taken from the queue that is in HT by then is discarded.
 *   - queue order: ISL ascending (F descending), then the step that produced the
 *     entry (steps done before it), then i, all ascending.  A full queue takes a new
 *     entry only if it comes before its last entry, which it then drops; neighbours
 *     are considered in that order, so the queue after a step holds the K first of
 *     its old entries and the step's new ones.
 *   - when the queue runs empty, or HT has no free slot for the new S, the walker
 *     restarts from a fresh random S with HT and queue emptied; there is no other
 *     restart rule (Alg. 1 has none).
 *   - the best sequence is updated by every neighbour that enters the queue (a
 *     neighbour that does not enter it cannot beat the best: the best is at least as
 *     good as every queue entry).
 * Trace codes, one per step: the low 16 bits of the new S's fingerprint, with bit 16
 * set when the step ended in a restart after an HT overflow, or -1 when the queue ran
 * empty (restart); the ISL trace holds the ISL of S at the end of the step. */
typedef struct {
    int64_t isl, born;
    int32_t i;
    uint64_t fp;
    int8_t *s;
} lo_pq_entry;

typedef struct {
    int32_t cap, size;
    lo_pq_entry *e;
} lo_pq;

static int pq_before(const lo_pq_entry *a, const lo_pq_entry *b)
{
    if (a->isl != b->isl) return a->isl < b->isl;
    if (a->born != b->born) return a->born < b->born;
    return a->i < b->i;
}

static int32_t pq_extreme(const lo_pq *q, int want_last)
{
    int32_t k = 0;
    for (int32_t j = 1; j < q->size; ++j) {
        int b = pq_before(&q->e[j], &q->e[k]);
        if (want_last ? !b : b) k = j;
    }
    return k;
}

/* removes entry k, keeping the storage of every entry */
static void pq_remove(lo_pq *q, int32_t k)
{
    lo_pq_entry t = q->e[k];
    q->e[k] = q->e[q->size - 1];
    q->e[q->size - 1] = t;
    q->size -= 1;
}

static void bf_note(lo_walker *w, const int8_t *s, int64_t isl, int64_t steps_done)
{
    if (isl < w->best_isl) {
        w->best_isl = isl;
        memcpy(w->s_best, s, (size_t)w->L);
        w->res.best_step = steps_done;
    }
    if (w->res.target_step < 0 && target_met(w, isl)) w->res.target_step = steps_done;
}

/* One step (expansion of S); e = steps done before it.  Returns the trace code, or
 * -99 on an internal mismatch. */
/* xLastovka's second table (the reading used here): one 64-bit word per slot, slot =
 * fingerprint mod its size; a neighbour with fingerprint f is in the table when its slot
 * holds (gen << 40) | (~f mod 2^40), gen being HT's generation (so a restart empties
 * both); inserting keeps the larger of the old and the new word, which makes the table's
 * content independent of the order of the insertions within a step. */
#define LO_CACHE_LOW 0xFFFFFFFFFFull
static uint64_t cache_tag(const lo_walker *w, uint64_t f)
{
    return ((uint64_t)w->ht.gen << 40) | (~f & LO_CACHE_LOW);
}

static int32_t bf_step(lo_walker *w, lo_pq *q, int64_t e)
{
    int32_t L = w->L, n = w->n;
    if (lo_neighbor_delta(w->s, L, w->delta) != 0) return -99;
    if (w->cache) {
        /* neighbours held by the second table are skipped: not evaluated, not queued */
        for (int32_t i = 0; i < n; ++i) {
            uint64_t f = w->fp ^ w->zkey[i];
            w->tried[i] = w->cache[f & w->ht.mask] == cache_tag(w, f);
            w->res.cache_hits += w->tried[i];
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t j = i;
        while (j > 0 && cmp_pair(w->delta, i, w->order[j - 1]) < 0) {
            w->order[j] = w->order[j - 1];
            --j;
        }
        w->order[j] = i;
    }
    for (int32_t t = 0; t < n; ++t) {
        int32_t i = w->order[t];
        if (w->cache && w->tried[i]) continue;
        lo_pq_entry c = {w->isl + w->delta[i], e, i, w->fp ^ w->zkey[i], NULL};
        int32_t last = -1;
        if (q->size == q->cap) {
            last = pq_extreme(q, 1);
            if (!pq_before(&c, &q->e[last])) break;  /* the rest come later still */
        }
        if (ht_contains(&w->ht, c.fp)) continue;
        if (last >= 0) pq_remove(q, last);
        lo_pq_entry *d = &q->e[q->size++];
        c.s = d->s;
        *d = c;
        memcpy(d->s, w->s, (size_t)L);
        int32_t m = L - 1 - i;
        d->s[i] = (int8_t)(-d->s[i]);
        if (m != i) d->s[m] = (int8_t)(-d->s[m]);
        if (lo_isl(d->s, L) != d->isl) return -99;
        bf_note(w, d->s, d->isl, e + 1);
    }
    if (w->cache) {
        /* every neighbour evaluated in this step enters the second table */
        for (int32_t i = 0; i < n; ++i) {
            if (w->tried[i]) continue;
            uint64_t f = w->fp ^ w->zkey[i], tag = cache_tag(w, f);
            uint64_t *slot = &w->cache[f & w->ht.mask];
            if (tag > *slot) *slot = tag;
        }
    }
    for (;;) {
        if (q->size == 0) {
            restart(w, e + 1);
            return -1;
        }
        int32_t k = pq_extreme(q, 0);
        lo_pq_entry *d = &q->e[k];
        if (ht_contains(&w->ht, d->fp)) {
            pq_remove(q, k);
            continue;
        }
        memcpy(w->s, d->s, (size_t)L);
        w->isl = d->isl;
        w->fp = d->fp;
        pq_remove(q, k);
        int32_t code = (int32_t)(w->fp & 0xFFFFu);
        if (!ht_insert(&w->ht, w->fp)) {
            w->res.overflows += 1;
            q->size = 0;
            restart(w, e + 1);
            return code | LO_TRACE_RESTART;
        }
        return code;
    }
}

static int run_bestfirst(lo_walk_job *job, int64_t w_idx)
{
    int32_t L = job->L, n = (L + 1) / 2, K = job->pq_size;
    lo_walker w;
    lo_pq q;
    memset(&w, 0, sizeof(w));
    memset(&q, 0, sizeof(q));
    w.L = L;
    w.n = n;
    w.seed = job->seed;
    w.g = (uint32_t)(job->g0 + w_idx);
    w.cfg = job->cfg;
    w.zkey = job->zkey;
    w.x = (int8_t *)malloc((size_t)L);
    w.s = (int8_t *)malloc((size_t)L);
    w.s_best = (int8_t *)malloc((size_t)L);
    w.delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    w.order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    w.tried = (int8_t *)calloc((size_t)n, 1);
    w.ht.mask = (1ull << job->cfg->tabu_log2) - 1;
    w.ht.cap = job->cfg->probe_cap;
    if ((uint64_t)w.ht.cap > w.ht.mask + 1) w.ht.cap = (int32_t)(w.ht.mask + 1);
    w.ht.slot = (uint64_t *)calloc((size_t)(w.ht.mask + 1), sizeof(uint64_t));
    if (job->second_hash) w.cache = (uint64_t *)calloc((size_t)(w.ht.mask + 1), sizeof(uint64_t));
    w.ht.gen = 1;
    w.best_isl = INT64_MAX;
    w.res.target_step = -1;
    q.cap = K;
    q.e = (lo_pq_entry *)calloc((size_t)K, sizeof(lo_pq_entry));
    int8_t *store = (int8_t *)malloc((size_t)K * (size_t)L);
    int rc = 0;
    if (!w.x || !w.s || !w.s_best || !w.delta || !w.order || !w.ht.slot || !q.e || !store || !w.tried ||
        (job->second_hash && !w.cache)) {
        rc = -3;
        goto done;
    }
    for (int32_t k = 0; k < K; ++k) q.e[k].s = store + (size_t)k * (size_t)L;
    start(&w, 0);
    for (int64_t t = 0; t < job->steps; ++t) {
        int32_t code = bf_step(&w, &q, t);
        if (code == -99) {
            rc = -2;
            break;
        }
        if (code == -1 || (code & LO_TRACE_RESTART)) q.size = 0;
        if (job->trace_code) {
            job->trace_code[w_idx * job->steps + t] = code;
            job->trace_isl[w_idx * job->steps + t] = (int32_t)w.isl;
        }
    }
    w.res.final_isl = (int32_t)w.isl;
    w.res.best_isl = (int32_t)w.best_isl;
    w.res.final_psl = (int32_t)lo_psl(w.s, L);
    w.res.best_psl = (int32_t)lo_psl(w.s_best, L);
    job->res[w_idx] = w.res;
    if (job->best_seq) memcpy(job->best_seq + w_idx * L, w.s_best, (size_t)L);
    if (job->final_seq) memcpy(job->final_seq + w_idx * L, w.s, (size_t)L);
done:
    free(w.x); free(w.s); free(w.s_best); free(w.delta); free(w.order); free(w.ht.slot); free(q.e); free(store);
    free(w.tried); free(w.cache);
    return rc;
}

/* Walkers g0 .. g0+count-1 of length L each take `steps` steps of the best-first
 * search with a queue of pq_size entries (cfg->patience is not used); arguments and
 * results as lo_walk. */
int lo_bestfirst(int32_t L, uint64_t seed, int64_t g0, int64_t count, int64_t steps, const lo_walk_cfg *cfg,
                 int32_t pq_size, lo_walk_result *res, int8_t *best_seq, int8_t *final_seq, int32_t *trace_code,
                 int32_t *trace_isl, int32_t nthreads)
{
    if (pq_size < 1) return -1;
    return walk_many(L, seed, g0, count, steps, cfg, pq_size, 0, 0, res, best_seq, final_seq, trace_code, trace_isl,
                     nthreads);
}

/* As lo_bestfirst with xLastovka's second table (see cache_tag): neighbours it holds are
 * skipped, every evaluated neighbour enters it; res[].cache_hits counts the skips. */
int lo_bestfirst_cached(int32_t L, uint64_t seed, int64_t g0, int64_t count, int64_t steps, const lo_walk_cfg *cfg,
                        int32_t pq_size, lo_walk_result *res, int8_t *best_seq, int8_t *final_seq,
                        int32_t *trace_code, int32_t *trace_isl, int32_t nthreads)
{
    if (pq_size < 1) return -1;
    return walk_many(L, seed, g0, count, steps, cfg, pq_size, 1, 0, res, best_seq, final_seq, trace_code, trace_isl,
                     nthreads);
}

/* ------------------------------------------------- exhaustive skew enumeration */

/* Every skew-symmetric sequence with the centre s_c = +1 (negating all of S keeps
 * Eq. 4 and the ISL): assignment a in [0, 2^(n-1)) sets x_i = -1 exactly when bit i
 * of a is set (i < c).  Reports the minimum ISL, how many assignments reach it and
 * the lowest such a, with its sequence.  Each ISL is Eq. 2 from scratch. */
typedef struct {
    int32_t L;
    uint64_t lo, hi;
    int64_t min_isl;
    uint64_t count, first;
} lo_enum_part;

static void *enum_thread(void *arg)
{
    lo_enum_part *p = (lo_enum_part *)arg;
    int32_t L = p->L, n = (L + 1) / 2;
    int8_t *x = (int8_t *)malloc((size_t)n), *s = (int8_t *)malloc((size_t)L);
    p->min_isl = INT64_MAX;
    p->count = 0;
    p->first = 0;
    for (uint64_t a = p->lo; a < p->hi; ++a) {
        for (int32_t i = 0; i < n - 1; ++i) x[i] = ((a >> i) & 1u) ? -1 : 1;
        x[n - 1] = 1;
        lo_skew_expand(x, L, s);
        int64_t e = lo_isl(s, L);
        if (e < p->min_isl) {
            p->min_isl = e;
            p->count = 1;
            p->first = a;
        } else if (e == p->min_isl) {
            p->count += 1;
        }
    }
    free(x);
    free(s);
    return NULL;
}

int lo_enumerate(int32_t L, int64_t *min_isl, uint64_t *count, uint64_t *first_assignment,
                 int8_t *best_seq, int32_t nthreads)
{
    if (L < 3 || (L & 1) == 0 || L > 79) return -1;
    int32_t n = (L + 1) / 2;
    uint64_t total = 1ull << (n - 1);
    if (nthreads <= 0) nthreads = (int32_t)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > total) nthreads = (int32_t)total;
    lo_enum_part *parts = (lo_enum_part *)calloc((size_t)nthreads, sizeof(lo_enum_part));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int32_t t = 0; t < nthreads; ++t) {
        parts[t].L = L;
        parts[t].lo = total * (uint64_t)t / (uint64_t)nthreads;
        parts[t].hi = total * (uint64_t)(t + 1) / (uint64_t)nthreads;
        pthread_create(&th[t], NULL, enum_thread, &parts[t]);
    }
    int64_t m = INT64_MAX;
    uint64_t cnt = 0, first = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (parts[t].hi == parts[t].lo) continue;
        if (parts[t].min_isl < m) {
            m = parts[t].min_isl;
            cnt = parts[t].count;
            first = parts[t].first;
        } else if (parts[t].min_isl == m) {
            cnt += parts[t].count;
        }
    }
    free(th);
    free(parts);
    *min_isl = m;
    *count = cnt;
    *first_assignment = first;
    if (best_seq) {
        int8_t *x = (int8_t *)malloc((size_t)n);
        for (int32_t i = 0; i < n - 1; ++i) x[i] = ((first >> i) & 1u) ? -1 : 1;
        x[n - 1] = 1;
        lo_skew_expand(x, L, best_seq);
        free(x);
    }
    return 0;
}
