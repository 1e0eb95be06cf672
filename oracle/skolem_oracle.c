/*
 * skolem_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU reference for the counting method of
 * "Counting Skolem Sequences" (Assarpour, Bar-Noy, Liu).  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load this file's
 * library.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, each function citing the passage it follows:
 *   orc_layout            -- the position set P and the differences d_k of the
 *                            three problems (Sec. 1.1 Skolem and Langford,
 *                            Sec. 1.2 hooked Skolem).
 *   orc_backtrack         -- Miller's enumeration (Sec. 2): pairs placed in
 *                            decreasing order, each at every position where
 *                            it fits, backtracking when a pair cannot be placed.
 *   orc_signed_sum        -- Algorithm 1 (Sec. 2.1) as stated: for every +-1
 *                            assignment X, sign(X) * prod_i sum_k x_k x_{k+i},
 *                            summed exactly (wrap-around 128-bit integers).
 *                            With half=1 the variable at max P is fixed to +1
 *                            (Lemma 2.2).
 *   orc_summand           -- the summand of Algorithm 1 for one assignment.
 *   orc_partial_sum_mod   -- the same summand over one block of assignments
 *                            (the low m free variables run, the rest fixed),
 *                            reduced modulo a given prime (Sec. 2.2: residues
 *                            modulo co-primes).
 *   orc_backtrack_hole, orc_signed_sum_hole, orc_partial_sum_mod_hole --
 *                            the same three for extended Skolem sequences
 *                            (Sec. 1.2: the hook anywhere): positions 1..2n+1
 *                            except one hole, differences 1..n.
 *   orc_ie_count          -- the inclusion-exclusion count (Sec. 2, the
 *                            third approach, after Larsen): over every set S
 *                            of avoided positions, (-1)^{|S|} times the
 *                            number of pairings of the universe (overlaps
 *                            allowed) that avoid S.
 *   orc_ie_partial_sum_mod -- the same sum over one block of sets, reduced
 *                            modulo a given prime.
 *   orc_philox4x32_10     -- the Philox-4x32-10 counter-based generator of
 *                            Salmon, Moraes, Dror, Shaw (SC'11), written from
 *                            its published definition.
 *   orc_pt_run            -- Algorithm 2 (Sec. 3): parallel tempering over the
 *                            simplified problem, energy = number of empty bins,
 *                            Metropolis moves and neighbour exchanges;
 *                            orc_pt_run_trips also counts the round trips of
 *                            configurations between the ends of the ladder.
 *   orc_simplified_energy_hist -- exhaustive enumeration of the simplified
 *                            problem of Sec. 3 (every pair k at any of its
 *                            start slots): the number N(E) of configurations
 *                            with E empty bins; Z(beta) = sum_E N(E) e^{-beta E}.
 *
 * Readings of the paper taken here (the paper is silent or inconsistent):
 *   - Langford differences d_k = k+1 (Sec. 1.1: two copies of k with k numbers
 *     between them, example 2,3,4,2,1,3,1,4).
 *   - Hooked Skolem: positions 1..2n-1 and 2n+1, d_k = k (Sec. 1.2).
 *   - Algorithm 2 accepts when a uniform u in [0,1) is below p (the printed
 *     "p <= random" contradicts p = min[1, e^{-beta dE}]).  In integers, with
 *     u = w / 2^32 for a 32-bit word w: accept iff w < ceil(p * 2^32).
 *   - Exchanges alternate: at iteration t the pairs (j, j+1) with j = t mod 2
 *     (rungs counted from 0) are tried.
 *   - A move picks k uniformly and a new start slot uniformly among the other
 *     start slots of pair k; a pair with a single start slot is not moved.
 *   - Statistics are taken from the state at the start of each iteration,
 *     then moves, then exchanges (the order of Algorithm 2); the first
 *     `burnin` iterations are not counted.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 s128;

#define ORC_MAXN 64      /* the paper's largest order: its closing S(64) estimate */
#define ORC_MAXSPAN (2 * ORC_MAXN + 2)

/* ------------------------------------------------------------------ layout */

/* Sec. 1.1 / 1.2.  present[1..span] marks the positions of P (1-indexed as in
 * the paper); d[1..n] are the differences.  Returns 0 or -1 for bad input. */
int orc_layout(int variant, int n, int *span, int *present, int *d)
{
    if (n < 1 || n > ORC_MAXN || variant < 0 || variant > 2) return -1;
    int s = (variant == 2) ? 2 * n + 1 : 2 * n;
    for (int i = 0; i <= s; i++) present[i] = (i >= 1);
    if (variant == 2) present[2 * n] = 0;          /* the hook: 2n is skipped */
    for (int k = 1; k <= n; k++) d[k] = (variant == 1) ? k + 1 : k;
    *span = s;
    return 0;
}

/* ------------------------------------------------------- O1: backtracking */

typedef struct {
    int n, span;
    int present[ORC_MAXSPAN + 1];
    int d[ORC_MAXN + 1];
    int label[ORC_MAXSPAN + 1];     /* 0 = empty, else the pair placed there */
    uint64_t count;
    int8_t *list;
    uint64_t max_list;
} bt_state;

static void bt_place(bt_state *st, int k)
{
    if (k == 0) {                                  /* every pair placed */
        if (st->list && st->count < st->max_list) {
            int8_t *row = st->list + st->count * (uint64_t)st->span;
            for (int i = 1; i <= st->span; i++) row[i - 1] = (int8_t)st->label[i];
        }
        st->count++;
        return;
    }
    int d = st->d[k];
    for (int a = 1; a + d <= st->span; a++) {      /* leftmost fit first */
        int b = a + d;
        if (!st->present[a] || !st->present[b]) continue;
        if (st->label[a] || st->label[b]) continue;
        st->label[a] = st->label[b] = k;
        bt_place(st, k - 1);                       /* next smaller pair */
        st->label[a] = st->label[b] = 0;           /* move this pair on */
    }
}

/* Number of pairings with reflections counted as distinct.  If list != NULL
 * the first max_list pairings are written as rows of span labels (0 marks
 * the skipped position of the hooked problem). */
int orc_backtrack(int variant, int n, uint64_t *count, int8_t *list, uint64_t max_list)
{
    bt_state *st = (bt_state *)calloc(1, sizeof(bt_state));
    if (!st) return -1;
    if (orc_layout(variant, n, &st->span, st->present, st->d)) { free(st); return -1; }
    st->n = n;
    st->list = list;
    st->max_list = max_list;
    bt_place(st, n);
    *count = st->count;
    free(st);
    return 0;
}

/* ----------------------------------------------- O2: Algorithm 1 directly */

typedef struct {
    int n, span, nvar;
    int present[ORC_MAXSPAN + 1];
    int d[ORC_MAXN + 1];
    int var_pos[ORC_MAXSPAN];       /* enumerated variable i -> position */
    int fixed_top;                  /* position held at +1 (half mode) or 0 */
    uint64_t lo, hi;                /* this worker's range of assignments */
    u128 sum;
} ss_job;

/* sign(X) * prod_{i=1..n} sum_k x_k x_{k+d_i}, as a wrap-around 128-bit value.
 * x[] holds +1/-1 at the positions of P and 0 elsewhere. */
static u128 summand_u128(const ss_job *j, const int *x)
{
    int sign = 1;
    for (int p = 1; p <= j->span; p++)
        if (j->present[p]) sign *= x[p];
    u128 prod = 1;
    for (int i = 1; i <= j->n; i++) {
        int di = j->d[i];
        long sum = 0;
        for (int k = 1; k + di <= j->span; k++) sum += (long)x[k] * x[k + di];
        prod *= (u128)(s128)sum;
    }
    return sign > 0 ? prod : (u128)0 - prod;
}

static void *ss_worker(void *arg)
{
    ss_job *j = (ss_job *)arg;
    int x[ORC_MAXSPAN + 2];
    u128 acc = 0;
    for (uint64_t X = j->lo; X < j->hi; X++) {
        memset(x, 0, sizeof(x));
        for (int i = 0; i < j->nvar; i++) x[j->var_pos[i]] = ((X >> i) & 1) ? -1 : 1;
        if (j->fixed_top) x[j->fixed_top] = 1;
        acc += summand_u128(j, x);
    }
    j->sum = acc;
    return NULL;
}

/* Algorithm 1: S = sum over X of sign(X) F(n, X).  out[0..1] = S as a
 * two's-complement 128-bit integer (exact while |S| < 2^127).  half=1 fixes
 * the variable at max P to +1 (Lemma 2.2), which halves S. */
int orc_signed_sum(int variant, int n, int half, int nthreads, uint64_t *out)
{
    ss_job base;
    memset(&base, 0, sizeof(base));
    if (orc_layout(variant, n, &base.span, base.present, base.d)) return -1;
    base.n = n;
    int top = 0;
    for (int p = 1; p <= base.span; p++) if (base.present[p]) top = p;
    for (int p = 1; p <= base.span; p++) {
        if (!base.present[p]) continue;
        if (half && p == top) continue;
        base.var_pos[base.nvar++] = p;
    }
    base.fixed_top = half ? top : 0;
    if (base.nvar > 62) return -1;
    uint64_t total = (uint64_t)1 << base.nvar;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > total) nthreads = (int)total;
    ss_job *jobs = (ss_job *)calloc((size_t)nthreads, sizeof(ss_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = base;
        jobs[t].lo = total / nthreads * t;
        jobs[t].hi = (t == nthreads - 1) ? total : total / nthreads * (t + 1);
        if (nthreads == 1) ss_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, ss_worker, &jobs[t]);
    }
    u128 s = 0;
    for (int t = 0; t < nthreads; t++) {
        if (nthreads > 1) pthread_join(th[t], NULL);
        s += jobs[t].sum;
    }
    free(jobs);
    free(th);
    out[0] = (uint64_t)s;
    out[1] = (uint64_t)(s >> 64);
    return 0;
}

/* ------------------------------------------- one summand, for properties */

/* sign(X) * F(n, X) for one assignment: x[1..span] (+1/-1 on P, ignored
 * elsewhere).  Written to out[0..1] as a two's-complement 128-bit integer
 * (exact while |F| < 2^127). */
int orc_summand(int variant, int n, const int *x_in, uint64_t *out)
{
    ss_job j;
    memset(&j, 0, sizeof(j));
    if (orc_layout(variant, n, &j.span, j.present, j.d)) return -1;
    j.n = n;
    int x[ORC_MAXSPAN + 2];
    memset(x, 0, sizeof(x));
    for (int p = 1; p <= j.span; p++) {
        if (!j.present[p]) continue;
        if (x_in[p] != 1 && x_in[p] != -1) return -1;
        x[p] = x_in[p];
    }
    u128 v = summand_u128(&j, x);
    out[0] = (uint64_t)v;
    out[1] = (uint64_t)(v >> 64);
    return 0;
}

/* -------------------------------------- one block of the sum, modulo p */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p)
{
    return (uint64_t)(((u128)a * b) % p);
}

static uint64_t to_res(long v, uint64_t p)
{
    long r = v % (long)p;
    return (uint64_t)(r < 0 ? r + (long)p : r);
}

/* The free variables are the positions 1..2n-1 (every variable of P except
 * max P, which Lemma 2.2 fixes to +1).  Free variable i (0-based) is position
 * i+1.  This block runs over the low m free variables and fixes the others
 * from q: free variable m+b is -1 iff bit b of q is set.  Returns
 * sum_block sign(X) F(n, X) mod p in [0, p). */
int orc_partial_sum_mod(int variant, int n, int m, uint64_t q, uint64_t p, uint64_t *out)
{
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1];
    if (orc_layout(variant, n, &span, present, d)) return -1;
    int nfree = 2 * n - 1;
    if (m < 0 || m > nfree || m > 40 || p < 3 || p > ((uint64_t)1 << 62)) return -1;
    if (nfree - m > 64) return -1;             /* q holds the fixed variables */
    int top = 0;
    for (int i = 1; i <= span; i++) if (present[i]) top = i;
    int x[ORC_MAXSPAN + 2];
    uint64_t acc = 0;
    for (uint64_t w = 0; w < ((uint64_t)1 << m); w++) {
        memset(x, 0, sizeof(x));
        for (int i = 0; i < nfree; i++) {
            int bit = (i < m) ? (int)((w >> i) & 1) : (int)((q >> (i - m)) & 1);
            x[i + 1] = bit ? -1 : 1;
        }
        x[top] = 1;
        int sign = 1;
        for (int i = 1; i <= span; i++) if (present[i]) sign *= x[i];
        uint64_t prod = 1;
        for (int k = 1; k <= n; k++) {
            long s = 0;
            for (int a = 1; a + d[k] <= span; a++) s += (long)x[a] * x[a + d[k]];
            prod = mulmod(prod, to_res(s, p), p);
        }
        if (sign < 0) prod = prod ? p - prod : 0;
        acc = (acc + prod) % p;
    }
    *out = acc;
    return 0;
}

/* ------------------------------- extended Skolem sequences (one hole) */

/* Sec. 1.2: extended Skolem sequences (Abrham and Kotzig) distribute the
 * numbers over 1..2n+1 with one position -- the hole -- left empty, pairs of
 * k at distance k.  hole = 2n is the hooked problem, hole = n+1 Rosa's (the
 * skip in the middle), hole = 2n+1 or 1 the Skolem problem on 2n positions. */
static int layout_hole(int n, int hole, int *span, int *present, int *d)
{
    if (n < 1 || n > ORC_MAXN || hole < 1 || hole > 2 * n + 1) return -1;
    *span = 2 * n + 1;
    for (int i = 0; i <= *span; i++) present[i] = (i >= 1 && i != hole);
    for (int k = 1; k <= n; k++) d[k] = k;
    return 0;
}

int orc_backtrack_hole(int n, int hole, uint64_t *count)
{
    bt_state *st = (bt_state *)calloc(1, sizeof(bt_state));
    if (!st) return -1;
    if (layout_hole(n, hole, &st->span, st->present, st->d)) { free(st); return -1; }
    st->n = n;
    bt_place(st, n);
    *count = st->count;
    free(st);
    return 0;
}

/* Algorithm 1 over the ±1 assignments of the 2n positions of that P, with
 * the variable at max P held at +1 (Lemma 2.2): the half-sum S as a
 * two's-complement 128-bit integer, out[0..1]. */
int orc_signed_sum_hole(int n, int hole, uint64_t *out)
{
    ss_job j;
    memset(&j, 0, sizeof(j));
    if (layout_hole(n, hole, &j.span, j.present, j.d)) return -1;
    j.n = n;
    int top = 0;
    for (int p = 1; p <= j.span; p++) if (j.present[p]) top = p;
    for (int p = 1; p <= j.span; p++)
        if (j.present[p] && p != top) j.var_pos[j.nvar++] = p;
    j.fixed_top = top;
    if (j.nvar > 40) return -1;
    j.lo = 0;
    j.hi = (uint64_t)1 << j.nvar;
    ss_worker(&j);
    out[0] = (uint64_t)j.sum;
    out[1] = (uint64_t)(j.sum >> 64);
    return 0;
}

/* One block of that half-sum modulo p: the free variables are the positions
 * of P below max P in increasing order (variable i = the i-th of them); the
 * low m run over both values, variable m+b is -1 iff bit b of q is set. */
int orc_partial_sum_mod_hole(int n, int hole, int m, uint64_t q, uint64_t p, uint64_t *out)
{
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1], pos[ORC_MAXSPAN];
    if (layout_hole(n, hole, &span, present, d)) return -1;
    int top = 0, nfree = 0;
    for (int i = 1; i <= span; i++) if (present[i]) top = i;
    for (int i = 1; i <= span; i++) if (present[i] && i != top) pos[nfree++] = i;
    if (m < 0 || m > nfree || m > 40 || nfree - m > 63 || p < 3 || p > ((uint64_t)1 << 62))
        return -1;
    int x[ORC_MAXSPAN + 2];
    uint64_t acc = 0;
    for (uint64_t w = 0; w < ((uint64_t)1 << m); w++) {
        memset(x, 0, sizeof(x));
        for (int i = 0; i < nfree; i++) {
            int bit = (i < m) ? (int)((w >> i) & 1) : (int)((q >> (i - m)) & 1);
            x[pos[i]] = bit ? -1 : 1;
        }
        x[top] = 1;
        int sign = 1;
        for (int i = 1; i <= span; i++) if (present[i]) sign *= x[i];
        uint64_t prod = 1;
        for (int k = 1; k <= n; k++) {
            long s = 0;
            for (int a = 1; a + d[k] <= span; a++) s += (long)x[a] * x[a + d[k]];
            prod = mulmod(prod, to_res(s, p), p);
        }
        if (sign < 0) prod = prod ? p - prod : 0;
        acc = (acc + prod) % p;
    }
    *out = acc;
    return 0;
}

/* ------------------------ O6: inclusion-exclusion over avoided positions */

/* Sec. 2 (third approach): let the universe be every way of placing each
 * pair k at two positions a, a+d_k of P, overlaps allowed, and A_i the
 * placements that leave position i empty.  The sequences are the placements
 * that leave no position empty, so by inclusion-exclusion their number
 * (reflections distinct) is
 *     sum over S subset of P of (-1)^{|S|} |A_S|,
 * A_S being the placements that avoid every position of S.  A placement
 * avoids S iff every pair lies inside T = P \ S, so |A_S| is the product over
 * k of the number of pairs (a, a+d_k) with both ends in T.
 * The sets T are enumerated through the positions of P in increasing order:
 * "variable i" (0-based) is the i-th position of P, in T iff bit i of the
 * enumerated word is set. */
static void ie_positions(int span, const int *present, int *pos, int *np)
{
    int c = 0;
    for (int i = 1; i <= span; i++) if (present[i]) pos[c++] = i;
    *np = c;
}

/* prod_k #{a : a, a+d_k in T}, T given by in_t[1..span] (1 = in T). */
static u128 ie_term(int n, int span, const int *d, const int *in_t)
{
    u128 prod = 1;
    for (int k = 1; k <= n; k++) {
        uint64_t pairs = 0;
        for (int a = 1; a + d[k] <= span; a++) pairs += (uint64_t)(in_t[a] && in_t[a + d[k]]);
        prod *= (u128)pairs;
    }
    return prod;
}

/* The count of sequences, reflections distinct, as out[0..1] (128 bits).
 * Wrap-around 128-bit arithmetic gives the exact sum whenever the result
 * is below 2^128, whatever the partial sums.  Limited to |P| <= 40. */
int orc_ie_count(int variant, int n, uint64_t *out)
{
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1], pos[ORC_MAXSPAN], np;
    if (orc_layout(variant, n, &span, present, d)) return -1;
    ie_positions(span, present, pos, &np);
    if (np > 40) return -1;
    int in_t[ORC_MAXSPAN + 2];
    u128 acc = 0;
    for (uint64_t w = 0; w < ((uint64_t)1 << np); w++) {
        memset(in_t, 0, sizeof(in_t));
        int size_t_ = 0;
        for (int i = 0; i < np; i++)
            if ((w >> i) & 1) { in_t[pos[i]] = 1; size_t_++; }
        u128 t = ie_term(n, span, d, in_t);
        if ((np - size_t_) & 1) acc -= t;          /* (-1)^{|S|}, |S| = |P| - |T| */
        else acc += t;
    }
    out[0] = (uint64_t)acc;
    out[1] = (uint64_t)(acc >> 64);
    return 0;
}

/* The same sum over one block of sets, modulo p: variables 0..m-1 run over
 * both values, variable m+b is fixed to bit b of q.  Returns the block sum
 * mod p in [0, p). */
int orc_ie_partial_sum_mod(int variant, int n, int m, uint64_t q, uint64_t p, uint64_t *out)
{
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1], pos[ORC_MAXSPAN], np;
    if (orc_layout(variant, n, &span, present, d)) return -1;
    ie_positions(span, present, pos, &np);
    if (m < 0 || m > np || m > 40 || p < 3 || p > ((uint64_t)1 << 62)) return -1;
    if (np - m < 64 && (q >> (np - m)) != 0) return -1;
    int in_t[ORC_MAXSPAN + 2];
    uint64_t acc = 0;
    for (uint64_t w = 0; w < ((uint64_t)1 << m); w++) {
        memset(in_t, 0, sizeof(in_t));
        int size_t_ = 0;
        for (int i = 0; i < np; i++) {
            int bit = (i < m) ? (int)((w >> i) & 1) : (int)((q >> (i - m)) & 1);
            if (bit) { in_t[pos[i]] = 1; size_t_++; }
        }
        u128 t = ie_term(n, span, d, in_t);
        uint64_t r = (uint64_t)(t % p);
        if (((np - size_t_) & 1) && r) r = p - r;
        acc = (acc + r) % p;
    }
    *out = acc;
    return 0;
}

/* ------------------------------------------------------ Philox-4x32-10 */

/* Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * ten rounds of two 32x32->64 multiplications with the Weyl key schedule. */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ----------------------------------------- O3: Algorithm 2 (tempering) */

/* Random-number streams (one Philox block each):
 *   init   : counter (k, rung, ladder, 1) word 0 -> start slot of pair k
 *   move   : counter (t, rung, ladder, 2) words 0,1,2 -> pair, slot, accept
 *   swap   : counter (t, j,    ladder, 2) word 3 -> exchange of (j, j+1)
 *            (the word rung j's move leaves unused)
 * key = (seed & 0xffffffff, seed >> 32). */

static uint64_t accept_threshold(double x)   /* x = beta * dE > 0 */
{
    double p = exp(-x);
    double t = ceil(ldexp(p, 32));
    if (t >= 4294967296.0) return (uint64_t)1 << 32;
    return (uint64_t)t;
}

typedef struct {
    int slot[ORC_MAXN + 1];           /* start bin (0-based) of pair k */
    int occ[ORC_MAXSPAN];             /* balls per bin */
    int E;                            /* number of empty bins */
    int dir;                          /* the last end of the ladder it sat at: 0 none
                                         yet, 1 rung 0 (beta = 0), 2 rung M-1 */
} pt_conf;

static void conf_recount(pt_conf *c, int n, const int *d, int bins)
{
    memset(c->occ, 0, sizeof(c->occ));
    for (int k = 1; k <= n; k++) { c->occ[c->slot[k]]++; c->occ[c->slot[k] + d[k]]++; }
    c->E = 0;
    for (int b = 0; b < bins; b++) c->E += (c->occ[b] == 0);
}

/* hist: M x (2n+1) counts of E per rung (temperature index) after burn-in.
 * acc_move[M], acc_swap[M]: accepted moves per rung, accepted exchanges per
 * lower rung of a pair (both may be NULL).  final_slots: L x M x n start slots
 * at the end, per ladder and temperature (may be NULL).  round_trips (may be
 * NULL): how often, over all ladders, a configuration came back to rung 0
 * after reaching rung M-1 since it was last at rung 0 -- a walk from the
 * hottest end of the ladder to the coldest and back, the usual measure of
 * how well the exchanges carry configurations through the temperatures.  Each
 * iteration first looks at the configurations at the two ends (rung 0: count
 * a return if it had reached rung M-1, then mark it; rung M-1: mark it if it
 * came from rung 0); returns are counted from iteration `burnin` on.
 * Variants 0 (Skolem) and 1 (Langford) only: bins are the 2n positions. */
int orc_pt_run_trips(int variant, int n, int M, const double *beta, int L, uint64_t iters,
                     uint64_t burnin, uint64_t seed, uint64_t *hist, uint64_t *acc_move,
                     uint64_t *acc_swap, uint8_t *final_slots, uint64_t *round_trips)
{
    if (variant < 0 || variant > 1 || n < 2 || n > ORC_MAXN || M < 1 || M > 64 || L < 1)
        return -1;
    if (iters > 0xffffffffull) return -1;
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1];
    orc_layout(variant, n, &span, present, d);
    int bins = 2 * n;
    int nslot[ORC_MAXN + 1];
    for (int k = 1; k <= n; k++) {
        nslot[k] = bins - d[k];
        if (nslot[k] < 1) return -1;
    }
    /* acceptance thresholds for moves (dE = 1, 2) and exchanges (dE = 1..2n) */
    uint64_t *tmove = (uint64_t *)calloc((size_t)M * 3, sizeof(uint64_t));
    uint64_t *tswap = (uint64_t *)calloc((size_t)M * (bins + 1), sizeof(uint64_t));
    pt_conf *conf = (pt_conf *)calloc((size_t)M, sizeof(pt_conf));
    if (!tmove || !tswap || !conf) { free(tmove); free(tswap); free(conf); return -1; }
    for (int j = 0; j < M; j++) {
        for (int de = 1; de <= 2; de++) tmove[j * 3 + de] = accept_threshold(beta[j] * (double)de);
        if (j + 1 < M)
            for (int de = 1; de <= bins; de++)
                tswap[j * (bins + 1) + de] = accept_threshold((beta[j + 1] - beta[j]) * (double)de);
    }
    memset(hist, 0, sizeof(uint64_t) * (size_t)M * (bins + 1));
    if (acc_move) memset(acc_move, 0, sizeof(uint64_t) * (size_t)M);
    if (acc_swap) memset(acc_swap, 0, sizeof(uint64_t) * (size_t)M);
    if (round_trips) *round_trips = 0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};

    for (int l = 0; l < L; l++) {
        for (int j = 0; j < M; j++) {                 /* a random configuration */
            for (int k = 1; k <= n; k++) {
                uint32_t c[4] = {(uint32_t)k, (uint32_t)j, (uint32_t)l, 1u}, r[4];
                orc_philox4x32_10(c, key, r);
                conf[j].slot[k] = (int)(((uint64_t)r[0] * (uint64_t)nslot[k]) >> 32);
            }
            conf_recount(&conf[j], n, d, bins);
            conf[j].dir = 0;
        }
        for (uint64_t t = 0; t < iters; t++) {
            if (M >= 2) {                             /* the ends of the ladder */
                if (conf[0].dir == 2 && t >= burnin && round_trips) (*round_trips)++;
                conf[0].dir = 1;
                if (conf[M - 1].dir == 1) conf[M - 1].dir = 2;
            }
            if (t >= burnin)                          /* Ratio(j) statistics */
                for (int j = 0; j < M; j++) hist[j * (bins + 1) + conf[j].E]++;
            for (int j = 0; j < M; j++) {             /* Metropolis moves */
                uint32_t c[4] = {(uint32_t)t, (uint32_t)j, (uint32_t)l, 2u}, r[4];
                orc_philox4x32_10(c, key, r);
                int k = 1 + (int)(((uint64_t)r[0] * (uint64_t)n) >> 32);
                if (nslot[k] < 2) continue;
                pt_conf *C = &conf[j];
                int s_old = C->slot[k];
                int s_new = (int)(((uint64_t)r[1] * (uint64_t)(nslot[k] - 1)) >> 32);
                if (s_new >= s_old) s_new++;
                int E0 = C->E;
                /* take the pair out, then put it at its new slot */
                if (--C->occ[s_old] == 0) C->E++;
                if (--C->occ[s_old + d[k]] == 0) C->E++;
                if (C->occ[s_new]++ == 0) C->E--;
                if (C->occ[s_new + d[k]]++ == 0) C->E--;
                int dE = C->E - E0;
                int accept = (dE <= 0) || ((uint64_t)r[2] < tmove[j * 3 + dE]);
                if (accept) {
                    C->slot[k] = s_new;
                    if (acc_move) acc_move[j]++;
                } else {                              /* undo */
                    if (--C->occ[s_new] == 0) C->E++;
                    if (--C->occ[s_new + d[k]] == 0) C->E++;
                    if (C->occ[s_old]++ == 0) C->E--;
                    if (C->occ[s_old + d[k]]++ == 0) C->E--;
                }
            }
            for (int j = (int)(t & 1); j + 1 < M; j += 2) {   /* exchanges */
                /* the fourth word of rung j's block of this iteration */
                uint32_t c[4] = {(uint32_t)t, (uint32_t)j, (uint32_t)l, 2u}, r[4];
                orc_philox4x32_10(c, key, r);
                int de = conf[j].E - conf[j + 1].E;
                int accept = (de <= 0) || ((uint64_t)r[3] < tswap[j * (bins + 1) + de]);
                if (accept) {
                    pt_conf tmp = conf[j];
                    conf[j] = conf[j + 1];
                    conf[j + 1] = tmp;
                    if (acc_swap) acc_swap[j]++;
                }
            }
        }
        if (final_slots)
            for (int j = 0; j < M; j++)
                for (int k = 1; k <= n; k++)
                    final_slots[((uint64_t)l * M + j) * n + (k - 1)] = (uint8_t)conf[j].slot[k];
    }
    free(tmove);
    free(tswap);
    free(conf);
    return 0;
}

int orc_pt_run(int variant, int n, int M, const double *beta, int L, uint64_t iters,
               uint64_t burnin, uint64_t seed, uint64_t *hist, uint64_t *acc_move,
               uint64_t *acc_swap, uint8_t *final_slots)
{
    return orc_pt_run_trips(variant, n, M, beta, L, iters, burnin, seed, hist, acc_move,
                            acc_swap, final_slots, NULL);
}

/* ------------------------------ O4: exact energy counts, tiny problems */

static void eh_rec(int k, int n, const int *d, const int *nslot, int bins, int *occ,
                   uint64_t *N)
{
    if (k > n) {
        int E = 0;
        for (int b = 0; b < bins; b++) E += (occ[b] == 0);
        N[E]++;
        return;
    }
    for (int s = 0; s < nslot[k]; s++) {
        occ[s]++;
        occ[s + d[k]]++;
        eh_rec(k + 1, n, d, nslot, bins, occ, N);
        occ[s]--;
        occ[s + d[k]]--;
    }
}

/* N[E] for E = 0..2n over every configuration of the simplified problem of
 * Sec. 3 (pair k at any start slot of the 2n bins, overlaps allowed). */
int orc_simplified_energy_hist(int variant, int n, uint64_t *N)
{
    if (variant < 0 || variant > 1 || n < 1 || n > 9) return -1;
    int span, present[ORC_MAXSPAN + 1], d[ORC_MAXN + 1];
    orc_layout(variant, n, &span, present, d);
    int bins = 2 * n, nslot[ORC_MAXN + 1], occ[ORC_MAXSPAN] = {0};
    for (int k = 1; k <= n; k++) {
        nslot[k] = bins - d[k];
        if (nslot[k] < 1) return -1;
    }
    memset(N, 0, sizeof(uint64_t) * (size_t)(bins + 1));
    eh_rec(1, n, d, nslot, bins, occ, N);
    return 0;
}
