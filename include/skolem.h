/*
 * skolem.h -- C ABI of libskolem.so, a GB300 (sm_103a) library that counts
 * Skolem, Langford and hooked Skolem pairings exactly, after "Counting Skolem
 * Sequences" (Assarpour, Bar-Noy, Liu), Sec. 2, and approximately by
 * parallel tempering, Sec. 3.
 *
 * Problems (variant):
 *   SK_SKOLEM   -- Sec. 1.1: split {1..2n} into n pairs (a_k, b_k) with
 *                  b_k - a_k = k.
 *   SK_LANGFORD -- Sec. 1.1: arrange 1,1,2,2,..,n,n so the two copies of k have
 *                  k numbers between them (positions k+1 apart).
 *   SK_HOOKED   -- Sec. 1.2: split {1..2n-1, 2n+1} into n pairs with
 *                  differences 1..n.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status (SK_OK = 0 or a negative SK_E*
 *     code) and writes its out-parameters only on SK_OK.
 *   - The caller owns every pointer it passes; the library never returns
 *     memory it allocated.  Pointers documented as "host" are host memory;
 *     pointers documented as "device" are device memory of the current CUDA
 *     device (for example torch tensors' data pointers).
 *   - `stream` fields are cudaStream_t values passed as void*; NULL selects a
 *     stream private to the library.  Calls are synchronous with respect to
 *     the host unless stated otherwise.
 *   - Zero is a valid count: n outside the existence classes returns 0 with
 *     SK_OK (Sec. 1.1: Skolem pairings exist iff n = 0,1 mod 4, Langford iff
 *     n = 0,3 mod 4).
 *   - The library needs a CUDA device of compute capability 10.3; without one
 *     every computing call returns SK_ECUDA.  There is no CPU fallback.
 */
#ifndef SKOLEM_H
#define SKOLEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SK_SKOLEM = 0, SK_LANGFORD = 1, SK_HOOKED = 2 };

enum {
  SK_OK = 0,
  SK_EINVAL = -1,     /* bad argument: variant, n, pointer, option */
  SK_ERANGE = -2,     /* the moduli cannot represent the value */
  SK_ECUDA = -3,      /* CUDA error or no usable device */
  SK_ENOMEM = -4,     /* device or host allocation failed */
  SK_ETIMEOUT = -5,   /* a bounded device loop gave up (error word set) */
  SK_EMISMATCH = -6,  /* a consistency check failed (check prime, 2^{2n-1}
                         divisibility, sign, parity of the count) */
  SK_ECKPT = -7       /* checkpoint file unreadable, corrupt or for another job */
};

/* Output conventions of the exact count.  Sec. 1.3: OEIS A059106 / A014552
 * (Tables 4, 5, 7, 8 of the paper) identify a sequence with its reflection;
 * A004075 / A176127 count both.  Lemma 2.1 yields the latter. */
enum { SK_COUNT_REFLECTIONS_IDENTIFIED = 0, SK_COUNT_ALL = 1 };

/* Largest n with a compiled exact kernel.  The position set of every variant
 * fits one 64-bit mask up to n = 31 (hooked Skolem spans 2n+1 = 63
 * positions), and the three 62-bit moduli (M ~ 2^186) hold the signed sum
 * C 2^{2n-1} with room to spare (|H| < 2^146 at n = 31).  Counting the
 * 2^{2n-1} terms of n >= 26 takes GPU-days; the work-item calls below reach
 * every order. */
#define SK_MAX_N 31

/* Arithmetic form of the term products (both give identical residues).
 * SK_ARITH_LIMBS: every term's product is formed exactly, as signed
 * radix-2^31 digits (|prod c_k| <= prod_k L_k, L_k = number of pairs at
 * distance d_k), and added into exact 64-bit words per digit; each work
 * item's sum is reduced modulo the primes once.  SK_ARITH_MONTGOMERY: every term's product is formed modulo
 * each prime by signed Montgomery steps (R = 2^32); compiled for three
 * moduli only (nprimes = 3). */
enum { SK_ARITH_LIMBS = 0, SK_ARITH_MONTGOMERY = 1 };

/* Symmetries used by the exact count.
 * SK_SYMMETRY_NEGATION (default): Lemma 2.2 only -- the summand is unchanged
 * when every x negates, so x_{max P} = +1 and 2^{2n-1} terms are summed.
 * SK_SYMMETRY_NEGATION_EVEN: Lemmas 2.2 and 2.4 -- negating the x at the even
 * positions multiplies the summand by s = (-1)^{e + o}, e = number of even
 * positions in P, o = number of odd distances d_k (s = +1 exactly for Skolem
 * n = 0,1, Langford n = 0,3 and hooked Skolem n = 2,3 (mod 4), the classes
 * in which pairings exist).  s = -1: the sum is 0 and no term is evaluated.
 * s = +1: one more variable is fixed to +1 (x_{2n-1} for Skolem and
 * Langford, through the negation of the odd positions; x_{2n-2} for hooked
 * Skolem, whose fixed position 2n+1 is odd) and 2^{2n-2} terms are summed;
 * the result (residues, coefficient) is the same.  Needs n >= 4; smaller
 * orders use SK_SYMMETRY_NEGATION (the report says which was used). */
/* SK_SYMMETRY_REVERSAL (Skolem and Langford; hooked Skolem: SK_EINVAL):
 * Lemmas 2.2 and 2.3 -- the summand is unchanged under reversal
 * i -> 2n+1-i, so of two assignments that are mirror images (with x_{2n}
 * kept at +1: reversed if x_1 = +1, reversed and negated if x_1 = -1) one is
 * summed twice and the other skipped; palindromic ones are summed once.  The
 * walk runs over positions 2..h+1 and their mirror images; a work item fixes
 * x_1 and the middle positions, and of each pair of mirror-image items one
 * is evaluated with weight 2 (decided by the first 8 mirror pairs of the
 * middle, from the outside in).  About (1/2 + 2^-9) of the 2^{2n-1} terms
 * are evaluated; walk_bits (if given) must be even, at least twice the
 * unrolled inner width and at most 2n-2.  The result is the same.  Needs
 * n >= 6; smaller orders use SK_SYMMETRY_NEGATION (the report says which
 * was used).  Exact-digit form only (arith = SK_ARITH_LIMBS).
 * SK_SYMMETRY_REVERSAL_EVEN (Skolem and Langford): Lemmas 2.2, 2.3 and 2.4
 * together.  Outside the existence classes the sum is 0 (Lemma 2.4's sign).
 * Inside them, negating the odd positions keeps the summand, flips x_1 and
 * keeps x_{2n}; it maps the mirrored walk's positions onto themselves and so
 * carries every work item with x_1 = +1 onto one with x_1 = -1 of equal sum:
 * only the x_1 = +1 items are evaluated and the sum is doubled, about a
 * quarter of the 2^{2n-1} terms.  Same walk-width rules as
 * SK_SYMMETRY_REVERSAL; n < 6 falls back to SK_SYMMETRY_NEGATION_EVEN (n >=
 * 4) or SK_SYMMETRY_NEGATION. */
enum {
  SK_SYMMETRY_NEGATION = 0,
  SK_SYMMETRY_NEGATION_EVEN = 1,
  SK_SYMMETRY_REVERSAL = 2,
  SK_SYMMETRY_REVERSAL_EVEN = 3
};
#define SK_MAX_PRIMES 4

typedef struct { uint64_t lo, hi; } sk_u128;   /* unsigned 128-bit integer */

/* Options of the exact count; zero-initialise and set what you need. */
typedef struct sk_count_opts {
  int nprimes;                 /* 0 -> 3.  3: CRT over 3 moduli.  4: the 4th
                                  modulus checks the CRT result. */
  uint64_t primes[SK_MAX_PRIMES]; /* 0 -> built-in 62-bit primes.  Each must be
                                  odd, in (2^62 - 2^31, 2^62) (the kernel's
                                  Montgomery step uses a high limb of 2^30),
                                  pairwise coprime. */
  int convention;              /* SK_COUNT_REFLECTIONS_IDENTIFIED (default) or
                                  SK_COUNT_ALL */
  int walk_bits;               /* m: Gray-walk bits per work item; 0 -> planner */
  int block_threads;           /* 32..256, multiple of 32; 0 -> 256 */
  int grid;                    /* CTAs; 0 -> SMs x resident CTAs per SM */
  void *stream;                /* cudaStream_t or NULL */
  const char *checkpoint_path; /* NULL: no checkpoint.  Else completed chunks
                                  are appended to this file and skipped when
                                  the same job is run again. */
  uint64_t chunk_items;        /* work items per launch; 0 -> all in one launch
                                  (or ~10 s of work when checkpointing) */
  uint64_t max_chunks;         /* stop (status SK_OK, report->complete = 0)
                                  after this many new chunks; 0 = no limit */
  int arith;                   /* SK_ARITH_LIMBS (default) or SK_ARITH_MONTGOMERY */
  int symmetry;                /* SK_SYMMETRY_NEGATION (default) or
                                  SK_SYMMETRY_NEGATION_EVEN */
} sk_count_opts;

typedef struct sk_count_report {
  int nprimes;
  uint64_t primes[SK_MAX_PRIMES];
  uint64_t residues[SK_MAX_PRIMES]; /* H mod p_i, H = sum of Lemma 2.1 over the
                                       2^{2n-1} assignments with x_{max P} = +1 */
  sk_u128 coefficient;         /* pairings with reflections distinct */
  uint64_t terms;              /* terms evaluated: 2^{2n-1} (Lemma 2.2),
                                  2^{2n-2} (Lemma 2.4, s = +1) or 0 (s = -1) */
  uint64_t items;              /* work items (terms / 2^m) */
  int walk_bits;               /* m */
  int inner_bits;              /* unrolled Gray bits */
  int arith;                   /* arithmetic form used */
  int block_threads, grid;
  uint64_t chunks_total, chunks_done, chunks_resumed;
  int complete;                /* 1 when every chunk is done */
  double kernel_ms;            /* device time of the launches of this call */
  double wall_ms;              /* host time of the whole call */
  int symmetry;                /* SK_SYMMETRY_* actually used */
} sk_count_report;

/* The plan skolem_count_ex would run for these options, without running it
 * (host code only, no device): rep receives the moduli, walk and inner bits,
 * arithmetic form, block size and grid (0: one wave), symmetry used, work
 * items, terms and chunks_total (the launches of a checkpointed run); the
 * fields that depend on the sums stay 0.  A zero class of Lemma 2.4 reports 0
 * items and terms and complete = 1.  Same argument checks as
 * skolem_count_ex. */
int sk_count_plan(int variant, int n, const sk_count_opts *opts, sk_count_report *rep);

/* Exact count of `variant` of order n (Lemma 2.1 with Lemma 2.2, evaluated in
 * Gray-code order, Sec. 2.1; residues modulo co-primes and the Chinese
 * remainder theorem, Sec. 2.2).  out (host): the count in the default
 * convention (reflections identified for Skolem and Langford; the hooked
 * count as is).  1 <= n <= SK_MAX_N. */
int skolem_count(int variant, int n, sk_u128 *out);

/* As skolem_count with options and an optional report (host pointers; opts
 * and rep may be NULL).  With a checkpoint path the call may stop early
 * (opts->max_chunks) and resume later; out is written only when complete. */
int skolem_count_ex(int variant, int n, const sk_count_opts *opts, sk_u128 *out,
                    sk_count_report *rep);

/* ------------------------------------------------------------ batches */

typedef struct sk_job { int variant; int n; } sk_job;

/* SK_BATCH_PERSISTENT: every job in one persistent launch (captured in a CUDA
 * graph unless no_graph) pulling 32-item chunks from a device queue, largest
 * job first.  SK_BATCH_PER_JOB: one launch per job, back to back on the
 * stream (the baseline). */
enum { SK_BATCH_PERSISTENT = 0, SK_BATCH_PER_JOB = 1 };

typedef struct sk_batch_opts {
  int nprimes;                    /* 0 -> 3; as in sk_count_opts */
  uint64_t primes[SK_MAX_PRIMES]; /* 0 -> built-in */
  int convention;                 /* SK_COUNT_* for every job */
  int mode;                       /* SK_BATCH_PERSISTENT (default) or SK_BATCH_PER_JOB */
  int no_graph;                   /* persistent mode: 0 (default) captures the
                                     launch in a CUDA graph and replays it;
                                     1 launches it directly */
  int repeats;                    /* runs of the whole batch (>= 1; 0 -> 1); the
                                     report gives the last and the fastest */
  int autotune;                   /* 1: tune walk width (and block size) per
                                     (variant, n) before the run, untimed */
  int block_threads;              /* 0 -> 256 or the tuned value */
  int walk_bits[SK_MAX_N + 1];    /* per n; 0 -> tuned or planner default */
  void *stream;                   /* cudaStream_t or NULL */
} sk_batch_opts;

typedef struct sk_batch_report {
  double kernel_ms;               /* device time of the last repeat */
  double kernel_ms_min;           /* fastest repeat */
  double wall_ms;                 /* host time of the whole call */
  double prepare_ms;              /* planning, tuning, graph capture */
  uint64_t terms;                 /* sum over jobs of 2^{2n-1} */
  uint64_t chunks;                /* 32-item chunks of the queue */
  int launches;                   /* kernel launches per repeat */
  int grid, block_threads;
} sk_batch_report;

/* Exact counts of njobs jobs (host array; 1 <= njobs <= 4096; each job as in
 * skolem_count).  outs (host, njobs): the counts in opts->convention;
 * status (host, njobs, may be NULL): per-job SK status (a job whose CRT checks
 * fail gets SK_EMISMATCH; the call then returns SK_EMISMATCH too).  opts and
 * rep may be NULL.  The persistent mode is an engineering addition (the paper
 * runs one job per GPU launch, Sec. 2.2). */
int skolem_count_batch(const sk_job *jobs, int njobs, const sk_batch_opts *opts, sk_u128 *outs,
                       int *status, sk_batch_report *rep);

typedef struct sk_tune_result {
  int walk_bits;                  /* fastest m */
  int block_threads;              /* fastest block size */
  double terms_per_s;             /* its rate on the sample */
  int candidates;                 /* configurations timed */
} sk_tune_result;

/* Times candidate walk widths m (planner default and +-2, +-4, within the
 * valid range) and block sizes (128, 256) of the exact-limb kernel for one
 * (variant, n) on the first work items (2^33 terms at most) and returns the
 * fastest.  The result is also cached in the library and used by
 * skolem_count_batch when opts->autotune is set.  opts may be NULL (only
 * nprimes/primes/stream are read). */
int skolem_autotune(int variant, int n, const sk_batch_opts *opts, sk_tune_result *out);

/* ------------------------------------------------------ approximate count */

/* Move proposals of the tempering chains.  SK_PT_PLAIN: Sec. 3 -- pair k
 * uniform, its new start slot uniform among its other slots.  SK_PT_LEARNED:
 * the move (k, slot) drawn from the softmax of a trained network over the
 * bin occupancies, with the Metropolis-Hastings correction (not in the
 * paper). */
enum { SK_PT_PLAIN = 0, SK_PT_LEARNED = 1 };

#define SK_PT_MAX_RUNGS 64
#define SK_PT_MAX_RUNGS_LEARNED 32

typedef struct sk_pt_opts {
  int rungs;              /* M temperatures, 1..64 (the learned proposal: 2..32);
                             0 -> 32.  Up to 32 rungs a ladder is one warp, lane
                             j serving rung j; 33..64 rungs span two warps, whose
                             rungs 31 and 32 exchange through shared memory */
  int ladders;            /* independent ladders run side by side; 0 -> 4096 */
  uint64_t seed;          /* Philox key */
  double burnin_frac;     /* leading fraction of iterations not counted;
                             0 -> 0.1, negative -> none */
  const double *beta;     /* host, `rungs` non-decreasing inverse temperatures
                             starting at 0; NULL -> pilot-tuned ladder */
  double beta_max;        /* top of the tuned ladder; 0 -> 32 */
  int proposal;           /* SK_PT_PLAIN (default) or SK_PT_LEARNED */
  const void *model;      /* SK_PT_LEARNED: a model from sk_mlp_create */
  void *stream;           /* cudaStream_t or NULL */
  int round_trips;        /* nonzero: count round trips (SK_PT_PLAIN; a few
                             percent more kernel time) */
} sk_pt_opts;

typedef struct sk_pt_report {
  int rungs, ladders;
  uint64_t iterations, burnin;
  double beta[SK_PT_MAX_RUNGS];      /* ladder used */
  double ratio[SK_PT_MAX_RUNGS];     /* E[z_{j+1}/z_j] per rung (Table 6's
                                        last column) */
  double acc_move[SK_PT_MAX_RUNGS];  /* accepted moves per rung (W1) */
  double acc_swap[SK_PT_MAX_RUNGS];  /* accepted exchanges of (j, j+1) (W2) */
  double estimate;
  double kernel_ms, tune_ms, wall_ms;
  /* Relative standard error of `estimate` from the spread of the estimates
   * of min(16, ladders) equal groups of consecutive ladders (sample standard deviation of the group
   * estimates / their mean / sqrt(groups)); statistical only, it does not see a ladder
   * that has not equilibrated.  0 with fewer than 2 groups (ladders < 2) and
   * for the learned proposal; NaN when the group estimates average to 0. */
  double rel_stderr;
  /* With opts->round_trips: how often, over all ladders and after burn-in,
   * a configuration came back to rung 0 having reached rung M-1 since it was
   * last there (a trip from the hottest end of the ladder to the coldest and
   * back); 0 otherwise. */
  uint64_t round_trips;
} sk_pt_report;

/* Approximate count by parallel tempering (Sec. 3, Algorithm 2): budget =
 * iterations per ladder (each one move per rung plus one exchange phase),
 * 1 <= budget < 2^32.  out (host): 1/2 Z(0) prod_j Ratio(j), reflections
 * identified, with Z(0) = prod_k (2n - d_k).  Skolem and Langford,
 * 2 <= n <= 64 (the learned proposal: n <= 40).  Deterministic for a given
 * seed.  Above n = 40 a ladder's tables (16-bit energy histogram of 2n+1
 * rows, start slots, bin counts) need more shared memory than 28 warps per
 * SM can hold, so fewer ladders are resident at once and a run of 4096
 * ladders takes more than one wave. */
int pt_estimate(int variant, int n, uint64_t budget, double *out);
int pt_estimate_ex(int variant, int n, uint64_t budget, const sk_pt_opts *opts, double *out,
                   sk_pt_report *rep);

/* The raw tempering run behind pt_estimate, for checks against a reference:
 * L ladders of M rungs (1..64) with the given ladder beta (host, M values) for
 * `iters` iterations, statistics after `burnin`.  Host outputs: hist
 * (M x (2n+1), counts of the energy E at each rung), acc_move / acc_swap
 * (M, may be NULL), final_slots (L x M x n start bins of pair k = 1..n at
 * each rung at the end, may be NULL). */
int sk_pt_run(int variant, int n, int M, const double *beta, int L, uint64_t iters,
              uint64_t burnin, uint64_t seed, uint64_t *hist, uint64_t *acc_move,
              uint64_t *acc_swap, uint8_t *final_slots);

/* sk_pt_run that also counts round trips along the ladder: round_trips
 * (host, one value, required) = how often, over all ladders, a configuration
 * came back to rung 0 having reached rung M-1 since it was last at rung 0.
 * Each iteration first looks at the configurations at the two ends (at rung
 * 0: count a return if it had reached rung M-1, then mark it as at rung 0;
 * at rung M-1: mark it if it came from rung 0); returns are counted from
 * iteration `burnin` on.  The other outputs are those of sk_pt_run, bit for
 * bit. */
int sk_pt_run_trips(int variant, int n, int M, const double *beta, int L, uint64_t iters,
                    uint64_t burnin, uint64_t seed, uint64_t *hist, uint64_t *acc_move,
                    uint64_t *acc_swap, uint8_t *final_slots, uint64_t *round_trips);

/* The estimator of pt_estimate on host histograms; host code only, no device
 * needed.  hist: `groups` >= 1 histograms of M x (2n+1) energy counts (groups x
 * M x (2n+1), host), e.g. sk_pt_run's over separate sets of ladders.  out:
 * 1/2 Z(0) prod_j Ratio(j) of their sum (as pt_estimate); ratios (M, may be
 * NULL): the Ratio(j) of the sum; rel_stderr (may be NULL): with groups >= 2
 * the relative standard error of out from the spread of the group estimates
 * (as sk_pt_report.rel_stderr), else 0.  Same variant / n / ladder checks as
 * pt_estimate (SK_EINVAL). */
int sk_pt_estimate_hist(int variant, int n, int M, const double *beta, int groups,
                        const uint64_t *hist, double *out, double *ratios, double *rel_stderr);

/* The pilot-tuned ladder pt_estimate uses when opts->beta is NULL. */
int sk_pt_tune_ladder(int variant, int n, int rungs, double beta_max, uint64_t seed,
                      double *beta);

/* ---------------------------------------------- learned move proposal */

/* The move-proposal network of SK_PT_LEARNED (not in the paper): the 2n bin
 * occupancies -> 256 ReLU -> 256 ReLU -> one logit per move (k, s), moves
 * ordered by pair k then start slot s = 0..2n-d_k-1.  BF16 weights with FP32
 * accumulation on the tensor cores, FP32 master weights, trained with Adam on
 * the cross entropy against t(m) ~ exp(-beta* dE(m)) over the valid moves of
 * each state (every move except a pair's current slot).
 * Parameter layout on the host (float, row-major): W1 [2n][256], b1 [256],
 * W2 [256][256], b2 [256], W3 [256][n_moves], b3 [n_moves]. */

/* Creates a model for (variant, n) (Skolem or Langford, 2 <= n <= 40) with
 * workspace for max_batch states (a multiple of 128), He-normal weights from
 * `seed`.  *model receives an opaque handle owned by the caller; release it
 * with sk_mlp_destroy. */
int sk_mlp_create(int variant, int n, int max_batch, uint64_t seed, void **model);
void sk_mlp_destroy(void *model);
/* Number of moves (logits) and of host parameters. */
int sk_mlp_dims(const void *model, int *n_moves, int *n_params);
int sk_mlp_set_params(void *model, const float *params);   /* host, n_params */
int sk_mlp_get_params(const void *model, float *params);   /* host, n_params */
/* Logits of B <= max_batch states.  slots (host, B x n): start slot of pair
 * k = 1..n of each state; logits (host, B x n_moves). */
int sk_mlp_forward(void *model, const uint8_t *slots, int B, float *logits);
/* The same logits as the tempering chains read them: rounded to bf16
 * (nearest even; the bit patterns, host, B x n_moves), from the forward that
 * stores only the move table's columns.  Same arguments and errors as
 * sk_mlp_forward. */
int sk_mlp_forward_bf16(void *model, const uint8_t *slots, int B, uint16_t *logits);
/* Mean loss of a batch (B a multiple of 128) and its gradient (host,
 * n_params, same layout as the parameters); the model is not updated. */
int sk_mlp_loss_grad(void *model, const uint8_t *slots, int B, float beta_star, float *loss,
                     float *grads);
/* Adam (Kingma & Ba 2015: lr, betas 0.9 / 0.999, eps 1e-8, bias-corrected
 * moments) on `count` states (host, count x n), `epochs` passes in
 * minibatches of `batch` (multiple of 128) in an order shuffled by `seed`,
 * or in the given order when seed == SK_MLP_KEEP_ORDER.  Each minibatch is
 * one step: forward, loss and gradients (as sk_mlp_loss_grad), the update of
 * the FP32 masters and moments, and the refresh of the BF16 weight copies.
 * final_loss: mean loss of the last epoch; ms: device time (both may be
 * NULL). */
#define SK_MLP_KEEP_ORDER UINT64_MAX
int sk_mlp_train(void *model, const uint8_t *states, uint64_t count, int epochs, int batch,
                 float lr, float beta_star, uint64_t seed, float *final_loss, double *ms);
/* Training state of a model, each array (host, n_params floats, the
 * parameter layout; any may be NULL): Adam's first and second moments, and
 * the parameters the forward pass uses -- the BF16 copies of W1, W2, W3
 * widened to float, and the FP32 biases.  *t (may be NULL): Adam steps taken
 * since sk_mlp_create or the last sk_mlp_set_params (which zeroes the
 * moments). */
int sk_mlp_get_train_state(const void *model, float *adam_m, float *adam_v, float *used,
                           int64_t *t);
/* Selects the GEMM path of a model's forward and backward: 1 (default) the
 * 5th-generation tensor cores (tcgen05, accumulators in tensor memory; the
 * backward's weight gradients summed over a K split in a fixed order, so a
 * gradient is the same bits every call), 0 warp-level mma.sync.
 * sk_mlp_check returns SK_ETIMEOUT if a tensor-core wait of the model ever
 * gave up (the results of that call are then invalid). */
int sk_mlp_set_gemm(void *model, int use_tensor_memory_path);
int sk_mlp_check(void *model);
/* The learned tempering run behind pt_estimate_ex with SK_PT_LEARNED, with
 * the outputs of sk_pt_run (no final states).  Needs a model of the same
 * (variant, n) whose max_batch >= L * M rounded up to 128.  The exchanges of
 * each iteration run on a second stream the call creates, joined to the
 * run's stream by events; the call returns after both have finished. */
int sk_pt_run_learned(int variant, int n, int M, const double *beta, int L, uint64_t iters,
                      uint64_t burnin, uint64_t seed, const void *model, uint64_t *hist,
                      uint64_t *acc_move, uint64_t *acc_swap);

/* Residues of single work items, for sampled checks at full size.  Item q of
 * walk width m fixes the free variables m..2n-2 (bit b of q set means
 * x_{m+b+1} = -1) and runs the low m through all values; its sum is
 * sum sign(X) F(n, X) over that block (Lemma 2.1's summand).  For items
 * q_lo .. q_lo+count-1, out (host, count x nprimes, row-major) receives each
 * block sum modulo each prime.  primes (host): nprimes in {3, 4} moduli as in
 * sk_count_opts.  count <= 2^20. */
int skolem_item_residues(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                         int nprimes, const uint64_t *primes, uint64_t *out);

/* The host step after the sum, for a sum computed in parts -- disjoint
 * ranges of work items on different GPUs, each part's item residues added
 * modulo each prime -- with no device: residues (host, parts x nprimes,
 * row-major, each in [0, p_i)) are added modulo each prime into the residues
 * of the whole sum over the 2^{2n-1} assignments of Lemma 2.2 (the parts must
 * cover every work item once), then rebuilt by the CRT with skolem_count_ex's
 * checks (lower half of the CRT range, divisibility by 2^{2n-1}, agreement
 * with a fourth prime) and put in `convention` (SK_COUNT_*).  primes: NULL
 * for the defaults, else nprimes moduli as in sk_count_opts.  SK_EMISMATCH
 * when a check fails, e.g. a residue that is wrong modulo one prime but not
 * the others; a part left out or added twice is in general NOT caught (work
 * item sums are themselves multiples of 2^{2n-1}), so covering every item
 * exactly once is the caller's part.  SK_EINVAL for bad arguments. */
int sk_count_from_residues(int variant, int n, int convention, int nprimes,
                           const uint64_t *primes, uint64_t parts, const uint64_t *residues,
                           sk_u128 *out);

/* ------------------------------------------- extended Skolem sequences */

/* The exact count of extended Skolem sequences (Sec. 1.2 names them, after
 * Abrham and Kotzig): the numbers 1..n in pairs at distance k over the
 * positions 1..2n+1 with one position -- `hole`, 1 <= hole <= 2n+1 -- left
 * empty.  hole = 2n is the hooked problem, hole = n+1 Rosa's (the skip in
 * the middle), holes 1 and 2n+1 the Skolem problem.  Lemma 2.1 on that
 * position set, the half-sum of Lemma 2.2, residues and CRT as in
 * skolem_count_ex (same options and report; symmetry must be
 * SK_SYMMETRY_NEGATION).  Reversal maps the sequences of hole h onto those
 * of hole 2n+2-h: a hole below n+1 is counted on its mirror image, and
 * reflections are identified (SK_COUNT_REFLECTIONS_IDENTIFIED) only for
 * holes 1, n+1 and 2n+1, whose position sets it maps onto themselves; any
 * other hole returns the count as it is.  The hole is held out of the walk:
 * a hole inside the unrolled inner block (n <= 4, holes near the middle)
 * returns SK_EINVAL, as does a walk_bits above the (mirrored) hole's bit. */
int sk_count_extended(int n, int hole, const sk_count_opts *opts, sk_u128 *out,
                      sk_count_report *rep);

/* Residues of single work items of that count for holes n+1..2n+1: the free
 * variables are the positions of P below max P in increasing order; item q
 * of walk width m fixes those beyond the first m (bit b of q -> variable
 * m+b) and runs the first m.  Otherwise as skolem_item_residues. */
int sk_extended_item_residues(int n, int hole, int m, uint64_t q_lo, uint64_t count, int nprimes,
                              const uint64_t *primes, uint64_t *out);

/* ------------------------------------------ inclusion-exclusion count */

/* Largest n with a compiled inclusion-exclusion kernel. */
#define SK_MAX_IE_N 24

/* The count by inclusion-exclusion over avoided positions -- the third
 * counting approach of Sec. 2 (after Larsen) -- as an exact cross-check of
 * skolem_count_ex that shares none of Lemma 2.1's arithmetic: with N_k(T)
 * the number of pairs (a, a+d_k) inside T, the sequences (reflections
 * distinct) number sum over T subset of P of (-1)^{|P|-|T|} prod_k N_k(T),
 * 2^{2n} terms (no symmetry halves them), summed on the GPU as residues
 * modulo the primes and rebuilt by the CRT (the result must lie in the lower
 * half of the CRT range and agree with a fourth prime when one is given).
 * Same arguments, output conventions and report as skolem_count_ex; opts
 * (may be NULL) must keep arith = SK_ARITH_LIMBS and symmetry =
 * SK_SYMMETRY_NEGATION (others: SK_EINVAL); checkpoints work as there (the
 * method is part of the file's header).  1 <= n <= SK_MAX_IE_N. */
int sk_count_inclusion_exclusion(int variant, int n, const sk_count_opts *opts, sk_u128 *out,
                                 sk_count_report *rep);

/* Residues of single work items of the inclusion-exclusion sum.  The 2n
 * variables are the positions of P in increasing order (variable i is in T
 * iff bit i of the set is 1); item q of walk width m fixes variables m..2n-1
 * (bit b of q -> variable m+b) and runs variables 0..m-1 through all values;
 * out (host, count x nprimes, row-major) receives each block sum modulo each
 * prime.  q_lo + count <= 2^{2n-m}, count <= 2^20; primes as in
 * skolem_item_residues. */
int sk_ie_item_residues(int variant, int n, int m, uint64_t q_lo, uint64_t count, int nprimes,
                        const uint64_t *primes, uint64_t *out);

/* skolem_item_residues with a choice of arithmetic form (SK_ARITH_*). */
int skolem_item_residues_ex(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                            int nprimes, const uint64_t *primes, int arith, uint64_t *out);

/* Largest `count` accepted by skolem_item_residues_noalloc: its static device
 * scratch holds this many work items x SK_MAX_PRIMES residues (512 KiB) plus
 * one 256-byte launch record. */
#define SK_NOALLOC_MAX_ITEMS 16384

/* skolem_item_residues for callers that cannot let the library allocate
 * device memory (a framework whose caching allocator owns the device budget,
 * or a host loop that cannot absorb the device-wide synchronisation of
 * cudaFree).  The paper has no counterpart; this is an engineering variant.
 * Same arguments and results as skolem_item_residues, plus `stream`
 * (cudaStream_t or NULL for the legacy default stream; the call synchronises
 * it).  It calls no cudaMalloc / cudaFree and creates no stream or event: its
 * device scratch is one static array of fixed size in the library, held by
 * every GPU that loads the library until exit.  The first call on a device
 * looks up that array's device address (make it before any stream capture).
 * Every call shares the array: calls that overlap on the GPU race.  count >
 * SK_NOALLOC_MAX_ITEMS returns SK_EINVAL. */
int skolem_item_residues_noalloc(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                                 int nprimes, const uint64_t *primes, void *stream,
                                 uint64_t *out);

/* INT32 throughput of the current device, the denominator of the exact
 * kernel's roofline (that path is integer-ALU bound).  mode 0: independent
 * 32-bit multiply-adds; mode 1: multiply-adds interleaved with three-input
 * logic ops.  ops_per_s (host): 32-bit operations per second; ms (host, may
 * be NULL): duration of the timed launch. */
int sk_int32_peak(int mode, double *ops_per_s, double *ms);

/* The built-in moduli (host, 4 entries): the four largest primes below 2^62. */
void sk_default_primes(uint64_t *out4);

/* Text for a status code (static storage). */
const char *sk_strerror(int status);

/* Library version (major * 10000 + minor * 100 + patch). */
int sk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SKOLEM_H */
