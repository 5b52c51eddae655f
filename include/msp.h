/*
 * msp.h -- C ABI of the GB300 (sm_103a) market-split lattice solver.
 *
 * Problem (Sec. 1, feasibility form fMSP): given A in Z^{m x n} and d in Z^m,
 * list the x in {0,1}^n with A x = d.  Method (Sec. 2, Algorithm 1): embed
 * the instance in the lattice of Eq. (2), LLL-reduce it, keep the n-m+1
 * reduced vectors whose first m entries vanish (a basis of ker[A | -d]),
 * Gram-Schmidt them (Eq. (4)), and enumerate exhaustively with the norm bound
 * (first pruning condition) and the Hoelder bound of Theorem 2, checking
 * every leaf exactly against Theorem 1.
 *
 * Every computational step runs in CUDA kernels on the device; the host side
 * of this library only validates arguments, sizes buffers and launches.
 *
 * Conventions for all entry points
 *   - A context owns every device buffer it allocates and releases them in
 *     msp_destroy().  Inputs are copied: the caller keeps its buffers.
 *   - All device work is queued on the stream given to msp_create() (NULL =
 *     the legacy default stream).  Functions that return results to host
 *     memory synchronise that stream before returning.
 *   - Functions never abort the process.  They return an msp_status; per
 *     instance failures are reported in msp_stats.status and make the batch
 *     call return the first nonzero per-instance status.
 *   - Calling a function before the one it depends on returns MSP_ESTATE.
 *   - Sizes: 1 <= m <= 32, 1 <= n <= 127 (so n + 1 <= 128 lattice
 *     coordinates after extraction), m <= n, |a_ij| < 2^31, |d_i| < 2^40.
 */
#ifndef MSP_H
#define MSP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSP_API __attribute__((visibility("default")))
#else
#define MSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSP_OK = 0,
    MSP_EINVAL = 1,      /* bad argument (size, pointer, option)                 */
    MSP_ENOMEM = 2,      /* device or host allocation failed                     */
    MSP_ECUDA = 3,       /* a CUDA runtime call failed (see msp_last_error)      */
    MSP_EOVERFLOW = 4,   /* an integer left its exact range (basis, N d, u)     */
    MSP_ERANK = 5,       /* kept vectors do not span ker[A|-d]: N too small      */
    MSP_ETIMEOUT = 6,    /* time cap reached; results are partial                */
    MSP_ETRUNC = 7,      /* solution buffer too small; counts stay exact         */
    MSP_ESTATE = 8,      /* call order violated                                  */
    MSP_ECAP = 9,        /* LLL iteration cap, or opts.lds_max, reached          */
    MSP_EQUEUE = 10      /* work queue capacity exceeded                         */
} msp_status;

typedef enum { MSP_ALL = 0, MSP_FIRST = 1 } msp_mode;      /* all solutions / stop at one  */
/* Order of the search.  PLAIN: depth-first (Algorithm 1) over the subtrees
 * in depth-first order.  LEARNED: the subtrees ranked by the scorer
 * (msp_set_scorer); the walk inside a subtree stays depth-first.  LDS:
 * limited discrepancy search (Sec. 3): iterations k = 0, 1, 2, ... each walk
 * Algorithm 1 but try a value only while the discrepancy cost of the path
 * (the sum over its levels of the value's cost, opts.lds_rank; the first
 * value of a level, the rounded centre, costs 0) stays at most k, and report
 * the leaves whose path costs exactly k; MSP_FIRST stops an instance at its
 * first solution, MSP_ALL when an iteration held no value back (every
 * solution is then reported exactly once).  LDS_LEARNED: limited
 * discrepancy search whose iterations take their subtrees in the scorer's
 * order (as LEARNED does; the same nodes and solutions as LDS, possibly
 * sooner). */
typedef enum { MSP_PLAIN = 0, MSP_LEARNED = 1, MSP_LDS = 2, MSP_LDS_LEARNED = 3 } msp_order;
typedef enum { MSP_HOST = 0, MSP_DEVICE = 1 } msp_memory;  /* where A and d live           */

/* Options.  msp_default_opts() fills the defaults given in brackets. */
typedef struct {
    int64_t N;             /* [1024] scale of the A-rows of Eq. (2) (Sec. 2: 2^10)      */
    double delta;          /* [0.99] LLL Lovasz parameter                                */
    double eta;            /* [0.51] LLL size-reduction bound on |mu|                    */
    int64_t lll_max_iter;  /* [2e6] LLL iteration cap (MSP_ECAP when reached)            */
    int hoelder;           /* [0] 0: Hoelder test with the one-direction cut of Sec. 2;   */
                           /*     1: Hoelder test skips only the failing value; 2: off    */
    int sym;               /* [1] 1: enumerate one of v, -v (first nonzero u > 0);        */
                           /*     0: both signs, keep leaves whose last entry is +1       */
    int use_eps;           /* [1] slack eps = (n+1) 2^-20 on both tests (0: none)         */
    int lanes;             /* [0] lanes per subtree walker: 4, 8, 16 or 32; 0 picks 8 when */
                           /*     the widest instance of the batch has n + 1 <= 64, else  */
                           /*     16 (msp_lanes tells the choice).  Also fixes the        */
                           /*     summation order of ||w||_1 (G interleaved partial sums  */
                           /*     combined pairwise), so node counts depend on it         */
    int split_depth;       /* [24] maximum number of top levels the splitter expands      */
    int split_target;      /* [0] stop splitting once an instance has this many subtree   */
                           /*     prefixes (0: 8 x the number of walkers / instances)     */
    int split_capacity;    /* [0] prefixes stored per instance (0: 4 x split_target)      */
    int warps_per_block;   /* [8] enumerator block size in warps, 1 to 8                  */
    int blocks_per_sm;     /* [0] enumerator blocks per SM (0: as many as can be resident; */
                           /*     larger values are capped at that)                     */
    int64_t sol_capacity;  /* [1<<20] solutions stored (over all instances)               */
    double max_seconds;    /* [600] safety cap on every enumeration's device time; the     */
                           /*       walkers stop and report MSP_ETIMEOUT when it passes   */
    int64_t donation_capacity; /* [1<<16] slots of the ring through which busy walkers */
                           /*       hand sibling ranges to idle ones (0: no donation)      */
    int log_features;      /* [0] 1: compute the 32 features of every subtree prefix      */
                           /*     (msp_export_features), e.g. to train the scorer         */
    int lds_budget;        /* [-1] MSP_LDS: >= 0 runs only the iteration with this budget */
                           /*      (at most 255)                                          */
    int lds_max;           /* [127] MSP_LDS: last budget tried (at most 255); an instance */
                           /*       not finished by then reports MSP_ECAP.  With          */
                           /*       lds_rank = 0 the budget 127 always exhausts a tree    */
                           /*       (its paths have at most 127 levels)                   */
    int first_split_target; /* [16384] split target of MSP_FIRST when split_target = 0: */
                           /*       small subtrees let a good queue order pay off        */
    int bkz_beta;          /* [0] >= 2: BKZ-beta of the kernel basis after LLL (Sec. 2   */
                           /*     names LLL or BKZ for step 1); 0: LLL only              */
    int bkz_max_tours;     /* [16] BKZ tours at most (a tour without insertion ends it) */
    int replicas;          /* [1] searches per instance, each on its own random order of */
                           /*     the variables (Sec. 4: shuffled input bases); in       */
                           /*     MSP_FIRST the first replica to find a solution stops  */
                           /*     the others.  Statistics and solutions are per caller's */
                           /*     instance; the export calls index the internal         */
                           /*     instances (instance i, replica k: i * replicas + k).   */
                           /*     At most 64.                                            */
    uint64_t replica_seed; /* [0x5EED5EED5EED5EED] replica k > 0 of instance i shuffles   */
                           /*     its columns by Fisher-Yates (j = n-1 .. 1, swap j with */
                           /*     z mod (j+1)) fed by splitmix64 from                    */
                           /*     replica_seed ^ (i << 32) ^ k; replica 0 is unshuffled  */
    int lds_rank;          /* [1] MSP_LDS: discrepancy cost of a value -- 1: its position */
                           /*     p in its level's walk (p = 0 for the rounded centre),  */
                           /*     0: one for every value after the first (Sec. 3 calls  */
                           /*     a discrepancy a deviation from the heuristic order)    */
    int fuse;              /* [0] 1: msp_run_async / msp_graph_capture of an all-        */
                           /*     solutions, depth-first, binary step reduce, split and   */
                           /*     enumerate in one cooperative launch -- the blocks       */
                           /*     prepare the instances (LLL, tables, split) and walkers  */
                           /*     start on each instance as soon as it is published, so  */
                           /*     the slowest reductions overlap the enumeration of the  */
                           /*     others.  Same nodes and solutions as 0 (separate        */
                           /*     launches); msp_phase_ms then reports the reduction and  */
                           /*     split as 0 and the whole launch as the enumeration.     */
                           /*     Off by default: on GB300 the fused walker is slower    */
                           /*     than the overlap gains (605 against 522 ms per step of */
                           /*     the 64-instance batch)                                  */
} msp_opts;

/* Per-instance results of an enumeration. */
typedef struct {
    int64_t nodes;         /* evaluated nodes: one per candidate (t, u_t) whose norm   */
                           /* ||w^(t)||^2 was computed (split part + subtrees)          */
    int64_t passed;        /* nodes that passed the norm test                          */
    int64_t leaves;        /* passed nodes at level 0 (exact Theorem 1 check)          */
    int64_t solutions;     /* x with A x = d found (exact count even if truncated)     */
    int64_t prefixes;      /* subtrees created by the splitter                         */
    int32_t split_level;   /* lowest level fixed by the splitter                       */
    int32_t kernel_rank;   /* number of kept vectors d = n - rank + 1                   */
    int64_t lll_iterations;
    int64_t lll_swaps;
    int64_t split_nodes;   /* part of `nodes` evaluated by the splitter               */
    int64_t split_passed;  /* part of `passed` evaluated by the splitter              */
    int64_t center_fma;    /* fmas spent by the walkers on the centres y_t            */
    int64_t fallbacks;     /* Hoelder tests too close to call from the exact integer  */
                           /* filter, decided by rebuilding the FP64 vector           */
    int64_t donations;     /* batch total only: sibling ranges handed between walkers */
    double walker_util;    /* batch total only: fraction of walker time spent walking */
    double first_ms;       /* MSP_FIRST: device time from the start of the enumeration */
                           /* to this instance's first verified solution (-1: none)   */
    int32_t status;        /* msp_status of this instance                              */
    int32_t lds_budget;    /* MSP_LDS: budget of the iteration that solved (MSP_FIRST) or */
                           /* finished (MSP_ALL) this instance; -1 otherwise            */
    double ms;             /* wall time of the enumeration call (whole batch)          */
    int64_t bkz_tours;     /* BKZ tours run (0 without BKZ)                            */
    int64_t bkz_inserts;   /* block shortest vectors inserted                         */
    int64_t bkz_nodes;     /* enumeration nodes of the block searches                 */
} msp_stats;

typedef struct msp_ctx msp_ctx;

/* Fill *opts with the defaults listed above. */
MSP_API void msp_default_opts(msp_opts *opts);

/* Create a context on the current CUDA device.  opts may be NULL (defaults);
 * stream is a cudaStream_t (NULL: default stream).  *out receives the
 * context or NULL on failure. */
MSP_API msp_status msp_create(msp_ctx **out, const msp_opts *opts, void *stream);

/* Release every device buffer of the context and the context itself.
 * Synchronises the context's stream first.  NULL is ignored. */
MSP_API void msp_destroy(msp_ctx *ctx);

/* Step a1 -- lattice of Eq. (2) (Sec. 2), binary bounds (r_max = c_j = 1),
 * for a batch of `count` instances.
 *   dims  host int32[count][2] = (m_i, n_i)
 *   A     int32, the A_i row-major (m_i x n_i) back to back
 *   d     int64, the d_i back to back
 *   mem   MSP_HOST: A, d are host pointers (copied host->device on the
 *         stream); MSP_DEVICE: device pointers, read before the next
 *         synchronising call returns.
 * Allocates (or reuses) the batch's device buffers, then builds each
 * instance's (m+n+1) x (n+1) generator on the device.  Any later call
 * works on this batch until the next msp_build_lattice(). */
MSP_API msp_status msp_build_lattice(msp_ctx *ctx, int count, const int32_t *dims,
                             const int32_t *A, const int64_t *d, int mem);

/* The general problem of Sec. 2: A x = d with 0 <= x_j <= r_j (bounds l
 * are removed beforehand by x := x - l, d := d - A l).  Same as
 * msp_build_lattice with the upper bounds
 *   r     host int32, the r_i (n_i entries each) back to back, always host
 *         memory; NULL: every bound is 1 (the binary problem).
 * The lattice of Eq. (2) uses r_max = lcm(r_1 .. r_n) and c_j = r_max / r_j;
 * the enumeration bounds become R = (n+1) r_max^2 and r_max ||w||_1 and the
 * leaf test of Theorem 1 reads x_j = (v_j + r_max) / (2 c_j).  Limits
 * (MSP_EINVAL otherwise): 1 <= r_j <= 255, r_max <= 1024, and the
 * solution of an instance must fit 128 bits: sum_j bitwidth(r_j) <= 128.
 * msp_solutions() then returns x_j in 0 .. r_j. */
MSP_API msp_status msp_build_lattice_bounds(msp_ctx *ctx, int count, const int32_t *dims,
                                    const int32_t *A, const int64_t *d, const int32_t *r, int mem);

/* Steps a2-a3 -- Alg. 1 steps 1-3: LLL-reduce every generator (exact
 * integer basis, exact int64 Gram matrix, FP64 Gram-Schmidt), keep the
 * reduced vectors whose first m entries are zero, drop those rows and
 * compute the FP64 Gram-Schmidt tables mu, ||bhat||^2, bhat (Eq. (4)).
 * Asynchronous; per-instance errors (MSP_EOVERFLOW, MSP_ERANK, MSP_ECAP)
 * surface in msp_enumerate's statistics. */
MSP_API msp_status msp_reduce(msp_ctx *ctx);

/* Steps a4-a7 -- Algorithm 1: split the top levels into subtree prefixes,
 * optionally reorder them by the learned scorer (MSP_LEARNED; falls back
 * to MSP_PLAIN when no scorer is loaded), enumerate every subtree on the
 * device and check every leaf exactly (Theorem 1).  MSP_FIRST finishes
 * each instance (with its replicas) at its first verified solution: its
 * remaining subtrees are skipped while the other instances of the batch go
 * on, and the launch ends once every instance is solved or its tree is
 * exhausted.  time_cap_s > 0 bounds the
 * enumeration's wall time (MSP_ETIMEOUT, partial results).
 * stats: NULL or count entries (one per instance).  total: NULL or one
 * entry summed over the batch.  Synchronises the stream. */
MSP_API msp_status msp_enumerate(msp_ctx *ctx, int mode, int order, double time_cap_s,
                         msp_stats *stats, msp_stats *total);

/* Asynchronous variant: queue a whole step (reduce + split + enumerate +
 * collect) for the current batch without synchronising, so that it can be
 * timed with events or captured in a CUDA graph.  Read the results with
 * msp_wait(). */
MSP_API msp_status msp_run_async(msp_ctx *ctx, int mode, int order);

/* Capture one whole step of the current batch -- lattice rebuilt from the
 * stored A and d, reduction, split, order, enumeration, solution collection
 * -- into a CUDA graph owned by the context.  Requires one completed
 * enumeration of the batch first (so every buffer exists); replaces any
 * previous graph.  msp_graph_launch() replays it on the context's stream
 * without host work between the kernels; read results with msp_wait().
 * The graph reads A and d from the context's device copies, so a later
 * msp_build_lattice() with a batch of the same layout (same count and same
 * (m, n) per instance) keeps it valid and the next replay solves the new
 * batch; a different layout discards it (msp_graph_launch then returns
 * MSP_ESTATE until the next capture). */
MSP_API msp_status msp_graph_capture(msp_ctx *ctx, int mode, int order);
MSP_API msp_status msp_graph_launch(msp_ctx *ctx);

/* Lanes per walker in effect for the current batch (0 before
 * msp_build_lattice). */
MSP_API int msp_lanes(const msp_ctx *ctx);

/* Synchronise and read the statistics of the last msp_run_async(). */
MSP_API msp_status msp_wait(msp_ctx *ctx, msp_stats *stats, msp_stats *total);

/* Solutions of instance `inst` after msp_enumerate / msp_wait: writes up to
 * cap rows of n bytes (x_j: 0/1, or 0 .. r_j with msp_build_lattice_bounds),
 * lexicographically sorted, into host memory x,
 * and the full count into *count.  cap = 0 (x may be NULL) only queries the
 * count.  Returns MSP_ETRUNC when the count exceeds cap or the context's
 * solution capacity. */
MSP_API msp_status msp_solutions(msp_ctx *ctx, int inst, uint8_t *x, size_t cap, size_t *count);

/* Export instance `inst`'s reduced kernel basis and Gram-Schmidt tables to
 * host memory (for inspection and tests).  dims_out[0] = kernel rank dd,
 * dims_out[1] = n + 1.  Any pointer may be NULL to skip it; otherwise
 * basis holds dd*(n+1) int32, mu dd*dd doubles (mu[i][j], row-major, 1 on
 * the diagonal), B dd doubles, bhat dd*(n+1) doubles. */
MSP_API msp_status msp_export_gso(msp_ctx *ctx, int inst, int32_t *dims_out, int32_t *basis,
                          double *mu, double *B, double *bhat);

/* Export instance `inst`'s full LLL-reduced basis: (n+1) x (m+n+1) int64,
 * one reduced vector per row, into host memory. */
MSP_API msp_status msp_export_reduced(msp_ctx *ctx, int inst, int64_t *basis);

/* Export the subtree prefixes of instance `inst` made by the last split
 * (the tree partition of Sec. 4), in depth-first order: up to cap rows of
 * dd int32 u values (entries below the split level are 0), their partial
 * norms rho, and the log of the last enumeration -- nodes evaluated in each
 * subtree (negative if the walk was cut short) and solutions found in it.
 * *count receives the number of prefixes and *split_level the lowest fixed
 * level.  Any array may be NULL. */
MSP_API msp_status msp_export_prefixes(msp_ctx *ctx, int inst, int32_t *u, double *rho, int64_t *nodes,
                                       int32_t *sols, size_t cap, size_t *count, int32_t *split_level);

/* Device time in milliseconds of the phases of the last enumeration,
 * measured with CUDA events on the context's stream: out[0] reduction
 * (LLL + Gram-Schmidt, if msp_reduce or msp_run_async queued it), out[1]
 * split, out[2] enumeration kernel, out[3] solution collection. */
MSP_API msp_status msp_phase_ms(msp_ctx *ctx, double *out);

/* ---- subtree scorer (not in the paper) -----------------------------------
 * In MSP_FIRST mode the subtrees of a batch are taken in rank order,
 * interleaving the instances: rank = depth-first position (MSP_PLAIN) or the
 * position by descending priority of a 3-layer MLP (MSP_LEARNED).  The order
 * never changes the pruning: MSP_ALL returns the same solutions and node
 * counts under either order.  Network 32 -> 64 -> 64 -> 8, ReLU, bfloat16
 * tensor-core products with float32 accumulation; parameters are float32:
 * W1[32][64] b1[64] W2[64][64] b2[64] W3[64][8] b3[8] (row = input).
 * Outputs y0 = logit of P(the subtree holds a solution), y1 = predicted
 * log(1 + nodes of the subtree); priority = log sigmoid(y0) - y1. */

/* Number of float32 parameters of the scorer (6792). */
MSP_API int msp_mlp_param_count(void);

/* Use the scorer with these parameters (host memory, copied) for
 * MSP_LEARNED; NULL removes it (MSP_LEARNED then falls back to MSP_PLAIN). */
MSP_API msp_status msp_set_scorer(msp_ctx *ctx, const float *theta);

/* After an enumeration with opts.log_features (or a learned order): the 32
 * features of each prefix of instance `inst`, in depth-first order (the
 * order of msp_export_prefixes), into host memory (cap rows of 32 floats);
 * *count = number of prefixes. */
MSP_API msp_status msp_export_features(msp_ctx *ctx, int inst, float *feat, size_t cap, size_t *count);

/* Scorer kernels on device memory (all pointers are device pointers; each
 * call synchronises the context's stream):
 *   forward: y[n][8] = mlp(x[n][32])
 *   grad:    gradient of the mean loss over the n rows (target[n][2] =
 *            (found 0/1, log(1 + nodes)); loss per row pos_weight*BCE for
 *            found rows, BCE otherwise, + 0.1 (y1 - target1)^2) into grad,
 *            mean loss into *loss
 *   train:   `steps` Adam steps (lr, betas 0.9/0.999, eps 1e-8) on
 *            mini-batches of 128 rows drawn with replacement by a
 *            counter-based generator from `seed`; theta is updated in place;
 *            losses (NULL or steps floats) receives each step's mean loss. */
MSP_API msp_status msp_mlp_forward(msp_ctx *ctx, const float *theta, const float *x, int64_t n, float *y);
MSP_API msp_status msp_mlp_grad(msp_ctx *ctx, const float *theta, const float *x, const float *target, int64_t n,
                                float pos_weight, float *grad, float *loss);
MSP_API msp_status msp_mlp_train(msp_ctx *ctx, float *theta, const float *x, const float *target, int64_t n,
                                 int steps, float lr, float pos_weight, uint64_t seed, float *losses);

/* Measure this GPU's FP64 fused multiply-add throughput: a kernel of
 * independent FMA chains on every SM, timed with CUDA events on the
 * context's stream.  *dfma_per_s receives FMA instructions (lanes) per
 * second.  Used as the measured peak of the enumeration roofline. */
MSP_API msp_status msp_fp64_peak(msp_ctx *ctx, double *dfma_per_s);

/* Lattice reduction without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a
 * library allocate device memory -- a host application whose allocator owns
 * the whole GPU (a pool that reserved the device up front, or a process under
 * a hard device-memory cap), or a latency-critical caller that cannot afford
 * the device-wide synchronisation an allocation may cause.
 *
 * It builds the lattice of Eq. (2) for one instance and LLL-reduces it with
 * the same kernels and the same arithmetic as msp_build_lattice() +
 * msp_reduce(), so the result equals msp_export_reduced() of that path.
 *   m, n      1 <= m <= 32, m <= n <= 127; larger sizes return MSP_EINVAL
 *   A, d      device pointers: A int32 m x n row-major, d int64[m] (inputs)
 *   N, delta, eta, max_iter   as in msp_opts; the LLL loop's device-time
 *             cap is msp_opts' default max_seconds, 600 s (MSP_ECAP after)
 *   basis     device pointer, int64 (n+1) x (m+n+1) (output, one reduced
 *             vector per row)
 *   stream    cudaStream_t (NULL: default stream); the call synchronises it
 * Returns MSP_OK, MSP_EINVAL, MSP_EOVERFLOW, MSP_ECAP or MSP_ECUDA.
 *
 * Scratch: a file-scope device array of 395,520 bytes (Gram matrix,
 * Gram-Schmidt rows, descriptor for n + 1 <= 128) that every GPU loading this
 * library holds until the process exits.  No cudaMalloc or cudaFree is
 * called.  The first call on a device looks up the array's device address
 * with that device current (one-time set-up); make that first call before
 * any stream capture.  All calls share the one array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  Each call rewrites everything it reads from the array. */
MSP_API msp_status msp_reduce_lattice_noalloc(int m, int n, const int32_t *A, const int64_t *d, int64_t N,
                                              double delta, double eta, int64_t max_iter, int64_t *basis,
                                              void *stream);

/* Human-readable name of a status code, and the context's last error text. */
MSP_API const char *msp_status_string(int status);
MSP_API const char *msp_last_error(const msp_ctx *ctx);

/* Number of CUDA kernels launched by this context since creation. */
MSP_API int64_t msp_kernel_launches(const msp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MSP_H */
