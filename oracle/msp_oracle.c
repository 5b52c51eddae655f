/*
 * msp_oracle.c -- plain, slow, scalar CPU oracle for the lattice method of
 * "Solving the Market Split Problem with Lattice Enumeration" (Wassermann).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * shares no code, header, table or constant generator with it.
 *
 * What it computes, step by step (paper references in brackets):
 *   1. lattice build        generator matrix of Eq. (2), binary case
 *                           r_max = c_j = 1                     [Sec. 2]
 *   2. LLL                  integral basis, exact int64 Gram matrix,
 *                           FP64 Gram-Schmidt recomputed per row from the
 *                           Gram matrix, one size-reduction pass per row
 *                           (repeated until nothing changes in the LLL
 *                           inside BKZ; reading R10)
 *                                                    [Sec. 2, Alg. 1 step 1]
 *   3. extraction           keep the vectors whose first m entries are zero,
 *                           drop those m rows          [Sec. 2, Alg. 1 step 2]
 *   4. Gram-Schmidt         Eq. (4) on the kept basis   [Alg. 1 step 3]
 *   5. enumeration          Algorithm 1: centre y_t, zig-zag next(), the
 *                           norm test (first pruning condition), the Hoelder
 *                           test of Theorem 2 with the one-direction cut,
 *                           exact leaf test of Theorem 1  [Sec. 2, Alg. 1]
 *   6. BKZ                  blockwise Korkine-Zolotarev reduction of the
 *                           kernel basis (the alternative to LLL that Sec. 2
 *                           names for step 1): block-wise shortest vectors
 *                           by enumeration, inserted, then LLL   [Sec. 2]
 *
 * Readings where the paper is silent or ambiguous (all fixed here and used
 * identically by the GPU path, which implements them independently):
 *   R1  next() is applied after every return from the recursive call and
 *       after every leaf (the pseudocode omits it).
 *   R2  u^1 = round-half-even(-y_t); zig-zag side s = +1 if -y_t >= u^1,
 *       else -1; u^{2k} = u^1 + s k, u^{2k+1} = u^1 - s k.
 *   R3  First Hoelder failure: take the regular next value u' and from then
 *       on step by sign(u' - u^1); a second Hoelder failure, or any norm
 *       failure, returns.
 *   R4  Tests carry a slack eps = R 2^-20 (prune iff rho > R + eps, resp.
 *       rho > ||w||_1 + eps) so that FP64 rounding can never drop a solution
 *       (every solution sits exactly on both bounds).  eps = 0 is available.
 *   R5  Leaf: the integer vector v = sum u_j b_j is checked exactly
 *       (Theorem 1): last entry +-r_max (sign-normalised to +r_max), all
 *       others in [-r_max, r_max], then A x = d with x_c = (v_c + r_max) /
 *       (2 c_c); binary: r_max = c_c = 1, v = +-1, x = (v + 1)/2.  General
 *       bounds: R = (n+1) r_max^2, the Hoelder bound is r_max ||w||_1 (the
 *       product formed first, then the slack added).
 *   R6  Symmetry: v and -v are both lattice points.  In "sym" mode levels
 *       whose prefix above is all zero try u = 0, 1, 2, ... only (the first
 *       nonzero coefficient from the top is positive).  "literal" mode runs
 *       the plain zig-zag everywhere and keeps only leaves with last = +1.
 *   R7  The homogenising coordinate (Theorem 1's w_0 = r_max) is stored last.
 *   R8  A node is one evaluation of the norm of w for a candidate (t, u_t).
 *   R9  Arithmetic order (every step one IEEE operation, no contraction):
 *         y_t  = fold i = d-1 .. t+1 of acc = fma(u_i, mu[i][t], acc), acc0 = 0
 *         x    = (double)u_t + y_t
 *         rho  = fma(x*x, B_t, rho_{t+1})
 *         w_c  = fma(x, bhat[t][c], w'_c)
 *         |w|_1: G interleaved partial sums s_l = sum_{c = l mod G} |w_c|
 *               (ascending c), then pairwise s_l += s_{l+off}, off = G/2..1.
 *       G ("lanes") is a parameter; G = 1 is the sequential sum.
 *   R10 N = 2^10 (Sec. 2); delta = 0.99, eta = 0.51 (the paper gives neither);
 *       inside LLL mu_kj = r_kj (1/B_j) with the reciprocal formed once per
 *       row, in the enumeration tables mu = r / B (Eq. (4) as written).  Size
 *       reduction of a row: one pass j = k-1 .. 0 on its freshly computed
 *       Gram-Schmidt row, updated in place; the LLL inside BKZ repeats the
 *       pass until nothing changes (see oracle_lll).
 *   R11 The construction of the paper's instance library is not described.
 *       The configurations plant a binary x and set d = A x; the stand-ins
 *       for the rows of the paper's timing table use the centred right-hand
 *       side d_i = floor(sum_j a_ij / 2).  The oracle takes A and d as given.
 *   R12 Limited discrepancy search (Sec. 3, after Harvey and Ginsberg): a
 *       discrepancy is a deviation from the heuristic order of a level's
 *       walk, whose first value u^1 is the rounded centre (0 on the all-zero
 *       levels of sym mode).  The paper does not say what a deviation to a
 *       later value of a many-valued level costs; two readings:
 *         rank (lds_rank = 1, the default): the value at position p of the
 *           level's walk (p = 0 for u^1, counting every value the walk
 *           takes, the one-direction phase after a Hoelder failure
 *           included) costs p discrepancies;
 *         flat (lds_rank = 0): every value other than u^1 costs one.
 *       The cost of a path is the sum over its levels.  Iteration k walks
 *       Algorithm 1 but tries a value only while the path's cost stays at
 *       most k, and reports a leaf only when the cost is exactly k, so
 *       iterations k = 0, 1, 2, ... report every solution exactly once.
 *       Nodes are counted as in R8 (the nodes of lower cost are visited
 *       again).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum { OR_OK = 0, OR_EOVERFLOW = 1, OR_ECAP = 2, OR_ENOMEM = 3, OR_EINVAL = 4 };

/* Entries of the basis are kept below 2^58 so that a 128-bit sum of
 * L <= 2^10 products of two entries cannot overflow. */
#define OR_ENTRY_LIMIT ((int64_t)1 << 58)

/* ------------------------------------------------------------------------ */
/* 1. Lattice build (Sec. 2, Eq. (2)).                                        */
/* Bounds 0 <= x_j <= r_j (l = 0 after the substitution of Sec. 2);          */
/* r_max = lcm(r_1..r_n), c_j = r_max / r_j; binary: r = NULL, all ones.     */
/* The generator has m+n+1 rows and n+1 columns; column j is basis vector j.  */
/* We store it as K = n+1 vectors of length L = m+n+1, vector-major:          */
/*   vector 0   = (-N d_1..-N d_m, -r_max (n times), +r_max)                  */
/*   vector j   = (N a_1j..N a_mj, 2 c_j e_j, 0),  j = 1..n                   */
/* ------------------------------------------------------------------------ */
static int64_t gcd64(int64_t a, int64_t b)
{
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

/* r_max = lcm of the bounds (1 for r = NULL); 0 when a bound is below 1 or
 * the lcm exceeds 2^20. */
int64_t oracle_rmax(int n, const int32_t *r)
{
    int64_t l = 1;
    if (!r) return 1;
    for (int j = 0; j < n; ++j) {
        if (r[j] < 1) return 0;
        l = l / gcd64(l, r[j]) * r[j];
        if (l > ((int64_t)1 << 20)) return 0;
    }
    return l;
}

int oracle_build_lattice_bounds(int m, int n, const int32_t *A, const int64_t *d, const int32_t *r,
                                int64_t N, int64_t *basis)
{
    if (m < 1 || n < 1 || N < 1) return OR_EINVAL;
    const int64_t rmax = oracle_rmax(n, r);
    if (rmax < 1) return OR_EINVAL;
    const int K = n + 1, L = m + n + 1;
    memset(basis, 0, sizeof(int64_t) * (size_t)K * (size_t)L);
    for (int i = 0; i < m; ++i) {
        i128 v = -(i128)N * (i128)d[i];
        if (v >= OR_ENTRY_LIMIT || v <= -OR_ENTRY_LIMIT) return OR_EOVERFLOW;
        basis[i] = (int64_t)v;
    }
    for (int j = 0; j < n; ++j) basis[m + j] = -rmax;
    basis[m + n] = rmax;
    for (int j = 1; j <= n; ++j) {
        int64_t *b = basis + (size_t)j * L;
        for (int i = 0; i < m; ++i) b[i] = N * (int64_t)A[(size_t)i * n + (j - 1)];
        b[m + (j - 1)] = 2 * (rmax / (r ? r[j - 1] : 1));
    }
    return OR_OK;
}

int oracle_build_lattice(int m, int n, const int32_t *A, const int64_t *d,
                         int64_t N, int64_t *basis)
{
    return oracle_build_lattice_bounds(m, n, A, d, NULL, N, basis);
}

/* ------------------------------------------------------------------------ */
/* 2. LLL reduction (Sec. 2; Alg. 1 step 1).                                  */
/* ------------------------------------------------------------------------ */
static int dot_exact(const int64_t *a, const int64_t *b, int L, int64_t *out)
{
    i128 s = 0;
    for (int i = 0; i < L; ++i) s += (i128)a[i] * (i128)b[i];
    if (s > (i128)INT64_MAX || s < (i128)INT64_MIN) return OR_EOVERFLOW;
    *out = (int64_t)s;
    return OR_OK;
}

/* Gram-Schmidt row k from the exact Gram matrix G (K x K, full):
 *   r_kj = G_kj - sum_{i<j} mu_ji r_ki,  mu_kj = r_kj * (1 / r_jj),
 *   r_kk = G_kk - sum_{i<k} mu_ki r_ki,  B_k = r_kk,  invB_k = 1 / B_k.
 * This is Eq. (4) written with r_kj = <b_k, bhat_j>; inside the reduction
 * mu is formed with the reciprocal of B_j, computed once per row. */
static void gso_row(int k, int K, const int64_t *G, double *mu, double *r, double *B, double *invB)
{
    for (int j = 0; j < k; ++j) {
        double acc = (double)G[(size_t)k * K + j];
        for (int i = 0; i < j; ++i)
            acc = fma(-mu[(size_t)j * K + i], r[(size_t)k * K + i], acc);
        r[(size_t)k * K + j] = acc;
        mu[(size_t)k * K + j] = acc * invB[j];
    }
    double acc = (double)G[(size_t)k * K + k];
    for (int i = 0; i < k; ++i)
        acc = fma(-mu[(size_t)k * K + i], r[(size_t)k * K + i], acc);
    r[(size_t)k * K + k] = acc;
    B[k] = acc;
    invB[k] = 1.0 / acc;
}

static int gram_row(int k, int K, int L, const int64_t *b, int64_t *G)
{
    for (int i = 0; i < K; ++i) {
        int64_t g;
        int st = dot_exact(b + (size_t)k * L, b + (size_t)i * L, L, &g);
        if (st) return st;
        G[(size_t)k * K + i] = g;
        G[(size_t)i * K + k] = g;
    }
    return OR_OK;
}

/* delta-LLL with size-reduction parameter eta.  b is K vectors of length L,
 * reduced in place.  Returns OR_OK, OR_EOVERFLOW or OR_ECAP (iteration cap).
 * Size reduction of row k (R10): its Gram-Schmidt row is computed from the
 * exact Gram matrix, then mu_kj for j = k-1 .. 0 is reduced in one pass,
 * the reductions updating the row in place (fma); the Gram row of b_k is
 * recomputed exactly.  lazy != 0 (the LLL inside BKZ) repeats the pass on a
 * freshly computed row until nothing changes, so the stored rows of a
 * finished run always equal a fresh computation. */
static int lll_core(int K, int L, int64_t *b, double delta, double eta, int64_t max_iter,
                    int64_t *iters_out, int64_t *swaps_out, int lazy)
{
    int st = OR_OK;
    int64_t *G = (int64_t *)calloc((size_t)K * K, sizeof(int64_t));
    double *mu = (double *)calloc((size_t)K * K, sizeof(double));
    double *r = (double *)calloc((size_t)K * K, sizeof(double));
    double *B = (double *)calloc((size_t)K, sizeof(double));
    double *invB = (double *)calloc((size_t)K, sizeof(double));
    int64_t iters = 0, swaps = 0;
    if (!G || !mu || !r || !B || !invB) { st = OR_ENOMEM; goto done; }

    for (int k = 0; k < K; ++k)
        if ((st = gram_row(k, K, L, b, G))) goto done;
    gso_row(0, K, G, mu, r, B, invB);

    int k = 1;
    while (k < K) {
        if (++iters > max_iter) { st = OR_ECAP; goto done; }
        /* size reduction (lazy: reduce, recompute the row exactly, repeat) */
        for (int pass = 0;; ++pass) {
            if (pass > 1000) { st = OR_ECAP; goto done; }
            gso_row(k, K, G, mu, r, B, invB);
            int changed = 0;
            for (int j = k - 1; j >= 0; --j) {
                double mkj = mu[(size_t)k * K + j];
                if (fabs(mkj) > eta) {
                    double qd = rint(mkj);
                    if (fabs(qd) > 4503599627370496.0) { st = OR_EOVERFLOW; goto done; }
                    int64_t q = (int64_t)qd;
                    for (int i = 0; i < j; ++i)
                        mu[(size_t)k * K + i] = fma(-qd, mu[(size_t)j * K + i], mu[(size_t)k * K + i]);
                    mu[(size_t)k * K + j] = mkj - qd;
                    int64_t *bk = b + (size_t)k * L;
                    const int64_t *bj = b + (size_t)j * L;
                    for (int c = 0; c < L; ++c) {
                        i128 v = (i128)bk[c] - (i128)q * (i128)bj[c];
                        if (v >= OR_ENTRY_LIMIT || v <= -OR_ENTRY_LIMIT) { st = OR_EOVERFLOW; goto done; }
                        bk[c] = (int64_t)v;
                    }
                    changed = 1;
                }
            }
            if (!changed) break;
            if ((st = gram_row(k, K, L, b, G))) goto done;
            if (!lazy) break;
        }
        /* Lovasz condition B_k >= (delta - mu_{k,k-1}^2) B_{k-1} */
        double mk = mu[(size_t)k * K + (k - 1)];
        double t1 = mk * mk;
        double t2 = delta - t1;
        double rhs = t2 * B[k - 1];
        if (B[k] < rhs) {
            int64_t *bk = b + (size_t)k * L, *bm = b + (size_t)(k - 1) * L;
            for (int c = 0; c < L; ++c) { int64_t t = bk[c]; bk[c] = bm[c]; bm[c] = t; }
            for (int i = 0; i < K; ++i) {      /* swap rows k-1, k of G */
                int64_t t = G[(size_t)k * K + i];
                G[(size_t)k * K + i] = G[(size_t)(k - 1) * K + i];
                G[(size_t)(k - 1) * K + i] = t;
            }
            for (int i = 0; i < K; ++i) {      /* swap columns k-1, k of G */
                int64_t t = G[(size_t)i * K + k];
                G[(size_t)i * K + k] = G[(size_t)i * K + (k - 1)];
                G[(size_t)i * K + (k - 1)] = t;
            }
            ++swaps;
            if (k - 1 == 0) gso_row(0, K, G, mu, r, B, invB);
            k = (k > 1) ? k - 1 : 1;
        } else {
            ++k;
        }
    }
done:
    if (iters_out) *iters_out = iters;
    if (swaps_out) *swaps_out = swaps;
    free(G); free(mu); free(r); free(B); free(invB);
    return st;
}

int oracle_lll(int K, int L, int64_t *b, double delta, double eta, int64_t max_iter,
               int64_t *iters_out, int64_t *swaps_out)
{
    return lll_core(K, L, b, delta, eta, max_iter, iters_out, swaps_out, 0);
}

/* ------------------------------------------------------------------------ */
/* 3. Extraction (Sec. 2; Alg. 1 step 2): keep, in order, the reduced vectors */
/* whose first m entries are all zero, and drop those m rows.                 */
/* Returns the number kept; kern receives kept x (n+1) entries.               */
/* A kept entry outside int32 sets *overflow.                                  */
/* ------------------------------------------------------------------------ */
int oracle_extract(int m, int n, const int64_t *basis, int32_t *kern, int *overflow)
{
    const int K = n + 1, L = m + n + 1, dim = n + 1;
    int kept = 0;
    *overflow = 0;
    for (int k = 0; k < K; ++k) {
        const int64_t *b = basis + (size_t)k * L;
        int zero = 1;
        for (int i = 0; i < m; ++i) if (b[i] != 0) { zero = 0; break; }
        if (!zero) continue;
        for (int c = 0; c < dim; ++c) {
            int64_t v = b[m + c];
            if (v > INT32_MAX || v < INT32_MIN) *overflow = 1;
            kern[(size_t)kept * dim + c] = (int32_t)v;
        }
        ++kept;
    }
    return kept;
}

/* ------------------------------------------------------------------------ */
/* 4. Gram-Schmidt of the kept basis (Eq. (4); Alg. 1 step 3).                */
/* mu is dd x dd (lower triangle used), B has dd entries, bhat is dd x dim.   */
/* ------------------------------------------------------------------------ */
int oracle_gso(int dd, int dim, const int32_t *kb, double *mu, double *B, double *bhat)
{
    int64_t *G = (int64_t *)malloc(sizeof(int64_t) * (size_t)dd * dd);
    double *r = (double *)calloc((size_t)dd * dd, sizeof(double));
    if (!G || !r) { free(G); free(r); return OR_ENOMEM; }
    for (int i = 0; i < dd; ++i)
        for (int j = 0; j < dd; ++j) {
            i128 s = 0;
            for (int c = 0; c < dim; ++c)
                s += (i128)kb[(size_t)i * dim + c] * (i128)kb[(size_t)j * dim + c];
            if (s > (i128)INT64_MAX || s < (i128)INT64_MIN) { free(G); free(r); return OR_EOVERFLOW; }
            G[(size_t)i * dd + j] = (int64_t)s;
        }
    memset(mu, 0, sizeof(double) * (size_t)dd * dd);
    for (int i = 0; i < dd; ++i) {
        for (int j = 0; j < i; ++j) {
            double acc = (double)G[(size_t)i * dd + j];
            for (int k = 0; k < j; ++k)
                acc = fma(-mu[(size_t)j * dd + k], r[(size_t)i * dd + k], acc);
            r[(size_t)i * dd + j] = acc;
            mu[(size_t)i * dd + j] = acc / B[j];
        }
        double acc = (double)G[(size_t)i * dd + i];
        for (int k = 0; k < i; ++k)
            acc = fma(-mu[(size_t)i * dd + k], r[(size_t)i * dd + k], acc);
        r[(size_t)i * dd + i] = acc;
        B[i] = acc;
        mu[(size_t)i * dd + i] = 1.0;
    }
    /* bhat_i = b_i - sum_{j<i} mu_ij bhat_j, coordinate by coordinate */
    for (int i = 0; i < dd; ++i)
        for (int c = 0; c < dim; ++c) {
            double acc = (double)kb[(size_t)i * dim + c];
            for (int j = 0; j < i; ++j)
                acc = fma(-mu[(size_t)i * dd + j], bhat[(size_t)j * dim + c], acc);
            bhat[(size_t)i * dim + c] = acc;
        }
    free(G); free(r);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 5. Enumeration: Algorithm 1.                                               */
/* ------------------------------------------------------------------------ */
enum { HOELDER_CUT = 0, HOELDER_FILTER = 1, HOELDER_OFF = 2 };

typedef struct {
    int hoelder;        /* HOELDER_CUT (paper), _FILTER (skip value only), _OFF */
    int sym;            /* 1: sym mode (R6), 0: literal mode                    */
    int lanes;          /* G of the |w|_1 summation order (R9), power of two    */
    int use_eps;        /* 1: slack eps = R 2^-20 (R4); 0: paper-literal         */
    int first;          /* stop at the first solution                            */
    int split_level;    /* >= 0: record prefixes passing at this level instead  */
                        /* of descending (top-k split); -1: off                 */
    int sub_level;      /* >= 0: enumerate only the subtree below a prefix whose */
                        /* values u[sub_level+1 .. dd-1] are given; -1: off       */
    int lds;            /* >= 0: one limited-discrepancy iteration with this     */
                        /* budget (R12); -1: plain depth-first search            */
    int lds_rank;       /* 1: a value's discrepancy is its position in its       */
                        /* level's walk (the k-th value tried costs k-1); 0:     */
                        /* every value after the first costs one (R12)           */
} oracle_enum_opts;

typedef struct {
    int64_t nodes, passed, leaves;
    int64_t nsol;       /* number of solutions found (may exceed sol_cap) */
    int64_t nprefix;    /* number of split prefixes found (may exceed cap) */
    int64_t lds_cuts;   /* values not tried because of the discrepancy budget */
    int stopped;
} oracle_enum_stats;

typedef struct {
    int dd, dim, m, n;
    const double *mu, *B, *bhat;
    const int32_t *kb, *A;
    const int64_t *d;
    const int32_t *r;   /* bounds (NULL: binary) */
    int64_t rmax;
    oracle_enum_opts o;
    double Rb, eps;
    int32_t *u;
    /* outputs */
    uint8_t *sol; int64_t sol_cap;
    int32_t *pre_u; double *pre_rho; int64_t pre_cap;
    oracle_enum_stats s;
    int64_t *vbuf; uint8_t *xbuf;
} enum_state;

/* y_t = sum_{i=t+1}^{dd-1} u_i mu_it, folded from the top (R9) */
static double center(const enum_state *e, int t)
{
    double acc = 0.0;
    for (int i = e->dd - 1; i > t; --i)
        acc = fma((double)e->u[i], e->mu[(size_t)i * e->dd + t], acc);
    return acc;
}

/* |w|_1 in the canonical G-lane order (R9) */
static double norm1(const double *w, int dim, int G)
{
    double s[64];
    for (int l = 0; l < G; ++l) s[l] = 0.0;
    for (int c = 0; c < dim; ++c) s[c % G] = s[c % G] + fabs(w[c]);
    for (int off = G / 2; off >= 1; off /= 2)
        for (int l = 0; l < off; ++l) s[l] = s[l] + s[l + off];
    return s[0];
}

/* zig-zag sequence around the centre (R2): index i >= 1 */
static long zigzag(long u1, int s, long i)
{
    return (i % 2 == 0) ? u1 + (long)s * (i / 2) : u1 - (long)s * ((i - 1) / 2);
}

/* Leaf test of Theorem 1 on v = sum_j u_j b_j (R5).  Returns 1 on a solution
 * and writes x. */
static int leaf_check(enum_state *e)
{
    const int dd = e->dd, dim = e->dim, n = e->n, m = e->m;
    int64_t *v = e->vbuf;
    for (int c = 0; c < dim; ++c) {
        int64_t acc = 0;
        for (int j = 0; j < dd; ++j) acc += (int64_t)e->u[j] * (int64_t)e->kb[(size_t)j * dim + c];
        v[c] = acc;
    }
    /* Theorem 1: last entry r_max, all others in [-r_max, r_max];
     * x_c = (v_c + r_max) / (2 c_c) */
    const int64_t rmax = e->rmax;
    int64_t last = v[dim - 1];
    if (e->o.sym) {
        if (last == -rmax) { for (int c = 0; c < dim; ++c) v[c] = -v[c]; last = rmax; }
    }
    if (last != rmax) return 0;
    for (int c = 0; c < n; ++c) {
        const int64_t cc = 2 * (rmax / (e->r ? e->r[c] : 1));
        if (v[c] > rmax || v[c] < -rmax || (v[c] + rmax) % cc != 0) return 0;
        e->xbuf[c] = (uint8_t)((v[c] + rmax) / cc);
    }
    for (int i = 0; i < m; ++i) {          /* independent verification A x = d */
        int64_t acc = 0;
        for (int c = 0; c < n; ++c) acc += (int64_t)e->A[(size_t)i * n + c] * e->xbuf[c];
        if (acc != e->d[i]) return 0;
    }
    return 1;
}

/* Discrepancy of the value at position pos (0-based) of a level's walk,
 * u the value and u1 the first one (R12). */
static int value_cost(const enum_state *e, long pos, long u, long u1)
{
    return e->o.lds_rank ? (int)pos : (u != u1);
}

/* enum(t, w') of Algorithm 1.  wp = w^{(t+1)}, rho_p = ||w^{(t+1)}||^2. */
static void enum_level(enum_state *e, int t, const double *wp, double rho_p, int disc)
{
    const int dd = e->dd, dim = e->dim;
    double w[dim];
    long pos = 0;                                  /* position of u in this level's walk */

    int zero_prefix = 1;
    for (int i = t + 1; i < dd; ++i) if (e->u[i] != 0) { zero_prefix = 0; break; }

    int onedirection = 0;
    long dir = 0;
    const double y = center(e, t);                 /* y_t */
    const double cstar = -y;
    long u1 = (long)rint(cstar);                   /* u_t <- round(-y_t) */
    int s = (cstar >= (double)u1) ? 1 : -1;
    long zi = 1;
    if (zero_prefix && e->o.sym) { u1 = 0; onedirection = 1; dir = 1; }
    long u = u1;

    for (;;) {
        const int cost = value_cost(e, pos, u, u1);
        if (e->o.lds >= 0 && cost > 0 && disc + cost > e->o.lds) {   /* budget spent (R12) */
            e->s.lds_cuts++;
            return;
        }
        e->u[t] = (int32_t)u;
        const double x = (double)u + y;            /* sum_{i>=t} u_i mu_it */
        const double xx = x * x;
        const double rho = fma(xx, e->B[t], rho_p);
        e->s.nodes++;
        if (rho > e->Rb) return;                   /* first pruning condition */
        e->s.passed++;
        if (t > 0) {
            for (int c = 0; c < dim; ++c) w[c] = fma(x, e->bhat[(size_t)t * dim + c], wp[c]);
            int fail = 0;
            if (e->o.hoelder != HOELDER_OFF) {
                const double h = (double)e->rmax * norm1(w, dim, e->o.lanes) + e->eps;
                fail = rho > h;                    /* second pruning condition */
            }
            if (fail && e->o.hoelder == HOELDER_CUT) {
                if (onedirection) return;
                zi += 1;                           /* one more regular next() */
                u = zigzag(u1, s, zi);
                dir = (u > u1) ? 1 : -1;
                onedirection = 1;
                pos += 1;
                continue;
            }
            if (!fail) {
                if (e->o.split_level == t) {
                    int64_t p = e->s.nprefix++;
                    if (p < e->pre_cap) {
                        for (int i = 0; i < dd; ++i)
                            e->pre_u[(size_t)p * dd + i] = (i >= t) ? e->u[i] : 0;
                        e->pre_rho[p] = rho;
                    }
                } else {
                    enum_level(e, t - 1, w, rho, disc + cost);  /* step forward */
                    if (e->s.stopped) return;
                }
            }
        } else {
            e->s.leaves++;
            if ((e->o.lds < 0 || disc + cost == e->o.lds) && leaf_check(e)) {
                int64_t q = e->s.nsol++;
                if (q < e->sol_cap) memcpy(e->sol + (size_t)q * e->n, e->xbuf, (size_t)e->n);
                if (e->o.first) { e->s.stopped = 1; return; }
            }
        }
        if (onedirection) u += dir;                 /* next(u_t) */
        else { zi += 1; u = zigzag(u1, s, zi); }
        pos += 1;
    }
}

/* Position of the value target in the walk of level t (the same sequence of
 * values and tests enum_level takes, without descending), given the centre
 * y, w^{(t+1)} and its norm; -1 if the walk never reaches it. */
static long level_position(const enum_state *e, int t, double y, const double *wp, double rho_p,
                           int zero_prefix, long target)
{
    const int dim = e->dim;
    double w[dim];
    const double cstar = -y;
    long u1 = (long)rint(cstar);
    const int s = (cstar >= (double)u1) ? 1 : -1;
    int onedirection = 0;
    long dir = 0, zi = 1, pos = 0;
    if (zero_prefix && e->o.sym) { u1 = 0; onedirection = 1; dir = 1; }
    long u = u1;
    for (;;) {
        if (u == target) return pos;
        const double x = (double)u + y;
        const double xx = x * x;
        const double rho = fma(xx, e->B[t], rho_p);
        if (rho > e->Rb) return -1;
        if (t > 0 && e->o.hoelder == HOELDER_CUT) {
            for (int c = 0; c < dim; ++c) w[c] = fma(x, e->bhat[(size_t)t * dim + c], wp[c]);
            const double h = (double)e->rmax * norm1(w, dim, e->o.lanes) + e->eps;
            if (rho > h) {
                if (onedirection) return -1;
                zi += 1;
                u = zigzag(u1, s, zi);
                dir = (u > u1) ? 1 : -1;
                onedirection = 1;
                pos += 1;
                continue;
            }
        }
        if (onedirection) u += dir;
        else { zi += 1; u = zigzag(u1, s, zi); }
        pos += 1;
    }
}

/* Enumerate the tree of Algorithm 1 (or the subtree below a prefix).
 * prefix_u: when o->sub_level >= 0, values u[sub_level+1..dd-1] (entries
 * below are ignored); w^{(sub_level+1)} and its norm are rebuilt from them
 * with the same operations the full enumeration performs on the way down. */
int oracle_enumerate_bounds(int dd, int dim, const double *mu, const double *B, const double *bhat,
                            const int32_t *kb, int m, int n, const int32_t *A, const int64_t *d,
                            const int32_t *r, const oracle_enum_opts *o, const int32_t *prefix_u,
                            uint8_t *sol, int64_t sol_cap,
                            int32_t *pre_u, double *pre_rho, int64_t pre_cap,
                            oracle_enum_stats *out)
{
    if (dd < 1 || dim != n + 1) return OR_EINVAL;
    const int64_t rmax = oracle_rmax(n, r);
    if (rmax < 1) return OR_EINVAL;
    if (o->lanes < 1 || o->lanes > 64 || (o->lanes & (o->lanes - 1))) return OR_EINVAL;
    enum_state e;
    memset(&e, 0, sizeof e);
    e.dd = dd; e.dim = dim; e.m = m; e.n = n;
    e.mu = mu; e.B = B; e.bhat = bhat; e.kb = kb; e.A = A; e.d = d;
    e.r = r; e.rmax = rmax;
    e.o = *o;
    const double R = (double)(dim * rmax * rmax);   /* R = (n+1) r_max^2 */
    e.eps = o->use_eps ? R * 0x1p-20 : 0.0;
    e.Rb = R + e.eps;
    e.sol = sol; e.sol_cap = sol_cap;
    e.pre_u = pre_u; e.pre_rho = pre_rho; e.pre_cap = pre_cap;
    e.u = (int32_t *)calloc((size_t)dd, sizeof(int32_t));
    e.vbuf = (int64_t *)calloc((size_t)dim, sizeof(int64_t));
    e.xbuf = (uint8_t *)calloc((size_t)n, 1);
    double *w0 = (double *)calloc((size_t)dim, sizeof(double));
    if (!e.u || !e.vbuf || !e.xbuf || !w0) {
        free(e.u); free(e.vbuf); free(e.xbuf); free(w0);
        return OR_ENOMEM;
    }
    int top = dd - 1;
    double rho0 = 0.0;
    int disc0 = 0;
    if (o->sub_level >= 0) {
        if (o->sub_level >= dd - 1) { free(e.u); free(e.vbuf); free(e.xbuf); free(w0); return OR_EINVAL; }
        int zero_prefix = 1;
        for (int t = dd - 1; t > o->sub_level; --t) {
            e.u[t] = prefix_u[t];
            const double y = center(&e, t);
            const long first = (zero_prefix && o->sym) ? 0 : (long)rint(-y);   /* u^1 of level t */
            if (o->lds >= 0 && o->lds_rank) {
                const long p = level_position(&e, t, y, w0, rho0, zero_prefix, e.u[t]);
                if (p < 0) { free(e.u); free(e.vbuf); free(e.xbuf); free(w0); return OR_EINVAL; }
                disc0 += (int)p;
            } else {
                disc0 += (e.u[t] != first);
            }
            zero_prefix = zero_prefix && (e.u[t] == 0);
            const double x = (double)e.u[t] + y;
            const double xx = x * x;
            rho0 = fma(xx, B[t], rho0);
            for (int c = 0; c < dim; ++c) w0[c] = fma(x, bhat[(size_t)t * dim + c], w0[c]);
        }
        top = o->sub_level;
    }
    enum_level(&e, top, w0, rho0, disc0);
    *out = e.s;
    free(e.u); free(e.vbuf); free(e.xbuf); free(w0);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 6. BKZ-beta on the kernel basis (Sec. 2 allows block reduction in place  */
/* of LLL for step 1 and gives no parameters).                               */
/* Readings (R14):                                                           */
/*   - BKZ runs on the kept kernel basis after LLL and extraction (the same */
/*     lattice the enumeration walks; the rows scaled by N play no part).   */
/*   - A tour visits k = 0 .. dd-2 with the block [k, h), h = min(k+beta,   */
/*     dd).  The block's shortest nonzero projected vector is found by     */
/*     Schnorr-Euchner enumeration (no Hoelder test: it is a general       */
/*     shortest vector search) with the bound delta * B_k, strict, shrunk  */
/*     to every improvement; ties keep the first found.  The tree has the  */
/*     same order and arithmetic as R2/R6/R9: zig-zag around the rounded   */
/*     centre, u >= 0 on all-zero top levels.                              */
/*   - An improvement u (primitive) is inserted by unimodular steps on the */
/*     rows k .. h-1: from the last row down, each pair (c_{i-1}, c_i) with */
/*     coefficients (a, b), g = gcd(a, b) = s a + t b, becomes            */
/*     ((a/g) c_{i-1} + (b/g) c_i, -t c_{i-1} + s c_i), moving the         */
/*     coefficient g one row up; then row k equals the inserted vector and */
/*     the whole basis is LLL-reduced again (delta, eta = 0.51).           */
/*   - Tours repeat until one inserts nothing, or max_tours.               */
/*   - Gram-Schmidt data of the whole basis from the exact Gram matrix in   */
/*     the LLL's form (mu_ij = r_ij (1/B_j)), rebuilt before each block.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dd, h, k;
    const double *mu, *B;
    double A;            /* current bound (strict) */
    int32_t *u, *best;
    int found;
    int64_t nodes;
} svp_state;

static void svp_level(svp_state *e, int t, double rho_p)
{
    const int dd = e->dd, h = e->h;
    int zero_prefix = 1;
    for (int i = t + 1; i < h; ++i) if (e->u[i] != 0) { zero_prefix = 0; break; }
    double acc = 0.0;
    for (int i = h - 1; i > t; --i) acc = fma((double)e->u[i], e->mu[(size_t)i * dd + t], acc);
    const double y = acc, cstar = -y;
    long u1 = (long)rint(cstar);
    const int s = (cstar >= (double)u1) ? 1 : -1;
    long zi = 1, u = u1;
    if (zero_prefix) u = u1 = 0;
    for (;;) {
        const double x = (double)u + y;
        const double rho = fma(x * x, e->B[t], rho_p);
        e->nodes++;
        if (!(rho < e->A)) return;
        e->u[t] = (int32_t)u;
        if (t == e->k) {
            if (!(zero_prefix && u == 0)) {      /* nonzero vector: an improvement */
                e->A = rho;
                memcpy(e->best + e->k, e->u + e->k, sizeof(int32_t) * (size_t)(h - e->k));
                e->found = 1;
            }
        } else {
            svp_level(e, t - 1, rho);
        }
        e->u[t] = 0;
        if (zero_prefix) ++u;
        else { ++zi; u = (zi % 2 == 0) ? u1 + (long)s * (zi / 2) : u1 - (long)s * ((zi - 1) / 2); }
    }
}

static int64_t egcd64(int64_t a, int64_t b, int64_t *sa, int64_t *tb)
{
    int64_t r0 = a < 0 ? -a : a, r1 = b < 0 ? -b : b, s0 = 1, s1 = 0, t0 = 0, t1 = 1;
    while (r1 != 0) {
        const int64_t q = r0 / r1, r2 = r0 - q * r1, s2 = s0 - q * s1, t2 = t0 - q * t1;
        r0 = r1; r1 = r2; s0 = s1; s1 = s2; t0 = t1; t1 = t2;
    }
    *sa = a < 0 ? -s0 : s0;
    *tb = b < 0 ? -t0 : t0;
    return r0;
}

/* b: dd x dim int64, BKZ-reduced in place.  Returns OR_OK, OR_EOVERFLOW,
 * OR_ECAP or OR_ENOMEM.  stats: tours run, insertions, enumeration nodes. */
int oracle_bkz(int dd, int dim, int64_t *b, int beta, double delta, int max_tours, int64_t lll_max_iter,
               int64_t *tours_out, int64_t *inserts_out, int64_t *nodes_out)
{
    if (dd < 1 || beta < 2) return OR_EINVAL;
    int st = OR_OK;
    int64_t tours = 0, inserts = 0, nodes = 0;
    double *mu = (double *)calloc((size_t)dd * dd, sizeof(double));
    double *r = (double *)calloc((size_t)dd * dd, sizeof(double));
    double *B = (double *)calloc((size_t)dd, sizeof(double));
    double *invB = (double *)calloc((size_t)dd, sizeof(double));
    int64_t *G = (int64_t *)calloc((size_t)dd * dd, sizeof(int64_t));
    int64_t *rows = (int64_t *)calloc((size_t)dd * dim, sizeof(int64_t));
    int32_t *u = (int32_t *)calloc((size_t)dd, sizeof(int32_t));
    int32_t *best = (int32_t *)calloc((size_t)dd, sizeof(int32_t));
    int64_t *a = (int64_t *)calloc((size_t)dd, sizeof(int64_t));
    if (!mu || !r || !B || !invB || !G || !rows || !u || !best || !a) { st = OR_ENOMEM; goto done; }
    for (int tour = 0; tour < max_tours; ++tour) {
        int inserted = 0;
        ++tours;
        for (int k = 0; k + 1 < dd; ++k) {
            const int h = (k + beta < dd) ? k + beta : dd;
            /* GSO of the current basis from the exact Gram matrix, in the
             * LLL's form (mu_ij = r_ij (1/B_j), R14) */
            for (int i = 0; i < dd; ++i)
                for (int j = 0; j <= i; ++j) {
                    int64_t g;
                    if ((st = dot_exact(b + (size_t)i * dim, b + (size_t)j * dim, dim, &g))) goto done;
                    G[(size_t)i * dd + j] = g;
                    G[(size_t)j * dd + i] = g;
                }
            for (int i = 0; i < dd; ++i) gso_row(i, dd, G, mu, r, B, invB);
            /* shortest nonzero vector of the projected block */
            svp_state e;
            memset(&e, 0, sizeof e);
            e.dd = dd; e.h = h; e.k = k; e.mu = mu; e.B = B;
            e.A = delta * B[k];
            e.u = u; e.best = best;
            memset(u, 0, sizeof(int32_t) * (size_t)dd);
            svp_level(&e, h - 1, 0.0);
            nodes += e.nodes;
            if (!e.found) continue;
            /* insertion by unimodular row steps (R14) */
            memcpy(rows, b + (size_t)k * dim, sizeof(int64_t) * (size_t)(h - k) * dim);
            for (int i = k; i < h; ++i) a[i - k] = best[i];
            for (int i = h - k - 1; i > 0; --i) {
                if (a[i] == 0) continue;
                int64_t *c0 = rows + (size_t)(i - 1) * dim, *c1 = rows + (size_t)i * dim;
                if (a[i - 1] == 0) {
                    for (int c = 0; c < dim; ++c) { int64_t t = c0[c]; c0[c] = c1[c]; c1[c] = t; }
                    a[i - 1] = a[i];
                    a[i] = 0;
                    continue;
                }
                int64_t sa, tb;
                const int64_t g = egcd64(a[i - 1], a[i], &sa, &tb);
                const int64_t p = a[i - 1] / g, q = a[i] / g;
                for (int c = 0; c < dim; ++c) {
                    const i128 v0 = (i128)p * c0[c] + (i128)q * c1[c];
                    const i128 v1 = -(i128)tb * c0[c] + (i128)sa * c1[c];
                    if (v0 >= OR_ENTRY_LIMIT || v0 <= -OR_ENTRY_LIMIT || v1 >= OR_ENTRY_LIMIT ||
                        v1 <= -OR_ENTRY_LIMIT) { st = OR_EOVERFLOW; goto done; }
                    c0[c] = (int64_t)v0;
                    c1[c] = (int64_t)v1;
                }
                a[i - 1] = g;
                a[i] = 0;
            }
            if (a[0] != 1 && a[0] != -1) continue;   /* not primitive: cannot be a basis vector */
            if (a[0] == -1) for (int c = 0; c < dim; ++c) rows[c] = -rows[c];
            memcpy(b + (size_t)k * dim, rows, sizeof(int64_t) * (size_t)(h - k) * dim);
            if ((st = lll_core(dd, dim, b, delta, 0.51, lll_max_iter, NULL, NULL, 1))) goto done;
            ++inserts;
            inserted = 1;
        }
        if (!inserted) break;
    }
done:
    if (tours_out) *tours_out = tours;
    if (inserts_out) *inserts_out = inserts;
    if (nodes_out) *nodes_out = nodes;
    free(mu); free(r); free(B); free(invB); free(G); free(rows); free(u); free(best); free(a);
    return st;
}

int oracle_enumerate(int dd, int dim, const double *mu, const double *B, const double *bhat,
                     const int32_t *kb, int m, int n, const int32_t *A, const int64_t *d,
                     const oracle_enum_opts *o, const int32_t *prefix_u,
                     uint8_t *sol, int64_t sol_cap,
                     int32_t *pre_u, double *pre_rho, int64_t pre_cap,
                     oracle_enum_stats *out)
{
    return oracle_enumerate_bounds(dd, dim, mu, B, bhat, kb, m, n, A, d, NULL, o, prefix_u, sol, sol_cap,
                                   pre_u, pre_rho, pre_cap, out);
}

/* Version tag so tests can check they loaded this file's build. */
int oracle_version(void) { return 1; }
