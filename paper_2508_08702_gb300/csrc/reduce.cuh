// reduce.cuh -- steps a1-a3 of the hot path as device functions: the
// lattice of Eq. (2), LLL (Alg. 1 step 1: exact int64 basis and Gram matrix,
// int128 products, FP64 Gram-Schmidt), the kept vectors with zero top rows
// and the Gram-Schmidt tables of Eq. (4) (Alg. 1 steps 2-3), BKZ of the kernel
// basis, and the fixed-point tables of the walkers' Hoelder filter.
// lattice.cu wraps them in one-warp-per-instance launches; enum.cu calls
// them from the fused launch, where warp 0 of a block prepares an instance
// before the block's warps join the walkers.
//
// One warp works on one instance: the reduction is a sequential loop over
// basis positions, so the parallelism is over coordinates / columns inside a
// step and over the instances of a batch.  Every floating-point operation
// is an explicit IEEE intrinsic (no contraction), in the fixed order:
//   r_kj = G_kj - sum_{i<j} mu_ji r_ki  (ascending i, one fma per term),
//   B_k = r_kk  (same fold with mu_ki); inside the reduction
//   mu_kj = r_kj * (1 / r_jj) with the reciprocal formed once per row, in
//   the enumeration tables mu_kj = r_kj / r_jj (Eq. (4) as written),
// size reduction of b_k against b_j in one pass j = k-1 .. 0 where
// |mu_kj| > eta, with q = rint(mu_kj), mu_ki <- fma(-q, mu_ji, mu_ki) (i < j),
// mu_kj <- mu_kj - q, then the Gram row of b_k recomputed exactly (the LLL
// inside BKZ redoes the row and repeats the pass until nothing changes);
// Lovasz: swap iff B_k < (delta - mu_{k,k-1}^2) B_{k-1}, each operation
// rounded.
#pragma once
#include "common.cuh"

namespace msp {

constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kEntryLimit = (int64_t)1 << 58;   // |entries| < 2^58: 128-bit dots cannot overflow

// Integer-pipe forms of FP64 steps of the block search (an FP64 instruction
// costs ~64 cycles on GB300), each exact for every input it sees there:
// int -> double for |v| < 2^31
__device__ __forceinline__ double svp_i2d(int v) {
    if (v == 0) return 0.0;
    const unsigned a = v < 0 ? (unsigned)(-v) : (unsigned)v;
    const int lz = __clz(a);
    const unsigned long long m = ((unsigned long long)a << (lz + 21)) & 0x000fffffffffffffULL;
    return __longlong_as_double((long long)(((unsigned long long)(v < 0) << 63) |
                                            ((unsigned long long)(1023 + 31 - lz) << 52) | m));
}

// a < b for a >= +0 (or NaN) and b > 0: the unsigned order of the bit patterns
// (a NaN compares not-less, as in FP64)
__device__ __forceinline__ bool svp_less(double a, double b) {
    return (unsigned long long)__double_as_longlong(a) < (unsigned long long)__double_as_longlong(b);
}

// c = -y rounded to nearest, ties to even (rint), and the side s = +1 if
// c >= rint(c) else -1; returns true when |rint(c)| > 1e9
__device__ __forceinline__ bool svp_round(double y, int& u1, int& s) {
    const unsigned long long c = (unsigned long long)__double_as_longlong(y) ^ 0x8000000000000000ULL;
    const bool neg = (c >> 63) != 0;
    const int e = (int)((c >> 52) & 0x7ff);
    const unsigned long long frac = c & 0x000fffffffffffffULL;
    if (e >= 1023 + 30) return true;   // |c| >= 2^30 (or inf, NaN): |rint(c)| > 1e9
    unsigned long long mag;
    bool up, exact;
    const int shift = 1075 - e;        // >= 22
    if (e == 0 || shift > 63) {        // |c| < 2^-11: rounds to 0
        mag = 0;
        up = false;
        exact = (e == 0 && frac == 0);
    } else {
        const unsigned long long m = frac | 0x0010000000000000ULL;
        const unsigned long long ip = m >> shift;
        const unsigned long long rem = m & ((1ULL << shift) - 1ULL);
        const unsigned long long half = 1ULL << (shift - 1);
        up = rem > half || (rem == half && (ip & 1ULL));
        exact = rem == 0;
        mag = ip + (up ? 1ULL : 0ULL);
    }
    if (mag > 1000000000ULL) return true;
    u1 = neg ? -(int)mag : (int)mag;
    s = neg ? ((up || exact) ? 1 : -1) : (up ? -1 : 1);
    return false;
}


// ---------------------------------------------------------------------------
// Replicas (Sec. 4: the input order shuffled at random, one search per
// order; the first to find a solution answers the instance).  Replica k > 0
// of an instance permutes its variables by Fisher-Yates, j = n-1 .. 1 swapping
// position j with position z mod (j+1), z the successive outputs of
// splitmix64 (Steele, Lea and Flood) started at seed ^ (group << 32) ^ k.
// perm[j] = the caller's column that becomes column j; A's columns and the
// bounds are permuted in place.  Replica 0 keeps the caller's order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64_next(unsigned long long& state) {
    unsigned long long z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}


__device__ __forceinline__ int64_t dot_exact(const int64_t* __restrict__ a, const int64_t* __restrict__ b,
                                             int L, bool& ovf) {
    __int128 s = 0;
    for (int c = 0; c < L; ++c) s += (__int128)a[c] * (__int128)b[c];
    if (s > (__int128)INT64_MAX || s < (__int128)INT64_MIN) ovf = true;
    return (int64_t)s;
}

// The same exact dot product when every entry is below 2^24 in magnitude
// (small != 0): 128 products of 48 bits sum below 2^55, so int64 is exact.
__device__ __forceinline__ int64_t dot_small(const int64_t* __restrict__ a, const int64_t* __restrict__ b, int L,
                                             bool small, bool& ovf) {
    if (!small || L > 128) return dot_exact(a, b, L, ovf);
    int64_t s = 0;
    for (int c = 0; c < L; ++c) s += a[c] * b[c];
    return s;
}

// warp-uniform: are all entries of rows [r0, r1) below 2^24 in magnitude?
__device__ __forceinline__ bool rows_small(const int64_t* __restrict__ b, int r0, int r1, int L) {
    bool ok = true;
    for (int e = (threadIdx.x & 31) + r0 * L; e < r1 * L; e += 32) ok &= (b[e] < (1 << 24) && b[e] > -(1 << 24));
    return __all_sync(kFull, ok);
}

__device__ __forceinline__ double pick4(const double (&a)[4], int q) {
    return q == 0 ? a[0] : q == 1 ? a[1] : q == 2 ? a[2] : a[3];
}

// Row k of the Gram-Schmidt data from the exact Gram matrix.  Lane l owns the
// columns j = l + 32 q (q < 4).  mu_at(j, i) returns mu_ji for j < k; it
// should read a layout where fixed i and consecutive j are adjacent (the
// lanes of a step then read one coalesced row).
// Results: rrow[i] = r_ki (when rrow is given), murow[i * mstride] = mu_ki
// (i < k), *Bk = r_kk.
// With invB (the reduction), mu_ki = r_ki * invB[i] and invB[k] = 1 / r_kk is
// stored; without it (Eq. (4) for the enumeration tables), mu_ki = r_ki / B[i].
template <class MuAt>
__device__ __forceinline__ void gso_row_warp(int k, const int64_t* __restrict__ Grow, MuAt mu_at,
                                             const double* __restrict__ B, double* rrow, double* murow,
                                             int mstride, double* Bk, int lane, double* invB = nullptr) {
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        acc[q] = (j <= k) ? __ll2double_rn(Grow[j]) : 0.0;
    }
    // column blocks q0 .. nq-1 hold the columns i < j <= k of a step: the
    // others are skipped by warp-uniform branches (an FP64 warp instruction
    // costs the same with no active lane as with 32)
    // (steps i of block qb broadcast from acc[qb]: the block index is a
    // compile-time constant, so no select sits on the serial chain)
    const int nq = (k >> 5) + 1;
#pragma unroll
    for (int qb = 0; qb < 4; ++qb) {
        if (qb >= nq) break;
        const int iend = min(k, 32 * qb + 32);
        for (int i = 32 * qb; i < iend; ++i) {
            const double rki = __shfl_sync(kFull, acc[qb], i & 31);
            const double muki = invB ? __dmul_rn(rki, invB[i]) : __ddiv_rn(rki, B[i]);
            const int q0 = (i + 1) >> 5;
#pragma unroll
            for (int q = qb; q < 4; ++q) {
                if (q >= q0 && q < nq) {
                    const int j = lane + 32 * q;
                    if (j > i && j <= k) acc[q] = __fma_rn(-(j < k ? mu_at(j, i) : muki), rki, acc[q]);
                }
            }
            if (lane == 0) {
                if (rrow) rrow[i] = rki;
                murow[(int64_t)i * mstride] = muki;
            }
        }
    }
    const double rkk = __shfl_sync(kFull, pick4(acc, k >> 5), k & 31);
    if (lane == 0) {
        if (rrow) rrow[k] = rkk;
        *Bk = rkk;
        if (invB) invB[k] = __ddiv_rn(1.0, rkk);
    }
    __syncwarp();
}

// delta-LLL of K vectors of length L (int64, vector-major, in place) by one
// warp: exact Gram matrix G (K x K), FP64 Gram-Schmidt rows recomputed from
// it (mu: K x K; invB, B: K), size reduction, Lovasz swaps.  Size reduction
// of row k: one pass j = k-1 .. 0 on its fresh Gram-Schmidt row, updated in
// place; lazy (the LLL inside BKZ) repeats the pass on a fresh row until
// nothing changes, so the stored rows of a finished run equal a fresh
// computation (which the restart below relies on).
// Returns a status; iterations and swaps are added to the counters.
//
// Restart (k0 > 0): G is the Gram matrix of the current basis and rows
// 0 .. k0-1 are an LLL fixed point whose Gram-Schmidt rows (mu, r, invB, B)
// are in place -- a run from scratch would pass them unchanged, so starting
// at k0 gives the same result.
static __device__ int32_t lll_warp(int64_t* __restrict__ b, int64_t* __restrict__ G, double* __restrict__ mu,
                            double* __restrict__ r, double* __restrict__ invB, double* __restrict__ B, int K, int L,
                            double delta, double eta, int64_t max_iter, unsigned long long deadline_ns,
                            int64_t& iters, int64_t& swaps, int k0 = 0, bool lazy = false) {
    const int lane = threadIdx.x & 31;
    // mu stored transposed: mu[i * K + j] = mu_ji (coalesced Gram-Schmidt rows)
    auto mu_at = [&](int j, int i) { return mu[(int64_t)i * K + j]; };
    (void)r;
    int32_t st = ST_OK;
    int64_t it = 0;
    bool small = rows_small(b, 0, K, L);
    if (k0 <= 0) {   // exact Gram matrix
        bool ovf = false;
        for (int e = lane; e < K * K; e += 32) {
            const int i = e / K, j = e % K;
            if (j <= i) {
                const int64_t g = dot_small(b + (int64_t)i * L, b + (int64_t)j * L, L, small, ovf);
                G[(int64_t)i * K + j] = g;
                G[(int64_t)j * K + i] = g;
            }
        }
        if (__any_sync(kFull, ovf)) st = ST_EOVERFLOW;
        __syncwarp();
        if (st == ST_OK) gso_row_warp(0, G, mu_at, B, nullptr, mu, K, &B[0], lane, invB);
    }

    int k = k0 > 1 ? k0 : 1;
    while (st == ST_OK && k < K) {
        if (++it > max_iter) { st = ST_ECAP; break; }
        if ((it & 255) == 0) {   // device-clock safety cap (uniform across the warp)
            const unsigned long long now = __shfl_sync(kFull, global_time_ns(), 0);
            if (now > deadline_ns) { st = ST_ECAP; break; }
        }
        // lazy size reduction of b_k
        for (int pass = 0;; ++pass) {
            if (pass > 1000) { st = ST_ECAP; break; }
            gso_row_warp(k, G + (int64_t)k * K, mu_at, B, nullptr, mu + k, K, &B[k], lane, invB);
            bool changed = false, ovf = false;
            // j = k-1 .. 0: the next j to reduce is the largest one at or
            // below jtop whose current |mu_kj| exceeds eta -- found for 32
            // columns at a time by a ballot (the values in between stay
            // below eta: only a reduction at a larger j changes them)
            const long long eta_bits = __double_as_longlong(eta);
            for (int jtop = k - 1; jtop >= 0;) {
                int j = -1;
                for (int base = jtop & ~31; base >= 0; base -= 32) {
                    const int jj = base + lane;
                    bool big = false;
                    if (jj <= jtop) {   // |mu| > eta on the bit pattern (no NaN passes, as in FP64)
                        const long long ab = __double_as_longlong(mu[(int64_t)jj * K + k]) & 0x7fffffffffffffffLL;
                        big = ab > eta_bits && ab <= 0x7ff0000000000000LL;
                    }
                    const unsigned bal = __ballot_sync(kFull, big);
                    if (bal) { j = base + 31 - __clz(bal); break; }
                }
                if (j < 0) break;
                jtop = j - 1;
                {
                    const double mkj = mu[(int64_t)j * K + k];
                    const double qd = rint(mkj);
                    if (fabs(qd) > 4503599627370496.0) { ovf = true; break; }
                    const int64_t q = (int64_t)qd;
                    for (int i = lane; i < j; i += 32)
                        mu[(int64_t)i * K + k] = __fma_rn(-qd, mu[(int64_t)i * K + j], mu[(int64_t)i * K + k]);
                    int64_t* bk = b + (int64_t)k * L;
                    const int64_t* bj = b + (int64_t)j * L;
                    for (int c = lane; c < L; c += 32) {
                        const __int128 v = (__int128)bk[c] - (__int128)q * (__int128)bj[c];
                        if (v >= kEntryLimit || v <= -kEntryLimit) ovf = true;
                        bk[c] = (int64_t)v;
                    }
                    __syncwarp();
                    if (lane == 0) mu[(int64_t)j * K + k] = __dsub_rn(mkj, qd);
                    __syncwarp();
                    changed = true;
                    if (__any_sync(kFull, ovf)) break;
                }
            }
            if (__any_sync(kFull, ovf)) { st = ST_EOVERFLOW; break; }
            if (!changed) break;
            small = small && rows_small(b, k, k + 1, L);
            for (int i = lane; i < K; i += 32) {
                const int64_t g = dot_small(b + (int64_t)k * L, b + (int64_t)i * L, L, small, ovf);
                G[(int64_t)k * K + i] = g;
                G[(int64_t)i * K + k] = g;
            }
            if (__any_sync(kFull, ovf)) { st = ST_EOVERFLOW; break; }
            __syncwarp();
            if (!lazy) break;   // one pass; the lazy variant re-checks a fresh row
        }
        if (st != ST_OK) break;
        // Lovasz condition
        const double mk = mu[(int64_t)(k - 1) * K + k];
        const double t1 = __dmul_rn(mk, mk);
        const double t2 = __dsub_rn(delta, t1);
        const double rhs = __dmul_rn(t2, B[k - 1]);
        if (B[k] < rhs) {
            int64_t* bk = b + (int64_t)k * L;
            int64_t* bm = b + (int64_t)(k - 1) * L;
            for (int c = lane; c < L; c += 32) {
                const int64_t t = bk[c]; bk[c] = bm[c]; bm[c] = t;
            }
            for (int i = lane; i < K; i += 32) {
                const int64_t t = G[(int64_t)k * K + i];
                G[(int64_t)k * K + i] = G[(int64_t)(k - 1) * K + i];
                G[(int64_t)(k - 1) * K + i] = t;
            }
            __syncwarp();
            for (int i = lane; i < K; i += 32) {
                const int64_t t = G[(int64_t)i * K + k];
                G[(int64_t)i * K + k] = G[(int64_t)i * K + (k - 1)];
                G[(int64_t)i * K + (k - 1)] = t;
            }
            __syncwarp();
            ++swaps;
            if (k - 1 == 0) gso_row_warp(0, G, mu_at, B, nullptr, mu, K, &B[0], lane, invB);
            k = (k > 1) ? k - 1 : 1;
        } else {
            ++k;
        }
    }
    iters += it;
    return st;
}

// Step a2: delta-LLL of the generator lattice, one warp per instance.
// The per-instance steps below are warp-level functions (a full warp calls
// them; lane = threadIdx.x mod 32): one warp per instance in their own
// launches, or warp 0 of a block of the fused enumeration launch.
static __device__ __noinline__ void lll_inst(const Pools& P, int inst, double delta, double eta, int64_t max_iter,
                                      unsigned long long max_ns) {
    InstDesc& I = P.inst[inst];
    if (I.status != ST_OK) return;
    const int K = I.K, L = I.L;
    double* mu = P.mu + I.offMu;
    int64_t iters = 0, swaps = 0;
    const int32_t st = lll_warp(P.basis + I.offBasis, P.gram + I.offGram, mu, mu + (int64_t)K * K,
                                mu + (int64_t)2 * K * K, P.Bl + I.offBl, K, L, delta, eta, max_iter,
                                __shfl_sync(kFull, global_time_ns(), 0) + max_ns, iters, swaps);
    if ((threadIdx.x & 31) == 0) {
        I.lll_iters = iters;
        I.lll_swaps = swaps;
        if (st != ST_OK) set_status(I, st);
    }
}


// rank of an r x c integer matrix modulo p = 2^31 - 1 (lane 0 only)
static __device__ int rank_mod_p(int64_t* M, int rows, int cols) {
    const int64_t p = 2147483647LL;
    for (int e = 0; e < rows * cols; ++e) M[e] = ((M[e] % p) + p) % p;
    int rank = 0;
    for (int c = 0; c < cols && rank < rows; ++c) {
        int piv = -1;
        for (int i = rank; i < rows; ++i) if (M[i * cols + c] != 0) { piv = i; break; }
        if (piv < 0) continue;
        for (int j = 0; j < cols; ++j) { int64_t t = M[rank * cols + j]; M[rank * cols + j] = M[piv * cols + j]; M[piv * cols + j] = t; }
        // inverse of the pivot by Fermat
        int64_t inv = 1, base = M[rank * cols + c], e = p - 2;
        while (e) { if (e & 1) inv = inv * base % p; base = base * base % p; e >>= 1; }
        for (int i = 0; i < rows; ++i) {
            if (i == rank || M[i * cols + c] == 0) continue;
            const int64_t f = M[i * cols + c] * inv % p;
            for (int j = 0; j < cols; ++j) M[i * cols + j] = ((M[i * cols + j] - f * M[rank * cols + j]) % p + p) % p;
        }
        ++rank;
    }
    return rank;
}

// Step a3: extraction and Gram-Schmidt of the kernel basis, one warp per
// instance.  gso_only: the kernel basis is already in place (after BKZ);
// only the Gram-Schmidt tables are recomputed.
static __device__ __noinline__ void extract_gso_inst(const Pools& P, int inst, int gso_only) {
    InstDesc& I = P.inst[inst];
    const int lane = threadIdx.x & 31;
    if (I.status != ST_OK) return;
    const int m = I.m, K = I.K, L = I.L, dim = I.n + 1;
    int32_t* kb = P.kb + I.offKb;
    int dd = I.dd;
    if (!gso_only) {
    const int64_t* b = P.basis + I.offBasis;
    // kept flags (vectors whose first m entries vanish), in reduced order
    unsigned kept_mask[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = lane + 32 * q;
        bool z = false;
        if (k < K) {
            z = true;
            for (int c = 0; c < m; ++c) if (b[(int64_t)k * L + c] != 0) { z = false; break; }
        }
        kept_mask[q] = __ballot_sync(kFull, z);
    }
    dd = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) dd += __popc(kept_mask[q]);
    const int mp = K - dd;   // vectors with a nonzero top part

    // The kept vectors span ker[A | -d] iff the top parts of the others are
    // linearly independent; rank modulo a prime is a lower bound of the
    // rational rank, so full rank mod p certifies independence.
    int32_t st = ST_OK;
    if (mp > m || mp > kMaxM) st = ST_ERANK;
    if (st == ST_OK && lane == 0 && mp > 0) {
        int64_t* M = P.gram + I.offGram;   // scratch: the Gram matrix is rebuilt below
        int r = 0;
        for (int k = 0; k < K; ++k) {
            if ((kept_mask[k >> 5] >> (k & 31)) & 1u) continue;
            for (int c = 0; c < m; ++c) M[r * m + c] = b[(int64_t)k * L + c];
            ++r;
        }
        if (rank_mod_p(M, mp, m) != mp) st = ST_ERANK;
    }
    st = __shfl_sync(kFull, st, 0);
    // copy the kept vectors without their top rows
    bool ovf = false;
    for (int k = 0; k < K && st == ST_OK; ++k) {
        if (!((kept_mask[k >> 5] >> (k & 31)) & 1u)) continue;
        int idx = 0;
        for (int q = 0; q < (k >> 5); ++q) idx += __popc(kept_mask[q]);
        idx += __popc(kept_mask[k >> 5] & ((1u << (k & 31)) - 1u));
        for (int c = lane; c < dim; c += 32) {
            const int64_t v = b[(int64_t)k * L + m + c];
            if (v >= (1 << 20) || v <= -(1 << 20)) ovf = true;
            kb[(int64_t)idx * dim + c] = (int32_t)v;
        }
    }
    if (__any_sync(kFull, ovf)) st = ST_EOVERFLOW;
    __syncwarp();
    if (st != ST_OK) {
        if (lane == 0) set_status(I, st);
        return;
    }
    }   // !gso_only
    // exact Gram matrix of the kernel basis (entries < 2^20 -> no overflow)
    int64_t* G = P.gram + I.offGram;
    for (int e = lane; e < dd * dd; e += 32) {
        const int i = e / dd, j = e % dd;
        int64_t s = 0;
        for (int c = 0; c < dim; ++c) s += (int64_t)kb[(int64_t)i * dim + c] * kb[(int64_t)j * dim + c];
        G[(int64_t)i * dd + j] = s;
    }
    __syncwarp();
    double* muT = P.muT + I.offMuT;   // muT[t][i] = mu_it, dd x dd
    double* Bt = P.B + I.offB;
    double* rrow = P.mu + I.offMu;    // scratch row
    double* murow = rrow + K;         // scratch row
    auto mu_at = [&](int j, int i) { return muT[(int64_t)i * dd + j]; };
    for (int i = 0; i < dd; ++i) {
        gso_row_warp(i, G + (int64_t)i * dd, mu_at, Bt, rrow, murow, 1, &Bt[i], lane);
        for (int j = lane; j < dd; j += 32)
            muT[(int64_t)j * dd + i] = (j < i) ? murow[j] : (j == i ? 1.0 : 0.0);
        __syncwarp();
    }
    // every ||bhat_t||^2 must be positive and finite, or the norm test of
    // the enumeration could never end a level
    bool bad = false;
    for (int i = lane; i < dd; i += 32) bad |= !(Bt[i] > 0.0 && Bt[i] < 1e300);
    if (__any_sync(kFull, bad)) {
        if (lane == 0) set_status(I, ST_EOVERFLOW);
        return;
    }
    // bhat_i = b_i - sum_{j<i} mu_ij bhat_j, per coordinate, ascending j
    double* bhat = P.bhat + I.offBhat;
    for (int i = 0; i < dd; ++i) {
        for (int c = lane; c < dim; c += 32) {
            double acc = (double)kb[(int64_t)i * dim + c];
            for (int j = 0; j < i; ++j)
                acc = __fma_rn(-muT[(int64_t)j * dd + i], bhat[(int64_t)j * dim + c], acc);
            bhat[(int64_t)i * dim + c] = acc;
        }
        __syncwarp();
    }
    if (lane == 0) { I.dd = dd; I.dim = dim; }
}


// ---------------------------------------------------------------------------
// BKZ-beta of the kernel basis (Sec. 2 offers block reduction as the
// alternative to LLL for step 1), one warp per instance, after extraction.  A tour visits the
// blocks [k, h), h = min(k + beta, dd), k = 0 .. dd-2: the Gram-Schmidt data
// of the whole basis is rebuilt (exact Gram matrix, Eq. (4) divided form),
// the block's shortest nonzero projected vector is searched by
// Schnorr-Euchner enumeration (lane 0; bound delta B_k, strict, shrunk to
// each improvement; zig-zag order and u >= 0 on all-zero top levels as in
// the main enumeration; no Hoelder test), and an improvement u is inserted
// by unimodular row steps -- from the last row of the block upwards, rows
// (c, c') with coefficients (a, b), g = gcd(a, b) = s a + t b, become
// ((a/g) c + (b/g) c', -t c + s c') -- after which the whole basis is
// LLL-reduced again.  Tours repeat until one inserts nothing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t egcd64(int64_t a, int64_t b, int64_t& sa, int64_t& tb) {
    int64_t r0 = a < 0 ? -a : a, r1 = b < 0 ? -b : b, s0 = 1, s1 = 0, t0 = 0, t1 = 1;
    while (r1 != 0) {
        const int64_t q = r0 / r1, r2 = r0 - q * r1, s2 = s0 - q * s1, t2 = t0 - q * t1;
        r0 = r1; r1 = r2; s0 = s1; s1 = s2; t0 = t1; t1 = t2;
    }
    sa = a < 0 ? -s0 : s0;
    tb = b < 0 ? -t0 : t0;
    return r0;
}

static __device__ __noinline__ void bkz_inst(const Pools& P, int inst, const BkzScratch& S, int beta, double delta, int max_tours,
                                      int64_t lll_max_iter, unsigned long long max_ns) {
    InstDesc& I = P.inst[inst];
    const int lane = threadIdx.x & 31;
    if (I.status != ST_OK) return;
    const int dd = I.dd, dim = I.dim, K = S.Kmax, D = S.dimMax;
    char* sp = S.base + (int64_t)inst * S.stride;
    int64_t* b = reinterpret_cast<int64_t*>(sp);                 // dd x dim
    int64_t* rows = b + (int64_t)K * D;                           // block copy
    int64_t* G = rows + (int64_t)K * D;                           // dd x dd, exact Gram of b
    double* mu2 = reinterpret_cast<double*>(G + (int64_t)K * K);  // Gram-Schmidt rows, LLL's form, transposed
    double* r2 = mu2 + (int64_t)K * K;                            // (unused by the reciprocal form)
    double* invB2 = r2 + (int64_t)K * K;
    double* B2 = invB2 + K;
    double* yv = B2 + K;                                          // SVP: centre per level
    double* rhoP = yv + K;                                        // SVP: parent norm per level
    int64_t* a = reinterpret_cast<int64_t*>(rhoP + K);            // insertion coefficients
    int32_t* u = reinterpret_cast<int32_t*>(a + K);
    int32_t* best = u + K;
    int32_t* u1v = best + K;
    int32_t* ziv = u1v + K;
    int32_t* flg = ziv + K;                                       // bit 0 zero prefix, bit 1 negative side
    int32_t* kb = P.kb + I.offKb;
    const unsigned long long deadline = __shfl_sync(kFull, global_time_ns(), 0) + max_ns;   // uniform

    for (int e = lane; e < dd * dim; e += 32) b[e] = kb[e];
    __syncwarp();
    int32_t st = ST_OK;
    int64_t tours = 0, inserts = 0, nodes = 0, iters = 0, swaps = 0;
    bool small = rows_small(b, 0, dd, dim);
    {   // exact Gram matrix; kept up to date row by row below
        bool ovf = false;
        for (int e = lane; e < dd * dd; e += 32) {
            const int i = e / dd, j = e % dd;
            if (j <= i) {
                const int64_t g = dot_small(b + (int64_t)i * dim, b + (int64_t)j * dim, dim, small, ovf);
                G[(int64_t)i * dd + j] = g;
                G[(int64_t)j * dd + i] = g;
            }
        }
        if (__any_sync(kFull, ovf)) st = ST_EOVERFLOW;
        __syncwarp();
    }
    // Gram-Schmidt rows of the whole basis in the LLL's form (mu2, invB2, B2;
    // mu2 transposed): fresh here, and kept fresh by the LLL runs below (the
    // lazy LLL leaves every row as a fresh computation from the Gram matrix)
    auto mu2_at = [&](int j, int i) { return mu2[(int64_t)i * dd + j]; };
    if (st == ST_OK)
        for (int i = 0; i < dd; ++i)
            gso_row_warp(i, G + (int64_t)i * dd, mu2_at, B2, nullptr, mu2 + i, dd, &B2[i], lane, invB2);
    bool lll_state = false;  // b is an LLL fixed point (a first LLL run has happened)
    for (int tour = 0; tour < max_tours && st == ST_OK; ++tour) {
        ++tours;
        bool inserted = false;
        for (int k = 0; k + 1 < dd && st == ST_OK; ++k) {
            const int h = min(k + beta, dd);
            {
                bool badB = false;   // a level with B_t <= 0 would never end its zig-zag
                for (int i = lane; i < dd; i += 32) badB |= !(B2[i] > 0.0 && B2[i] < 1e300);
                if (__any_sync(kFull, badB)) { st = ST_EOVERFLOW; break; }
            }
            // shortest nonzero vector of the projected block (lane 0)
            int found = 0;
            if (lane == 0) {
                double A = __dmul_rn(delta, B2[k]);
                for (int i = 0; i < dd; ++i) u[i] = 0;
                int t = h - 1;
                rhoP[t] = 0.0;
                bool enter = true;
                long long nloc = 0;
                for (;;) {
                    int cur;
                    if (enter) {
                        // zero prefix above t: the parent's flag and its current value
                        const bool zp = (t == h - 1) || ((flg[t + 1] & 1) && u[t + 1] == 0);
                        double acc = 0.0;
                        for (int i = h - 1; i > t; --i) acc = __fma_rn(svp_i2d(u[i]), mu2[(int64_t)t * dd + i], acc);
                        yv[t] = acc;
                        int uu = 0, sgn = 1;   // rint(-acc) and its side
                        if (svp_round(acc, uu, sgn)) { st = ST_EOVERFLOW; break; }
                        if (zp) uu = 0;
                        u1v[t] = uu;
                        ziv[t] = 1;
                        flg[t] = (zp ? 1 : 0) | (sgn < 0 ? 2 : 0);
                        cur = uu;
                        enter = false;
                    } else {
                        // next value of level t
                        u[t] = 0;
                        if (flg[t] & 1) {
                            cur = u1v[t] + ziv[t];   // 0, 1, 2, ... (zi counts the steps)
                            ++ziv[t];
                        } else {
                            const int zi = ++ziv[t];
                            const int sgn = (flg[t] & 2) ? -1 : 1;
                            cur = (zi % 2 == 0) ? u1v[t] + sgn * (zi / 2) : u1v[t] - sgn * ((zi - 1) / 2);
                        }
                    }
                    const double x = __dadd_rn(svp_i2d(cur), yv[t]);
                    const double rho = __fma_rn(__dmul_rn(x, x), B2[t], rhoP[t]);   // >= +0 (B_t > 0)
                    ++nloc;
                    if ((nloc & 4095) == 0 && global_time_ns() > deadline) { st = ST_ECAP; break; }
                    if (!svp_less(rho, A)) {   // level exhausted: back to the parent
                        u[t] = 0;
                        if (t == h - 1) break;
                        ++t;
                        continue;
                    }
                    u[t] = cur;
                    if (t == k) {
                        if (!((flg[t] & 1) && cur == 0)) {
                            A = rho;
                            for (int i = k; i < h; ++i) best[i] = u[i];
                            found = 1;
                        }
                    } else {
                        rhoP[t - 1] = rho;
                        --t;
                        enter = true;
                    }
                }
                nodes += nloc;
            }
            st = __shfl_sync(kFull, st, 0);
            found = __shfl_sync(kFull, found, 0);
            if (st != ST_OK || !found) continue;
            // insertion by unimodular row steps
            const int nb = h - k;
            for (int e = lane; e < nb * dim; e += 32) rows[e] = b[(int64_t)k * dim + e];
            if (lane == 0) for (int i = 0; i < nb; ++i) a[i] = best[k + i];
            __syncwarp();
            bool bad = false;
            for (int i = nb - 1; i > 0; --i) {
                const int64_t ai = a[i], am = a[i - 1];
                if (ai == 0) continue;
                int64_t* c0 = rows + (int64_t)(i - 1) * dim;
                int64_t* c1 = rows + (int64_t)i * dim;
                if (am == 0) {
                    for (int c = lane; c < dim; c += 32) { const int64_t t0 = c0[c]; c0[c] = c1[c]; c1[c] = t0; }
                    __syncwarp();
                    if (lane == 0) { a[i - 1] = ai; a[i] = 0; }
                    __syncwarp();
                    continue;
                }
                int64_t sa, tb;
                const int64_t g = egcd64(am, ai, sa, tb);
                const int64_t p = am / g, q = ai / g;
                for (int c = lane; c < dim; c += 32) {
                    const __int128 v0 = (__int128)p * c0[c] + (__int128)q * c1[c];
                    const __int128 v1 = -(__int128)tb * c0[c] + (__int128)sa * c1[c];
                    if (v0 >= kEntryLimit || v0 <= -kEntryLimit || v1 >= kEntryLimit || v1 <= -kEntryLimit) bad = true;
                    c0[c] = (int64_t)v0;
                    c1[c] = (int64_t)v1;
                }
                __syncwarp();
                if (lane == 0) { a[i - 1] = g; a[i] = 0; }
                __syncwarp();
            }
            if (__any_sync(kFull, bad)) { st = ST_EOVERFLOW; break; }
            const int64_t a0 = a[0];
            if (a0 != 1 && a0 != -1) continue;   // not primitive (cannot happen for a shortest vector)
            for (int e = lane; e < nb * dim; e += 32)
                b[(int64_t)k * dim + e] = (a0 == -1 && e < dim) ? -rows[e] : rows[e];
            __syncwarp();
            // Gram rows of the replaced block
            small = small && rows_small(b, k, h, dim);
            bool ovf = false;
            for (int e = lane; e < nb * dd; e += 32) {
                const int i = k + e / dd, j = e % dd;
                const int64_t gv = dot_small(b + (int64_t)i * dim, b + (int64_t)j * dim, dim, small, ovf);
                G[(int64_t)i * dd + j] = gv;
                G[(int64_t)j * dd + i] = gv;
            }
            if (__any_sync(kFull, ovf)) { st = ST_EOVERFLOW; break; }
            __syncwarp();
            // LLL of the whole basis: once a first run has made the basis an
            // LLL fixed point, the rows above k are untouched, so later runs
            // restart at k
            st = lll_warp(b, G, mu2, r2, invB2, B2, dd, dim, delta, 0.51, lll_max_iter, deadline, iters, swaps,
                          lll_state ? k : 0, true);
            lll_state = true;
            small = rows_small(b, 0, dd, dim);
            ++inserts;
            inserted = true;
        }
        if (!inserted) break;
    }
    // back to the int32 kernel basis (the enumeration's entries stay below 2^20)
    bool ovf = false;
    for (int e = lane; e < dd * dim && st == ST_OK; e += 32) {
        if (b[e] >= (1 << 20) || b[e] <= -(1 << 20)) ovf = true;
        else kb[e] = (int32_t)b[e];
    }
    if (__any_sync(kFull, ovf) && st == ST_OK) st = ST_EOVERFLOW;
    if (lane == 0) {
        I.bkz_tours = tours;
        I.bkz_inserts = inserts;
        I.bkz_nodes = nodes;
        if (st != ST_OK) set_status(I, st);
    }
}


// Fixed-point parameters of the exact integer filter used by the walkers
// for the Hoelder test (one warp per instance, after extract_gso_kernel):
//   sx: |x| <= sqrt((R + eps) / B_t) on every node that passes the norm test,
//       so trunc(x 2^sx) fits in 31 bits;
//   sb: |bhat_tc| <= sqrt(B_t), so round(bhat 2^sb) fits in 31 bits;
//   sx + sb <= 50, and with R = (n+1) r_max^2 and ||w||_1 <= (n+1) r_max + 1
//   on passing nodes: ||w||_1 2^(sx+sb-27) < 2^31 (the walkers' int32 sum),
//   r_max ||w||_1 2^(sx+sb) < 2^62 and (R + eps) 2^(sx+sb) < 2^62.
__device__ __forceinline__ int ceil_log2(double v) {
    int e;
    const double f = frexp(v, &e);   // v = f 2^e, 0.5 <= f < 1
    return (f == 0.5) ? e - 1 : e;
}

static __device__ __noinline__ void prep_fixed_inst(const Pools& P, int inst, int use_eps, int dimPad) {
    InstDesc& I = P.inst[inst];
    const int lane = threadIdx.x & 31;
    if (I.status != ST_OK) return;
    const int dd = I.dd, dim = I.dim;
    const double* Bt = P.B + I.offB;
    const double* bhat = P.bhat + I.offBhat;
    const double R = (double)dim * (double)I.rmax * (double)I.rmax;
    const double Rb = R + (use_eps ? R * 0x1p-20 : 0.0);
    double xm = 0.0, bm = 0.0;
    for (int t = lane; t < dd; t += 32) xm = fmax(xm, sqrt(Rb / Bt[t]));
    for (int e = lane; e < dd * dim; e += 32) bm = fmax(bm, fabs(bhat[e]));
    for (int off = 16; off >= 1; off >>= 1) {
        xm = fmax(xm, __shfl_xor_sync(kFull, xm, off));
        bm = fmax(bm, __shfl_xor_sync(kFull, bm, off));
    }
    int ex, eb;
    frexp(xm * 1.0001 + 1.0, &ex);   // xm < 2^ex
    frexp(bm * 1.0001 + 1.0, &eb);
    int sx = min(25, 30 - ex), sb = min(25, 30 - eb);
    {   // caps of the sums (binary problems with n + 1 <= 128 stay at 50)
        const double l1max = (double)dim * (double)I.rmax + 1.0;
        int smax = 58 - ceil_log2(l1max);
        smax = min(smax, 62 - ceil_log2(l1max * (double)I.rmax));
        smax = min(smax, 62 - ceil_log2(Rb + 1.0));
        if (sx + sb > smax) sb = max(8, smax - sx);
        if (sx + sb > smax) sx = smax - sb;
    }
    if (sx < 8 || sb < 8 || sx + sb < 20) {   // values too large for a useful filter
        if (lane == 0) set_status(I, ST_EOVERFLOW);
        return;
    }
    int32_t* bq = P.bq + I.offBq;
    int64_t* nbq = P.nbq + I.offNbq;
    const double scale = ldexp(1.0, sb);
    for (int t = 0; t < dd; ++t) {
        long long s = 0;
        for (int c = lane; c < dimPad; c += 32) {
            const int v = (c < dim) ? __double2int_rn(bhat[(int64_t)t * dim + c] * scale) : 0;
            bq[(int64_t)t * dimPad + c] = v;
            s += (v < 0) ? -(long long)v : (long long)v;
        }
        for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
        if (lane == 0) nbq[t] = s;
    }
    if (lane == 0) { I.sx = sx; I.sb = sb; }
}


}  // namespace msp
