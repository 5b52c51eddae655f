// lattice.cu -- steps a1-a3 of the hot path on the device:
//   build_lattice_kernel   generator of Eq. (2), binary bounds (Sec. 2)
//   lll_kernel             LLL reduction (Alg. 1 step 1): exact int64 basis and
//                          Gram matrix (int128 products), FP64 Gram-Schmidt
//   extract_gso_kernel     kept vectors with zero top rows (Alg. 1 step 2) and
//                          the Gram-Schmidt tables of Eq. (4) (Alg. 1 step 3)
//
// One warp works on one instance: the reduction is a sequential loop over
// basis positions, so the parallelism is over coordinates / columns inside a
// step and over the instances of a batch.  Every floating-point operation
// is an explicit IEEE intrinsic (no contraction), in the fixed order:
//   r_kj = G_kj - sum_{i<j} mu_ji r_ki  (ascending i, one fma per term),
//   mu_kj = r_kj / r_jj,  B_k = r_kk  (same fold with mu_ki),
// size reduction of b_k against b_j for j = k-1 .. 0 while |mu_kj| > eta,
// with q = rint(mu_kj), mu_ki <- fma(-q, mu_ji, mu_ki) (i < j), mu_kj <- mu_kj - q,
// then the Gram row of b_k recomputed exactly and the row redone; Lovasz:
// swap iff B_k < (delta - mu_{k,k-1}^2) B_{k-1}, each operation rounded.
#include "common.cuh"

namespace msp {

constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kEntryLimit = (int64_t)1 << 58;   // |entries| < 2^58: 128-bit dots cannot overflow

__global__ void __launch_bounds__(128) build_lattice_kernel(Pools P, int64_t N) {
    InstDesc& I = P.inst[blockIdx.x];
    const int m = I.m, n = I.n, K = I.K, L = I.L;
    int64_t* b = P.basis + I.offBasis;
    const int32_t* A = P.A + I.offA;
    const int64_t* d = P.d + I.offd;
    bool ovf = false;
    for (int e = threadIdx.x; e < K * L; e += blockDim.x) {
        const int k = e / L, c = e % L;
        __int128 v = 0;
        if (k == 0) {
            if (c < m) v = -(__int128)N * (__int128)d[c];
            else v = (c < m + n) ? -1 : 1;
        } else {
            if (c < m) v = (__int128)N * (__int128)A[(int64_t)c * n + (k - 1)];
            else if (c == m + (k - 1)) v = 2;
        }
        if (v >= kEntryLimit || v <= -kEntryLimit) ovf = true;
        b[e] = (int64_t)v;
    }
    if (ovf) set_status(I, ST_EOVERFLOW);
}

__device__ __forceinline__ int64_t dot_exact(const int64_t* __restrict__ a, const int64_t* __restrict__ b,
                                             int L, bool& ovf) {
    __int128 s = 0;
    for (int c = 0; c < L; ++c) s += (__int128)a[c] * (__int128)b[c];
    if (s > (__int128)INT64_MAX || s < (__int128)INT64_MIN) ovf = true;
    return (int64_t)s;
}

__device__ __forceinline__ double pick4(const double (&a)[4], int q) {
    return q == 0 ? a[0] : q == 1 ? a[1] : q == 2 ? a[2] : a[3];
}

// Row k of the Gram-Schmidt data from the exact Gram matrix.  Lane l owns the
// columns j = l + 32 q (q < 4).  mu_at(j, i) returns mu_ji for j < k.
// Results: rrow[i] = r_ki, murow[i] = mu_ki (i < k), *Bk = r_kk.
// With invB (the reduction), mu_ki = r_ki * invB[i] and invB[k] = 1 / r_kk is
// stored; without it (Eq. (4) for the enumeration tables), mu_ki = r_ki / B[i].
template <class MuAt>
__device__ __forceinline__ void gso_row_warp(int k, const int64_t* __restrict__ Grow, MuAt mu_at,
                                             const double* __restrict__ B, double* rrow, double* murow,
                                             double* Bk, int lane, double* invB = nullptr) {
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        acc[q] = (j <= k) ? __ll2double_rn(Grow[j]) : 0.0;
    }
    for (int i = 0; i < k; ++i) {
        const double rki = __shfl_sync(kFull, pick4(acc, i >> 5), i & 31);
        const double muki = invB ? __dmul_rn(rki, invB[i]) : __ddiv_rn(rki, B[i]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            if (j > i && j < k) acc[q] = __fma_rn(-mu_at(j, i), rki, acc[q]);
            else if (j == k) acc[q] = __fma_rn(-muki, rki, acc[q]);
        }
        if (lane == 0) {
            if (rrow) rrow[i] = rki;
            murow[i] = muki;
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

// Step a2: delta-LLL, one warp per instance (blockDim.x == 32).
__global__ void __launch_bounds__(32) lll_kernel(Pools P, double delta, double eta, int64_t max_iter,
                                                 unsigned long long max_ns) {
    InstDesc& I = P.inst[blockIdx.x];
    const int lane = threadIdx.x;
    if (I.status != ST_OK) return;
    const unsigned long long t_start = global_time_ns();
    const int K = I.K, L = I.L;
    int64_t* b = P.basis + I.offBasis;
    int64_t* G = P.gram + I.offGram;
    double* mu = P.mu + I.offMu;
    double* r = mu + (int64_t)K * K;
    double* invB = r + (int64_t)K * K;
    double* B = P.Bl + I.offBl;
    auto mu_at = [&](int j, int i) { return mu[(int64_t)j * K + i]; };
    int32_t st = ST_OK;
    int64_t iters = 0, swaps = 0;

    // exact Gram matrix
    {
        bool ovf = false;
        for (int e = lane; e < K * K; e += 32) {
            const int i = e / K, j = e % K;
            if (j <= i) {
                const int64_t g = dot_exact(b + (int64_t)i * L, b + (int64_t)j * L, L, ovf);
                G[(int64_t)i * K + j] = g;
                G[(int64_t)j * K + i] = g;
            }
        }
        if (__any_sync(kFull, ovf)) st = ST_EOVERFLOW;
        __syncwarp();
    }
    if (st == ST_OK) gso_row_warp(0, G, mu_at, B, r, mu, &B[0], lane, invB);

    int k = 1;
    while (st == ST_OK && k < K) {
        if (++iters > max_iter) { st = ST_ECAP; break; }
        if ((iters & 255) == 0) {   // device-clock safety cap (uniform across the warp)
            const unsigned long long now = __shfl_sync(kFull, global_time_ns(), 0);
            if (now - t_start > max_ns) { st = ST_ECAP; break; }
        }
        // lazy size reduction of b_k
        for (int pass = 0;; ++pass) {
            if (pass > 1000) { st = ST_ECAP; break; }
            gso_row_warp(k, G + (int64_t)k * K, mu_at, B, r + (int64_t)k * K, mu + (int64_t)k * K, &B[k], lane,
                         invB);
            bool changed = false, ovf = false;
            for (int j = k - 1; j >= 0; --j) {
                const double mkj = mu[(int64_t)k * K + j];
                if (fabs(mkj) > eta) {
                    const double qd = rint(mkj);
                    if (fabs(qd) > 4503599627370496.0) { ovf = true; break; }
                    const int64_t q = (int64_t)qd;
                    for (int i = lane; i < j; i += 32)
                        mu[(int64_t)k * K + i] = __fma_rn(-qd, mu[(int64_t)j * K + i], mu[(int64_t)k * K + i]);
                    int64_t* bk = b + (int64_t)k * L;
                    const int64_t* bj = b + (int64_t)j * L;
                    for (int c = lane; c < L; c += 32) {
                        const __int128 v = (__int128)bk[c] - (__int128)q * (__int128)bj[c];
                        if (v >= kEntryLimit || v <= -kEntryLimit) ovf = true;
                        bk[c] = (int64_t)v;
                    }
                    __syncwarp();
                    if (lane == 0) mu[(int64_t)k * K + j] = __dsub_rn(mkj, qd);
                    __syncwarp();
                    changed = true;
                    if (__any_sync(kFull, ovf)) break;
                }
            }
            if (__any_sync(kFull, ovf)) { st = ST_EOVERFLOW; break; }
            if (!changed) break;
            for (int i = lane; i < K; i += 32) {
                const int64_t g = dot_exact(b + (int64_t)k * L, b + (int64_t)i * L, L, ovf);
                G[(int64_t)k * K + i] = g;
                G[(int64_t)i * K + k] = g;
            }
            if (__any_sync(kFull, ovf)) { st = ST_EOVERFLOW; break; }
            __syncwarp();
        }
        if (st != ST_OK) break;
        // Lovasz condition
        const double mk = mu[(int64_t)k * K + (k - 1)];
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
            if (k - 1 == 0) gso_row_warp(0, G, mu_at, B, r, mu, &B[0], lane, invB);
            k = (k > 1) ? k - 1 : 1;
        } else {
            ++k;
        }
    }
    if (lane == 0) {
        I.lll_iters = iters;
        I.lll_swaps = swaps;
        if (st != ST_OK) set_status(I, st);
    }
}

// rank of an r x c integer matrix modulo p = 2^31 - 1 (lane 0 only)
__device__ int rank_mod_p(int64_t* M, int rows, int cols) {
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

// Step a3: extraction and Gram-Schmidt of the kernel basis, one warp per instance.
__global__ void __launch_bounds__(32) extract_gso_kernel(Pools P) {
    InstDesc& I = P.inst[blockIdx.x];
    const int lane = threadIdx.x;
    if (I.status != ST_OK) return;
    const int m = I.m, K = I.K, L = I.L, dim = I.n + 1;
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
    int dd = 0;
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
    int32_t* kb = P.kb + I.offKb;
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
        gso_row_warp(i, G + (int64_t)i * dd, mu_at, Bt, rrow, murow, &Bt[i], lane);
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

// Fixed-point parameters of the exact integer filter used by the walkers
// for the Hoelder test (one warp per instance, after extract_gso_kernel):
//   sx: |x| <= sqrt((R + eps) / B_t) on every node that passes the norm test,
//       so trunc(x 2^sx) fits in 31 bits;
//   sb: |bhat_tc| <= sqrt(B_t), so round(bhat 2^sb) fits in 31 bits;
//   sx + sb <= 50 keeps |w|_1 2^(sx+sb) <= sqrt(n+1) |w|_2 2^50 inside int64.
__global__ void __launch_bounds__(32) prep_fixed_kernel(Pools P, int use_eps, int dimPad) {
    InstDesc& I = P.inst[blockIdx.x];
    const int lane = threadIdx.x;
    if (I.status != ST_OK) return;
    const int dd = I.dd, dim = I.dim;
    const double* Bt = P.B + I.offB;
    const double* bhat = P.bhat + I.offBhat;
    const double Rb = (double)dim + (use_eps ? (double)dim * 0x1p-20 : 0.0);
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
    const int sx = min(25, 30 - ex), sb = min(25, 30 - eb);
    if (sx < 8 || sb < 8) {          // values too large for a useful filter
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
