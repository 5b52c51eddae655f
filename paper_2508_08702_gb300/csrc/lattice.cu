// lattice.cu -- steps a1-a3 of the hot path on the device, one launch per
// step (the device functions are in reduce.cuh):
//   build_lattice_kernel   generator of Eq. (2) (Sec. 2)
//   permute_kernel         shuffled column orders of the replicas (Sec. 4)
//   lll_kernel             LLL reduction (Alg. 1 step 1), one warp per instance
//   extract_gso_kernel     kept vectors and Gram-Schmidt tables (Alg. 1 steps 2-3)
//   bkz_kernel             BKZ-beta of the kernel basis (Sec. 2), one warp per instance
//   prep_fixed_kernel      fixed-point tables of the walkers' Hoelder filter
#include "reduce.cuh"

namespace msp {

// Step a1: generator of Eq. (2) with bounds 0 <= x_j <= r_j: column 0 is
// (-N d, -r_max (n times), r_max), column j is (N a_j, 2 c_j e_j, 0).
__global__ void __launch_bounds__(128) build_lattice_kernel(Pools P, int64_t N) {
    InstDesc& I = P.inst[blockIdx.x];
    const int m = I.m, n = I.n, K = I.K, L = I.L;
    int64_t* b = P.basis + I.offBasis;
    const int32_t* A = P.A + I.offA;
    const int64_t* d = P.d + I.offd;
    const int32_t* r = P.r ? P.r + I.offR : nullptr;   // no bounds given: the binary problem
    const int64_t rmax = r ? I.rmax : 1;
    bool ovf = false;
    for (int e = threadIdx.x; e < K * L; e += blockDim.x) {
        const int k = e / L, c = e % L;
        __int128 v = 0;
        if (k == 0) {
            if (c < m) v = -(__int128)N * (__int128)d[c];
            else v = (c < m + n) ? -rmax : rmax;
        } else {
            if (c < m) v = (__int128)N * (__int128)A[(int64_t)c * n + (k - 1)];
            else if (c == m + (k - 1)) v = 2 * (r ? rmax / r[k - 1] : 1);   // 2 c_j, c_j = r_max / r_j
        }
        if (v >= kEntryLimit || v <= -kEntryLimit) ovf = true;
        b[e] = (int64_t)v;
    }
    if (ovf) set_status(I, ST_EOVERFLOW);
}

__global__ void __launch_bounds__(128) permute_kernel(Pools P, int32_t* perm, int32_t* rperm,
                                                      unsigned long long seed) {
    InstDesc& I = P.inst[blockIdx.x];
    const int m = I.m, n = I.n;
    int32_t* pi = perm + I.offR;
    __shared__ int32_t col[128];
    if (threadIdx.x == 0) {
        for (int j = 0; j < n; ++j) col[j] = j;
        if (I.replica > 0) {
            unsigned long long st = seed ^ ((unsigned long long)I.group << 32) ^ (unsigned long long)I.replica;
            for (int j = n - 1; j >= 1; --j) {
                const int k = (int)(splitmix64_next(st) % (unsigned long long)(j + 1));
                const int t = col[j]; col[j] = col[k]; col[k] = t;
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) pi[j] = col[j];
    if (I.replica == 0) return;
    // rows of A and the bounds, gathered through the permutation
    int32_t* A = const_cast<int32_t*>(P.A) + I.offA;
    int32_t* r = rperm + I.offR;
    __shared__ int32_t row[128];
    for (int i = 0; i < m; ++i) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = A[(int64_t)i * n + col[j]];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)i * n + j] = row[j];
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = r[col[j]];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) r[j] = row[j];
}

__global__ void __launch_bounds__(32) lll_kernel(Pools P, double delta, double eta, int64_t max_iter,
                                                 unsigned long long max_ns) {
    lll_inst(P, blockIdx.x, delta, eta, max_iter, max_ns);
}

__global__ void __launch_bounds__(32) extract_gso_kernel(Pools P, int gso_only) {
    extract_gso_inst(P, blockIdx.x, gso_only);
}

__global__ void __launch_bounds__(32) bkz_kernel(Pools P, BkzScratch S, int beta, double delta, int max_tours,
                                                 int64_t lll_max_iter, unsigned long long max_ns) {
    bkz_inst(P, blockIdx.x, S, beta, delta, max_tours, lll_max_iter, max_ns);
}

__global__ void __launch_bounds__(32) prep_fixed_kernel(Pools P, int use_eps, int dimPad) {
    prep_fixed_inst(P, blockIdx.x, use_eps, dimPad);
}

}  // namespace msp
