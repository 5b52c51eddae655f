// learn.cu -- the order in which the walkers take the subtrees (prefixes).
//
// features_kernel   32 features per prefix (shape of its projected vector,
//                   depth, the limited-discrepancy count of its path
//                   (Sec. 2.1), a Gaussian-heuristic size estimate of the
//                   subtree, the ||bhat||^2 profile of the levels below)
// score_keys_kernel the scorer's outputs -> sort keys
// bitonic_*         device sort of (key, value) pairs
// The first-solution mode interleaves the instances of a batch by rank, so
// every instance gets walkers at once; within an instance the rank is the
// depth-first position (plain order) or the scorer's priority (learned order).
// The order never changes which nodes are evaluated in the all-solutions
// mode, only when.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace msp {

constexpr int kFeat = 32;

// per instance: sum of log B_i below the split and 16 buckets of mean log(B_i / R)
__global__ void __launch_bounds__(32) profile_kernel(Pools P, float* prof) {
    const InstDesc& I = P.inst[blockIdx.x];
    float* out = prof + (int64_t)blockIdx.x * 17;
    const int lane = threadIdx.x;
    if (I.status != ST_OK || I.nprefix == 0) {
        for (int e = lane; e < 17; e += 32) out[e] = 0.f;
        return;
    }
    const int sl = I.split_level;
    const double* Bt = P.B + I.offB;
    const float R = (float)I.dim * (float)I.rmax * (float)I.rmax;
    float s = 0.f;
    for (int i = lane; i < sl; i += 32) s += logf((float)Bt[i]);
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[0] = s;
    if (lane < 16) {
        const int lo = lane * sl / 16, hi = (lane + 1) * sl / 16;
        float a = 0.f;
        for (int i = lo; i < hi; ++i) a += logf((float)Bt[i] / R);
        out[1 + lane] = hi > lo ? a / (float)(hi - lo) : 0.f;
    }
}

__device__ __forceinline__ int instance_of(const Pools& P, int64_t gid) {
    int lo = 0, hi = P.count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P.qbase[mid] <= gid) lo = mid; else hi = mid;
    }
    return lo;
}

// features of prefix gid (queue position before any reordering)
__global__ void features_kernel(Pools P, const float* __restrict__ prof, float* __restrict__ feat) {
    const int64_t total = P.qbase[P.count];
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int inst = instance_of(P, gid);
        const InstDesc& I = P.inst[inst];
        const int64_t j = gid - P.qbase[inst];
        const int64_t fo = frontier_index(P, inst, I.front_sel, j);
        const int dd = I.dd, dim = I.dim, sl = I.split_level, k = dd - sl;
        const float R = (float)dim * (float)I.rmax * (float)I.rmax;   // (n+1) r_max^2
        const float rho = (float)P.frho[fo];
        const double* w = P.fw + fo * P.dimPad;
        float l1 = 0.f, linf = 0.f, big = 0.f;
        for (int c = 0; c < dim; ++c) {
            const float a = fabsf((float)w[c]);
            l1 += a;
            linf = fmaxf(linf, a);
            big += a > 1.f ? 1.f : 0.f;
        }
        const float* pr = prof + (int64_t)inst * 17;
        const float rem = fmaxf(R - rho, 1e-6f);
        const float half = 0.5f * (float)sl;
        // log of the Gaussian-heuristic number of lattice points of the subtree
        const float logv = half * logf(3.14159265f * rem) - lgammaf(half + 1.f) - 0.5f * pr[0];
        float f[kFeat];
        f[0] = rho / R;
        f[1] = (l1 - rho) / R;
        f[2] = linf;
        f[3] = big / (float)dim;
        f[4] = (float)sl / (float)dd;
        f[5] = k > 0 ? (float)P.fdisc[fo] / (float)k : 0.f;
        f[6] = k > 0 ? P.fxsum[fo] / (float)k : 0.f;
        f[7] = logv / 16.f;
        f[8] = (float)I.m / (float)I.n;
        f[9] = log2f((float)I.nprefix + 1.f) / 20.f;
        f[10] = (float)j / (float)(I.nprefix > 0 ? I.nprefix : 1);
        f[11] = logf(rem) / 4.f;
#pragma unroll
        for (int b = 0; b < 16; ++b) f[12 + b] = pr[1 + b] / 4.f;
#pragma unroll
        for (int b = 28; b < kFeat; ++b) f[b] = 0.f;
        float* out = feat + gid * kFeat;
#pragma unroll
        for (int b = 0; b < kFeat; ++b) out[b] = f[b];
    }
}

__device__ __forceinline__ uint32_t ordered_bits(float x) {   // monotone float -> uint32
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// stage 1 (learned): key = (instance, descending priority), value = gid.
// priority = the scorer's logit of P(the subtree holds a solution); its
// node-count output is an auxiliary training target and does not enter the
// order (discounting by the predicted size found the solution later)
__global__ void score_keys_kernel(Pools P, const float* __restrict__ y, int64_t npad, unsigned long long* keys,
                                  unsigned long long* vals) {
    const int64_t total = P.qbase[P.count];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < total) {
            const int inst = instance_of(P, i);
            const float pri = y[i * 8];
            keys[i] = ((unsigned long long)inst << 32) | (unsigned long long)(~ordered_bits(pri));
            vals[i] = (unsigned long long)i;
        } else {
            keys[i] = ~0ULL;
            vals[i] = ~0ULL;
        }
    }
}

// stage 2: key = (rank within instance, instance), value = gid.  With a
// stage-1 result (sorted), rank = position - qbase[inst]; without one, rank =
// the depth-first position.
__global__ void rank_keys_kernel(Pools P, int64_t npad, const unsigned long long* s1vals, unsigned long long* keys,
                                 unsigned long long* vals) {
    const int64_t total = P.qbase[P.count];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < total) {
            const int64_t gid = s1vals ? (int64_t)s1vals[i] : i;
            const int inst = instance_of(P, i);   // positions keep the instance blocks
            const int64_t rank = i - P.qbase[inst];
            keys[i] = ((unsigned long long)rank << 20) | (unsigned long long)inst;
            vals[i] = (unsigned long long)gid;
        } else {
            keys[i] = ~0ULL;
            vals[i] = ~0ULL;
        }
    }
}

__global__ void bitonic_step_kernel(unsigned long long* keys, unsigned long long* vals, int64_t n, int64_t j,
                                    int64_t k) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i ^ j;
        if (l <= i) continue;
        const bool asc = (i & k) == 0;
        const unsigned long long ki = keys[i], kl = keys[l], vi = vals[i], vl = vals[l];
        const bool gt = ki > kl || (ki == kl && vi > vl);
        if (gt == asc) {
            keys[i] = kl; keys[l] = ki;
            vals[i] = vl; vals[l] = vi;
        }
    }
}

__global__ void copy_perm_kernel(Pools P, const unsigned long long* vals, int64_t* perm) {
    const int64_t total = P.qbase[P.count];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int64_t)vals[i];
}

static cudaError_t bitonic_sort(unsigned long long* keys, unsigned long long* vals, int64_t npad, cudaStream_t st,
                                int64_t* launches) {
    const int threads = 256;
    const int blocks = (int)((npad / 2 + threads - 1) / threads < 4096 ? (npad / 2 + threads - 1) / threads : 4096);
    for (int64_t k = 2; k <= npad; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            bitonic_step_kernel<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(keys, vals, npad, j, k);
            ++*launches;
        }
    return cudaGetLastError();
}

cudaError_t launch_features(const Pools& P, float* prof, float* feat, int sms, cudaStream_t st) {
    profile_kernel<<<P.count, 32, 0, st>>>(P, prof);
    features_kernel<<<sms * 8, 256, 0, st>>>(P, prof, feat);
    return cudaGetLastError();
}

// Queue order for the first-solution mode.  y = scorer outputs (learned) or
// null (plain).  npad: power of two >= number of prefixes; keys/vals: npad
// entries each; perm receives the order (queue position -> gid).
cudaError_t launch_order(const Pools& P, const float* y, int64_t npad, unsigned long long* keys,
                         unsigned long long* vals, unsigned long long* keys2, unsigned long long* vals2,
                         int64_t* perm, int sms, cudaStream_t st, int64_t* launches) {
    const int blocks = sms * 4;
    cudaError_t e = cudaSuccess;
    const unsigned long long* s1 = nullptr;
    if (y) {
        score_keys_kernel<<<blocks, 256, 0, st>>>(P, y, npad, keys, vals);
        ++*launches;
        if ((e = bitonic_sort(keys, vals, npad, st, launches)) != cudaSuccess) return e;
        s1 = vals;
    }
    rank_keys_kernel<<<blocks, 256, 0, st>>>(P, npad, s1, keys2, vals2);
    ++*launches;
    if ((e = bitonic_sort(keys2, vals2, npad, st, launches)) != cudaSuccess) return e;
    copy_perm_kernel<<<blocks, 256, 0, st>>>(P, vals2, perm);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace msp
