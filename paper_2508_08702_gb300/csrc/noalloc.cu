// noalloc.cu -- lattice reduction for callers that cannot allocate device memory.
//
// Who needs this: a host application whose allocator owns the whole GPU
// (a memory pool that reserved the device up front, or a process under a hard
// device-memory cap) cannot let a library call cudaMalloc behind its back, and
// latency-critical callers cannot afford the device-wide synchronisation an
// allocation may cause.  msp_reduce_lattice_noalloc() builds the lattice of
// one instance and LLL-reduces it with the same kernels as msp_reduce(), but
// its scratch (the exact Gram matrix, the Gram-Schmidt rows and the instance
// descriptor) lives in the file-scope array below, which every GPU that loads
// this library holds until the process exits.  The caller passes the inputs
// and the output buffer; nothing is allocated or freed.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/msp.h"
#include "common.cuh"

namespace msp {
__global__ void build_lattice_kernel(Pools P, int64_t N);
__global__ void lll_kernel(Pools P, double delta, double eta, int64_t max_iter, unsigned long long max_ns);
}  // namespace msp

using namespace msp;

namespace {

constexpr int kNoAllocMaxK = 128;   // n + 1 basis vectors at most (n <= 127)
constexpr size_t kDescBytes = 256;
constexpr size_t kGramBytes = (size_t)kNoAllocMaxK * kNoAllocMaxK * 8;
constexpr size_t kMuBytes = ((size_t)2 * kNoAllocMaxK * kNoAllocMaxK + kNoAllocMaxK) * 8;
constexpr size_t kBBytes = (size_t)kNoAllocMaxK * 8;
constexpr size_t kScratchBytes = kDescBytes + kGramBytes + kMuBytes + kBBytes;   // 395,520 bytes

static_assert(sizeof(InstDesc) <= kDescBytes, "the descriptor slot of the scratch is too small");

// The scratch.  In host code this name is only a host-side stand-in: the
// device address comes from cudaGetSymbolAddress (scratch_on_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device with that device current.
cudaError_t scratch_on_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" MSP_API msp_status msp_reduce_lattice_noalloc(int m, int n, const int32_t* A, const int64_t* d,
                                                         int64_t N, double delta, double eta, int64_t max_iter,
                                                         int64_t* basis, void* stream) {
    if (m < 1 || m > kMaxM || n < 1 || n + 1 > kNoAllocMaxK || m > n || !A || !d || !basis) return MSP_EINVAL;
    if (N < 1 || N > (1LL << 30) || !(delta > 0.25 && delta < 1.0) || !(eta >= 0.5 && eta < 1.0) || max_iter < 1)
        return MSP_EINVAL;
    unsigned char* base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) {
        cudaGetLastError();
        return MSP_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int K = n + 1, L = m + n + 1;
    // a fresh descriptor every call: the status word must start at zero
    InstDesc I;
    std::memset(&I, 0, sizeof I);
    I.m = m; I.n = n; I.K = K; I.L = L; I.dim = n + 1;
    Pools P;
    std::memset(&P, 0, sizeof P);
    P.inst = reinterpret_cast<InstDesc*>(base);
    P.count = 1;
    P.A = A;
    P.d = d;
    P.basis = basis;
    P.gram = reinterpret_cast<int64_t*>(base + kDescBytes);
    P.mu = reinterpret_cast<double*>(base + kDescBytes + kGramBytes);
    P.Bl = reinterpret_cast<double*>(base + kDescBytes + kGramBytes + kMuBytes);
    cudaError_t e = cudaMemcpyAsync(P.inst, &I, sizeof I, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        build_lattice_kernel<<<1, 128, 0, st>>>(P, N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        // the same device-time cap as msp_reduce with default options (600 s)
        lll_kernel<<<1, 32, 0, st>>>(P, delta, eta, max_iter, 600ULL * 1000000000ULL);
        e = cudaGetLastError();
    }
    InstDesc out;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out, P.inst, sizeof out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MSP_ECUDA;
    }
    return (msp_status)out.status;
}
