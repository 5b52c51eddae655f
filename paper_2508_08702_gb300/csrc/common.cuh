// common.cuh -- device-side data layout shared by the sm_103a kernels of the
// market-split lattice solver.  Host orchestration lives in api.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msp {

constexpr int kMaxM = 32;      // rows of A
constexpr int kMaxDim = 128;   // n + 1 lattice coordinates after extraction
constexpr int kMaxK = 128;     // basis vectors n + 1

// per-instance status codes (same values as msp_status in include/msp.h)
enum : int32_t {
    ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_EOVERFLOW = 4, ST_ERANK = 5,
    ST_ETIMEOUT = 6, ST_ETRUNC = 7, ST_ESTATE = 8, ST_ECAP = 9, ST_EQUEUE = 10
};

// Descriptor of one instance of a batch; offsets are element offsets into
// the pools of Pools below.  Descriptors, and every per-instance region of
// the tables the walkers read, start on their own 128-byte lines: in the
// fused launch an instance is prepared while walkers on other SMs already
// read the tables of others, and a line shared by two instances could sit
// in an SM's L1 with the bytes of the one not yet prepared.
struct __align__(128) InstDesc {
    int32_t m, n, K, L;      // K = n + 1 basis vectors of length L = m + n + 1
    int32_t dd, dim;         // kernel rank (set by the extractor), dim = n + 1
    int32_t status;
    int32_t split_level;     // lowest level fixed by the splitter
    int32_t front_sel;       // frontier buffer holding the final prefixes
    int32_t rmax;            // lcm of the bounds 0 <= x_j <= r_j (1: binary), Sec. 2
    int64_t offR;            // n int32         upper bounds r_j; also the column permutation
    int32_t group, replica;  // the caller's instance and the replica of it (shuffled columns)
    int64_t nprefix;         // number of prefixes (subtrees)
    int64_t offA, offd;      // A (int32, m*n), d (int64, m)
    int64_t offBasis;        // K*L int64   LLL basis, vector-major
    int64_t offGram;         // K*K int64   exact Gram matrix
    int64_t offMu;           // 2*K*K+K f64 LLL mu, r and 1/B
    int64_t offBl;           // K f64       LLL ||bhat||^2
    int64_t offKb;           // K*dim int32 kept (kernel) basis
    int64_t offMuT;          // K*K f64     muT[t][i] = mu[i][t]
    int64_t offB;            // K f64       ||bhat_t||^2
    int64_t offBhat;         // K*dim f64   bhat[t][c]
    int64_t lll_iters, lll_swaps;
    int64_t bkz_tours, bkz_inserts, bkz_nodes;   // BKZ of the kernel basis (0 without BKZ)
    // fixed-point filter of the Hoelder test (set by prep_fixed_kernel)
    int32_t sx, sb;          // scales: Xq = trunc(x 2^sx), Bq = round(bhat 2^sb)
    int64_t offBq;           // K*dimPad int32   Bq[t][c]
    int64_t offNbq;          // K int64          sum_c |Bq[t][c]|
};

struct InstCounters {
    unsigned long long nodes, passed, leaves, nsol;
    unsigned long long split_nodes, split_passed;   // part done by the splitter
    unsigned long long center_fma;                  // centre-fold fmas of the walkers
    unsigned long long fallbacks;                   // Hoelder tests decided by the FP64 rebuild
    unsigned long long first_ns;                    // first-solution mode: time of the first solution
    unsigned long long lds_cuts;                    // values held back by the discrepancy budget
};

// A found solution: x_c is bit (127 - c) of the 128-bit key (hi:lo), so that
// numeric key order equals lexicographic order of x as a byte string.
struct SolRec {
    int32_t inst;
    int32_t pad;
    unsigned long long hi, lo;
};

struct Pools {
    InstDesc* inst;
    InstCounters* cnt;
    int count;
    int Kmax, dimMax, dimPad;          // maxima over the batch; dimPad = dimMax rounded to 32
    const int32_t* A;
    const int64_t* d;
    int64_t* basis;
    int64_t* gram;
    double* mu;
    double* Bl;
    int32_t* kb;
    double* muT;
    double* B;
    double* bhat;
    int32_t* bq;                       // fixed-point bhat (see InstDesc::offBq)
    int64_t* nbq;
    // splitter frontier: [count][2][F] prefixes of (u[Kmax] int32, rho, w[dimPad])
    int32_t* fu;
    double* frho;
    double* fw;
    int32_t* fdisc;                    // per prefix: discrepancy cost of the path (limited discrepancy search)
    float* fxsum;                      // per prefix: sum over its levels of |x|
    int64_t F;
    // work queue
    int64_t* qbase;                    // count + 1 exclusive prefix sums of nprefix
    const int64_t* qperm;              // optional queue order (learned); may be null
    int64_t* plog_nodes;               // per prefix: nodes evaluated in its subtree
    int32_t* plog_sols;                // per prefix: solutions found in its subtree
    // donated sibling ranges (work handed from busy walkers to idle ones)
    char* don;                         // don_cap slots of don_stride bytes
    unsigned long long* don_seq;       // per slot sequence number (bounded MPMC ring)
    int64_t don_cap, don_stride;
    // solutions
    SolRec* sols;
    int64_t sol_cap;
    struct Ctrl* ctrl;
    const unsigned char* skip;         // optional, per instance: 1 = no subtrees in this launch
    const int32_t* r;                  // upper bounds of x per variable (all instances)
    unsigned* gsolved;                 // per group (caller's instance): a replica found a solution
    unsigned long long* gfirst_ns;     // per group: time of that first solution
};

// bits of the field that holds x_j in a solution key (x_j <= r_j)
__host__ __device__ inline int bound_bits(int r) {
    int b = 0;
    while (r > 0) { ++b; r >>= 1; }
    return b;
}

// Control words of one enumeration, in device memory.
struct Ctrl {
    unsigned long long qhead;          // next static queue item
    unsigned long long dhead, dtail;   // donation queue: next to take / next free slot
    int idle;                          // walkers waiting for donated work
    int busy;                          // walkers holding work
    unsigned long long donations;      // sibling ranges handed over
    unsigned long long walk_cycles;    // sum over walkers of clock cycles spent walking
    unsigned long long life_cycles;    // sum over walkers of clock cycles alive
    unsigned long long nsol_total;     // solutions found (all instances)
    unsigned long long deadline_ns;    // globaltimer deadline, 0 = none
    unsigned int stop;                 // 1: every instance solved (first-solution mode), 2: time cap
    int32_t gstatus;                   // batch-wide status
    unsigned long long start_ns;       // globaltimer at the start of the enumeration
    int solved;                        // first-solution mode: instances with a solution
    int active;                        // instances with subtrees to enumerate
    // fused launch: instances join the queue as their blocks finish them
    unsigned long long qres;           // reservations: (instances << 40) | queue positions reserved
};

// Enumeration options passed to the split and enumeration kernels.
// Per-instance global scratch of the BKZ kernel: two K x D int64 blocks
// (basis, block copy), three K x K blocks (Gram; the LLL's mu and r), five
// K-vectors of 8 bytes and five of 4 bytes; the stride is rounded to 256
// bytes.
struct BkzScratch {
    char* base;
    int64_t stride;   // bytes per instance
    int Kmax, dimMax;
    __host__ __device__ static int64_t bytes(int Kmax, int dimMax) {
        const int64_t K = Kmax, D = dimMax;
        const int64_t raw = 8 * (2 * K * D + 3 * K * K + 5 * K) + 4 * 5 * K;
        return (raw + 255) / 256 * 256;
    }
};

// Fused launch: the enumeration kernel's blocks first prepare the instances
// of the batch (block b takes instances b, b + grid, ...: warp 0 reduces the
// lattice and builds the tables, then the whole block splits the top levels)
// and publish each one's subtrees to the queue; the walkers start on the
// published subtrees while other instances are still being prepared.
struct Pipe {
    int on;                            // 0: the instances were prepared by earlier launches
    double delta, eta;                 // LLL parameters
    int64_t lll_max_iter;
    unsigned long long max_ns;         // device-time cap of one reduction
    int bkz_beta, bkz_max_tours;       // BKZ of the kernel basis (beta < 2: none)
    BkzScratch S;
    int use_eps, dimPad;
    int split_depth;
    int64_t split_target;
    int64_t* fcnt;                     // split scratch (per instance, F entries)
    int64_t* rl;                       // publish list: [count] queue bases, [count] instances,
                                       // [count] ready flags (zeroed before the launch)
};

struct EnumCfg {
    int hoelder;     // 0: Hoelder test with the one-direction cut, 1: skip value only, 2: off
    int sym;         // 1: one of v, -v;  0: both signs
    int use_eps;     // slack eps = (n+1) 2^-20 on both tests
    int first;       // stop at the first solution
    int lds;         // >= 0: one limited-discrepancy iteration with this budget; -1: depth-first
    int lds_rank;    // discrepancy cost of a value: 1 its position in the level's walk, 0 one if not the first
};

__device__ __forceinline__ int64_t frontier_index(const Pools& P, int inst, int sel, int64_t j) {
    return ((int64_t)inst * 2 + sel) * P.F + j;
}

__device__ __forceinline__ unsigned long long global_time_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_status(InstDesc& I, int32_t st) {
    atomicCAS(&I.status, ST_OK, st);
}

}  // namespace msp
