// api.cu -- C ABI of include/msp.h: argument checks, device buffers, launches.
// Every computational step is a kernel in lattice.cu / enum.cu; this file
// only sizes buffers, queues work on the context's stream and copies
// results back.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/msp.h"
#include "common.cuh"

namespace msp {
__global__ void build_lattice_kernel(Pools P, int64_t N);
__global__ void lll_kernel(Pools P, double delta, double eta, int64_t max_iter, unsigned long long max_ns);
__global__ void extract_gso_kernel(Pools P, int gso_only);
__global__ void bkz_kernel(Pools P, BkzScratch S, int beta, double delta, int max_tours, int64_t lll_max_iter,
                           unsigned long long max_ns);
__global__ void prep_fixed_kernel(Pools P, int use_eps, int dimPad);
__global__ void permute_kernel(Pools P, int32_t* perm, int32_t* rperm, unsigned long long seed);
cudaError_t launch_split(const Pools& P, const EnumCfg& cfg, int lanes, int max_depth, int64_t target,
                         int64_t* fcnt, cudaStream_t st);
cudaError_t launch_enum(const Pools& P, const EnumCfg& cfg, int lanes, int blocks, int threads, char* scratch,
                        int Kmax, int dimPad, int variant, const Pipe& pipe, cudaStream_t st);
cudaError_t launch_collect(const Pools& P, int64_t* soff, unsigned long long* fill, SolRec* seg, SolRec* out,
                           cudaStream_t st);
cudaError_t launch_start(Ctrl* ctrl, unsigned long long cap_ns, int keep, cudaStream_t st);
cudaError_t launch_ring_init(unsigned long long* seq, int64_t cap, cudaStream_t st);
int64_t walker_bytes(int Kmax, int dimPad);
int64_t donation_slot_bytes(int Kmax, int dimPad);
int enum_blocks_per_sm(int lanes, int threads, int dimMax, int Kmax, int variant);
int enum_smem_bytes(int lanes, int threads, int Kmax);
cudaError_t launch_features(const Pools& P, float* prof, float* feat, int sms, cudaStream_t st);
cudaError_t launch_order(const Pools& P, const float* y, int64_t npad, unsigned long long* keys,
                         unsigned long long* vals, unsigned long long* keys2, unsigned long long* vals2,
                         int64_t* perm, int sms, cudaStream_t st, int64_t* launches);
cudaError_t mlp_forward(const float* theta, const float* X, int64_t n, float* Y, int sms, cudaStream_t st);
cudaError_t mlp_grad(const float* theta, const float* X, const float* target, int64_t n, float pos_weight,
                     float* grad, float* loss, cudaStream_t st);
cudaError_t mlp_train(float* theta, const float* X, const float* target, int64_t n, int steps, float lr,
                      float pos_weight, uint64_t seed, float* work, float* losses, cudaStream_t st);
int mlp_param_count();
cudaError_t fp64_peak(double* dfma_per_s, int sms, cudaStream_t st);
}  // namespace msp

using namespace msp;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct msp_ctx {
    msp_opts o;
    cudaStream_t st = nullptr;
    int dev = 0, sms = 0, smem_optin = 48 * 1024;
    int lanes = 8;                       // lanes per walker for the current batch
    std::string err;
    int64_t launches = 0;
    int state = 0;   // 0 empty, 1 lattice built, 2 reduced, 3 enumerated
    // batch
    int count = 0, Kmax = 0, dimMax = 0, dimPad = 0;
    int64_t F = 0;
    std::vector<InstDesc> hinst;
    std::vector<InstDesc> layout;        // descriptors as msp_build_lattice wrote them
    std::vector<int32_t> hr;             // bounds of all instances (host copy)
    bool bounded = false;                // some instance has r_max > 1
    int ucount = 0;                      // the caller's instances (count = ucount x replicas)
    std::vector<int32_t> hperm;          // column permutation of every replica (host copy)
    std::vector<msp_stats> stats;
    int last_mode = 0;
    double last_ms = 0.0;
    std::chrono::steady_clock::time_point t_start;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evr0 = nullptr, evr1 = nullptr;   // reduce
    cudaEvent_t evs1 = nullptr, eve1 = nullptr;   // split end, enumerate end
    bool reduce_timed = false;
    // device buffers
    Buf inst, cnt, A, d, basis, gram, mu, Bl, kb, muT, B, bhat, bq, nbq, fu, fdisc, fxsum, frho, fw, fcnt, qbase, sols, ctrl, soff,
        fill, seg, sout, scratch, plog_nodes, plog_sols, don, don_seq, feat, prof, yout, skeys, svals, skeys2,
        svals2, perm, theta, mlpwork, inst0, skip, bkzs, rb, gsolved, gfirst, colperm, rl;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cst = nullptr;          // private stream the step is captured on
    int graph_mode = 0;
    int64_t graph_launches = 0;
    Pools graph_P{};                     // buffers and layout the graph was captured on
    std::vector<InstDesc> graph_inst;
    std::vector<int32_t> lds_done;       // per instance: budget that solved / finished it (-1)
    bool last_lds = false;
    bool last_fused = false;             // the last enumeration also reduced and split (one launch)
    bool scorer_set = false;
    bool features_valid = false;
    std::vector<int64_t> soff_h;
    std::vector<SolRec> sout_h;
    bool sout_valid = false;
    Pools P{};
};

namespace {

msp_status fail(msp_ctx* c, msp_status s, const std::string& what) {
    if (c) c->err = what;
    return s;
}

msp_status cuda_fail(msp_ctx* c, cudaError_t e, const char* where) {
    return fail(c, MSP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Event record that also times a graph replay: inside a capture the record
// becomes a graph node (external record) instead of a capture-internal marker.
void record(msp_ctx* c, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, c->st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, c->st);
}

void drop_graph(msp_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_inst.clear();
}

msp_status ensure(msp_ctx* c, Buf& b, size_t bytes, const char* name) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return MSP_OK;
    if (b.p) {
        cudaStreamSynchronize(c->st);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MSP_ENOMEM, std::string("cudaMalloc ") + name + " (" + std::to_string(bytes) + " bytes): " +
                                       cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return MSP_OK;
}

template <class T>
T* ptr(Buf& b) {
    return static_cast<T*>(b.p);
}

void refresh_pools(msp_ctx* c) {
    Pools& P = c->P;
    P.inst = ptr<InstDesc>(c->inst);
    P.cnt = ptr<InstCounters>(c->cnt);
    P.count = c->count;
    P.Kmax = c->Kmax;
    P.dimMax = c->dimMax;
    P.dimPad = c->dimPad;
    P.A = ptr<int32_t>(c->A);
    P.d = ptr<int64_t>(c->d);
    P.basis = ptr<int64_t>(c->basis);
    P.gram = ptr<int64_t>(c->gram);
    P.mu = ptr<double>(c->mu);
    P.Bl = ptr<double>(c->Bl);
    P.kb = ptr<int32_t>(c->kb);
    P.muT = ptr<double>(c->muT);
    P.B = ptr<double>(c->B);
    P.bhat = ptr<double>(c->bhat);
    P.bq = ptr<int32_t>(c->bq);
    P.nbq = ptr<int64_t>(c->nbq);
    P.fu = ptr<int32_t>(c->fu);
    P.frho = ptr<double>(c->frho);
    P.fw = ptr<double>(c->fw);
    P.fdisc = ptr<int32_t>(c->fdisc);
    P.fxsum = ptr<float>(c->fxsum);
    P.F = c->F;
    P.qbase = ptr<int64_t>(c->qbase);
    P.qperm = nullptr;
    P.plog_nodes = ptr<int64_t>(c->plog_nodes);
    P.plog_sols = ptr<int32_t>(c->plog_sols);
    P.don = ptr<char>(c->don);
    P.don_seq = ptr<unsigned long long>(c->don_seq);
    P.don_cap = c->o.donation_capacity;
    P.don_stride = donation_slot_bytes(c->Kmax, c->dimPad);
    P.sols = ptr<SolRec>(c->sols);
    P.sol_cap = c->o.sol_capacity;
    P.ctrl = ptr<Ctrl>(c->ctrl);
    P.r = ptr<int32_t>(c->rb);
    P.gsolved = ptr<unsigned>(c->gsolved);
    P.gfirst_ns = ptr<unsigned long long>(c->gfirst);
}

int walkers_of(const msp_ctx* c, int blocks, int threads) { return blocks * threads / c->lanes; }

// Threads per enumeration block: the requested warps, reduced while the
// walkers' level state would not fit the shared memory a block may use.
void enum_launch_shape(const msp_ctx* c, int* blocks, int* threads) {
    int t = c->o.warps_per_block * 32;
    while (t > 32 && enum_smem_bytes(c->lanes, t, c->Kmax) > c->smem_optin) t -= 32;
    *threads = t;
    // blocks per SM: the option, at most as many as can be resident (the
    // walkers are persistent: a block that cannot start would only start
    // once others have finished)
    // (the fused launch's variant counts too, so both launches have the same
    // walkers: its blocks must all be resident at once)
    int fit = enum_blocks_per_sm(c->lanes, t, c->dimMax, c->Kmax, 0);
    const int fit3 = enum_blocks_per_sm(c->lanes, t, c->dimMax, c->Kmax, 3);
    if (fit3 > 0) fit = std::min(fit, fit3);
    fit = std::max(1, fit);
    int bps = c->o.blocks_per_sm;
    bps = bps <= 0 ? fit : std::min(bps, fit);
    *blocks = c->sms * bps;
}

// Buffers whose size follows the per-instance frontier capacity F (prefixes,
// their logs and features, the sort keys of the queue order).  Grow-only.
msp_status size_frontier(msp_ctx* c, int64_t F) {
    F = (F + 31) / 32 * 32;   // every instance's frontier region on its own 128-byte lines
    const size_t n = (size_t)c->count, K = (size_t)c->Kmax, D = (size_t)c->dimPad;
    const int64_t cap = (int64_t)n * F;
    int64_t npad = 1;
    while (npad < cap) npad <<= 1;
    msp_status s;
#define ENSURE(buf, bytes)                                               \
    if ((s = ensure(c, c->buf, (size_t)(bytes), #buf)) != MSP_OK) return s;
    ENSURE(fu, sizeof(int32_t) * n * 2 * F * K);
    ENSURE(frho, sizeof(double) * n * 2 * F);
    ENSURE(fw, sizeof(double) * n * 2 * F * D);
    ENSURE(fcnt, sizeof(int64_t) * n * F);
    ENSURE(fdisc, sizeof(int32_t) * n * 2 * F);
    ENSURE(fxsum, sizeof(float) * n * 2 * F);
    ENSURE(plog_nodes, sizeof(int64_t) * n * F);
    ENSURE(plog_sols, sizeof(int32_t) * n * F);
    ENSURE(feat, sizeof(float) * 32 * (size_t)cap);
    ENSURE(yout, sizeof(float) * 8 * (size_t)cap);
    ENSURE(skeys, sizeof(unsigned long long) * (size_t)npad);
    ENSURE(svals, sizeof(unsigned long long) * (size_t)npad);
    ENSURE(skeys2, sizeof(unsigned long long) * (size_t)npad);
    ENSURE(svals2, sizeof(unsigned long long) * (size_t)npad);
    ENSURE(perm, sizeof(int64_t) * (size_t)cap);
#undef ENSURE
    c->F = F;
    return MSP_OK;
}

// Split target of one enumeration: the option, else (first-solution mode) the
// finer first-solution split, else 8 subtrees per walker over the batch.
int64_t split_target_of(msp_ctx* c, int mode, int64_t walkers) {
    if (c->o.split_target > 0) return c->o.split_target;
    if (mode == MSP_FIRST && c->o.first_split_target > 0) return c->o.first_split_target;
    return std::max<int64_t>(64, 8 * walkers / std::max(c->count, 1));
}

// Grows the frontier to 4 x the split target of `mode` (unless the capacity
// is fixed by an option); a captured graph on the old buffers is dropped.
msp_status fit_frontier(msp_ctx* c, int mode, int64_t walkers) {
    if (c->o.split_capacity > 0) return MSP_OK;
    const int64_t want = 4 * split_target_of(c, mode, walkers);
    if (want <= c->F) return MSP_OK;
    msp_status s = size_frontier(c, want);
    if (s != MSP_OK) return s;
    refresh_pools(c);
    if (c->gexec && std::memcmp(&c->graph_P, &c->P, sizeof(Pools)) != 0) drop_graph(c);
    return MSP_OK;
}

msp_status check_launch(msp_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return MSP_OK;
}

}  // namespace

extern "C" {

void msp_default_opts(msp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->N = 1024;
    o->delta = 0.99;
    o->eta = 0.51;
    o->lll_max_iter = 2000000;
    o->hoelder = 0;
    o->sym = 1;
    o->use_eps = 1;
    o->lanes = 0;
    o->split_depth = 24;
    o->split_target = 0;
    o->split_capacity = 0;
    o->warps_per_block = 8;
    o->blocks_per_sm = 0;
    o->sol_capacity = 1 << 20;
    o->max_seconds = 600.0;
    o->donation_capacity = 1 << 16;
    o->log_features = 0;
    o->lds_budget = -1;
    o->lds_max = 127;
    o->lds_rank = 1;
    o->fuse = 0;
    o->first_split_target = 16384;
    o->bkz_beta = 0;
    o->bkz_max_tours = 16;
    o->replicas = 1;
    o->replica_seed = 0x5EED5EED5EED5EEDULL;
}

const char* msp_status_string(int s) {
    switch (s) {
        case MSP_OK: return "ok";
        case MSP_EINVAL: return "invalid argument";
        case MSP_ENOMEM: return "out of memory";
        case MSP_ECUDA: return "CUDA error";
        case MSP_EOVERFLOW: return "integer overflow";
        case MSP_ERANK: return "kept vectors do not span the kernel (N too small)";
        case MSP_ETIMEOUT: return "time cap reached";
        case MSP_ETRUNC: return "solution buffer too small";
        case MSP_ESTATE: return "call order violated";
        case MSP_ECAP: return "iteration cap reached (LLL, or the last budget of the discrepancy search)";
        case MSP_EQUEUE: return "work queue capacity exceeded";
        default: return "unknown status";
    }
}

const char* msp_last_error(const msp_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t msp_kernel_launches(const msp_ctx* c) { return c ? c->launches : 0; }

msp_status msp_create(msp_ctx** out, const msp_opts* opts, void* stream) {
    if (!out) return MSP_EINVAL;
    *out = nullptr;
    msp_ctx* c = new (std::nothrow) msp_ctx();
    if (!c) return MSP_ENOMEM;
    if (opts) c->o = *opts; else msp_default_opts(&c->o);
    const msp_opts& o = c->o;
    if (o.N < 1 || o.N > (1LL << 30) || !(o.delta > 0.25 && o.delta < 1.0) || !(o.eta >= 0.5 && o.eta < 1.0) ||
        o.hoelder < 0 || o.hoelder > 2 || (o.lanes != 0 && o.lanes != 4 && o.lanes != 8 && o.lanes != 16 && o.lanes != 32) ||
        o.split_depth < 0 || o.warps_per_block < 1 || o.warps_per_block > 8 || o.sol_capacity < 1 ||
        o.lll_max_iter < 1 || !(o.max_seconds > 0.0) || o.donation_capacity < 0 || o.lds_budget < -1 ||
        o.lds_budget > 255 || o.lds_max < 0 || o.lds_max > 255 || (o.lds_rank != 0 && o.lds_rank != 1) || o.first_split_target < 0 ||
        o.bkz_beta < 0 || o.bkz_beta == 1 || o.bkz_beta > 128 || o.bkz_max_tours < 1 || o.replicas < 1 ||
        o.replicas > 64) {
        delete c;
        return MSP_EINVAL;
    }
    c->st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->evr0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->evr1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->evs1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->eve1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return MSP_ECUDA;
    }
    *out = c;
    return MSP_OK;
}

void msp_destroy(msp_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    Buf* all[] = {&c->inst, &c->cnt, &c->A, &c->d, &c->basis, &c->gram, &c->mu, &c->Bl, &c->kb, &c->muT, &c->B,
                  &c->bhat, &c->bq, &c->nbq, &c->fdisc, &c->fxsum, &c->fu, &c->frho, &c->fw, &c->fcnt, &c->qbase, &c->sols, &c->ctrl, &c->soff,
                  &c->fill, &c->seg, &c->sout, &c->scratch, &c->plog_nodes, &c->plog_sols, &c->don,
                  &c->don_seq, &c->feat, &c->prof, &c->yout, &c->skeys, &c->svals, &c->skeys2, &c->svals2,
                  &c->perm, &c->theta, &c->mlpwork, &c->inst0, &c->skip, &c->bkzs, &c->rb, &c->gsolved,
                  &c->gfirst, &c->colperm, &c->rl};
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cst) cudaStreamDestroy(c->cst);
    for (Buf* b : all)
        if (b->p) cudaFree(b->p);
    for (cudaEvent_t ev : {c->ev0, c->ev1, c->evr0, c->evr1, c->evs1, c->eve1})
        if (ev) cudaEventDestroy(ev);
    delete c;
}

msp_status msp_build_lattice(msp_ctx* c, int count, const int32_t* dims, const int32_t* A, const int64_t* d,
                             int mem) {
    return msp_build_lattice_bounds(c, count, dims, A, d, nullptr, mem);
}

msp_status msp_build_lattice_bounds(msp_ctx* c, int count, const int32_t* dims, const int32_t* A,
                                    const int64_t* d, const int32_t* r, int mem) {
    if (!c) return MSP_EINVAL;
    if (count < 1 || !dims || !A || !d || (mem != MSP_HOST && mem != MSP_DEVICE))
        return fail(c, MSP_EINVAL, "msp_build_lattice: bad arguments");
    const int R = c->o.replicas;   // searches per caller's instance (shuffled column orders)
    const int total = count * R;
    std::vector<InstDesc> h(total);
    int64_t nA = 0, nd = 0, nBasis = 0, nGram = 0, nMu = 0, nK = 0, nKb = 0, nT = 0, nR = 0;
    int64_t uA = 0, ud = 0, uR = 0;   // offsets in the caller's arrays
    int Kmax = 0, dimMax = 0;
    std::vector<int32_t> hr;   // bounds of all internal instances (ones for binary problems)
    std::vector<int64_t> srcA(total), srcd(total);
    for (int g = 0; g < count; ++g) {
        const int m = dims[2 * g], n = dims[2 * g + 1];
        if (m < 1 || m > kMaxM || n < 1 || n + 1 > kMaxDim || m > n)
            return fail(c, MSP_EINVAL, "msp_build_lattice: instance " + std::to_string(g) + " has bad (m, n)");
        // bounds 0 <= x_j <= r_j (Sec. 2): r_max = lcm, key fields of bound_bits(r_j) bits
        int64_t rmax = 1;
        int keybits = 0;
        for (int j = 0; j < n; ++j) {
            const int32_t rj = r ? r[uR + j] : 1;
            if (rj < 1 || rj > 255)
                return fail(c, MSP_EINVAL, "msp_build_lattice: instance " + std::to_string(g) +
                                               ": bounds must lie in [1, 255]");
            int64_t a = rmax, b = rj;
            while (b) { const int64_t t = a % b; a = b; b = t; }
            rmax = rmax / a * rj;
            if (rmax > 1024)
                return fail(c, MSP_EINVAL, "msp_build_lattice: instance " + std::to_string(g) +
                                               ": lcm of the bounds exceeds 1024");
            keybits += bound_bits(rj);
        }
        if (keybits > 128)
            return fail(c, MSP_EINVAL, "msp_build_lattice: instance " + std::to_string(g) +
                                           ": more than 128 bits of x (sum of bit widths of the bounds)");
        for (int k = 0; k < R; ++k) {
            const int i = g * R + k;
            InstDesc& I = h[i];
            std::memset(&I, 0, sizeof I);
            I.group = g;
            I.replica = k;
            I.rmax = (int32_t)rmax;
            I.offR = nR;
            for (int j = 0; j < n; ++j) hr.push_back(r ? r[uR + j] : 1);
            nR += n;
            I.m = m; I.n = n; I.K = n + 1; I.L = m + n + 1; I.dim = n + 1;
            I.offA = nA; nA += (int64_t)m * n;
            I.offd = nd; nd += m;
            srcA[i] = uA;
            srcd[i] = ud;
            I.offBasis = nBasis; nBasis += (int64_t)I.K * I.L;
            I.offGram = nGram; nGram += (int64_t)I.K * I.K;
            I.offMu = nMu; nMu += (int64_t)2 * I.K * I.K + I.K;
            // (128-byte aligned regions, see InstDesc: 16 doubles, 32 int32)
            I.offBl = nK; I.offB = nK; nK += (I.K + 15) / 16 * 16;
            I.offKb = nKb; I.offBhat = nKb; nKb += ((int64_t)I.K * I.dim + 31) / 32 * 32;
            I.offMuT = nT; nT += ((int64_t)I.K * I.K + 15) / 16 * 16;
            Kmax = std::max(Kmax, I.K);
            dimMax = std::max(dimMax, I.dim);
        }
        uA += (int64_t)m * n;
        ud += m;
        uR += n;
    }
    c->ucount = count;
    count = total;   // from here on: the internal instances
    c->count = count;
    c->Kmax = Kmax;
    c->dimMax = dimMax;
    c->dimPad = (dimMax + 31) / 32 * 32;
    // automatic lanes: at most 8 coordinates per lane on 8-lane walkers,
    // else 16-lane walkers (wider lattices spill registers at 8 lanes)
    c->lanes = c->o.lanes ? c->o.lanes : (dimMax <= 64 ? 8 : 16);
    int64_t nBq = 0;
    for (int i = 0; i < count; ++i) {
        h[i].offBq = nBq;
        h[i].offNbq = (int64_t)i * ((Kmax + 15) / 16 * 16);
        nBq += (int64_t)h[i].K * c->dimPad;
    }
    // split sizes
    int blocks, threads;
    enum_launch_shape(c, &blocks, &threads);
    const int64_t walkers = walkers_of(c, blocks, threads);
    int64_t target = c->o.split_target > 0 ? c->o.split_target : std::max<int64_t>(64, 8 * walkers / count);
    const int64_t F = c->o.split_capacity > 0 ? std::max<int64_t>(c->o.split_capacity, 1) : 4 * target;
    msp_status s;
#define ENSURE(buf, bytes)                                               \
    if ((s = ensure(c, c->buf, (size_t)(bytes), #buf)) != MSP_OK) return s;
    ENSURE(inst, sizeof(InstDesc) * count);
    ENSURE(inst0, sizeof(InstDesc) * count);
    ENSURE(cnt, sizeof(InstCounters) * count);
    ENSURE(A, sizeof(int32_t) * nA);
    ENSURE(rb, sizeof(int32_t) * nR);
    ENSURE(d, sizeof(int64_t) * nd);
    ENSURE(basis, sizeof(int64_t) * nBasis);
    ENSURE(gram, sizeof(int64_t) * nGram);
    ENSURE(mu, sizeof(double) * nMu);
    ENSURE(Bl, sizeof(double) * nK);
    ENSURE(kb, sizeof(int32_t) * nKb);
    ENSURE(muT, sizeof(double) * nT);
    ENSURE(B, sizeof(double) * nK);
    ENSURE(bhat, sizeof(double) * nKb);
    ENSURE(bq, sizeof(int32_t) * nBq);
    ENSURE(nbq, sizeof(int64_t) * (size_t)count * ((Kmax + 15) / 16 * 16));
    ENSURE(don, (size_t)c->o.donation_capacity * donation_slot_bytes(Kmax, c->dimPad));
    ENSURE(don_seq, sizeof(unsigned long long) * (size_t)std::max<int64_t>(c->o.donation_capacity, 1));
    ENSURE(qbase, sizeof(int64_t) * (count + 1));
    ENSURE(sols, sizeof(SolRec) * (size_t)c->o.sol_capacity);
    ENSURE(ctrl, sizeof(Ctrl));
    ENSURE(soff, sizeof(int64_t) * (count + 1));
    ENSURE(fill, sizeof(unsigned long long) * count);
    ENSURE(seg, sizeof(SolRec) * (size_t)c->o.sol_capacity);
    ENSURE(sout, sizeof(SolRec) * (size_t)c->o.sol_capacity);
    ENSURE(scratch, (size_t)walkers * walker_bytes(Kmax, c->dimPad));
    ENSURE(prof, sizeof(float) * 17 * (size_t)count);
    ENSURE(colperm, sizeof(int32_t) * nR);
    ENSURE(gsolved, sizeof(unsigned) * c->ucount);
    ENSURE(gfirst, sizeof(unsigned long long) * c->ucount);
#undef ENSURE
    if ((s = size_frontier(c, F)) != MSP_OK) return s;
    refresh_pools(c);
    const cudaMemcpyKind kind = (mem == MSP_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (R == 1) {
        e = cudaMemcpyAsync(c->A.p, A, sizeof(int32_t) * nA, kind, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d.p, d, sizeof(int64_t) * nd, kind, c->st);
    } else {   // every replica starts from the caller's A and d
        for (int i = 0; i < count && e == cudaSuccess; ++i) {
            const InstDesc& I = h[i];
            e = cudaMemcpyAsync(ptr<int32_t>(c->A) + I.offA, A + srcA[i], sizeof(int32_t) * I.m * I.n, kind, c->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ptr<int64_t>(c->d) + I.offd, d + srcd[i], sizeof(int64_t) * I.m, kind, c->st);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->rb.p, hr.data(), sizeof(int32_t) * nR, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->inst0.p, h.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->inst.p, c->inst0.p, sizeof(InstDesc) * count, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // h is a host temporary
    if (e == cudaSuccess) e = cudaMemsetAsync(c->cnt.p, 0, sizeof(InstCounters) * count, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_build_lattice copies");
    c->hperm.assign(nR, 0);
    if (R > 1) {   // shuffled column orders of the replicas (and their bounds)
        permute_kernel<<<count, 128, 0, c->st>>>(c->P, ptr<int32_t>(c->colperm), ptr<int32_t>(c->rb),
                                                c->o.replica_seed);
        ++c->launches;
        if ((s = check_launch(c, "permute_kernel")) != MSP_OK) return s;
        e = cudaMemcpyAsync(c->hperm.data(), c->colperm.p, sizeof(int32_t) * nR, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), c->rb.p, sizeof(int32_t) * nR, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "permute");
    }
    c->hinst = h;
    c->layout = h;
    c->hr = hr;
    c->bounded = false;
    for (const InstDesc& I : h) c->bounded |= I.rmax > 1;
    // a captured step stays valid for new A, d of the same layout in the same buffers
    if (c->gexec && (std::memcmp(&c->graph_P, &c->P, sizeof(Pools)) != 0 || c->graph_inst.size() != h.size() ||
                     std::memcmp(c->graph_inst.data(), h.data(), sizeof(InstDesc) * h.size()) != 0))
        drop_graph(c);
    build_lattice_kernel<<<count, 128, 0, c->st>>>(c->P, c->o.N);
    ++c->launches;
    if ((s = check_launch(c, "build_lattice_kernel")) != MSP_OK) return s;
    c->state = 1;
    c->sout_valid = false;
    return MSP_OK;
}

msp_status msp_reduce(msp_ctx* c) {
    if (!c) return MSP_EINVAL;
    if (c->state < 1) return fail(c, MSP_ESTATE, "msp_reduce before msp_build_lattice");
    record(c, c->evr0);
    lll_kernel<<<c->count, 32, 0, c->st>>>(c->P, c->o.delta, c->o.eta, c->o.lll_max_iter,
                                           (unsigned long long)(c->o.max_seconds * 1e9));
    ++c->launches;
    msp_status s = check_launch(c, "lll_kernel");
    if (s != MSP_OK) return s;
    extract_gso_kernel<<<c->count, 32, 0, c->st>>>(c->P, 0);
    ++c->launches;
    if ((s = check_launch(c, "extract_gso_kernel")) != MSP_OK) return s;
    if (c->o.bkz_beta >= 2) {   // BKZ of the kernel basis, then its tables again
        BkzScratch S{nullptr, BkzScratch::bytes(c->Kmax, c->dimMax), c->Kmax, c->dimMax};
        if ((s = ensure(c, c->bkzs, (size_t)S.stride * c->count, "bkz scratch")) != MSP_OK) return s;
        S.base = ptr<char>(c->bkzs);
        bkz_kernel<<<c->count, 32, 0, c->st>>>(c->P, S, c->o.bkz_beta, c->o.delta, c->o.bkz_max_tours,
                                               c->o.lll_max_iter, (unsigned long long)(c->o.max_seconds * 1e9));
        ++c->launches;
        if ((s = check_launch(c, "bkz_kernel")) != MSP_OK) return s;
        extract_gso_kernel<<<c->count, 32, 0, c->st>>>(c->P, 1);
        ++c->launches;
        if ((s = check_launch(c, "extract_gso_kernel")) != MSP_OK) return s;
    }
    prep_fixed_kernel<<<c->count, 32, 0, c->st>>>(c->P, c->o.use_eps, c->dimPad);
    ++c->launches;
    if ((s = check_launch(c, "prep_fixed_kernel")) != MSP_OK) return s;
    record(c, c->evr1);
    c->reduce_timed = true;
    c->state = 2;
    return MSP_OK;
}

// A whole step can run as one fused launch (reduction and split inside the
// enumeration kernel) when the queue needs no global order: all solutions,
// depth-first, no feature log, binary bounds.
static bool fusable(const msp_ctx* c, int mode, int order) {
    if (!(c->o.fuse && mode == MSP_ALL && order == MSP_PLAIN && !c->o.log_features && !c->bounded)) return false;
    int blocks, threads;
    enum_launch_shape(c, &blocks, &threads);
    return enum_blocks_per_sm(c->lanes, threads, c->dimMax, c->Kmax, 3) * c->sms >= blocks;
}

// Queues one enumeration.  lds >= 0: one limited-discrepancy iteration with
// that budget; cont: a later iteration of the same search (counters, stored
// solutions, start time and deadline carry over).
static msp_status queue_enumerate(msp_ctx* c, int mode, int order, double time_cap_s, int lds = -1,
                                  bool cont = false, bool fused = false) {
    EnumCfg cfg{c->o.hoelder, c->o.sym, c->o.use_eps, mode == MSP_FIRST ? 1 : 0, lds, c->o.lds_rank};
    int blocks, threads;
    enum_launch_shape(c, &blocks, &threads);
    const int64_t walkers = walkers_of(c, blocks, threads);
    msp_status s = ensure(c, c->scratch, (size_t)walkers * walker_bytes(c->Kmax, c->dimPad), "scratch");
    if (s != MSP_OK) return s;
    if ((s = fit_frontier(c, mode, walkers)) != MSP_OK) return s;
    const int64_t target = std::min<int64_t>(split_target_of(c, mode, walkers), c->F);
    cudaError_t e = cont ? cudaSuccess : cudaMemsetAsync(c->cnt.p, 0, sizeof(InstCounters) * c->count, c->st);
    if (e == cudaSuccess && !cont) e = cudaMemsetAsync(c->gsolved.p, 0, sizeof(unsigned) * c->ucount, c->st);
    if (e == cudaSuccess && !cont) e = cudaMemsetAsync(c->gfirst.p, 0, sizeof(unsigned long long) * c->ucount, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->plog_nodes.p, 0, c->plog_nodes.bytes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->plog_sols.p, 0, c->plog_sols.bytes, c->st);
    if (e == cudaSuccess && c->o.donation_capacity > 0) e = launch_ring_init(ptr<unsigned long long>(c->don_seq), c->o.donation_capacity, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset counters");
    // the caller's cap, else the context's safety cap: no walk outlives it
    const double cap_s = time_cap_s > 0 ? std::min(time_cap_s, c->o.max_seconds) : c->o.max_seconds;
    const unsigned long long cap_ns = (unsigned long long)(cap_s * 1e9);
    Pipe pipe{};
    if (fused) {   // the reduction and the split run inside the enumeration launch
        if ((s = ensure(c, c->rl, sizeof(int64_t) * 3 * (size_t)c->count, "publish list")) != MSP_OK) return s;
        // ready flags of the publish list start at zero
        if ((e = cudaMemsetAsync(ptr<int64_t>(c->rl) + 2 * (size_t)c->count, 0, sizeof(int64_t) * (size_t)c->count,
                                 c->st)) != cudaSuccess)
            return cuda_fail(c, e, "publish list");
        pipe.on = 1;
        pipe.delta = c->o.delta;
        pipe.eta = c->o.eta;
        pipe.lll_max_iter = c->o.lll_max_iter;
        pipe.max_ns = (unsigned long long)(c->o.max_seconds * 1e9);
        pipe.bkz_beta = c->o.bkz_beta;
        pipe.bkz_max_tours = c->o.bkz_max_tours;
        if (c->o.bkz_beta >= 2) {
            BkzScratch S{nullptr, BkzScratch::bytes(c->Kmax, c->dimMax), c->Kmax, c->dimMax};
            if ((s = ensure(c, c->bkzs, (size_t)S.stride * c->count, "bkz scratch")) != MSP_OK) return s;
            S.base = ptr<char>(c->bkzs);
            pipe.S = S;
        }
        pipe.use_eps = c->o.use_eps;
        pipe.dimPad = c->dimPad;
        pipe.split_depth = c->o.split_depth;
        pipe.split_target = target;
        pipe.fcnt = ptr<int64_t>(c->fcnt);
        pipe.rl = ptr<int64_t>(c->rl);
        record(c, c->evr0);   // (reduction and split: inside the enumeration's time)
        record(c, c->evr1);
        c->reduce_timed = true;
    }
    if (!cont) record(c, c->ev0);
    if ((e = launch_start(ptr<Ctrl>(c->ctrl), cap_ns, cont ? 1 : 0, c->st)) != cudaSuccess)
        return cuda_fail(c, e, "start");
    ++c->launches;
    Pools Ps = c->P;
    Ps.skip = lds >= 0 ? ptr<unsigned char>(c->skip) : nullptr;
    if (!fused) {
        if ((e = launch_split(Ps, cfg, c->lanes, c->o.split_depth, target, ptr<int64_t>(c->fcnt), c->st)) !=
            cudaSuccess)
            return cuda_fail(c, e, "split");
        c->launches += 2;
    }
    // subtree features and queue order: the first-solution mode interleaves the
    // instances by rank (depth-first rank, or the scorer's rank when learned)
    const bool learned = (order == MSP_LEARNED || order == MSP_LDS_LEARNED) && c->scorer_set;
    const bool want_features = c->o.log_features || learned;
    Pools Pq = c->P;
    c->features_valid = false;
    if (want_features) {
        if ((e = launch_features(c->P, ptr<float>(c->prof), ptr<float>(c->feat), c->sms, c->st)) != cudaSuccess)
            return cuda_fail(c, e, "features");
        c->launches += 2;
        c->features_valid = true;
    }
    if (mode == MSP_FIRST || learned) {
        const int64_t cap = (int64_t)c->count * c->F;
        int64_t npad = 1;
        while (npad < cap) npad <<= 1;
        const float* y = nullptr;
        if (learned) {
            if ((e = mlp_forward(ptr<float>(c->theta), ptr<float>(c->feat), cap, ptr<float>(c->yout), c->sms, c->st)) !=
                cudaSuccess)
                return cuda_fail(c, e, "scorer");
            ++c->launches;
            y = ptr<float>(c->yout);
        }
        if ((e = launch_order(c->P, y, npad, ptr<unsigned long long>(c->skeys), ptr<unsigned long long>(c->svals),
                              ptr<unsigned long long>(c->skeys2), ptr<unsigned long long>(c->svals2),
                              ptr<int64_t>(c->perm), c->sms, c->st, &c->launches)) != cudaSuccess)
            return cuda_fail(c, e, "order");
        Pq.qperm = ptr<int64_t>(c->perm);
    }
    if (!cont) record(c, c->evs1);
    // walker variant: general bounds, binary discrepancy search, or plain
    const int variant = fused ? 3 : (c->bounded ? 2 : (lds >= 0 ? 1 : 0));
    if ((e = launch_enum(Pq, cfg, c->lanes, blocks, threads, ptr<char>(c->scratch), c->Kmax, c->dimPad,
                         variant, pipe, c->st)) !=
        cudaSuccess)
        return cuda_fail(c, e, "enumerate");
    ++c->launches;
    record(c, c->eve1);
    if ((e = launch_collect(c->P, ptr<int64_t>(c->soff), ptr<unsigned long long>(c->fill), ptr<SolRec>(c->seg),
                            ptr<SolRec>(c->sout), c->st)) != cudaSuccess)
        return cuda_fail(c, e, "collect");
    c->launches += 4;
    record(c, c->ev1);
    c->last_mode = mode;
    c->last_lds = lds >= 0;
    c->last_fused = fused;
    c->state = 3;
    c->sout_valid = false;
    return MSP_OK;
}

// Limited discrepancy search (Sec. 3): iterations with budgets 0, 1, 2, ...
// (or the one budget of opts.lds_budget).  Between iterations the host reads
// the per-instance counters: an instance is finished once it has a solution
// (MSP_FIRST) or once an iteration held no value back for want of budget
// (its tree is exhausted); finished instances get no subtrees afterwards.
static msp_status run_lds(msp_ctx* c, int mode, int order, double time_cap_s) {
    const int n = c->count;
    msp_status s = ensure(c, c->skip, (size_t)n, "skip");
    if (s != MSP_OK) return s;
    std::vector<unsigned char> skip(n, 0);
    std::vector<unsigned long long> cuts_seen(n, 0);
    std::vector<InstCounters> cn(n);
    std::vector<InstDesc> h(n);
    c->lds_done.assign(n, -1);
    const int k0 = c->o.lds_budget >= 0 ? c->o.lds_budget : 0;
    const int k1 = c->o.lds_budget >= 0 ? c->o.lds_budget : c->o.lds_max;
    cudaError_t e = cudaMemsetAsync(c->skip.p, 0, (size_t)n, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "lds skip");
    for (int k = k0; k <= k1; ++k) {
        if ((s = queue_enumerate(c, mode, order, time_cap_s, k, k != k0)) != MSP_OK) return s;
        Ctrl ctl;
        e = cudaStreamSynchronize(c->st);
        if (e == cudaSuccess) e = cudaMemcpy(cn.data(), c->cnt.p, sizeof(InstCounters) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), c->inst.p, sizeof(InstDesc) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&ctl, c->ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "lds iteration");
        std::vector<unsigned> gs(c->ucount, 0);
        e = cudaMemcpy(gs.data(), c->gsolved.p, sizeof(unsigned) * c->ucount, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "lds iteration");
        bool all_done = true;
        for (int i = 0; i < n; ++i) {
            if (skip[i]) continue;
            const unsigned long long cuts = cn[i].lds_cuts - cuts_seen[i];
            cuts_seen[i] = cn[i].lds_cuts;
            const bool finished = h[i].status != ST_OK || (mode == MSP_FIRST && gs[h[i].group]) || cuts == 0;
            if (finished) {
                skip[i] = 1;
                c->lds_done[i] = k;
            } else {
                all_done = false;
            }
        }
        if (all_done || ctl.stop == 2 || k == k1) break;
        e = cudaMemcpyAsync(c->skip.p, skip.data(), (size_t)n, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // skip is a host temporary
        if (e != cudaSuccess) return cuda_fail(c, e, "lds skip");
    }
    return MSP_OK;
}

msp_status msp_run_async(msp_ctx* c, int mode, int order) {
    if (!c) return MSP_EINVAL;
    if (c->state < 1) return fail(c, MSP_ESTATE, "msp_run_async before msp_build_lattice");
    if (mode != MSP_ALL && mode != MSP_FIRST) return fail(c, MSP_EINVAL, "bad mode");
    if (order != MSP_PLAIN && order != MSP_LEARNED)
        return fail(c, MSP_EINVAL, "msp_run_async: order must be MSP_PLAIN or MSP_LEARNED (MSP_LDS: msp_enumerate)");
    if (fusable(c, mode, order)) return queue_enumerate(c, mode, order, 0.0, -1, false, true);
    msp_status s = msp_reduce(c);
    if (s != MSP_OK) return s;
    return queue_enumerate(c, mode, order, 0.0);
}

// One whole step on the device-resident batch: descriptors reset from the
// pristine copy, lattice rebuilt from the stored A and d, reduction, split,
// order, enumeration, collection.  No host synchronisation inside.
static msp_status queue_step(msp_ctx* c, int mode, int order) {
    cudaError_t e = cudaMemcpyAsync(c->inst.p, c->inst0.p, sizeof(InstDesc) * c->count, cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "reset descriptors");
    build_lattice_kernel<<<c->count, 128, 0, c->st>>>(c->P, c->o.N);
    ++c->launches;
    msp_status s = check_launch(c, "build_lattice_kernel");
    if (s != MSP_OK) return s;
    if (fusable(c, mode, order)) return queue_enumerate(c, mode, order, 0.0, -1, false, true);
    if ((s = msp_reduce(c)) != MSP_OK) return s;
    return queue_enumerate(c, mode, order, 0.0);
}

msp_status msp_graph_capture(msp_ctx* c, int mode, int order) {
    if (!c) return MSP_EINVAL;
    if (c->state < 3) return fail(c, MSP_ESTATE, "msp_graph_capture: run one enumeration of the batch first");
    if (mode != MSP_ALL && mode != MSP_FIRST) return fail(c, MSP_EINVAL, "bad mode");
    if (order != MSP_PLAIN && order != MSP_LEARNED)
        return fail(c, MSP_EINVAL, "msp_graph_capture: order must be MSP_PLAIN or MSP_LEARNED");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_graph_capture sync");
    drop_graph(c);
    {   // every buffer the step touches exists before the capture starts
        int blocks, threads;
        enum_launch_shape(c, &blocks, &threads);
        msp_status s0 = fit_frontier(c, mode, walkers_of(c, blocks, threads));
        if (s0 != MSP_OK) return s0;
    }
    // the caller's stream may be the legacy default stream, which cannot be
    // captured: capture on a private stream, replay on the caller's
    if (!c->cst && (e = cudaStreamCreateWithFlags(&c->cst, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(c, e, "capture stream");
    const int64_t launches0 = c->launches;
    cudaStream_t user = c->st;
    c->st = c->cst;
    e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { c->st = user; return cuda_fail(c, e, "cudaStreamBeginCapture"); }
    msp_status s = queue_step(c, mode, order);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->st, &g);
    c->st = user;
    if (s != MSP_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(c, e, "cudaGraphInstantiate"); }
    c->graph = g;
    c->graph_P = c->P;
    c->graph_inst = c->layout;
    c->graph_launches = c->launches - launches0;
    c->launches = launches0;
    c->graph_mode = mode;
    return MSP_OK;
}

msp_status msp_graph_launch(msp_ctx* c) {
    if (!c) return MSP_EINVAL;
    if (!c->gexec) return fail(c, MSP_ESTATE, "msp_graph_launch before msp_graph_capture");
    cudaError_t e = cudaGraphLaunch(c->gexec, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    c->launches += c->graph_launches;
    c->last_mode = c->graph_mode;
    c->state = 3;
    c->sout_valid = false;
    return MSP_OK;
}

// The stored solutions of internal instance i, decoded (x_j in a field of
// bound_bits(r_j) bits, most significant first, from key bit 127 down) and
// put back in the caller's column order (replica k > 0 permuted them).
static msp_status decode_instance(msp_ctx* c, int i, std::vector<std::vector<uint8_t>>& out) {
    const int64_t lo = c->soff_h[i], have = c->soff_h[i + 1] - lo;
    std::vector<SolRec> rec((size_t)std::max<int64_t>(have, 0));
    if (have > 0) {
        cudaError_t e = cudaMemcpy(rec.data(), ptr<SolRec>(c->sout) + lo, sizeof(SolRec) * have, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "msp_solutions copy");
    }
    const InstDesc& I = c->layout[i];
    const int n = I.n;
    const int32_t* rr = c->hr.data() + I.offR;
    const int32_t* pi = c->hperm.data() + I.offR;
    const bool permuted = c->ucount != c->count && I.replica > 0;
    for (const SolRec& q : rec) {
        std::vector<uint8_t> x(n);
        int off = 0;
        for (int j = 0; j < n; ++j) {
            const int w = bound_bits(rr[j]);
            const int sh = 128 - off - w;
            const unsigned long long v =
                sh >= 64 ? (q.hi >> (sh - 64)) : ((q.lo >> sh) | (sh > 0 ? q.hi << (64 - sh) : 0ULL));
            x[permuted ? pi[j] : j] = (uint8_t)(v & ((1ULL << w) - 1ULL));
            off += w;
        }
        out.push_back(std::move(x));
    }
    return MSP_OK;
}

// All replicas' solutions of the caller's instance g, sorted and distinct.
static msp_status group_solutions(msp_ctx* c, int g, std::vector<std::vector<uint8_t>>& out) {
    const int R = c->count / c->ucount;
    for (int k = 0; k < R; ++k) {
        msp_status s = decode_instance(c, g * R + k, out);
        if (s != MSP_OK) return s;
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return MSP_OK;
}

msp_status msp_wait(msp_ctx* c, msp_stats* stats, msp_stats* total) {
    if (!c) return MSP_EINVAL;
    if (c->state < 3) return fail(c, MSP_ESTATE, "msp_wait before an enumeration");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "enumeration");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->last_ms = ms;
    std::vector<InstDesc> h(c->count);
    std::vector<InstCounters> cn(c->count);
    Ctrl ctl;
    c->soff_h.assign(c->count + 1, 0);
    e = cudaMemcpy(h.data(), c->inst.p, sizeof(InstDesc) * c->count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(cn.data(), c->cnt.p, sizeof(InstCounters) * c->count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ctl, c->ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->soff_h.data(), c->soff.p, sizeof(int64_t) * (c->count + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading results");
    c->hinst = h;
    c->stats.assign(c->count, msp_stats{});
    msp_status first_bad = MSP_OK;
    msp_stats tot{};
    const bool trunc = (int64_t)ctl.nsol_total > c->o.sol_capacity;
    for (int i = 0; i < c->count; ++i) {
        msp_stats& S = c->stats[i];
        S.nodes = (int64_t)cn[i].nodes;
        S.passed = (int64_t)cn[i].passed;
        S.leaves = (int64_t)cn[i].leaves;
        S.solutions = (int64_t)cn[i].nsol;
        S.prefixes = h[i].nprefix;
        S.split_level = h[i].split_level;
        S.kernel_rank = h[i].dd;
        S.lll_iterations = h[i].lll_iters;
        S.lll_swaps = h[i].lll_swaps;
        S.bkz_tours = h[i].bkz_tours;
        S.bkz_inserts = h[i].bkz_inserts;
        S.bkz_nodes = h[i].bkz_nodes;
        S.split_nodes = (int64_t)cn[i].split_nodes;
        S.split_passed = (int64_t)cn[i].split_passed;
        S.center_fma = (int64_t)cn[i].center_fma;
        S.fallbacks = (int64_t)cn[i].fallbacks;
        S.first_ms = (c->last_mode == MSP_FIRST && cn[i].nsol > 0) ? (double)cn[i].first_ns * 1e-6 : -1.0;
        S.lds_budget = (c->last_lds && i < (int)c->lds_done.size()) ? c->lds_done[i] : -1;
        int32_t st = h[i].status;
        if (st == MSP_OK && ctl.stop == 2) st = MSP_ETIMEOUT;
        // the iterated discrepancy search reached opts.lds_max with the tree not exhausted
        if (st == MSP_OK && c->last_lds && c->o.lds_budget < 0 && S.lds_budget < 0) st = MSP_ECAP;
        if (st == MSP_OK && trunc) st = MSP_ETRUNC;
        S.status = st;
        S.ms = ms;
        if (st != MSP_OK && first_bad == MSP_OK) first_bad = (msp_status)st;
        tot.nodes += S.nodes;
        tot.passed += S.passed;
        tot.leaves += S.leaves;
        tot.solutions += S.solutions;
        tot.prefixes += S.prefixes;
        tot.lll_iterations += S.lll_iterations;
        tot.lll_swaps += S.lll_swaps;
        tot.bkz_tours += S.bkz_tours;
        tot.bkz_inserts += S.bkz_inserts;
        tot.bkz_nodes += S.bkz_nodes;
        tot.split_nodes += S.split_nodes;
        tot.split_passed += S.split_passed;
        tot.center_fma += S.center_fma;
        tot.fallbacks += S.fallbacks;
    }
    tot.status = first_bad;
    tot.ms = ms;
    tot.donations = (int64_t)ctl.donations;
    tot.walker_util = ctl.life_cycles ? (double)ctl.walk_cycles / (double)ctl.life_cycles : 0.0;
    if (c->ucount != c->count) {   // replicas: one record per caller's instance
        c->sout_valid = false;
        std::vector<unsigned> gs(c->ucount, 0);
        std::vector<unsigned long long> gf(c->ucount, 0);
        e = cudaMemcpy(gs.data(), c->gsolved.p, sizeof(unsigned) * c->ucount, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gf.data(), c->gfirst.p, sizeof(unsigned long long) * c->ucount,
                                             cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "reading group results");
        const int R = c->count / c->ucount;
        std::vector<msp_stats> u(c->ucount, msp_stats{});
        tot.solutions = 0;
        for (int g = 0; g < c->ucount; ++g) {
            msp_stats& U = u[g];
            U = c->stats[(size_t)g * R];   // sizes, split level, rank: replica 0
            U.status = MSP_OK;
            U.lds_budget = -1;
            for (int k = 0; k < R; ++k) {
                const msp_stats& S = c->stats[(size_t)g * R + k];
                if (k > 0) {
                    U.nodes += S.nodes; U.passed += S.passed; U.leaves += S.leaves; U.prefixes += S.prefixes;
                    U.lll_iterations += S.lll_iterations; U.lll_swaps += S.lll_swaps;
                    U.bkz_tours += S.bkz_tours; U.bkz_inserts += S.bkz_inserts; U.bkz_nodes += S.bkz_nodes;
                    U.split_nodes += S.split_nodes; U.split_passed += S.split_passed;
                    U.center_fma += S.center_fma; U.fallbacks += S.fallbacks;
                }
                if (S.status != MSP_OK && U.status == MSP_OK) U.status = S.status;
                U.lds_budget = std::max(U.lds_budget, S.lds_budget);
            }
            U.first_ms = (c->last_mode == MSP_FIRST && gs[g]) ? (double)gf[g] * 1e-6 : -1.0;
            std::vector<std::vector<uint8_t>> xs;
            msp_status sg = group_solutions(c, g, xs);
            if (sg != MSP_OK) return sg;
            U.solutions = (int64_t)xs.size();
            tot.solutions += U.solutions;
        }
        c->stats = u;
    }
    if (stats) std::memcpy(stats, c->stats.data(), sizeof(msp_stats) * c->stats.size());
    if (total) *total = tot;
    return first_bad;
}

msp_status msp_enumerate(msp_ctx* c, int mode, int order, double time_cap_s, msp_stats* stats, msp_stats* total) {
    if (!c) return MSP_EINVAL;
    if (c->state < 2) return fail(c, MSP_ESTATE, "msp_enumerate before msp_reduce");
    if (mode != MSP_ALL && mode != MSP_FIRST) return fail(c, MSP_EINVAL, "bad mode");
    if (order != MSP_PLAIN && order != MSP_LEARNED && order != MSP_LDS && order != MSP_LDS_LEARNED)
        return fail(c, MSP_EINVAL, "bad order");
    const bool lds = order == MSP_LDS || order == MSP_LDS_LEARNED;
    msp_status s = lds ? run_lds(c, mode, order, time_cap_s) : queue_enumerate(c, mode, order, time_cap_s);
    if (s != MSP_OK) return s;
    return msp_wait(c, stats, total);
}

int msp_lanes(const msp_ctx* c) { return (c && c->state >= 1) ? c->lanes : 0; }

int msp_mlp_param_count(void) { return mlp_param_count(); }

msp_status msp_set_scorer(msp_ctx* c, const float* theta) {
    if (!c) return MSP_EINVAL;
    if (!theta) { c->scorer_set = false; return MSP_OK; }
    msp_status s = ensure(c, c->theta, sizeof(float) * mlp_param_count(), "theta");
    if (s != MSP_OK) return s;
    cudaError_t e = cudaMemcpyAsync(c->theta.p, theta, sizeof(float) * mlp_param_count(), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_set_scorer");
    c->scorer_set = true;
    return MSP_OK;
}

msp_status msp_export_features(msp_ctx* c, int inst, float* feat, size_t cap, size_t* count) {
    if (!c || !count) return MSP_EINVAL;
    if (c->state < 3 || !c->features_valid) return fail(c, MSP_ESTATE, "msp_export_features: no features logged");
    if (inst < 0 || inst >= c->count) return fail(c, MSP_EINVAL, "instance index out of range");
    cudaError_t e = cudaStreamSynchronize(c->st);
    int64_t q[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(q, ptr<int64_t>(c->qbase) + inst, sizeof q, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_features");
    *count = (size_t)(q[1] - q[0]);
    const int64_t take = std::min<int64_t>(q[1] - q[0], (int64_t)cap);
    if (feat && take > 0) {
        e = cudaMemcpy(feat, ptr<float>(c->feat) + q[0] * 32, sizeof(float) * 32 * take, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_features copy");
    }
    return MSP_OK;
}

msp_status msp_mlp_forward(msp_ctx* c, const float* theta, const float* x, int64_t n, float* y) {
    if (!c || !theta || !x || !y || n < 0) return MSP_EINVAL;
    cudaError_t e = mlp_forward(theta, x, n, y, c->sms, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_mlp_forward");
    ++c->launches;
    return MSP_OK;
}

msp_status msp_mlp_grad(msp_ctx* c, const float* theta, const float* x, const float* target, int64_t n,
                        float pos_weight, float* grad, float* loss) {
    if (!c || !theta || !x || !target || !grad || !loss || n < 1) return MSP_EINVAL;
    cudaError_t e = mlp_grad(theta, x, target, n, pos_weight, grad, loss, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_mlp_grad");
    ++c->launches;
    return MSP_OK;
}

msp_status msp_mlp_train(msp_ctx* c, float* theta, const float* x, const float* target, int64_t n, int steps,
                         float lr, float pos_weight, uint64_t seed, float* losses) {
    if (!c || !theta || !x || !target || n < 1 || steps < 1 || !(lr > 0.f)) return MSP_EINVAL;
    msp_status s = ensure(c, c->mlpwork, sizeof(float) * 3 * mlp_param_count(), "mlpwork");
    if (s != MSP_OK) return s;
    cudaError_t e = mlp_train(theta, x, target, n, steps, lr, pos_weight, seed, ptr<float>(c->mlpwork), losses, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_mlp_train");
    ++c->launches;
    return MSP_OK;
}

msp_status msp_fp64_peak(msp_ctx* c, double* dfma_per_s) {
    if (!c || !dfma_per_s) return MSP_EINVAL;
    cudaError_t e = fp64_peak(dfma_per_s, c->sms, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_fp64_peak");
    c->launches += 4;
    return MSP_OK;
}

msp_status msp_phase_ms(msp_ctx* c, double* out) {
    if (!c || !out) return MSP_EINVAL;
    if (c->state < 3) return fail(c, MSP_ESTATE, "msp_phase_ms before an enumeration");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_phase_ms");
    float r = 0.f, s = 0.f, n = 0.f, k = 0.f;
    if (c->reduce_timed) cudaEventElapsedTime(&r, c->evr0, c->evr1);
    cudaEventElapsedTime(&s, c->ev0, c->evs1);
    cudaEventElapsedTime(&n, c->evs1, c->eve1);
    cudaEventElapsedTime(&k, c->eve1, c->ev1);
    out[0] = r; out[1] = s; out[2] = n; out[3] = k;
    return MSP_OK;
}

msp_status msp_solutions(msp_ctx* c, int inst, uint8_t* x, size_t cap, size_t* count) {
    if (!c || !count) return MSP_EINVAL;
    if (c->state < 3 || c->stats.empty()) return fail(c, MSP_ESTATE, "msp_solutions before msp_wait");
    if (inst < 0 || inst >= (int)c->stats.size()) return fail(c, MSP_EINVAL, "instance index out of range");
    const int64_t found = c->stats[inst].solutions;
    *count = (size_t)found;
    if (cap == 0) return MSP_OK;
    if (!x) return MSP_EINVAL;
    if (c->ucount != c->count) {   // replicas: the union of the replicas' solutions, caller's order
        std::vector<std::vector<uint8_t>> xs;
        msp_status s = group_solutions(c, inst, xs);
        if (s != MSP_OK) return s;
        const size_t take = std::min(xs.size(), cap);
        for (size_t k = 0; k < take; ++k) std::memcpy(x + k * xs[k].size(), xs[k].data(), xs[k].size());
        return (take < (size_t)found) ? MSP_ETRUNC : MSP_OK;
    }
    const int64_t lo = c->soff_h[inst];
    const int64_t have = c->soff_h[inst + 1] - lo;   // stored records of this instance
    const int64_t take = std::min<int64_t>(have, (int64_t)cap);
    std::vector<SolRec> rec(take);
    if (take > 0) {
        cudaError_t e = cudaMemcpy(rec.data(), ptr<SolRec>(c->sout) + lo, sizeof(SolRec) * take, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "msp_solutions copy");
    }
    const int n = c->hinst[inst].n;
    const int32_t* rr = c->hr.data() + c->layout[inst].offR;
    for (int64_t k = 0; k < take; ++k) {
        int off = 0;   // x_j: bound_bits(r_j) bits, most significant first, from key bit 127 down
        for (int j = 0; j < n; ++j) {
            const int w = bound_bits(rr[j]);
            const int sh = 128 - off - w;
            unsigned long long v = sh >= 64 ? (rec[k].hi >> (sh - 64))
                                            : ((rec[k].lo >> sh) | (sh > 0 ? rec[k].hi << (64 - sh) : 0ULL));
            x[(size_t)k * n + j] = (uint8_t)(v & ((1ULL << w) - 1ULL));
            off += w;
        }
    }
    return (take < found) ? MSP_ETRUNC : MSP_OK;
}

msp_status msp_export_gso(msp_ctx* c, int inst, int32_t* dims_out, int32_t* basis, double* mu, double* B,
                          double* bhat) {
    if (!c) return MSP_EINVAL;
    if (c->state < 2) return fail(c, MSP_ESTATE, "msp_export_gso before msp_reduce");
    if (inst < 0 || inst >= c->count) return fail(c, MSP_EINVAL, "instance index out of range");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_gso sync");
    InstDesc I;
    e = cudaMemcpy(&I, ptr<InstDesc>(c->inst) + inst, sizeof I, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_gso");
    if (I.status != MSP_OK) return (msp_status)I.status;
    const int dd = I.dd, dim = I.dim;
    if (dims_out) { dims_out[0] = dd; dims_out[1] = dim; }
    if (basis) e = cudaMemcpy(basis, ptr<int32_t>(c->kb) + I.offKb, sizeof(int32_t) * dd * dim, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && B) e = cudaMemcpy(B, ptr<double>(c->B) + I.offB, sizeof(double) * dd, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && bhat)
        e = cudaMemcpy(bhat, ptr<double>(c->bhat) + I.offBhat, sizeof(double) * dd * dim, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mu) {
        std::vector<double> t((size_t)dd * dd);
        e = cudaMemcpy(t.data(), ptr<double>(c->muT) + I.offMuT, sizeof(double) * dd * dd, cudaMemcpyDeviceToHost);
        for (int i = 0; i < dd; ++i)
            for (int j = 0; j < dd; ++j) mu[(size_t)i * dd + j] = (j <= i) ? t[(size_t)j * dd + i] : 0.0;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_gso copies");
    return MSP_OK;
}

msp_status msp_export_reduced(msp_ctx* c, int inst, int64_t* basis) {
    if (!c || !basis) return MSP_EINVAL;
    if (c->state < 2) return fail(c, MSP_ESTATE, "msp_export_reduced before msp_reduce");
    if (inst < 0 || inst >= c->count) return fail(c, MSP_EINVAL, "instance index out of range");
    cudaError_t e = cudaStreamSynchronize(c->st);
    InstDesc I;
    if (e == cudaSuccess) e = cudaMemcpy(&I, ptr<InstDesc>(c->inst) + inst, sizeof I, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(basis, ptr<int64_t>(c->basis) + I.offBasis, sizeof(int64_t) * I.K * I.L, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_reduced");
    return (msp_status)I.status;
}

msp_status msp_export_prefixes(msp_ctx* c, int inst, int32_t* u, double* rho, int64_t* nodes, int32_t* sols,
                               size_t cap, size_t* count, int32_t* split_level) {
    if (!c || !count) return MSP_EINVAL;
    if (c->state < 3) return fail(c, MSP_ESTATE, "msp_export_prefixes before an enumeration");
    if (inst < 0 || inst >= c->count) return fail(c, MSP_EINVAL, "instance index out of range");
    cudaError_t e = cudaStreamSynchronize(c->st);
    InstDesc I;
    if (e == cudaSuccess) e = cudaMemcpy(&I, ptr<InstDesc>(c->inst) + inst, sizeof I, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_prefixes");
    *count = (size_t)I.nprefix;
    if (split_level) *split_level = I.split_level;
    const int64_t take = std::min<int64_t>(I.nprefix, (int64_t)cap);
    const int64_t base = ((int64_t)inst * 2 + I.front_sel) * c->F;
    if (u && take > 0) {
        std::vector<int32_t> tmp((size_t)take * c->Kmax);
        e = cudaMemcpy(tmp.data(), ptr<int32_t>(c->fu) + base * c->Kmax, sizeof(int32_t) * tmp.size(),
                       cudaMemcpyDeviceToHost);
        for (int64_t p = 0; p < take; ++p)
            for (int i = 0; i < I.dd; ++i) u[(size_t)p * I.dd + i] = tmp[(size_t)p * c->Kmax + i];
    }
    if (e == cudaSuccess && rho && take > 0)
        e = cudaMemcpy(rho, ptr<double>(c->frho) + base, sizeof(double) * take, cudaMemcpyDeviceToHost);
    // the subtree log is indexed by queue position
    if (e == cudaSuccess && (nodes || sols) && take > 0) {
        int64_t q0 = 0;
        e = cudaMemcpy(&q0, ptr<int64_t>(c->qbase) + inst, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && nodes)
            e = cudaMemcpy(nodes, ptr<int64_t>(c->plog_nodes) + q0, sizeof(int64_t) * take, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && sols)
            e = cudaMemcpy(sols, ptr<int32_t>(c->plog_sols) + q0, sizeof(int32_t) * take, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "msp_export_prefixes copies");
    return MSP_OK;
}

}  // extern "C"
