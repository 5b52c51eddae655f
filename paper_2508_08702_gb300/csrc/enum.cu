// enum.cu -- steps a4-a7 of the hot path (Algorithm 1) on the device:
//   split_kernel     expands the top levels of each instance's search tree
//                    breadth-first with the exact rules of Algorithm 1 and
//                    leaves the surviving prefixes as independent subtrees
//                    (the tree partition of Sec. 4), in depth-first order
//   queue_kernel     global work queue over all instances' prefixes
//   enum_kernel      persistent walkers: a group of G lanes runs the depth-
//                    first search of one subtree at a time; lane l owns the
//                    coordinates c = l (mod G) of the projected vectors w
//   collect kernels  solutions sorted per instance
//
// Arithmetic of a node (t, u) at level t, given the parent's w' = w^(t+1)
// and rho' = ||w'||^2 (first pruning condition, Sec. 2):
//   y_t  = fold i = d-1 .. t+1 of acc = fma(u_i, mu_it, acc)      (centre)
//   x    = u + y_t;  rho = fma(x*x, B_t, rho')                      (norm)
//   prune when rho > R + eps, R = (n+1) r_max^2
//   t > 0: w = fma(x, bhat_t, w') per coordinate;  ||w||_1 as G lane
//   partials (ascending coordinates) combined pairwise; Hoelder test of
//   Theorem 2: fail when rho > ||w||_1 + eps.  First failure: one more
//   zig-zag value, then walk only in that direction; second failure or a
//   norm failure: step back.
//   t = 0: exact integer check of v = sum_j u_j b_j (Theorem 1).
// Limited discrepancy search (Sec. 3): a value other than the first of its
// level's walk (u^1, the rounded centre) is a discrepancy, costing its
// position p in the walk (rank reading) or one (flat reading); an iteration
// with budget k tries a value only while the path's cost stays at most k and
// reports a leaf only when the cost is exactly k.
// The centre uses the partial-sum cache of Gama-Nguyen-Regev: sigma[t][i]
// holds the fold down to index i, J[t] the highest level changed since, so
// only the changed tail of the fold is redone -- the same operations in
// the same order as the full fold.
#include "common.cuh"
#include "reduce.cuh"

namespace msp {

enum { HOELDER_CUT = 0, HOELDER_FILTER = 1, HOELDER_OFF = 2 };
constexpr int kUMax = 1 << 15;   // |u| bound: levels store u as int16

__device__ __forceinline__ int zigzag(int u1, int s, int i) {
    return (i & 1) == 0 ? u1 + s * (i >> 1) : u1 - s * ((i - 1) >> 1);
}

// R = (n+1) r_max^2 (Sec. 2) and the slack of reading R4, R 2^-20
__device__ __forceinline__ double bound_R(const InstDesc& I) {
    return (double)I.dim * (double)I.rmax * (double)I.rmax;
}

__device__ __forceinline__ double slack_of(double R, int use_eps) {
    return use_eps ? R * 0x1p-20 : 0.0;
}

// ---------------------------------------------------------------------------
// Splitter: one block per instance.
// ---------------------------------------------------------------------------

// Sibling loop of one parent at level t (one thread).  With WRITE, children
// that pass both tests are written at out index base, base+1, ...
template <int G, bool WRITE>
__device__ int64_t expand_parent(const Pools& P, const EnumCfg& cfg, int inst, int dd, int dim, int t,
                                 const int32_t* __restrict__ pu, double prho, const double* __restrict__ pw,
                                 int pdisc, float pxsum, int out_sel, int64_t base, unsigned long long& nodes,
                                 unsigned long long& passed, unsigned long long& cuts, bool& ovf) {
    const InstDesc& I = P.inst[inst];
    const double* muT = P.muT + I.offMuT;
    const double* Bt = P.B + I.offB;
    const double* bhat = P.bhat + I.offBhat;
    const double R = bound_R(I);
    const double eps = slack_of(R, cfg.use_eps);
    const double Rb = R + eps;
    const double rmaxd = (double)I.rmax;

    double y = 0.0;
    bool zp = true;
    for (int i = dd - 1; i > t; --i) {
        y = __fma_rn((double)pu[i], muT[(int64_t)t * dd + i], y);
        zp = zp && (pu[i] == 0);
    }
    const double cstar = -y;
    const double r1 = rint(cstar);
    if (fabs(r1) >= (double)kUMax) { ovf = true; return 0; }
    int u1 = (int)r1;
    const int s = (cstar >= r1) ? 1 : -1;
    bool onedir = false;
    int dir = 0, zi = 1;
    if (zp && cfg.sym) { u1 = 0; onedir = true; dir = 1; }
    int u = u1;
    int pos = 0;   // position of u in this level's walk
    int64_t nch = 0;
    for (;;) {
        const int cost = cfg.lds_rank ? pos : (u != u1 ? 1 : 0);
        if (cfg.lds >= 0 && cost > 0 && pdisc + cost > cfg.lds) {   // discrepancy budget spent
            if (WRITE) ++cuts;
            break;
        }
        if (u >= kUMax || u <= -kUMax) { ovf = true; break; }
        const double x = __dadd_rn((double)u, y);
        const double rho = __fma_rn(__dmul_rn(x, x), Bt[t], prho);
        if (WRITE) ++nodes;
        if (rho > Rb) break;
        if (WRITE) ++passed;
        double sl[G];
#pragma unroll
        for (int l = 0; l < G; ++l) sl[l] = 0.0;
        for (int c0 = 0; c0 < dim; c0 += G) {
#pragma unroll
            for (int l = 0; l < G; ++l) {
                const int c = c0 + l;
                if (c < dim) sl[l] = __dadd_rn(sl[l], fabs(__fma_rn(x, bhat[(int64_t)t * dim + c], pw[c])));
            }
        }
#pragma unroll
        for (int off = G / 2; off >= 1; off >>= 1) {
#pragma unroll
            for (int l = 0; l < off; ++l) sl[l] = __dadd_rn(sl[l], sl[l + off]);
        }
        bool fail = false;
        if (cfg.hoelder != HOELDER_OFF) fail = rho > __dadd_rn(__dmul_rn(rmaxd, sl[0]), eps);
        if (fail && cfg.hoelder == HOELDER_CUT) {
            if (onedir) break;
            ++zi;
            u = zigzag(u1, s, zi);
            dir = (u > u1) ? 1 : -1;
            onedir = true;
            ++pos;
            continue;
        }
        if (!fail) {
            if (WRITE) {
                const int64_t o = frontier_index(P, inst, out_sel, base + nch);
                int32_t* ou = P.fu + o * P.Kmax;
                for (int i = 0; i < P.Kmax; ++i) ou[i] = (i > t && i < dd) ? pu[i] : 0;
                ou[t] = u;
                P.frho[o] = rho;
                P.fdisc[o] = pdisc + cost;
                P.fxsum[o] = pxsum + (float)fabs(x);
                double* ow = P.fw + o * P.dimPad;
                for (int c = 0; c < dim; ++c) ow[c] = __fma_rn(x, bhat[(int64_t)t * dim + c], pw[c]);
            }
            ++nch;
        }
        if (onedir) u += dir;
        else { ++zi; u = zigzag(u1, s, zi); }
        ++pos;
    }
    return nch;
}

// exclusive scan of cnt[0..n) in place (block-wide); returns the total
__device__ int64_t block_exclusive_scan(int64_t* cnt, int64_t n) {
    __shared__ int64_t part[1024 + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t chunk = (n + nt - 1) / nt;
    const int64_t lo = tid * chunk, hi = min(n, lo + chunk);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int i = 0; i < nt; ++i) { const int64_t v = part[i]; part[i] = run; run += v; }
        part[nt] = run;
    }
    __syncthreads();
    int64_t run = part[tid];
    for (int64_t i = lo; i < hi; ++i) { const int64_t v = cnt[i]; cnt[i] = run; run += v; }
    const int64_t total = part[nt];
    __syncthreads();
    return total;
}

// The split of one instance by a whole block (any number of threads).
template <int G>
__device__ __noinline__ void split_inst(const Pools& P, const EnumCfg& cfg, int inst, int max_depth, int64_t target,
                                        int64_t* fcnt) {
    InstDesc& I = P.inst[inst];
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = (I.status == ST_OK) && !(P.skip && P.skip[inst]);
    __syncthreads();
    if (!s_ok) {
        if (threadIdx.x == 0) { I.nprefix = 0; I.split_level = 0; I.front_sel = 0; }
        return;
    }
    const int dd = I.dd, dim = I.dim;
    int64_t* cnt = fcnt + (int64_t)inst * P.F;
    // root parent: nothing fixed, w = 0, rho = 0
    {
        const int64_t o = frontier_index(P, inst, 0, 0);
        for (int i = threadIdx.x; i < P.Kmax; i += blockDim.x) P.fu[o * P.Kmax + i] = 0;
        for (int c = threadIdx.x; c < P.dimPad; c += blockDim.x) P.fw[o * P.dimPad + c] = 0.0;
        if (threadIdx.x == 0) { P.frho[o] = 0.0; P.fdisc[o] = 0; P.fxsum[o] = 0.f; }
    }
    __syncthreads();
    int sel = 0, t = dd - 1, depth = 0;
    int64_t count = 1;
    unsigned long long nodes = 0, passed = 0, cuts = 0;
    bool ovf = false;
    __shared__ int s_ovf;
    while (depth < max_depth && t >= 1 && count < target) {
        for (int64_t p = threadIdx.x; p < count; p += blockDim.x) {
            const int64_t o = frontier_index(P, inst, sel, p);
            unsigned long long dn = 0, dp = 0, dc = 0;
            cnt[p] = expand_parent<G, false>(P, cfg, inst, dd, dim, t, P.fu + o * P.Kmax, P.frho[o],
                                             P.fw + o * P.dimPad, P.fdisc[o], 0.f, sel ^ 1, 0, dn, dp, dc, ovf);
        }
        if (threadIdx.x == 0) s_ovf = 0;
        __syncthreads();
        if (ovf) s_ovf = 1;
        __syncthreads();
        if (s_ovf) break;
        const int64_t total = block_exclusive_scan(cnt, count);
        if (total > P.F) break;   // keep the current level as the prefixes
        for (int64_t p = threadIdx.x; p < count; p += blockDim.x) {
            const int64_t o = frontier_index(P, inst, sel, p);
            expand_parent<G, true>(P, cfg, inst, dd, dim, t, P.fu + o * P.Kmax, P.frho[o], P.fw + o * P.dimPad,
                                   P.fdisc[o], P.fxsum[o], sel ^ 1, cnt[p], nodes, passed, cuts, ovf);
        }
        __syncthreads();
        sel ^= 1;
        count = total;
        --t;
        ++depth;
        if (count == 0) break;
    }
    if (nodes) {
        atomicAdd(&P.cnt[inst].nodes, nodes);
        atomicAdd(&P.cnt[inst].split_nodes, nodes);
    }
    if (passed) {
        atomicAdd(&P.cnt[inst].passed, passed);
        atomicAdd(&P.cnt[inst].split_passed, passed);
    }
    if (cuts) atomicAdd(&P.cnt[inst].lds_cuts, cuts);
    if (threadIdx.x == 0) {
        I.split_level = t + 1;
        I.front_sel = sel;
        I.nprefix = count;
    }
    if (ovf) set_status(I, ST_EOVERFLOW);
}

template <int G>
__global__ void __launch_bounds__(256) split_kernel(Pools P, EnumCfg cfg, int max_depth, int64_t target,
                                                    int64_t* fcnt) {
    split_inst<G>(P, cfg, blockIdx.x, max_depth, target, fcnt);
}

// resets the control words and arms the time cap on the device clock;
// keep != 0 continues a search (the next limited-discrepancy iteration): the
// start time, the deadline and the stored solutions carry over
__global__ void start_kernel(Ctrl* c, unsigned long long cap_ns, int keep) {
    c->qhead = 0;
    c->dhead = 0;
    c->dtail = 0;
    c->idle = 0;
    c->busy = 0;
    c->donations = 0;
    c->stop = 0;
    c->gstatus = 0;
    if (!keep) {
        c->walk_cycles = 0;
        c->life_cycles = 0;
        c->nsol_total = 0;
        c->start_ns = global_time_ns();
        c->deadline_ns = cap_ns ? c->start_ns + cap_ns : 0ULL;
    }
    c->solved = 0;
    c->active = 0;
    c->qres = 0;
}

// exclusive prefix sums of the per-instance prefix counts (one thread)
__global__ void queue_kernel(Pools P) {
    int64_t run = 0;
    int active = 0, last = -1;   // groups with work (a group's replicas are contiguous)
    for (int i = 0; i < P.count; ++i) {
        P.qbase[i] = run;
        const int64_t k = (P.inst[i].status == ST_OK) ? P.inst[i].nprefix : 0;
        run += k;
        if (k > 0 && P.inst[i].group != last) { ++active; last = P.inst[i].group; }
    }
    P.ctrl->active = active;
    P.qbase[P.count] = run;
    P.ctrl->qhead = 0;
}

// ---------------------------------------------------------------------------
// Enumerator: persistent walkers of G lanes.
// ---------------------------------------------------------------------------

// Global scratch of one walker: the FP64 root vector w^(t0+1) of its walk
// (the canonical start of the exact fallback) and the centre cache sigma:
// sigma[t][i] holds the fold of the centre of level t down to index i.
struct WalkerLayout {
    int Kmax, dimPad;
    __host__ __device__ int64_t bytes() const {
        return (int64_t)dimPad * 8 + (int64_t)Kmax * (Kmax + 1) * 8;
    }
};

// Level state of one walker in shared memory: for each level t on the
// current path, the value u being explored there (also as a double), the
// zig-zag state, the quantised x, the centre y_t, the parent's norm
// rho_{t+1}, the discrepancy cost above and the position of u in the level's
// walk.  One base pointer; the arrays follow each other.
struct Levels {
    unsigned char* base;
    int K;
    __device__ __forceinline__ double& y(int t) const { return reinterpret_cast<double*>(base)[t]; }
    __device__ __forceinline__ double& rho(int t) const { return reinterpret_cast<double*>(base)[K + t]; }
    __device__ __forceinline__ double& ud(int t) const { return reinterpret_cast<double*>(base)[2 * K + t]; }
    __device__ __forceinline__ int& xq(int t) const { return reinterpret_cast<int*>(base + 24 * K)[t]; }
    __device__ __forceinline__ short& u(int t) const { return reinterpret_cast<short*>(base + 28 * K)[t]; }
    __device__ __forceinline__ short& u1(int t) const { return reinterpret_cast<short*>(base + 30 * K)[t]; }
    __device__ __forceinline__ short& zi(int t) const { return reinterpret_cast<short*>(base + 32 * K)[t]; }
    __device__ __forceinline__ unsigned char& meta(int t) const { return base[34 * K + t]; }
    __device__ __forceinline__ unsigned char& J(int t) const { return base[35 * K + t]; }
    // discrepancy cost of the path above level t (limited discrepancy search)
    __device__ __forceinline__ unsigned char& dab(int t) const { return base[36 * K + t]; }
    // position of u(t) in the walk of level t (rank reading; at most the budget)
    __device__ __forceinline__ unsigned char& pos(int t) const { return base[37 * K + t]; }
    // the queue item (prefix) of the current walk
    __device__ __forceinline__ int64_t& gid() const { return *reinterpret_cast<int64_t*>(base + (38 * K + 7) / 8 * 8); }
    // fused launch: the queue position taken but not yet published (-1: none)
    __device__ __forceinline__ int64_t& ticket() const {
        return *reinterpret_cast<int64_t*>(base + (38 * K + 7) / 8 * 8 + 8);
    }
};

__host__ __device__ inline int level_bytes(int Kmax) { return ((38 * Kmax + 7) / 8 * 8 + 16 + 15) / 16 * 16; }

__device__ __forceinline__ Levels levels_at(unsigned char* base, int Kmax) {
    Levels L;
    L.base = base;
    L.K = Kmax;
    return L;
}

// Header of a donated sibling range: the untried values at level t of a
// walk, continued by another walker exactly where the donor stopped.  The
// slot continues with int32 u[Kmax] (values above t) and the canonical FP64
// w^(t+1) (double[dimPad]).
struct DonHdr {
    int32_t inst, t, u, u1, zi, meta, dab, pos;
    int64_t gid;
    double y, rhoP;
};

__host__ __device__ inline int64_t donation_stride(int Kmax, int dimPad) {
    return ((int64_t)sizeof(DonHdr) + (int64_t)Kmax * 4 + 15) / 16 * 16 + (int64_t)dimPad * 8;
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    const int gi = (threadIdx.x & 31) / G;
    return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
}

// sum of a per-lane counter over the lanes of a group (every lane gets it)
template <int G>
__device__ __forceinline__ unsigned long long group_sum(unsigned v, unsigned gmask) {
    unsigned long long s = v;
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) s += __shfl_xor_sync(gmask, s, off, G);
    return s;
}

// exact int -> double without the FP64 pipe (|v| < 2^31)
__device__ __forceinline__ double i2d_exact(int v) {
    if (v == 0) return 0.0;
    const unsigned a = v < 0 ? (unsigned)(-v) : (unsigned)v;
    const int lz = __clz(a);
    const unsigned long long m = ((unsigned long long)a << (lz + 21)) & 0x000fffffffffffffULL;
    const unsigned long long bits = ((unsigned long long)(v < 0) << 63) |
                                    ((unsigned long long)(1023 + 31 - lz) << 52) | m;
    return __longlong_as_double((long long)bits);
}

// trunc(|x| 2^s) with the sign of x, by integer operations on the bits
__device__ __forceinline__ long long fix_trunc(double x, int s) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const long long mant = (b & 0x000fffffffffffffLL) | 0x0010000000000000LL;
    const int sh = 1075 - s - e;
    long long q;
    if (e == 0 || sh >= 63) q = 0;
    else if (sh <= 0) q = mant << (-sh);
    else q = mant >> sh;
    return b < 0 ? -q : q;
}

// The start of a level's zig-zag from its centre y, on the bit pattern of
// c = -y with integer operations only (an FP64 operation costs ~64 cycles of
// latency on this GPU): u1 = c rounded to nearest, ties to even (rint), and
// the side s = +1 if c >= u1 else -1.  Returns true when |u1| >= kUMax.
__device__ __forceinline__ bool centre_round(double y, int& u1, int& s) {
    const unsigned long long c = (unsigned long long)__double_as_longlong(y) ^ 0x8000000000000000ULL;   // -y
    const bool neg = (c >> 63) != 0;
    const int e = (int)((c >> 52) & 0x7ff);
    const unsigned long long frac = c & 0x000fffffffffffffULL;
    unsigned long long mag;
    bool up, exact;
    if (e >= 1023 + 16) return true;   // |c| >= 2^16
    const int shift = 1075 - e;        // >= 21: the integer part has at most 32 bits
    if (e == 0 || shift > 63) {        // |c| < 2^-11 (or zero, or subnormal): rounds to 0
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
    if (mag >= (unsigned long long)kUMax) return true;
    u1 = neg ? -(int)mag : (int)mag;
    s = neg ? ((up || exact) ? 1 : -1) : (up ? -1 : 1);
    return false;
}

// level meta bits
constexpr int kOneDir = 1, kNegS = 2, kZeroPrefix = 4, kDonated = 8;

// Rare paths of the walk, kept out of line so that they do not raise the
// register pressure of the hot loop.

// Exact Theorem 1 check of v = sum_j u_j b_j at a leaf (t = 0, u_0 = u);
// records a verified solution.  Returns 1 if it was one.
template <int G, int CPL>
__device__ __noinline__ int leaf_check(const Pools& P, const EnumCfg& cfg, int inst, const Levels& L, int u,
                                       unsigned gmask) {
    const InstDesc& I = P.inst[inst];
    const int dd = I.dd, dim = I.dim, n = I.n, m = I.m;
    const int32_t* __restrict__ kb = P.kb + I.offKb;
    const int lg = threadIdx.x & (G - 1);
    long long v[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        long long a = 0;
        if (c < dim) {
            a = (long long)u * kb[c];
            for (int j = 1; j < dd; ++j) a += (long long)L.u(j) * kb[(int64_t)j * dim + c];
        }
        v[q] = a;
    }
    long long mine = 0;
#pragma unroll
    for (int q = 0; q < CPL; ++q) if (q == (dim - 1) / G) mine = v[q];
    const long long last = __shfl_sync(gmask, mine, (dim - 1) % G, G);
    const long long sg = (cfg.sym && last == -1) ? -1 : 1;
    bool ok = (last * sg == 1);
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        const long long vc = v[q] * sg;
        if (c < n && vc != 1 && vc != -1) ok = false;
    }
    ok = __all_sync(gmask, ok);
    if (!ok) return 0;
    unsigned long long khi = 0, klo = 0;
    const int gi = (threadIdx.x & 31) / G;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        const bool one = (c < n) && (v[q] * sg == 1);
        unsigned bits = __ballot_sync(gmask, one) >> (gi * G);
        if (G < 32) bits &= (1u << (G & 31)) - 1u;
        for (int l = 0; l < G; ++l) {
            if ((bits >> l) & 1u) {
                const int cc = G * q + l;   // x_cc = 1 at key bit 127 - cc
                if (cc < 64) khi |= 1ULL << (63 - cc);
                else klo |= 1ULL << (127 - cc);
            }
        }
    }
    // independent verification A x = d
    const int32_t* Ai = P.A + I.offA;
    const int64_t* di = P.d + I.offd;
    for (int i = lg; i < m; i += G) {
        long long acc = 0;
        for (int c = 0; c < n; ++c) {
            const bool xc = c < 64 ? (khi >> (63 - c)) & 1ULL : (klo >> (127 - c)) & 1ULL;
            if (xc) acc += Ai[(int64_t)i * n + c];
        }
        if (acc != di[i]) ok = false;
    }
    ok = __all_sync(gmask, ok);
    if (ok && lg == 0) {
        const unsigned long long k = atomicAdd(&P.ctrl->nsol_total, 1ULL);
        if ((int64_t)k < P.sol_cap) {
            SolRec r;
            r.inst = inst; r.pad = 0; r.hi = khi; r.lo = klo;
            P.sols[k] = r;
        }
        const unsigned long long prev = atomicAdd(&P.cnt[inst].nsol, 1ULL);
        if (cfg.first) {
            const unsigned long long now = global_time_ns() - P.ctrl->start_ns;
            if (prev == 0) P.cnt[inst].first_ns = now;   // first solution of this replica
            if (atomicCAS(&P.gsolved[I.group], 0u, 1u) == 0u) {   // ... and of its group
                P.gfirst_ns[I.group] = now;
                if (atomicAdd(&P.ctrl->solved, 1) + 1 >= P.ctrl->active) atomicExch(&P.ctrl->stop, 1u);
            }
        }
    }
    return ok ? 1 : 0;
}

// The same check for the general bounds of Sec. 2 (any r_max >= 1): kept
// apart so that the binary walker's register budget is unchanged.
template <int G, int CPL>
__device__ __noinline__ int leaf_check_bounded(const Pools& P, const EnumCfg& cfg, int inst, const Levels& L, int u,
                                       unsigned gmask) {
    const InstDesc& I = P.inst[inst];
    const int dd = I.dd, dim = I.dim, n = I.n, m = I.m;
    const int32_t* __restrict__ kb = P.kb + I.offKb;
    const int lg = threadIdx.x & (G - 1);
    long long v[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        long long a = 0;
        if (c < dim) {
            a = (long long)u * kb[c];
            for (int j = 1; j < dd; ++j) a += (long long)L.u(j) * kb[(int64_t)j * dim + c];
        }
        v[q] = a;
    }
    long long mine = 0;
#pragma unroll
    for (int q = 0; q < CPL; ++q) if (q == (dim - 1) / G) mine = v[q];
    const long long last = __shfl_sync(gmask, mine, (dim - 1) % G, G);
    // Theorem 1: last entry r_max (sign-normalised), the others in
    // [-r_max, r_max]; x_c = (v_c + r_max) / (2 c_c), c_c = r_max / r_c
    const long long rm = I.rmax;
    const int32_t* __restrict__ rr = P.r + I.offR;
    const long long sg = (cfg.sym && last == -rm) ? -1 : 1;
    bool ok = (last * sg == rm);
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        const long long vc = v[q] * sg;
        if (c < n) {
            if (rm == 1) {
                if (vc != 1 && vc != -1) ok = false;
            } else {
                const long long c2 = 2 * (rm / rr[c]);
                if (vc > rm || vc < -rm || (vc + rm) % c2 != 0) ok = false;
            }
        }
    }
    ok = __all_sync(gmask, ok);
    if (!ok) return 0;
    // key: x_c in a field of bound_bits(r_c) bits, most significant first,
    // fields in coordinate order from key bit 127 down (binary: bit 127 - c)
    unsigned long long khi = 0, klo = 0;
    if (rm == 1) {
        const int gi = (threadIdx.x & 31) / G;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int c = lg + G * q;
            const bool one = (c < n) && (v[q] * sg == 1);
            unsigned bits = __ballot_sync(gmask, one) >> (gi * G);
            if (G < 32) bits &= (1u << (G & 31)) - 1u;
            for (int l = 0; l < G; ++l) {
                if ((bits >> l) & 1u) {
                    const int cc = G * q + l;   // x_cc = 1 at key bit 127 - cc
                    if (cc < 64) khi |= 1ULL << (63 - cc);
                    else klo |= 1ULL << (127 - cc);
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int c = lg + G * q;
            if (c >= n) continue;
            int off = 0;
            for (int j = 0; j < c; ++j) off += bound_bits(rr[j]);
            const int w = bound_bits(rr[c]);
            const unsigned long long x = (unsigned long long)((v[q] * sg + rm) / (2 * (rm / rr[c])));
            const int sh = 128 - off - w;   // position of the field's lowest bit
            if (sh >= 64) {
                khi |= x << (sh - 64);
            } else {
                klo |= x << sh;
                if (sh + w > 64) khi |= x >> (64 - sh);
            }
        }
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
            khi |= __shfl_xor_sync(gmask, khi, o, G);
            klo |= __shfl_xor_sync(gmask, klo, o, G);
        }
    }
    // independent verification A x = d, x read back from the key
    const int32_t* Ai = P.A + I.offA;
    const int64_t* di = P.d + I.offd;
    for (int i = lg; i < m; i += G) {
        long long acc = 0;
        int off = 0;
        for (int c = 0; c < n; ++c) {
            const int w = (rm == 1) ? 1 : bound_bits(rr[c]);
            const int sh = 128 - off - w;
            unsigned long long x = sh >= 64 ? (khi >> (sh - 64)) : ((klo >> sh) | (sh > 0 ? khi << (64 - sh) : 0ULL));
            x &= (1ULL << w) - 1ULL;
            acc += (long long)x * Ai[(int64_t)i * n + c];
            off += w;
        }
        if (acc != di[i]) ok = false;
    }
    ok = __all_sync(gmask, ok);
    if (ok && lg == 0) {
        const unsigned long long k = atomicAdd(&P.ctrl->nsol_total, 1ULL);
        if ((int64_t)k < P.sol_cap) {
            SolRec r;
            r.inst = inst; r.pad = 0; r.hi = khi; r.lo = klo;
            P.sols[k] = r;
        }
        const unsigned long long prev = atomicAdd(&P.cnt[inst].nsol, 1ULL);
        if (cfg.first) {
            const unsigned long long now = global_time_ns() - P.ctrl->start_ns;
            if (prev == 0) P.cnt[inst].first_ns = now;   // first solution of this replica
            if (atomicCAS(&P.gsolved[I.group], 0u, 1u) == 0u) {   // ... and of its group
                P.gfirst_ns[I.group] = now;
                if (atomicAdd(&P.ctrl->solved, 1) + 1 >= P.ctrl->active) atomicExch(&P.ctrl->stop, 1u);
            }
        }
    }
    return ok ? 1 : 0;
}

// Canonical FP64 ||w^(t)||_1 for the node (t, x): the chain of Algorithm 1
// rebuilt from the walk's root w^(t0+1) with the same fmas as the FP64
// method, summed in the G-lane order.
template <int G, int CPL>
__device__ __noinline__ double canonical_l1(const double* __restrict__ bhat, const double* __restrict__ root_w,
                                            const Levels& L, int t0, int t, double x, int dim, unsigned gmask) {
    const int lg = threadIdx.x & (G - 1);
    double sl = 0.0;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lg + G * q;
        if (c < dim) {
            double w = root_w[c];
            for (int j = t0; j > t; --j)
                w = __fma_rn(__dadd_rn(L.ud(j), L.y(j)), bhat[(int64_t)j * dim + c], w);
            w = __fma_rn(x, bhat[(int64_t)t * dim + c], w);
            sl = __dadd_rn(sl, fabs(w));
        }
    }
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) sl = __dadd_rn(sl, __shfl_xor_sync(gmask, sl, off, G));
    return sl;
}

// Hand the untried values of the highest open level h in (t, t0] to an idle
// walker.  Returns 1 if a slot was written.
template <int G>
__device__ __noinline__ int donate(const Pools& P, int inst, int64_t gid, const Levels& L, const double* root_w,
                                   const double* __restrict__ bhat, int t0, int t, int dd, int dim, int Kmax,
                                   int lds, int lds_rank, unsigned gmask) {
    const int lg = threadIdx.x & (G - 1);
    if (P.don_cap <= 0) return 0;
    int h = -1;
    for (int l = t0; l > t; --l)   // untried values of a level are discrepancies: they need budget
        if (!(L.meta(l) & kDonated) && (lds < 0 || L.dab(l) + (lds_rank ? L.pos(l) + 1 : 1) <= lds)) {
            h = l;
            break;
        }
    if (h < 0) return 0;
    // reserve ring index k (slot k mod cap); the slot is free once its
    // sequence number equals k (set by the consumer of index k - cap)
    long long slot = -1;
    if (lg == 0) {
        for (int tries = 0; tries < 64; ++tries) {
            const unsigned long long old = *(volatile unsigned long long*)&P.ctrl->dtail;
            const unsigned long long head = *(volatile unsigned long long*)&P.ctrl->dhead;
            if (old - head >= (unsigned long long)P.don_cap) break;   // ring full
            if (*(volatile unsigned long long*)&P.don_seq[old % P.don_cap] != old) break;   // slot still being read
            if (atomicCAS(&P.ctrl->dtail, old, old + 1) == old) { slot = (long long)old; break; }
        }
    }
    slot = __shfl_sync(gmask, slot, 0, G);
    if (slot < 0) return 0;
    const long long k = slot;
    slot = k % P.don_cap;
    char* sp = P.don + slot * P.don_stride;
    int32_t* su = reinterpret_cast<int32_t*>(sp + sizeof(DonHdr));
    double* sw = reinterpret_cast<double*>(sp + ((int64_t)sizeof(DonHdr) + (int64_t)Kmax * 4 + 15) / 16 * 16);
    if (lg == 0) {
        DonHdr hd;
        hd.inst = inst; hd.t = h; hd.u = L.u(h); hd.u1 = L.u1(h);
        hd.zi = L.zi(h); hd.meta = L.meta(h) & ~kDonated; hd.gid = gid;
        hd.dab = L.dab(h); hd.pos = L.pos(h);
        hd.y = L.y(h); hd.rhoP = L.rho(h);
        *reinterpret_cast<DonHdr*>(sp) = hd;
    }
    for (int i = h + 1 + lg; i < dd; i += G) su[i] = L.u(i);
    // canonical FP64 w^(h+1): the chain from the root down to level h+1
    for (int c = lg; c < dim; c += G) {
        double w = root_w[c];
        for (int j = t0; j > h; --j)
            w = __fma_rn(__dadd_rn(L.ud(j), L.y(j)), bhat[(int64_t)j * dim + c], w);
        sw[c] = w;
    }
    __threadfence();
    __syncwarp(gmask);
    if (lg == 0) {
        atomicExch(&P.don_seq[slot], (unsigned long long)k + 1);   // full for index k
        L.meta(h) |= kDonated;
        atomicAdd(&P.ctrl->donations, 1ULL);
    }
    __syncwarp(gmask);
    return 1;
}
// walk actions
constexpr int kNext = 0, kDescend = 1, kUp = 2, kEval = 3, kEnter = 4;

// Walk state of one group of G lanes.  Lane l owns the coordinates
// c = l + G q (q < CPL) of the integer vector
//   W = sum_j Xq_j Bq_j  ~  w^(t+1) 2^(sx+sb),
// which is exact and therefore reversible: stepping back to level t
// subtracts that level's term instead of reloading a stored vector.  E bounds
// (in units of 2^-(sx+sb)) the distance of the filter's ||w||_1 from the
// exact one: per level (n+1)(|Xq| + 1)/2 + sum_c |Bq_c| + 1, (n+1) for
// rounding the root, and (n+1) 2^kHiShift for summing T >> kHiShift.
// The Hoelder decision of the FP64 method, rho > ||w||_1 + eps, is taken from
// the filter whenever the margin exceeds the bound; otherwise the canonical
// FP64 w is rebuilt from the walk's root and the decision is the FP64 one.
//
// All groups of a warp run one flat loop in lockstep: every iteration each
// group performs one step of its own state machine (fetch work, or evaluate
// one node and move), so the groups re-converge at the top of every step
// and the three FP64 operations of a node (x, x^2, rho) are issued once per
// warp for all 32/G walkers -- the FP64 pipe charges per warp instruction.
constexpr int kHiShift = 27;   // sum |T| >> 27 in int32: ||w||_1 2^23 < 2^31

enum : int { kFetch = 0, kWalk = 1, kDone = 2 };

// Minimum resident blocks per SM requested from the register allocator:
// two blocks for groups of 8 or more lanes (measured best on GB300); the
// 4-lane groups carry 16+ coordinates per lane and keep one block.
#ifndef MSP_ENUM_MIN_BLOCKS
#define MSP_ENUM_MIN_BLOCKS(g) ((g) >= 8 ? 2 : 1)
#endif

// Fused launch: publish instance inst's subtrees (thread 0 of its block),
// without waiting for anyone.  One atomic reserves the entry r (instances
// counted in the high bits) and the queue positions base .. base + n - 1,
// so the bases grow with r; the entry is written, then flagged ready.  A
// walker holding position tk < the reserved total finds its entry by a
// binary search over rl[0 .. r_reserved) that reads only ready entries
// (else it keeps tk and looks again later).
__device__ __noinline__ void publish_instance(const Pools& P, const Pipe& pipe, int inst) {
    const InstDesc& I = P.inst[inst];
    const unsigned long long n = (I.status == ST_OK) ? (unsigned long long)I.nprefix : 0ULL;
    const unsigned long long old = atomicAdd(&P.ctrl->qres, (1ULL << 40) | n);
    const int r = (int)(old >> 40);
    const unsigned long long base = old & ((1ULL << 40) - 1ULL);
    pipe.rl[r] = (int64_t)base;
    pipe.rl[P.count + r] = inst;
    P.qbase[inst] = (int64_t)base;
    if (r + 1 == P.count) P.qbase[P.count] = (int64_t)(base + n);
    __threadfence();
    *(volatile int64_t*)&pipe.rl[2 * P.count + r] = 1;
}

// Fused launch: the entry of the published list whose range holds queue
// position tk (tk < the reserved total of the r_res reserved entries), or -1
// while an entry the search needs is not ready yet.
__device__ __forceinline__ int find_entry(const Pools& P, const Pipe& pipe, int64_t tk, int r_res) {
    const volatile int64_t* rl = pipe.rl;
    int lo = 0, hi = r_res;
    if (rl[2 * P.count] == 0) return -1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rl[2 * P.count + mid] == 0) return -1;
        if (rl[mid] <= tk) lo = mid; else hi = mid;
    }
    __threadfence();
    return lo;
}

// Fused launch: block b prepares instances b, b + grid, ...  Warp 0 runs
// the reduction steps (LLL, extraction and Gram-Schmidt, optional BKZ, the
// filter tables), the whole block splits the top levels, thread 0 publishes
// the subtrees.  The same device functions as the separate launches, so the
// prepared instance is bit for bit the same.
template <int G>
__device__ __noinline__ void prepare_instances(const Pools& P, const EnumCfg& cfg, const Pipe& pipe) {
    for (int inst = blockIdx.x; inst < P.count; inst += gridDim.x) {
        if (threadIdx.x < 32) {
            lll_inst(P, inst, pipe.delta, pipe.eta, pipe.lll_max_iter, pipe.max_ns);
            extract_gso_inst(P, inst, 0);
            if (pipe.bkz_beta >= 2) {
                bkz_inst(P, inst, pipe.S, pipe.bkz_beta, pipe.delta, pipe.bkz_max_tours, pipe.lll_max_iter,
                         pipe.max_ns);
                extract_gso_inst(P, inst, 1);
            }
            prep_fixed_inst(P, inst, pipe.use_eps, pipe.dimPad);
            __threadfence();
        }
        __syncthreads();
        split_inst<G>(P, cfg, inst, pipe.split_depth, pipe.split_target, pipe.fcnt);
        __syncthreads();
        if (threadIdx.x == 0) publish_instance(P, pipe, inst);
        __syncthreads();
    }
}

// Variants V of the walker: 0 plain (binary bounds, depth-first), 1 binary
// with the discrepancy bookkeeping of a limited-discrepancy iteration, 2
// general bounds (r_max >= 1; depth-first or discrepancy search), 3 plain in
// the fused launch (the blocks first prepare the instances, walkers take
// subtrees as instances are published).  EXT: the discrepancy bookkeeping is
// compiled in; BND: r_max is a run-time value and leaves take the general
// check; FUSED: the preparation and the published queue.  Each variant
// carries only the state and calls it needs, so the register budget stays
// with the hot loop.
template <int G, int CPL, int V>
__global__ void __launch_bounds__(256, MSP_ENUM_MIN_BLOCKS(G))
    enum_kernel(Pools P, EnumCfg cfg, char* scratch, WalkerLayout WL, Pipe pipe) {
    constexpr bool EXT = V == 1 || V == 2;
    constexpr bool BND = V == 2;
    constexpr bool FUSED = V == 3;
    extern __shared__ __align__(16) unsigned char smem[];
    if (FUSED) prepare_instances<G>(P, cfg, pipe);
    const int lg = threadIdx.x & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int wib = threadIdx.x / G;
    const int64_t walker = (int64_t)blockIdx.x * (blockDim.x / G) + wib;
    const int Kmax = WL.Kmax, dimPad = WL.dimPad;
    const Levels L = levels_at(smem + (int64_t)wib * level_bytes(Kmax), Kmax);
    char* ws = scratch + walker * WL.bytes();
    double* root_w = reinterpret_cast<double*>(ws);
    double* sigma = root_w + dimPad;
    Ctrl* ctrl = P.ctrl;
    const int64_t total = FUSED ? 0 : P.qbase[P.count];   // (fused launch: known only at the end)
    if (FUSED && lg == 0) L.ticket() = -1;

    // ---- per-walk state (uniform over the group's lanes) ----
    int state = kFetch;
    bool static_done = false;          // lane 0: the split queue is exhausted
    int idle_reg = 0;                  // counted in ctrl->idle (uniform over the group)
    int inst = 0, dd = 0, dim = 0, sx = 0, Sf = 0, t0 = 0, t = 0;
    long long Rbits = 0, eps_fix = 0;
    int ehalf = 0;
    long long rmax = 1;   // stays the constant 1 in the plain variant
    double eps = 0.0;
    const double* muT = nullptr;
    const double* Btab = nullptr;
    const int32_t* bqtab = nullptr;
    const int64_t* nbqtab = nullptr;
    double y = 0.0, rhoP = 0.0, Bt = 0.0;
    int u = 0, u1 = 0, s = 1, zi = 1, dir = 0, act = kEval;
    int dab = 0;                       // discrepancy cost of the path above level t
    int pos = 0;                       // position of u in the walk of level t
    bool onedir = false, zp = true;
    long long Epar = 0, nbq_t = 0;
    long long W[CPL];
    int bq[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) { W[q] = 0; bq[q] = 0; }
    unsigned nodes = 0, passed = 0, cfma = 0;   // per walk, flushed before they could overflow
    unsigned leaves = 0, fallbacks = 0, cuts = 0;
    int item_sols = 0;
    unsigned spins = 0;
    const long long life0 = clock64();
    long long walk0 = 0;

    for (;;) {
        // ================= fetch: one non-blocking attempt per step =========
        // (a walker already waiting for donated work polls every 32nd step)
        if (state == kFetch && (!idle_reg || ((++spins & 31) == 0))) {
            int64_t gid = 0;   // this step's queue item (kept in shared memory for the walk)
            int src = 0, quit = 0;
            long long id = 0;
            int fent = 0;      // fused launch: the published entry of the queue item
            if (lg == 0) {
                if (!static_done && !FUSED) {
                    const unsigned long long it = atomicAdd(&ctrl->qhead, 1ULL);
                    if ((int64_t)it < total) {
                        src = 1;
                        id = (long long)it;
                    } else {
                        static_done = true;
                    }
                } else if (!static_done) {
                    // fused launch: a queue position is valid once the instance
                    // whose range holds it is published; the walker keeps its
                    // position until then, or until every instance is published
                    // and the position lies past the end
                    int64_t tk = L.ticket();
                    if (tk < 0) tk = (int64_t)atomicAdd(&ctrl->qhead, 1ULL);
                    const unsigned long long qr = *(volatile unsigned long long*)&ctrl->qres;
                    const int r_res = (int)(qr >> 40);
                    const int64_t reserved = (int64_t)(qr & ((1ULL << 40) - 1ULL));
                    const int e = tk < reserved ? find_entry(P, pipe, tk, r_res) : -1;
                    if (e >= 0) {
                        src = 1;
                        id = (long long)tk;
                        fent = e;
                        tk = -1;
                    } else if (r_res >= P.count && tk >= reserved) {
                        static_done = true;
                        tk = -1;
                    } else if (global_time_ns() > ctrl->deadline_ns) {
                        // (no spin counter here: spins is per lane and must stay
                        // equal across the group -- it gates the group's fetch)
                        atomicExch(&ctrl->stop, 2u);
                        quit = 1;
                        tk = -1;
                    } else if (*(volatile unsigned*)&ctrl->stop) {
                        quit = 1;
                        tk = -1;
                    } else {
                        // still waiting: back off, so that thousands of waiting
                        // walkers do not hold the line of the reservation word
                        // (and the preparing warps' memory traffic) hostage
                        __nanosleep(4000);
                    }
                    L.ticket() = tk;
                }
                if (src == 0 && static_done) {
                    if (!idle_reg) { atomicAdd(&ctrl->idle, 1); idle_reg = 1; }
                    const unsigned long long h = *(volatile unsigned long long*)&ctrl->dhead;
                    const unsigned long long tl = *(volatile unsigned long long*)&ctrl->dtail;
                    if (h < tl && atomicCAS(&ctrl->dhead, h, h + 1) == h) {
                        src = 2;
                        id = (long long)h;
                    } else if (*(volatile unsigned*)&ctrl->stop) {
                        quit = 1;
                    } else if (h >= tl && *(volatile int*)&ctrl->busy == 0 &&
                               *(volatile unsigned long long*)&ctrl->dhead ==
                                   *(volatile unsigned long long*)&ctrl->dtail) {
                        quit = 1;   // nothing left anywhere
                    } else if ((spins & 255) == 0 && global_time_ns() > ctrl->deadline_ns) {
                        atomicExch(&ctrl->stop, 2u);
                        quit = 1;
                    }
                }
                if (src == 2) {   // the donor finishes writing the slot right after reserving it
                    const unsigned long long k = (unsigned long long)id;
                    id = (long long)(k % P.don_cap);
                    unsigned waited = 0;
                    while (*(volatile unsigned long long*)&P.don_seq[id] != k + 1) {
                        if ((++waited & 1023) == 0 && global_time_ns() > ctrl->deadline_ns) {
                            atomicExch(&ctrl->stop, 2u);
                            src = 0;
                            quit = 1;
                            break;
                        }
                    }
                    __threadfence();
                }
                if (src) {
                    atomicAdd(&ctrl->busy, 1);
                    if (idle_reg) { atomicSub(&ctrl->idle, 1); idle_reg = 0; }
                }
                if (quit && idle_reg) { atomicSub(&ctrl->idle, 1); idle_reg = 0; }
            }
            src = __shfl_sync(gmask, src, 0, G);
            id = __shfl_sync(gmask, id, 0, G);
            quit = __shfl_sync(gmask, quit, 0, G);
            idle_reg = __shfl_sync(gmask, idle_reg, 0, G);   // uniform over the group
            if (quit) state = kDone;
            if (src) {
                // ---- set up a walk ----
                if (src == 1) {
                    gid = P.qperm ? P.qperm[id] : (int64_t)id;
                    if (lg == 0) L.gid() = gid;
                    if (FUSED) {   // the published instance whose range holds gid
                        fent = __shfl_sync(gmask, fent, 0, G);
                        inst = (int)((const volatile int64_t*)pipe.rl)[P.count + fent];
                    } else {
                        int lo = 0, hi = P.count;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (P.qbase[mid] <= gid) lo = mid; else hi = mid;
                        }
                        inst = lo;
                    }
                } else {
                    const DonHdr* hd = reinterpret_cast<const DonHdr*>(P.don + id * P.don_stride);
                    inst = hd->inst;
                    gid = hd->gid;
                    if (lg == 0) L.gid() = gid;
                }
                int skip = 0;
                if (cfg.first && lg == 0) skip = *(volatile unsigned*)&P.gsolved[P.inst[inst].group] != 0;
                skip = __shfl_sync(gmask, skip, 0, G);
                if (skip) {   // instance already solved: drop the subtree
                    if (lg == 0) {
                        if (src == 2) {   // release the ring slot
                            __threadfence();
                            const unsigned long long k = *(volatile unsigned long long*)&P.don_seq[id] - 1;
                            atomicExch(&P.don_seq[id], k + (unsigned long long)P.don_cap);
                        }
                        atomicSub(&ctrl->busy, 1);
                    }
                    src = 0;
                }
            }
            if (src) {
                // a walk starts inside its instance's levels; anything else (a
                // descriptor or a donated slot out of range) ends as an error
                // instead of a walk through memory it does not own
                const InstDesc& I = P.inst[inst];
                const int tst = (src == 1) ? I.split_level - 1
                                           : reinterpret_cast<const DonHdr*>(P.don + id * P.don_stride)->t;
                if (I.dd <= 0 || I.dd > Kmax || I.dim <= 0 || I.dim > dimPad || tst < 0 || tst >= I.dd) {
                    if (lg == 0) {
                        set_status(P.inst[inst], ST_EOVERFLOW);
                        atomicSub(&ctrl->busy, 1);
                    }
                    src = 0;
                }
            }
            if (src) {
                const InstDesc& I = P.inst[inst];
                dd = I.dd;
                dim = I.dim;
                sx = I.sx;
                Sf = I.sx + I.sb;
                muT = P.muT + I.offMuT;
                Btab = P.B + I.offB;
                bqtab = P.bq + I.offBq;
                nbqtab = P.nbq + I.offNbq;
                if (BND) rmax = I.rmax;
                {
                    const double R = bound_R(I);
                    eps = slack_of(R, cfg.use_eps);
                    Rbits = __double_as_longlong(R + eps);
                    // eps 2^(sx+sb), exact: R 2^(sx+sb-20)
                    eps_fix = cfg.use_eps ? ((long long)dim * rmax * rmax) << (Sf - 20) : 0LL;
                }
                ehalf = dim;
                zp = true;
                if (src == 1) {
                    const int split_level = I.split_level;
                    t0 = split_level - 1;
                    const int64_t qb = FUSED ? *(const volatile int64_t*)&P.qbase[inst] : P.qbase[inst];
                    const int64_t fo = frontier_index(P, inst, I.front_sel, gid - qb);
                    const int32_t* pu = P.fu + fo * P.Kmax;
                    for (int i = split_level; i < dd; ++i) {
                        const int32_t v = pu[i];
                        if (lg == 0) { L.u(i) = (short)v; L.ud(i) = (double)v; }
                        zp = zp && (v == 0);
                    }
                    for (int c = lg; c < dim; c += G) root_w[c] = P.fw[fo * P.dimPad + c];
                    rhoP = P.frho[fo];
                    if (EXT) dab = P.fdisc[fo];
                } else {
                    const char* slot = P.don + id * P.don_stride;
                    const DonHdr hd = *reinterpret_cast<const DonHdr*>(slot);
                    const int32_t* su = reinterpret_cast<const int32_t*>(slot + sizeof(DonHdr));
                    const double* sw = reinterpret_cast<const double*>(
                        slot + ((int64_t)sizeof(DonHdr) + (int64_t)Kmax * 4 + 15) / 16 * 16);
                    t0 = hd.t;
                    for (int i = t0 + 1 + lg; i < dd; i += G) { L.u(i) = (short)su[i]; L.ud(i) = (double)su[i]; }
                    for (int c = lg; c < dim; c += G) root_w[c] = sw[c];
                    __syncwarp(gmask);
                    if (lg == 0) {   // slot read: free it for ring index (k + cap)
                        __threadfence();
                        const unsigned long long k = *(volatile unsigned long long*)&P.don_seq[id] - 1;
                        atomicExch(&P.don_seq[id], k + (unsigned long long)P.don_cap);
                    }
                    rhoP = hd.rhoP;
                    y = hd.y;
                    u = hd.u;
                    u1 = hd.u1;
                    onedir = hd.meta & kOneDir;
                    s = (hd.meta & kNegS) ? -1 : 1;
                    zp = (hd.meta & kZeroPrefix) != 0;
                    if (onedir) dir = hd.zi; else zi = hd.zi;
                    if (EXT) { dab = hd.dab; pos = hd.pos; }
                }
                for (int i = lg; i <= t0; i += G) L.J(i) = (unsigned char)(dd - 1);
                if (lg == 0) L.meta(t0) = 0;
                __syncwarp(gmask);
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const int c = lg + G * q;
                    W[q] = (c < dim) ? llrint(ldexp(root_w[c], Sf)) : 0LL;
                }
                Epar = (long long)ehalf;
                t = t0;
                Bt = Btab[t];
                nbq_t = nbqtab[t];
#pragma unroll
                for (int q = 0; q < CPL; ++q) bq[q] = (lg + G * q < dim) ? bqtab[(int64_t)t * dimPad + lg + G * q] : 0;
                nodes = passed = leaves = cfma = fallbacks = cuts = 0;
                item_sols = 0;
                state = kWalk;
                walk0 = clock64();
                if (src == 1) {
                    act = kEnter;
                } else {
                    act = kNext;   // the donor evaluated u already
                }
            }
        }

        // ================= walk: one node per step ==========================
        if (state == kWalk) {
            bool abort = false, quiet = false;
            __syncwarp(gmask);   // level state written by lane 0 in the previous step
            if (act == kEnter) {
                // Entering level t: the centre y_t by the cached fold, and the
                // start of the zig-zag.  Lane 0 folds level t's cache row from
                // its highest changed index Jt down to t + 1.  Lane l > 0 takes
                // the row of level t - l, whose pending indices are those of
                // the levels from t down to t - l (Q); when they all lie in
                // Jt .. t + 1 it folds that row over the same indices alongside
                // lane 0 (the u above t are fixed from here on), so entering
                // level t - l later folds only the indices added below t.  A
                // lane whose row has older changes above Jt keeps them pending
                // (J = Q) for later.  Every row is the same fold in the same
                // order as without the lanes' help, so every y_t is bit for
                // bit the same.
                const int tl = t - lg;                     // this lane's level
                int Q = (tl >= 0) ? (int)L.J(tl) : -1;
#pragma unroll
                for (int off = 1; off < G; off <<= 1) {
                    const int v = __shfl_up_sync(gmask, Q, off, G);
                    if (lg >= off) Q = max(Q, v);
                }
                const int Jt = __shfl_sync(gmask, Q, 0, G);
                const bool fold = tl >= 0 && Q <= Jt;
                double acc = 0.0;
                if (fold) {
                    double* srow = sigma + (int64_t)tl * (Kmax + 1);
                    const double* mrow = muT + (int64_t)tl * dd;
                    acc = (Q + 1 < dd) ? srow[Q + 1] : 0.0;
                    for (int i = Q; i > t; --i) {
                        acc = __fma_rn(L.ud(i), mrow[i], acc);
                        srow[i] = acc;
                    }
                    if (Q > t) cfma += (unsigned)(Q - t);
                }
                y = __shfl_sync(gmask, acc, 0, G);
                __syncwarp(gmask);
                if (tl >= 0) L.J(tl) = (unsigned char)(fold ? t : Q);   // rows valid above index J
                // the level below the lanes' reach inherits the pending index
                if (lg == G - 1 && fold && tl > 0 && L.J(tl - 1) < Q) L.J(tl - 1) = (unsigned char)Q;
                if (centre_round(y, u1, s)) { abort = true; u1 = 0; s = 1; }
                onedir = false; dir = 0; zi = 1;
                if (zp && cfg.sym) { u1 = 0; onedir = true; dir = 1; }
                u = u1;
                if (EXT) pos = 0;
            } else if (act == kNext) {
                if (onedir) u += dir;
                else { ++zi; u = zigzag(u1, s, zi); }
                if (EXT) ++pos;
                if (lg == 0 && t > 0 && L.J(t - 1) < t) L.J(t - 1) = (unsigned char)t;
            }
            __syncwarp(gmask);
            if ((nodes & 1023) == 1023) {
                // stop flag, time cap, and donation to idle walkers
                int st = 0, want = 0;
                if (lg == 0) {
                    st = *(volatile unsigned*)&ctrl->stop != 0;
                    if (!st && global_time_ns() > ctrl->deadline_ns) {
                        atomicExch(&ctrl->stop, 2u);
                        st = 1;
                    }
                    const int idle = *(volatile int*)&ctrl->idle;
                    if (idle > 0) {
                        const unsigned long long qd = *(volatile unsigned long long*)&ctrl->dtail -
                                                      *(volatile unsigned long long*)&ctrl->dhead;
                        want = qd < (unsigned long long)idle;
                    }
                }
                int solved = 0;
                if (cfg.first && lg == 0) solved = *(volatile unsigned*)&P.gsolved[P.inst[inst].group] != 0;
                if (__shfl_sync(gmask, st, 0, G)) abort = true;
                else if (__shfl_sync(gmask, solved, 0, G)) { abort = true; quiet = true; }
                else if (__shfl_sync(gmask, want, 0, G))
                    donate<G>(P, inst, L.gid(), L, root_w, P.bhat + P.inst[inst].offBhat, t0, t, dd, dim, Kmax,
                              EXT ? cfg.lds : -1, cfg.lds_rank, gmask);
                // the 32-bit walk counters are flushed long before they could wrap
                // (at most 1024 nodes and 1024 x 128 centre fmas between checks)
                if (nodes >= (1u << 30) || __any_sync(gmask, cfma >= (1u << 30))) {
                    const unsigned long long csum = group_sum<G>(cfma, gmask);
                    if (lg == 0) {
                        atomicAdd(&P.cnt[inst].nodes, (unsigned long long)nodes);
                        atomicAdd(&P.cnt[inst].passed, (unsigned long long)passed);
                        atomicAdd(&P.cnt[inst].leaves, (unsigned long long)leaves);
                        atomicAdd(&P.cnt[inst].center_fma, csum);
                        atomicAdd(&P.cnt[inst].fallbacks, (unsigned long long)fallbacks);
                        if (cuts) atomicAdd(&P.cnt[inst].lds_cuts, (unsigned long long)cuts);
                        atomicAdd(reinterpret_cast<unsigned long long*>(&P.plog_nodes[L.gid()]),
                                  (unsigned long long)nodes);
                    }
                    nodes = passed = cfma = 0;
                    leaves = fallbacks = cuts = 0;
                }
            }
            if (u >= kUMax || u <= -kUMax) {
                if (!abort && lg == 0) set_status(P.inst[inst], ST_EOVERFLOW);
                abort = true;
            }
            bool finished = abort;
            if (!abort) {
                // ---- node (t, u): centre, norm (FP64, the canonical operations) ----
                const double x = __dadd_rn(i2d_exact(u), y);
                const double rho = __fma_rn(__dmul_rn(x, x), Bt, rhoP);
                // discrepancy cost of this value (limited discrepancy search)
                const int cost = EXT ? (cfg.lds_rank ? pos : (u != u1 ? 1 : 0)) : 0;
                const bool over_budget = EXT && cfg.lds >= 0 && cost > 0 && dab + cost > cfg.lds;
                nodes += over_budget ? 0 : 1;
                cuts += over_budget ? 1 : 0;
                long long Ech = 0;
                int xq = 0;
                if (over_budget || __double_as_longlong(rho) > Rbits) {   // norm test on the bit patterns (rho >= 0)
                    act = kUp;
                } else {
                    ++passed;
                    if (t == 0) {
                        ++leaves;
                        if (!EXT || cfg.lds < 0 || dab + cost == cfg.lds)
                            item_sols += BND ? leaf_check_bounded<G, CPL>(P, cfg, inst, L, u, gmask)
                                             : leaf_check<G, CPL>(P, cfg, inst, L, u, gmask);
                        act = kNext;
                    } else {
                        // ---- Hoelder test (Theorem 2) through the exact integer filter ----
                        xq = (int)fix_trunc(x, sx);
                        int lsum = 0;
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            const long long Tq = W[q] + (long long)xq * (long long)bq[q];
                            lsum += abs((int)(Tq >> kHiShift));
                        }
#pragma unroll
                        for (int off = G / 2; off >= 1; off >>= 1) lsum += __shfl_xor_sync(gmask, lsum, off, G);
                        const long long axq = xq < 0 ? -(long long)xq : (long long)xq;
                        Ech = Epar + (((long long)ehalf * (axq + 1)) >> 1) + nbq_t + 1;
                        bool fail = false;
                        if (cfg.hoelder != HOELDER_OFF) {
                            // r_max ||w||_1 (Theorem 2 with r_max); r_max = 1 for binary problems
                            long long Lfix = (long long)lsum << kHiShift;
                            long long Ebase = Ech + (Ech >> 10) + ((long long)ehalf << kHiShift);
                            if (BND && rmax != 1) { Lfix *= rmax; Ebase *= rmax; }
                            const long long M = fix_trunc(rho, Sf) - Lfix - eps_fix;
                            const long long Etot = Ebase + (Lfix >> 32) + 64;
                            if (M > Etot) fail = true;
                            else if (M < -Etot) fail = false;
                            else {
                                ++fallbacks;
                                fail = rho > __dadd_rn(__dmul_rn((double)rmax,
                                                                 canonical_l1<G, CPL>(P.bhat + P.inst[inst].offBhat, root_w, L, t0, t, x, dim,
                                                                                      gmask)),
                                                       eps);
                            }
                        }
                        if (fail && cfg.hoelder == HOELDER_CUT) {
                            if (onedir) {
                                act = kUp;
                            } else {
                                // first failure: one more regular value, then one direction
                                ++zi;
                                u = zigzag(u1, s, zi);
                                dir = (u > u1) ? 1 : -1;
                                onedir = true;
                                if (EXT) ++pos;
                                if (lg == 0 && L.J(t - 1) < t) L.J(t - 1) = (unsigned char)t;
                                act = kEval;
                            }
                        } else {
                            act = fail ? kNext : kDescend;
                        }
                    }
                }
                // limited discrepancy search: once the next value of this level
                // is over the budget, so is every later one (the cost does not
                // fall along the walk) -- leave the level now (one cut, as when
                // the value is tried) instead of spending a step on it.  After a
                // kEval the next value is the one already set (position pos).
                if (EXT && cfg.lds >= 0 && (act == kNext || act == kEval) &&
                    dab + (cfg.lds_rank ? pos + (act == kNext ? 1 : 0) : 1) > cfg.lds) {
                    ++cuts;
                    act = kUp;
                }
                if (act == kDescend) {
                    // save level t; the child becomes the parent of level t-1
                    if (lg == 0) {
                        L.u(t) = (short)u;
                        L.ud(t) = i2d_exact(u);
                        L.u1(t) = (short)u1;
                        L.zi(t) = (short)(onedir ? dir : zi);
                        L.meta(t) = (unsigned char)((onedir ? kOneDir : 0) | (s < 0 ? kNegS : 0) | (zp ? kZeroPrefix : 0));
                        L.xq(t) = xq;
                        L.y(t) = y;
                        L.rho(t) = rhoP;
                        if (EXT) {
                            L.dab(t) = (unsigned char)dab;
                            L.pos(t) = (unsigned char)min(pos, 255);
                        }
                    }
                    if (EXT) dab += cost;
                    {
                        // the child's W = W + xq Bq, recomputed instead of keeping the
                        // candidate vector live across the node (registers); the opaque copy
                        // of xq keeps the compiler from reusing the earlier products
                        int xo;
                        asm volatile("mov.b32 %0, %1;" : "=r"(xo) : "r"(xq));
#pragma unroll
                        for (int q = 0; q < CPL; ++q) W[q] += (long long)xo * (long long)bq[q];
                    }
                    Epar = Ech;
                    rhoP = rho;
                    zp = zp && (u == 0);
                    --t;
                    Bt = Btab[t];
                    nbq_t = nbqtab[t];
#pragma unroll
                    for (int q = 0; q < CPL; ++q) bq[q] = (lg + G * q < dim) ? bqtab[(int64_t)t * dimPad + lg + G * q] : 0;
                    act = kEnter;
                } else if (act == kUp) {
                    // step back; subtract each level's term; donated levels are done
                    int meta = 0;
                    for (;;) {
                        if (t == t0) { finished = true; break; }
                        ++t;
                        meta = L.meta(t);
                        const int xqt = L.xq(t);
                        const long long axt = xqt < 0 ? -(long long)xqt : (long long)xqt;
                        nbq_t = nbqtab[t];
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            bq[q] = (lg + G * q < dim) ? bqtab[(int64_t)t * dimPad + lg + G * q] : 0;
                            W[q] -= (long long)xqt * (long long)bq[q];
                        }
                        Epar -= (((long long)ehalf * (axt + 1)) >> 1) + nbq_t + 1;
                        if (!(meta & kDonated)) {
                            // (LDS) a level whose next value is over the budget is left too
                            if (EXT && cfg.lds >= 0 &&
                                L.dab(t) + (cfg.lds_rank ? L.pos(t) + 1 : 1) > cfg.lds) {
                                ++cuts;
                                continue;
                            }
                            break;
                        }
                    }
                    if (!finished) {
                        u = L.u(t);
                        u1 = L.u1(t);
                        onedir = meta & kOneDir;
                        s = (meta & kNegS) ? -1 : 1;
                        zp = (meta & kZeroPrefix) != 0;
                        if (onedir) dir = L.zi(t); else zi = L.zi(t);
                        y = L.y(t);
                        rhoP = L.rho(t);
                        if (EXT) { dab = L.dab(t); pos = L.pos(t); }
                        Bt = Btab[t];
                        act = kNext;
                    }
                }
            }
            if (finished) {
                const unsigned long long csum = group_sum<G>(cfma, gmask);
                if (lg == 0) {
                    if (abort && !quiet && !(*(volatile unsigned*)&ctrl->stop)) set_status(P.inst[inst], ST_EOVERFLOW);
                    atomicAdd(&P.cnt[inst].nodes, (unsigned long long)nodes);
                    atomicAdd(&P.cnt[inst].passed, (unsigned long long)passed);
                    atomicAdd(&P.cnt[inst].leaves, (unsigned long long)leaves);
                    atomicAdd(&P.cnt[inst].center_fma, csum);
                    atomicAdd(&P.cnt[inst].fallbacks, (unsigned long long)fallbacks);
                    if (cuts) atomicAdd(&P.cnt[inst].lds_cuts, (unsigned long long)cuts);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&P.plog_nodes[L.gid()]), (unsigned long long)nodes);
                    if (item_sols) atomicAdd(&P.plog_sols[L.gid()], item_sols);
                    atomicAdd(&ctrl->walk_cycles, (unsigned long long)(clock64() - walk0));
                    atomicSub(&ctrl->busy, 1);
                }
                state = (abort && *(volatile unsigned*)&ctrl->stop) ? kDone : kFetch;
                state = __shfl_sync(gmask, state, 0, G);
            }
        }
        if (__all_sync(0xffffffffu, state == kDone)) break;
        if (__all_sync(0xffffffffu, state != kWalk)) __nanosleep(500);   // whole warp waiting for work
    }
    if (lg == 0) atomicAdd(&ctrl->life_cycles, (unsigned long long)(clock64() - life0));
}

// ---------------------------------------------------------------------------
// Solutions: per-instance segments sorted by key.
// ---------------------------------------------------------------------------
// counts of the stored records per instance
__global__ void sol_count_kernel(Pools P, unsigned long long* fill) {
    const int64_t stored = min((int64_t)P.ctrl->nsol_total, P.sol_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < stored; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&fill[P.sols[k].inst], 1ULL);
}

// soff = exclusive prefix sums of the stored counts; fill reset for the scatter
__global__ void sol_offsets_kernel(Pools P, int64_t* soff, unsigned long long* fill) {
    int64_t run = 0;
    for (int i = 0; i < P.count; ++i) {
        soff[i] = run;
        run += (int64_t)fill[i];
        fill[i] = 0;
    }
    soff[P.count] = run;
}

__global__ void sol_scatter_kernel(Pools P, const int64_t* soff, unsigned long long* fill, SolRec* seg) {
    const int64_t stored = min((int64_t)P.ctrl->nsol_total, P.sol_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < stored; k += (int64_t)gridDim.x * blockDim.x) {
        const SolRec r = P.sols[k];
        const unsigned long long pos = atomicAdd(&fill[r.inst], 1ULL);
        seg[soff[r.inst] + (int64_t)pos] = r;
    }
}

// rank of each record among its instance's records (key order, ties by slot)
__global__ void sol_rank_kernel(Pools P, const int64_t* soff, const SolRec* seg, SolRec* out) {
    const int64_t stored = soff[P.count];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < stored; k += (int64_t)gridDim.x * blockDim.x) {
        const SolRec r = seg[k];
        const int64_t lo = soff[r.inst], hi = soff[r.inst + 1];
        int64_t rank = 0;
        for (int64_t j = lo; j < hi; ++j) {
            const SolRec o = seg[j];
            rank += (o.hi < r.hi) || (o.hi == r.hi && (o.lo < r.lo || (o.lo == r.lo && j < k)));
        }
        out[lo + rank] = r;
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from api.cu).
// ---------------------------------------------------------------------------
// (G, CPL) instances: CPL = coordinates per lane, G * CPL >= n + 1
#define MSP_ENUM_SHAPES(X) X(4, 16) X(4, 32) X(8, 8) X(8, 16) X(16, 4) X(16, 6) X(16, 8) X(32, 4)

static int pick_cpl(int lanes, int dimMax) {
    const int need = (dimMax + lanes - 1) / lanes;
    const int opts[] = {4, 6, 8, 16, 32};
    for (int c : opts) {
        if (c < need) continue;
        switch (lanes * 100 + c) {
            case 416: case 432: case 808: case 816: case 1604: case 1606: case 1608: case 3204: return c;
            default: break;
        }
    }
    return 0;
}

int enum_smem_bytes(int lanes, int threads, int Kmax) { return (threads / lanes) * level_bytes(Kmax); }

cudaError_t launch_split(const Pools& P, const EnumCfg& cfg, int lanes, int max_depth, int64_t target,
                         int64_t* fcnt, cudaStream_t st) {
    switch (lanes) {
        case 4: split_kernel<4><<<P.count, 256, 0, st>>>(P, cfg, max_depth, target, fcnt); break;
        case 8: split_kernel<8><<<P.count, 256, 0, st>>>(P, cfg, max_depth, target, fcnt); break;
        case 16: split_kernel<16><<<P.count, 256, 0, st>>>(P, cfg, max_depth, target, fcnt); break;
        case 32: split_kernel<32><<<P.count, 256, 0, st>>>(P, cfg, max_depth, target, fcnt); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    queue_kernel<<<1, 1, 0, st>>>(P);
    return cudaGetLastError();
}

// ring slot k starts free for index k
__global__ void ring_init_kernel(unsigned long long* seq, int64_t cap) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += (int64_t)gridDim.x * blockDim.x)
        seq[k] = (unsigned long long)k;
}

cudaError_t launch_ring_init(unsigned long long* seq, int64_t cap, cudaStream_t st) {
    ring_init_kernel<<<64, 256, 0, st>>>(seq, cap);
    return cudaGetLastError();
}

cudaError_t launch_start(Ctrl* ctrl, unsigned long long cap_ns, int keep, cudaStream_t st) {
    start_kernel<<<1, 1, 0, st>>>(ctrl, cap_ns, keep);
    return cudaGetLastError();
}

// resident blocks per SM of the plain walker (variant 0) or of the fused
// launch's (variant 3, which also holds the splitter's static shared memory)
int enum_blocks_per_sm(int lanes, int threads, int dimMax, int Kmax, int variant) {
    int n = 0;
    const int cpl = pick_cpl(lanes, dimMax);
    const int smem = enum_smem_bytes(lanes, threads, Kmax);
#define MSP_OCC1(g, c, v)                                                                             \
    {                                                                                                 \
        if (cudaFuncSetAttribute(enum_kernel<g, c, v>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) \
                != cudaSuccess ||                                                                     \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, enum_kernel<g, c, v>, threads, smem) !=     \
                cudaSuccess) {                                                                        \
            cudaGetLastError();                                                                       \
            n = 0;                                                                                    \
        }                                                                                             \
    }
#define MSP_OCC(g, c)                                                                                 \
    if (lanes == g && cpl == c) {                                                                     \
        if (variant == 3) MSP_OCC1(g, c, 3)                                                           \
        else MSP_OCC1(g, c, 0)                                                                        \
    }
    MSP_ENUM_SHAPES(MSP_OCC)
#undef MSP_OCC
#undef MSP_OCC1
    return n;
}

int64_t walker_bytes(int Kmax, int dimPad) { return WalkerLayout{Kmax, dimPad}.bytes(); }

int64_t donation_slot_bytes(int Kmax, int dimPad) { return donation_stride(Kmax, dimPad); }

// pipe.on: the fused launch, cooperative so that every block is resident
// (walkers wait for instances that other blocks prepare)
cudaError_t launch_enum(const Pools& P, const EnumCfg& cfg, int lanes, int blocks, int threads, char* scratch,
                        int Kmax, int dimPad, int variant, const Pipe& pipe, cudaStream_t st) {
    WalkerLayout W{Kmax, dimPad};
    const int cpl = pick_cpl(lanes, P.dimMax);
    const int smem = enum_smem_bytes(lanes, threads, Kmax);
#define MSP_LAUNCH1(g, c, b)                                                                          \
    {                                                                                                 \
        /* the shared-memory attribute is set once, outside any stream capture */                     \
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;                                     \
        cudaStreamIsCapturing(st, &cs);                                                               \
        if (cs == cudaStreamCaptureStatusNone) {                                                      \
            cudaError_t e = cudaFuncSetAttribute(enum_kernel<g, c, b>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
            if (e != cudaSuccess) return e;                                                           \
        }                                                                                             \
        if (pipe.on) {                                                                                \
            cudaLaunchConfig_t lc = {};                                                               \
            lc.gridDim = dim3(blocks);                                                                \
            lc.blockDim = dim3(threads);                                                              \
            lc.dynamicSmemBytes = smem;                                                               \
            lc.stream = st;                                                                           \
            cudaLaunchAttribute at[1];                                                                \
            at[0].id = cudaLaunchAttributeCooperative;                                                \
            at[0].val.cooperative = 1;                                                                \
            lc.attrs = at;                                                                            \
            lc.numAttrs = 1;                                                                          \
            return cudaLaunchKernelEx(&lc, enum_kernel<g, c, b>, P, cfg, scratch, W, pipe);           \
        }                                                                                             \
        enum_kernel<g, c, b><<<blocks, threads, smem, st>>>(P, cfg, scratch, W, pipe);                \
        return cudaGetLastError();                                                                    \
    }
#define MSP_LAUNCH(g, c)                                                                              \
    if (lanes == g && cpl == c) {                                                                     \
        if (variant == 3) MSP_LAUNCH1(g, c, 3)                                                        \
        else if (variant == 2) MSP_LAUNCH1(g, c, 2)                                                   \
        else if (variant == 1) MSP_LAUNCH1(g, c, 1)                                                   \
        else MSP_LAUNCH1(g, c, 0)                                                                     \
    }
    MSP_ENUM_SHAPES(MSP_LAUNCH)
#undef MSP_LAUNCH
#undef MSP_LAUNCH1
    return cudaErrorInvalidValue;
}

cudaError_t launch_collect(const Pools& P, int64_t* soff, unsigned long long* fill, SolRec* seg, SolRec* out,
                           cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(fill, 0, sizeof(unsigned long long) * P.count, st);
    if (e != cudaSuccess) return e;
    sol_count_kernel<<<256, 256, 0, st>>>(P, fill);
    sol_offsets_kernel<<<1, 1, 0, st>>>(P, soff, fill);
    sol_scatter_kernel<<<256, 256, 0, st>>>(P, soff, fill, seg);
    sol_rank_kernel<<<256, 256, 0, st>>>(P, soff, seg, out);
    return cudaGetLastError();
}

}  // namespace msp
