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
// The centre uses the partial-sum cache of Gama-Nguyen-Regev: sigma[t][i]
// holds the fold down to index i, J[t] the highest level changed since, so
// only the changed tail of the fold is redone -- the same operations in
// the same order as the full fold.
#include "common.cuh"

namespace msp {

enum { HOELDER_CUT = 0, HOELDER_FILTER = 1, HOELDER_OFF = 2 };
constexpr int kUMax = 1 << 20;   // |u| bound keeping integer leaf sums exact

__device__ __forceinline__ int zigzag(int u1, int s, int i) {
    return (i & 1) == 0 ? u1 + s * (i >> 1) : u1 - s * ((i - 1) >> 1);
}

__device__ __forceinline__ double slack_of(int dim, int use_eps) {
    return use_eps ? (double)dim * 0x1p-20 : 0.0;
}

// ---------------------------------------------------------------------------
// Splitter: one block per instance.
// ---------------------------------------------------------------------------

// Sibling loop of one parent at level t (one thread).  With WRITE, children
// that pass both tests are written at out index base, base+1, ...
template <int G, bool WRITE>
__device__ int64_t expand_parent(const Pools& P, const EnumCfg& cfg, int inst, int dd, int dim, int t,
                                 const int32_t* __restrict__ pu, double prho, const double* __restrict__ pw,
                                 int out_sel, int64_t base, unsigned long long& nodes,
                                 unsigned long long& passed, bool& ovf) {
    const InstDesc& I = P.inst[inst];
    const double* muT = P.muT + I.offMuT;
    const double* Bt = P.B + I.offB;
    const double* bhat = P.bhat + I.offBhat;
    const double eps = slack_of(dim, cfg.use_eps);
    const double Rb = (double)dim + eps;

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
    int64_t nch = 0;
    for (;;) {
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
        if (cfg.hoelder != HOELDER_OFF) fail = rho > __dadd_rn(sl[0], eps);
        if (fail && cfg.hoelder == HOELDER_CUT) {
            if (onedir) break;
            ++zi;
            u = zigzag(u1, s, zi);
            dir = (u > u1) ? 1 : -1;
            onedir = true;
            continue;
        }
        if (!fail) {
            if (WRITE) {
                const int64_t o = frontier_index(P, inst, out_sel, base + nch);
                int32_t* ou = P.fu + o * P.Kmax;
                for (int i = 0; i < P.Kmax; ++i) ou[i] = (i > t && i < dd) ? pu[i] : 0;
                ou[t] = u;
                P.frho[o] = rho;
                double* ow = P.fw + o * P.dimPad;
                for (int c = 0; c < dim; ++c) ow[c] = __fma_rn(x, bhat[(int64_t)t * dim + c], pw[c]);
            }
            ++nch;
        }
        if (onedir) u += dir;
        else { ++zi; u = zigzag(u1, s, zi); }
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

template <int G>
__global__ void __launch_bounds__(256) split_kernel(Pools P, EnumCfg cfg, int max_depth, int64_t target,
                                                    int64_t* fcnt) {
    const int inst = blockIdx.x;
    InstDesc& I = P.inst[inst];
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = (I.status == ST_OK);
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
        if (threadIdx.x == 0) P.frho[o] = 0.0;
    }
    __syncthreads();
    int sel = 0, t = dd - 1, depth = 0;
    int64_t count = 1;
    unsigned long long nodes = 0, passed = 0;
    bool ovf = false;
    __shared__ int s_ovf;
    while (depth < max_depth && t >= 1 && count < target) {
        for (int64_t p = threadIdx.x; p < count; p += blockDim.x) {
            const int64_t o = frontier_index(P, inst, sel, p);
            unsigned long long dn = 0, dp = 0;
            cnt[p] = expand_parent<G, false>(P, cfg, inst, dd, dim, t, P.fu + o * P.Kmax, P.frho[o],
                                             P.fw + o * P.dimPad, sel ^ 1, 0, dn, dp, ovf);
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
                                   sel ^ 1, cnt[p], nodes, passed, ovf);
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
    if (threadIdx.x == 0) {
        I.split_level = t + 1;
        I.front_sel = sel;
        I.nprefix = count;
    }
    if (ovf) set_status(I, ST_EOVERFLOW);
}

// resets the control words and arms the time cap on the device clock
__global__ void start_kernel(Ctrl* c, unsigned long long cap_ns) {
    c->qhead = 0;
    c->dhead = 0;
    c->dtail = 0;
    c->idle = 0;
    c->busy = 0;
    c->nsol_total = 0;
    c->stop = 0;
    c->gstatus = 0;
    c->deadline_ns = cap_ns ? global_time_ns() + cap_ns : 0ULL;
}

// exclusive prefix sums of the per-instance prefix counts (one thread)
__global__ void queue_kernel(Pools P) {
    int64_t run = 0;
    for (int i = 0; i < P.count; ++i) {
        P.qbase[i] = run;
        run += (P.inst[i].status == ST_OK) ? P.inst[i].nprefix : 0;
    }
    P.qbase[P.count] = run;
    P.ctrl->qhead = 0;
}

// ---------------------------------------------------------------------------
// Enumerator: persistent walkers of G lanes.
// ---------------------------------------------------------------------------

struct WalkerLayout {
    int Kmax, dimPad;
    __host__ __device__ int64_t bytes() const {
        // level state: 5 int32 arrays + 2 double arrays; w stack; sigma cache
        const int64_t ints = ((int64_t)5 * Kmax * 4 + 15) / 16 * 16;
        return ints + (int64_t)2 * Kmax * 8 + (int64_t)Kmax * dimPad * 8 + (int64_t)Kmax * (Kmax + 1) * 8;
    }
};

// Header of a donated sibling range: the untried values at level t of a
// walk, continued by another walker exactly where the donor stopped.  The
// slot continues with int32 u[Kmax] (values above t) and double w[dimPad]
// (w^(t+1)).
struct DonHdr {
    int32_t inst, t, u, u1, zi, meta;
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

// level meta bits
constexpr int kOneDir = 1, kNegS = 2, kZeroPrefix = 4, kDonated = 8;
// walk actions
constexpr int kNext = 0, kDescend = 1, kUp = 2, kEval = 3;

template <int G>
__global__ void __launch_bounds__(256) enum_kernel(Pools P, EnumCfg cfg, char* scratch, WalkerLayout W) {
    constexpr int CPL = kMaxDim / G;
    const int lg = threadIdx.x & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int64_t walker = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    char* ws = scratch + walker * W.bytes();
    const int Kmax = W.Kmax, dimPad = W.dimPad, S = Kmax + 1;
    int32_t* lv_u = reinterpret_cast<int32_t*>(ws);
    int32_t* lv_u1 = lv_u + Kmax;
    int32_t* lv_zi = lv_u1 + Kmax;
    int32_t* lv_meta = lv_zi + Kmax;
    int32_t* lv_J = lv_meta + Kmax;
    double* lv_y = reinterpret_cast<double*>(ws + ((int64_t)5 * Kmax * 4 + 15) / 16 * 16);
    double* lv_rhoP = lv_y + Kmax;
    double* wstack = lv_rhoP + Kmax;
    double* sigma = wstack + (int64_t)Kmax * dimPad;
    Ctrl* ctrl = P.ctrl;

    const int64_t total = P.qbase[P.count];
    bool static_done = false;   // meaningful in lane 0 only
    for (;;) {
        // ---- obtain work: a split prefix, else a donated sibling range ----
        int src = 0;
        long long id = 0;
        if (lg == 0) {
            if (!static_done) {
                const unsigned long long it = atomicAdd(&ctrl->qhead, 1ULL);
                if ((int64_t)it < total) {
                    src = 1;
                    id = (long long)it;
                    atomicAdd(&ctrl->busy, 1);
                } else {
                    static_done = true;
                }
            }
            if (src == 0) {
                atomicAdd(&ctrl->idle, 1);
                for (;;) {
                    if (*(volatile unsigned*)&ctrl->stop) break;
                    const unsigned long long h = *(volatile unsigned long long*)&ctrl->dhead;
                    const unsigned long long tl = *(volatile unsigned long long*)&ctrl->dtail;
                    if (h < tl) {
                        if (atomicCAS(&ctrl->dhead, h, h + 1) == h) {
                            atomicAdd(&ctrl->busy, 1);
                            src = 2;
                            id = (long long)h;
                            break;
                        }
                        continue;
                    }
                    if (*(volatile int*)&ctrl->busy == 0 &&
                        *(volatile unsigned long long*)&ctrl->dhead == *(volatile unsigned long long*)&ctrl->dtail)
                        break;   // nothing left anywhere
                    if (global_time_ns() > ctrl->deadline_ns) {
                        atomicExch(&ctrl->stop, 2u);
                        break;
                    }
                    __nanosleep(1000);
                }
                atomicSub(&ctrl->idle, 1);
            }
            if (src == 2) {   // wait until the donor has written the slot
                while (!*(volatile unsigned*)&P.don_ready[id]) {
                    if (global_time_ns() > ctrl->deadline_ns) {
                        atomicExch(&ctrl->stop, 2u);
                        atomicSub(&ctrl->busy, 1);
                        src = 0;
                        break;
                    }
                    __nanosleep(100);
                }
                __threadfence();
            }
        }
        src = __shfl_sync(gmask, src, 0, G);
        id = __shfl_sync(gmask, id, 0, G);
        if (src == 0) break;

        // ---- set up the walk ----
        int inst;
        int64_t gid;
        int t0;
        double w_par[CPL], w_ch[CPL];
        double rhoP, y = 0.0;
        int u = 0, u1 = 0, s = 1, zi = 1, dir = 0;
        bool onedir = false, zp = true;
        int act;
        if (src == 1) {
            gid = P.qperm ? P.qperm[id] : (int64_t)id;
            int lo = 0, hi = P.count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (P.qbase[mid] <= gid) lo = mid; else hi = mid;
            }
            inst = lo;
        } else {
            const DonHdr* hd = reinterpret_cast<const DonHdr*>(P.don + id * P.don_stride);
            inst = hd->inst;
            gid = hd->gid;
        }
        const InstDesc& I = P.inst[inst];
        const int dd = I.dd, dim = I.dim, n = I.n, m = I.m;
        const double* __restrict__ muT = P.muT + I.offMuT;
        const double* __restrict__ Bt = P.B + I.offB;
        const double* __restrict__ bhat = P.bhat + I.offBhat;
        const int32_t* __restrict__ kb = P.kb + I.offKb;
        const double eps = slack_of(dim, cfg.use_eps);
        const double Rb = (double)dim + eps;
        if (src == 1) {
            const int split_level = I.split_level;
            t0 = split_level - 1;
            const int64_t fo = frontier_index(P, inst, I.front_sel, gid - P.qbase[inst]);
            const int32_t* pu = P.fu + fo * P.Kmax;
            for (int i = split_level; i < dd; ++i) {
                const int32_t v = pu[i];
                lv_u[i] = v;
                zp = zp && (v == 0);
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int c = lg + G * q;
                w_par[q] = (c < dim) ? P.fw[fo * P.dimPad + c] : 0.0;
            }
            rhoP = P.frho[fo];
            act = kEval;   // fresh level: enter it below
        } else {
            const char* slot = P.don + id * P.don_stride;
            const DonHdr hd = *reinterpret_cast<const DonHdr*>(slot);
            const int32_t* su = reinterpret_cast<const int32_t*>(slot + sizeof(DonHdr));
            const double* sw = reinterpret_cast<const double*>(
                slot + ((int64_t)sizeof(DonHdr) + (int64_t)Kmax * 4 + 15) / 16 * 16);
            t0 = hd.t;
            for (int i = t0 + 1; i < dd; ++i) lv_u[i] = su[i];
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int c = lg + G * q;
                w_par[q] = (c < dim) ? sw[c] : 0.0;
            }
            rhoP = hd.rhoP;
            y = hd.y;
            u = hd.u;
            u1 = hd.u1;
            onedir = hd.meta & kOneDir;
            s = (hd.meta & kNegS) ? -1 : 1;
            zp = (hd.meta & kZeroPrefix) != 0;
            if (onedir) dir = hd.zi; else zi = hd.zi;
            act = kNext;   // the donor evaluated u already
        }
        for (int i = lg; i <= t0; i += G) lv_J[i] = dd - 1;
        for (int i = lg; i < dd; i += G) sigma[(int64_t)i * S + dd] = 0.0;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int c = lg + G * q;
            w_ch[q] = 0.0;
            if (c < dim) wstack[(int64_t)t0 * dimPad + c] = w_par[q];
        }
        if (lg == 0) lv_meta[t0] = 0;
        __syncwarp(gmask);

        unsigned long long nodes = 0, passed = 0, leaves = 0, cfma = 0;
        int item_sols = 0;
        int t = t0;
        bool abort = false;

        // entering level t: centre by the cached fold, start of the zig-zag
        auto enter_level = [&]() {
            const int Jt = lv_J[t];
            double acc = sigma[(int64_t)t * S + Jt + 1];
            for (int i = Jt; i > t; --i) {
                acc = __fma_rn((double)lv_u[i], muT[(int64_t)t * dd + i], acc);
                sigma[(int64_t)t * S + i] = acc;
            }
            y = acc;
            cfma += (unsigned long long)(Jt - t);
            if (t > 0) lv_J[t - 1] = max(lv_J[t - 1], Jt);
            lv_J[t] = t;
            const double cstar = -y;
            const double r1 = rint(cstar);
            if (fabs(r1) >= (double)kUMax) abort = true;
            u1 = abort ? 0 : (int)r1;
            s = (cstar >= r1) ? 1 : -1;
            onedir = false; dir = 0; zi = 1;
            if (zp && cfg.sym) { u1 = 0; onedir = true; dir = 1; }
            u = u1;
            if (t > 0) lv_J[t - 1] = max(lv_J[t - 1], t);
        };
        if (src == 1) enter_level();

        while (!abort) {
            if (act == kNext) {
                if (onedir) u += dir;
                else { ++zi; u = zigzag(u1, s, zi); }
                if (t > 0) lv_J[t - 1] = max(lv_J[t - 1], t);
            }
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
                        const unsigned long long q = *(volatile unsigned long long*)&ctrl->dtail -
                                                     *(volatile unsigned long long*)&ctrl->dhead;
                        want = q < (unsigned long long)idle;
                    }
                }
                if (__shfl_sync(gmask, st, 0, G)) { abort = true; break; }
                if (__shfl_sync(gmask, want, 0, G)) {
                    int h = -1;
                    for (int l = t0; l > t; --l)
                        if (!(lv_meta[l] & kDonated)) { h = l; break; }
                    if (h >= 0) {
                        long long slot = -1;
                        if (lg == 0) {
                            for (int tries = 0; tries < 64; ++tries) {
                                const unsigned long long old = *(volatile unsigned long long*)&ctrl->dtail;
                                if ((int64_t)old >= P.don_cap) break;
                                if (atomicCAS(&ctrl->dtail, old, old + 1) == old) { slot = (long long)old; break; }
                            }
                        }
                        slot = __shfl_sync(gmask, slot, 0, G);
                        if (slot >= 0) {
                            char* sp = P.don + slot * P.don_stride;
                            int32_t* su = reinterpret_cast<int32_t*>(sp + sizeof(DonHdr));
                            double* sw = reinterpret_cast<double*>(
                                sp + ((int64_t)sizeof(DonHdr) + (int64_t)Kmax * 4 + 15) / 16 * 16);
                            if (lg == 0) {
                                DonHdr hd;
                                hd.inst = inst; hd.t = h; hd.u = lv_u[h]; hd.u1 = lv_u1[h];
                                hd.zi = lv_zi[h]; hd.meta = lv_meta[h] & ~kDonated; hd.gid = gid;
                                hd.y = lv_y[h]; hd.rhoP = lv_rhoP[h];
                                *reinterpret_cast<DonHdr*>(sp) = hd;
                            }
                            for (int i = h + 1 + lg; i < dd; i += G) su[i] = lv_u[i];
                            for (int c = lg; c < dim; c += G) sw[c] = wstack[(int64_t)h * dimPad + c];
                            __threadfence();
                            __syncwarp(gmask);
                            if (lg == 0) atomicExch(&P.don_ready[slot], 1u);
                            lv_meta[h] |= kDonated;
                            __syncwarp(gmask);
                        }
                    }
                }
            }
            if (u >= kUMax || u <= -kUMax) { abort = true; set_status(const_cast<InstDesc&>(I), ST_EOVERFLOW); break; }
            const double x = __dadd_rn((double)u, y);
            const double rho = __fma_rn(__dmul_rn(x, x), Bt[t], rhoP);
            ++nodes;
            if (!(rho <= Rb)) {   // norm test (a NaN never passes)
                act = kUp;
            } else {
                ++passed;
                if (t == 0) {
                    ++leaves;
                    // exact Theorem 1 check of v = sum_j u_j b_j
                    long long v[CPL];
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const int c = lg + G * q;
                        long long a = 0;
                        if (c < dim) {
                            a = (long long)u * kb[c];
                            for (int j = 1; j < dd; ++j) a += (long long)lv_u[j] * kb[(int64_t)j * dim + c];
                        }
                        v[q] = a;
                    }
                    long long mine = 0;
#pragma unroll
                    for (int q = 0; q < CPL; ++q) if (q == (dim - 1) / G) mine = v[q];
                    const long long last = __shfl_sync(gmask, mine, (dim - 1) % G, G);
                    const long long sg = (cfg.sym && last == -1) ? -1 : 1;
                    bool ok = (last * sg == 1);
                    unsigned long long khi = 0, klo = 0;
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const int c = lg + G * q;
                        const long long vc = v[q] * sg;
                        if (c < n && vc != 1 && vc != -1) ok = false;
                    }
                    ok = __all_sync(gmask, ok);
                    if (ok) {
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
                            const unsigned long long k = atomicAdd(&ctrl->nsol_total, 1ULL);
                            if ((int64_t)k < P.sol_cap) {
                                SolRec r;
                                r.inst = inst; r.pad = 0; r.hi = khi; r.lo = klo;
                                P.sols[k] = r;
                            }
                            atomicAdd(&P.cnt[inst].nsol, 1ULL);
                            if (cfg.first) atomicExch(&ctrl->stop, 1u);
                        }
                        if (ok) ++item_sols;
                    }
                    act = kNext;
                } else {
                    double sl = 0.0;
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const int c = lg + G * q;
                        if (c < dim) {
                            w_ch[q] = __fma_rn(x, bhat[(int64_t)t * dim + c], w_par[q]);
                            sl = __dadd_rn(sl, fabs(w_ch[q]));
                        }
                    }
#pragma unroll
                    for (int off = G / 2; off >= 1; off >>= 1)
                        sl = __dadd_rn(sl, __shfl_xor_sync(gmask, sl, off, G));
                    bool fail = false;
                    if (cfg.hoelder != HOELDER_OFF) fail = rho > __dadd_rn(sl, eps);
                    if (fail && cfg.hoelder == HOELDER_CUT) {
                        if (onedir) {
                            act = kUp;
                        } else {
                            // first failure: one more regular value, then one direction
                            ++zi;
                            u = zigzag(u1, s, zi);
                            dir = (u > u1) ? 1 : -1;
                            onedir = true;
                            lv_J[t - 1] = max(lv_J[t - 1], t);
                            act = kEval;
                        }
                    } else {
                        act = fail ? kNext : kDescend;
                    }
                }
            }
            if (act == kDescend) {
                // save level t, make the child the parent of level t-1
                lv_u[t] = u;
                lv_u1[t] = u1;
                lv_zi[t] = onedir ? dir : zi;
                lv_meta[t] = (onedir ? kOneDir : 0) | (s < 0 ? kNegS : 0) | (zp ? kZeroPrefix : 0);
                lv_y[t] = y;
                lv_rhoP[t] = rhoP;
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const int c = lg + G * q;
                    w_par[q] = w_ch[q];
                    if (c < dim) wstack[(int64_t)(t - 1) * dimPad + c] = w_ch[q];
                }
                rhoP = rho;
                zp = zp && (u == 0);
                --t;
                __syncwarp(gmask);
                enter_level();
                act = kEval;
                continue;
            }
            if (act == kUp) {
                // step back; levels whose remaining values were donated are done
                bool done = false;
                int meta = 0;
                do {
                    if (t == t0) { done = true; break; }
                    ++t;
                    meta = lv_meta[t];
                } while (meta & kDonated);
                if (done) break;
                u = lv_u[t];
                u1 = lv_u1[t];
                onedir = meta & kOneDir;
                s = (meta & kNegS) ? -1 : 1;
                zp = (meta & kZeroPrefix) != 0;
                if (onedir) dir = lv_zi[t]; else zi = lv_zi[t];
                y = lv_y[t];
                rhoP = lv_rhoP[t];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const int c = lg + G * q;
                    w_par[q] = (c < dim) ? wstack[(int64_t)t * dimPad + c] : 0.0;
                }
                __syncwarp(gmask);
                act = kNext;
            }
        }
        if (abort && lg == 0 && !(*(volatile unsigned*)&ctrl->stop)) set_status(const_cast<InstDesc&>(I), ST_EOVERFLOW);
        if (lg == 0) {
            atomicAdd(&P.cnt[inst].nodes, nodes);
            atomicAdd(&P.cnt[inst].passed, passed);
            atomicAdd(&P.cnt[inst].leaves, leaves);
            atomicAdd(&P.cnt[inst].center_fma, cfma);
            atomicAdd(reinterpret_cast<unsigned long long*>(&P.plog_nodes[gid]), nodes);
            if (item_sols) atomicAdd(&P.plog_sols[gid], item_sols);
            atomicSub(&ctrl->busy, 1);
        }
        __syncwarp(gmask);
        if (abort) {
            int st = 0;
            if (lg == 0) st = *(volatile unsigned*)&ctrl->stop != 0;
            if (__shfl_sync(gmask, st, 0, G)) break;
        }
    }
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
cudaError_t launch_split(const Pools& P, const EnumCfg& cfg, int lanes, int max_depth, int64_t target,
                         int64_t* fcnt, cudaStream_t st) {
    switch (lanes) {
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

cudaError_t launch_start(Ctrl* ctrl, unsigned long long cap_ns, cudaStream_t st) {
    start_kernel<<<1, 1, 0, st>>>(ctrl, cap_ns);
    return cudaGetLastError();
}

int enum_blocks_per_sm(int lanes, int threads) {
    int n = 0;
    switch (lanes) {
        case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, enum_kernel<8>, threads, 0); break;
        case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, enum_kernel<16>, threads, 0); break;
        case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, enum_kernel<32>, threads, 0); break;
        default: break;
    }
    return n;
}

int64_t walker_bytes(int Kmax, int dimPad) { return WalkerLayout{Kmax, dimPad}.bytes(); }

int64_t donation_slot_bytes(int Kmax, int dimPad) { return donation_stride(Kmax, dimPad); }

cudaError_t launch_enum(const Pools& P, const EnumCfg& cfg, int lanes, int blocks, int threads, char* scratch,
                        int Kmax, int dimPad, cudaStream_t st) {
    WalkerLayout W{Kmax, dimPad};
    switch (lanes) {
        case 8: enum_kernel<8><<<blocks, threads, 0, st>>>(P, cfg, scratch, W); break;
        case 16: enum_kernel<16><<<blocks, threads, 0, st>>>(P, cfg, scratch, W); break;
        case 32: enum_kernel<32><<<blocks, threads, 0, st>>>(P, cfg, scratch, W); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
