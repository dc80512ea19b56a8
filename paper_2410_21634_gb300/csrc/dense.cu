// Single-seed LocalGD with dense x and r in HBM (Eq. local-gd, Section 3.3).
//
// One round t = three launches on the solve stream:
//   k_prep      zero the round counters
//   k_frontier  S_t from the candidate list C_t: threshold test, r_u -> 0, x_u += c r_u,
//               per-edge share w_u, degree bin, FP64 round statistics; for the heat
//               kernel it also clears what is left of the finished layer t-1
//   k_push      every (u in S_t, v in N(u)): r_v += w_u by atomic add; a node whose
//               residual crosses its threshold during the round is appended to C_{t+1}
//               exactly once (contributions are >= 0, so the running value crosses once)
// C_t is therefore exactly S_t (plus the seed in round 0) and no round scans all n nodes
// (the remark after Corollary 3.6: thresholding must cost O(touched), not O(n)).
//
// Floating point: every expression of the round is written with explicit round-to-nearest
// intrinsics (never contracted into FMA) in the order x_u + c*rho, (coef*rho)/d_u,
// fl(eps_theta*d_u), so FP64 rounds match a sequential FP64 evaluation up to the order of
// the additions into each r_v.  FP32 mode stores x and r as float; shares are computed in
// FP64 and rounded once; thresholds are FP64 (stored as the float just above, which makes
// the float comparison equal to the FP64 one) and all statistics are FP64.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "detsort.cuh"

namespace cg = cooperative_groups;

namespace gde {

template <typename real> struct alignas(2 * sizeof(real)) RPair {
    real r;    // residual r_v
    real thr;  // fl(eps d_v) (FP32: rounded up to float)
};

struct Ctl {
    unsigned long long hub_packed;  // (hub count << 40) | hub volume
    unsigned int cnt_small;
    unsigned int cnt_med;
    unsigned int cand_out;
    unsigned int touched_out;
    unsigned int n_active;
    unsigned int pad;
    unsigned long long vol;
    double rS_l1;
    double scat;
    double retired;
    unsigned int overflow;
    unsigned int pad2;
};

constexpr int kHubVolBits = 40;
constexpr unsigned long long kHubVolMask = (1ull << kHubVolBits) - 1;

struct DenseWork {
    int precision = 0;
    int64_t n = 0;
    size_t rsz = 8;
    void *x = nullptr;
    void *rp = nullptr;       // RPair[n]     (PPR, Katz)
    void *rl[2] = {nullptr, nullptr};  // layers  (HK)
    int32_t *cand[2] = {nullptr, nullptr};
    int32_t *touched[2] = {nullptr, nullptr};
    int32_t *active = nullptr;
    int64_t *b_beg[3] = {nullptr, nullptr, nullptr};
    int32_t *b_deg[3] = {nullptr, nullptr, nullptr};
    void *b_w[3] = {nullptr, nullptr, nullptr};
    int64_t *hub_vstart = nullptr;
    Ctl *ctl = nullptr;
    Ctl *hctl = nullptr;  // pinned
    // Katz: the source entry x_s - 1 in FP64 (starts at -1, gains every residual pushed at s),
    // so that f_Katz = x - e_s keeps full precision at s (no cancellation against the unit)
    double *xsrc = nullptr;
    int32_t seed = -1;
    Bins bins;
    // deterministic scatter (sort + segmented reduce), allocated on first use
    void *wbuf = nullptr;            // real[n]
    uint32_t *sact[2] = {nullptr, nullptr};   // sorted active ids + temporary
    int64_t *vdeg = nullptr;         // degrees of the sorted active nodes, then their edge starts
    int64_t *vstart = nullptr;
    uint32_t *pkey[2] = {nullptr, nullptr};   // pair targets v
    void *pval[2] = {nullptr, nullptr};       // pair shares w
    void *dscratch = nullptr;
    int64_t *dtotal = nullptr;       // device scalar
    int64_t *htotal = nullptr;       // pinned
    int64_t pair_cap = 0;
    // host-side round state
    gde_kind kind = GDE_PPR;
    int64_t t = 0;
    unsigned ncand = 0;
    unsigned ntouched[2] = {0, 0};  // HK: touched-list length of the layer in each buffer
    int64_t last_active = 0;
    bool done = false;
};

// ------------------------------------------------------------ device helpers --


__device__ __forceinline__ double rabs(double v) { return fabs(v); }
__device__ __forceinline__ float rabs(float v) { return fabsf(v); }


// threshold fl(eps_theta * d) in the storage type; FP32 rounds up so that for a float r,
// r >= thr32  <=>  (double) r >= thr64
template <typename real> __device__ __forceinline__ real thr_store(double eps_theta, int32_t d);
template <> __device__ __forceinline__ double thr_store<double>(double e, int32_t d) {
    return __dmul_rn(e, (double)d);
}
template <> __device__ __forceinline__ float thr_store<float>(double e, int32_t d) {
    return __double2float_ru(__dmul_rn(e, (double)d));
}

// warp-aggregated append; entries past `cap` are dropped and flagged (never expected: each
// list receives every node at most once per round)
__device__ __forceinline__ void append_u32(unsigned *counter, int32_t *list, int32_t v,
                                           unsigned cap, unsigned *overflow) {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned)g.size());
    const unsigned i = g.shfl(base, 0) + g.thread_rank();
    if (i < cap) list[i] = v; else atomicOr(overflow, 1u);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// --------------------------------------------------------------------- init --

// scale of the generalised propagation's residual at a node: y_u = max(d_u, 1)^b r_u
__device__ __forceinline__ double gppr_scale(int32_t d, double b) {
    return pow((double)(d > 0 ? d : 1), b);
}

template <typename real>
__global__ void k_init_pairs(int64_t n, const int32_t *__restrict__ deg, real *__restrict__ x,
                             RPair<real> *__restrict__ rp, double eps, int32_t seed, double gbeta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = real(0);
        RPair<real> p;
        // unit source; the generalised propagation stores it scaled, y_s = S_s
        p.r = (i == seed) ? (gbeta != 0.0 ? from_f64<real>(gppr_scale(deg[i], gbeta)) : real(1)) : real(0);
        p.thr = thr_store<real>(eps, deg[i]);
        rp[i] = p;
    }
}

template <typename real>
__global__ void k_init_layers(int64_t n, real *__restrict__ x, real *__restrict__ r0,
                              real *__restrict__ r1, int32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = real(0);
        r0[i] = (i == seed) ? real(1) : real(0);
        r1[i] = real(0);
    }
}

__global__ void k_prep(Ctl *ctl, int32_t *cand0, int32_t *touched0, int32_t seed) {
    if (threadIdx.x == 0) memset(ctl, 0, sizeof(Ctl));
    if (cand0 && threadIdx.x == 0) cand0[0] = seed;
    if (touched0 && threadIdx.x == 0) touched0[0] = seed;
}

// ----------------------------------------------------------------- frontier --

template <typename real> struct FrontierArgs {
    const int64_t *off;
    const int32_t *cand;
    unsigned ncand;
    real *x;
    RPair<real> *rp;      // PPR/Katz
    real *rcur;           // HK current layer
    double eps_theta;     // HK: fl(theta_t eps)
    double cx;            // x_u += cx * rho  (PPR alpha, else 1)
    double coef;          // PPR 1-alpha, Katz beta, HK fl(tau/(t+1))
    double gbeta;         // generalised propagation: x_u += (cx * rho) / S_u (0: plain PPR)
    double *xsrc;         // Katz: x_seed - 1 in FP64, or NULL
    int32_t seed;
    int propagate;
    int32_t t1, t2;
    int64_t *b_beg[3];
    int32_t *b_deg[3];
    real *b_w[3];
    int64_t *hub_vstart;
    int32_t *active;
    Ctl *ctl;
    unsigned cap;         // capacity of every list (n)
    // HK: clear the finished layer's leftovers
    const int32_t *clear_list;
    unsigned nclear;
    real *rclear;
    real *wbuf;           // deterministic mode: per-node share of the pushed nodes (no bins)
};

template <typename real, int KIND>
__global__ void __launch_bounds__(kThreads) k_frontier(FrontierArgs<real> a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned my_active = 0;
    unsigned long long my_vol = 0;
    double my_rs = 0.0, my_scat = 0.0, my_ret = 0.0;

    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ci = tid; ci < a.ncand; ci += nthreads) {
        const int32_t u = a.cand[ci];
        const int64_t beg = a.off[u];
        const int32_t d = (int32_t)(a.off[u + 1] - beg);
        real rho;
        bool act;
        if (KIND == GDE_HK) {
            rho = a.rcur[u];
            const double thr = __dmul_rn(a.eps_theta, (double)d);
            act = (rho != real(0)) && (fabs((double)rho) >= thr);
        } else {
            const RPair<real> p = a.rp[u];
            rho = p.r;
            act = (rho != real(0)) && (rabs(rho) >= p.thr);
        }
        if (act) {
            if (KIND == GDE_HK) a.rcur[u] = real(0); else a.rp[u].r = real(0);
            const double rho64 = (double)rho;
            if (KIND == GDE_PPR && a.gbeta != 0.0)
                a.x[u] = radd<real>(a.x[u], from_f64<real>(__ddiv_rn(__dmul_rn(a.cx, rho64),
                                                                     gppr_scale(d, a.gbeta))));
            else if (KIND == GDE_PPR)
                a.x[u] = radd<real>(a.x[u], from_f64<real>(__dmul_rn(a.cx, rho64)));
            else
                a.x[u] = radd<real>(a.x[u], rho);
            if (KIND == GDE_KATZ && a.xsrc && u == a.seed) *a.xsrc = __dadd_rn(*a.xsrc, rho64);
            append_u32(&a.ctl->n_active, a.active, u, a.cap, &a.ctl->overflow);
            my_active += 1;
            my_vol += (unsigned long long)d;
            my_rs += fabs(rho64);
            if (a.propagate && d > 0) {
                double w64;
                if (KIND == GDE_KATZ)
                    w64 = __dmul_rn(a.coef, rho64);
                else
                    w64 = __ddiv_rn(__dmul_rn(a.coef, rho64), (double)d);
                const real w = from_f64<real>(w64);
                my_scat += __dmul_rn((double)w, (double)d);
                if (a.wbuf) {
                    a.wbuf[u] = w;
                } else if (d <= a.t1) {
                    cg::coalesced_group g = cg::coalesced_threads();
                    unsigned base = 0;
                    if (g.thread_rank() == 0) base = atomicAdd(&a.ctl->cnt_small, (unsigned)g.size());
                    const unsigned i = g.shfl(base, 0) + g.thread_rank();
                    a.b_beg[0][i] = beg; a.b_deg[0][i] = d; a.b_w[0][i] = w;
                } else if (d <= a.t2) {
                    cg::coalesced_group g = cg::coalesced_threads();
                    unsigned base = 0;
                    if (g.thread_rank() == 0) base = atomicAdd(&a.ctl->cnt_med, (unsigned)g.size());
                    const unsigned i = g.shfl(base, 0) + g.thread_rank();
                    a.b_beg[1][i] = beg; a.b_deg[1][i] = d; a.b_w[1][i] = w;
                } else {
                    // hub: one packed atomic gives both the slot and the start of this
                    // hub's edges in the concatenated hub adjacency, in the same order
                    cg::coalesced_group g = cg::coalesced_threads();
                    const unsigned long long dv = (unsigned long long)d;
                    const unsigned long long excl = cg::exclusive_scan(g, dv);
                    const unsigned long long tot = g.shfl(excl + dv, g.size() - 1);
                    unsigned long long old = 0;
                    if (g.thread_rank() == 0)
                        old = atomicAdd(&a.ctl->hub_packed,
                                        ((unsigned long long)g.size() << kHubVolBits) + tot);
                    old = g.shfl(old, 0);
                    const unsigned long long i = (old >> kHubVolBits) + g.thread_rank();
                    a.b_beg[2][i] = beg; a.b_deg[2][i] = d; a.b_w[2][i] = w;
                    a.hub_vstart[i] = (int64_t)((old & kHubVolMask) + excl);
                }
            }
        }
    }
    if (KIND == GDE_HK) {
        // leftovers of the finished layer (sub-threshold entries) are cleared so the buffer
        // can hold layer t+1; their mass is recorded
        for (int64_t j = tid; j < a.nclear; j += nthreads) {
            const int32_t v = a.clear_list[j];
            my_ret += fabs((double)a.rclear[v]);
            a.rclear[v] = real(0);
        }
    }
    // FP64 round statistics: warp then block reduction, one atomic per block and field
    __shared__ double s_d[3][kWarps];
    __shared__ unsigned long long s_v[kWarps];
    __shared__ unsigned s_a[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double rs = warp_sum(my_rs), sc = warp_sum(my_scat), rt = warp_sum(my_ret);
    unsigned long long vv = warp_sum(my_vol);
    unsigned aa = warp_sum(my_active);
    if (lane == 0) { s_d[0][wid] = rs; s_d[1][wid] = sc; s_d[2][wid] = rt; s_v[wid] = vv; s_a[wid] = aa; }
    __syncthreads();
    if (wid == 0) {
        rs = lane < kWarps ? s_d[0][lane] : 0.0;
        sc = lane < kWarps ? s_d[1][lane] : 0.0;
        rt = lane < kWarps ? s_d[2][lane] : 0.0;
        vv = lane < kWarps ? s_v[lane] : 0ull;
        aa = lane < kWarps ? s_a[lane] : 0u;
        rs = warp_sum(rs); sc = warp_sum(sc); rt = warp_sum(rt); vv = warp_sum(vv); aa = warp_sum(aa);
        if (lane == 0 && (aa | (rt != 0.0))) {
            atomicAdd(&a.ctl->rS_l1, rs);
            atomicAdd(&a.ctl->scat, sc);
            atomicAdd(&a.ctl->retired, rt);
            atomicAdd(&a.ctl->vol, vv);
        }
    }
}

// --------------------------------------------------------------------- push --

template <typename real> struct PushArgs {
    const int32_t *col;
    const int32_t *deg;
    const int64_t *b_beg[3];
    const int32_t *b_deg[3];
    const real *b_w[3];
    const int64_t *hub_vstart;
    RPair<real> *rp;       // PPR/Katz
    real *rnext;           // HK next layer
    double eps_theta_next; // HK: fl(theta_{t+1} eps)
    int32_t *cand_out;
    int32_t *touched_out;
    Ctl *ctl;
    int32_t chunk;
    unsigned cap;
};

template <typename real, int KIND>
__device__ __forceinline__ void scatter(const PushArgs<real> &a, int32_t v, real w) {
    if (KIND == GDE_HK) {
        const real old = atomicAdd(a.rnext + v, w);
        if (old == real(0) && w > real(0))
            append_u32(&a.ctl->touched_out, a.touched_out, v, a.cap, &a.ctl->overflow);
        const double thr = __dmul_rn(a.eps_theta_next, (double)a.deg[v]);
        const real nv = radd<real>(old, w);
        if ((double)old < thr && (double)nv >= thr) append_u32(&a.ctl->cand_out, a.cand_out, v, a.cap, &a.ctl->overflow);
    } else {
        RPair<real> *p = a.rp + v;
        const real old = atomicAdd(&p->r, w);
        const real thr = p->thr;
        const real nv = radd<real>(old, w);
        if (old < thr && nv >= thr) append_u32(&a.ctl->cand_out, a.cand_out, v, a.cap, &a.ctl->overflow);
    }
}

template <typename real, int KIND>
__global__ void __launch_bounds__(kThreads) k_push(PushArgs<real> a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long hp = a.ctl->hub_packed;
    const int64_t H = (int64_t)(hp >> kHubVolBits);
    const int64_t VH = (int64_t)(hp & kHubVolMask);

    // hubs: the concatenated hub adjacency is cut into equal chunks (merge-path), one warp
    // per chunk; consecutive lanes read consecutive columns
    if (VH > 0) {
        const int64_t nchunks = (VH + a.chunk - 1) / a.chunk;
        for (int64_t c = gw; c < nchunks; c += nw) {
            const int64_t e0 = c * a.chunk;
            const int64_t e1 = min(e0 + (int64_t)a.chunk, VH);
            int64_t lo = 0, hi = H;  // last h with vstart[h] <= e0
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (a.hub_vstart[mid] <= e0) lo = mid; else hi = mid;
            }
            int64_t h = lo;
            int64_t hs = a.hub_vstart[h];
            int64_t he = hs + a.b_deg[2][h];
            int64_t hb = a.b_beg[2][h];
            real hw = a.b_w[2][h];
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                while (e >= he) {
                    ++h;
                    hs = a.hub_vstart[h];
                    he = hs + a.b_deg[2][h];
                    hb = a.b_beg[2][h];
                    hw = a.b_w[2][h];
                }
                scatter<real, KIND>(a, a.col[hb + (e - hs)], hw);
            }
        }
    }
    // medium degrees: one warp per node
    const unsigned nmed = a.ctl->cnt_med;
    for (int64_t i = gw; i < nmed; i += nw) {
        const int64_t b = a.b_beg[1][i];
        const int32_t d = a.b_deg[1][i];
        const real w = a.b_w[1][i];
        for (int32_t k = lane; k < d; k += 32) scatter<real, KIND>(a, a.col[b + k], w);
    }
    // small degrees: one thread per node
    const unsigned nsm = a.ctl->cnt_small;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = a.b_beg[0][i];
        const int32_t d = a.b_deg[0][i];
        const real w = a.b_w[0][i];
        for (int32_t k = 0; k < d; k++) scatter<real, KIND>(a, a.col[b + k], w);
    }
}

// ------------------------------------------------------------------- output --

template <typename real>
__global__ void k_scale_copy(int64_t n, const real *__restrict__ x, real *__restrict__ dst,
                             double scale, int apply) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const real v = x[i];
        dst[i] = apply ? from_f64<real>(__dmul_rn(scale, (double)v)) : v;
    }
}

template <typename real>
__global__ void k_read_r_pairs(int64_t n, const RPair<real> *__restrict__ rp, real *__restrict__ dst,
                               const int32_t *__restrict__ deg, double gbeta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        // the generalised propagation's residual is kept scaled: r = y / S
        dst[i] = gbeta != 0.0 ? from_f64<real>(__ddiv_rn((double)rp[i].r, gppr_scale(deg[i], gbeta))) : rp[i].r;
}

// ---------------------------------------------------- deterministic scatter --
//
// Each round: the active ids are sorted, their edges are written out as (v, w_u) pairs in
// ascending u and CSR order, the pairs are sorted by v with a stable sort (so equal targets
// keep ascending u), and each target adds its run sequentially to the residual it had after
// the frontier phase.  That is the order of a sequential FP64 evaluation of Eq. (local-gd)
// that pushes S_t in ascending id, and the result does not depend on thread timing.

__global__ void k_det_degrees(int64_t na, const uint32_t *__restrict__ act, const int64_t *__restrict__ off,
                              int64_t *__restrict__ deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = act[i];
        deg[i] = off[u + 1] - off[u];
    }
}

template <typename real>
__global__ void k_det_expand(int64_t na, const uint32_t *__restrict__ act, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ col, const int64_t *__restrict__ vstart,
                             const real *__restrict__ wbuf, uint32_t *__restrict__ pkey, real *__restrict__ pval) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < na; i += nw) {
        const uint32_t u = act[i];
        const int64_t b = off[u], d = off[u + 1] - b, s = vstart[i];
        const real w = wbuf[u];
        for (int64_t k = lane; k < d; k += 32) {
            pkey[s + k] = (uint32_t)col[b + k];
            pval[s + k] = w;
        }
    }
}

// one thread per run of equal targets: sequential sum in pair order, then the threshold test
// on the run's start and end values (contributions are positive)
template <typename real, int KIND>
__global__ void k_det_apply(int64_t np, const uint32_t *__restrict__ pkey, const real *__restrict__ pval,
                            RPair<real> *rp, real *rnext, const int32_t *__restrict__ deg, double eps_theta_next,
                            int32_t *cand_out, int32_t *touched_out, Ctl *ctl, unsigned cap) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = pkey[p];
        if (p > 0 && pkey[p - 1] == v) continue;
        real r0, thr;
        double thr64 = 0.0;
        if (KIND == GDE_HK) {
            r0 = rnext[v];
            thr64 = __dmul_rn(eps_theta_next, (double)deg[v]);
        } else {
            r0 = rp[v].r;
            thr = rp[v].thr;
        }
        real r = r0;
        for (int64_t q = p; q < np && pkey[q] == v; q++) r = radd<real>(r, pval[q]);
        bool cross;
        if (KIND == GDE_HK) {
            rnext[v] = r;
            if (r0 == real(0) && r != real(0))
                append_u32(&ctl->touched_out, touched_out, (int32_t)v, cap, &ctl->overflow);
            cross = (double)r0 < thr64 && (double)r >= thr64;
        } else {
            rp[v].r = r;
            cross = r0 < thr && r >= thr;
        }
        if (cross) append_u32(&ctl->cand_out, cand_out, (int32_t)v, cap, &ctl->overflow);
    }
}

// ============================================================ host side =====

static unsigned grid_for(int64_t items, int64_t per_block = kThreads) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > kSMs * 64) b = kSMs * 64;
    return (unsigned)b;
}

DenseWork *dense_work_create(Graph &g, int precision) {
    DenseWork *w = new DenseWork();
    w->precision = precision;
    w->n = g.n;
    w->bins = g.bins;
    w->rsz = precision == GDE_FP64 ? 8 : 4;
    const int64_t n = g.n > 0 ? g.n : 1;
    try {
        w->x = dmalloc(w->rsz * n, "x");
        w->rp = dmalloc(2 * w->rsz * n, "residual");
        for (int k = 0; k < 2; k++) w->cand[k] = (int32_t *)dmalloc(4 * n, "candidates");
        w->active = (int32_t *)dmalloc(4 * n, "active set");
        for (int b = 0; b < 3; b++) {
            w->b_beg[b] = (int64_t *)dmalloc(8 * n, "bins");
            w->b_deg[b] = (int32_t *)dmalloc(4 * n, "bins");
            w->b_w[b] = dmalloc(w->rsz * n, "bins");
        }
        w->hub_vstart = (int64_t *)dmalloc(8 * n, "hub offsets");
        w->ctl = (Ctl *)dmalloc(sizeof(Ctl), "counters");
        w->xsrc = (double *)dmalloc(sizeof(double), "source entry");
        GDE_CUDA(cudaMallocHost((void **)&w->hctl, sizeof(Ctl)));
    } catch (...) {
        dense_work_destroy(w);
        throw;
    }
    return w;
}

static void ensure_det(DenseWork *w, Graph &g) {
    if (w->wbuf) return;
    const int64_t n = w->n > 0 ? w->n : 1;
    w->pair_cap = g.nnz > 0 ? g.nnz : 1;
    w->wbuf = dmalloc(w->rsz * n, "deterministic shares");
    w->sact[0] = (uint32_t *)dmalloc(4 * n, "sorted active");
    w->vdeg = (int64_t *)dmalloc(8 * n, "active degrees");
    w->vstart = (int64_t *)dmalloc(8 * n, "active edge starts");
    for (int k = 0; k < 2; k++) {
        w->pkey[k] = (uint32_t *)dmalloc(4 * (size_t)w->pair_cap, "pair targets");
        w->pval[k] = dmalloc(w->rsz * (size_t)w->pair_cap, "pair shares");
    }
    const int64_t big = w->pair_cap > n ? w->pair_cap : n;
    size_t sb = sort_scratch_bytes(big), cb = scan_scratch_bytes(n);
    w->dscratch = dmalloc(sb > cb ? sb : cb, "sort scratch");
    w->dtotal = (int64_t *)dmalloc(sizeof(int64_t), "pair count");
    GDE_CUDA(cudaMallocHost((void **)&w->htotal, sizeof(int64_t)));
}

static void ensure_layers(DenseWork *w) {
    if (w->rl[0]) return;
    const int64_t n = w->n > 0 ? w->n : 1;
    for (int k = 0; k < 2; k++) {
        w->rl[k] = dmalloc(w->rsz * n, "layers");
        w->touched[k] = (int32_t *)dmalloc(4 * n, "touched");
    }
}

void dense_work_destroy(DenseWork *w) {
    if (!w) return;
    dfree(w->x);
    dfree(w->rp);
    for (int k = 0; k < 2; k++) {
        dfree(w->rl[k]);
        dfree(w->cand[k]);
        dfree(w->touched[k]);
    }
    dfree(w->active);
    for (int b = 0; b < 3; b++) {
        dfree(w->b_beg[b]);
        dfree(w->b_deg[b]);
        dfree(w->b_w[b]);
    }
    dfree(w->hub_vstart);
    dfree(w->ctl);
    dfree(w->xsrc);
    dfree(w->wbuf);
    for (int k = 0; k < 2; k++) { dfree(w->sact[k]); dfree(w->pkey[k]); dfree(w->pval[k]); }
    dfree(w->vdeg); dfree(w->vstart); dfree(w->dscratch); dfree(w->dtotal);
    if (w->htotal) cudaFreeHost(w->htotal);
    if (w->hctl) cudaFreeHost(w->hctl);
    delete w;
}

__global__ void k_set_source(double *xsrc) { *xsrc = -1.0; }

// the output's source entry f_Katz,s = x_s - 1, from the FP64 source word
template <typename real>
__global__ void k_patch_source(real *dst, int32_t seed, const double *xsrc) {
    dst[seed] = from_f64<real>(*xsrc);
}

template <typename real>
static void begin_impl(Graph &g, DenseWork *w, const SolveParams &p, int32_t seed) {
    const unsigned grid = grid_for(g.n);
    if (layered(p.kind)) {
        ensure_layers(w);
        k_init_layers<real><<<grid, kThreads, 0, p.stream>>>(g.n, (real *)w->x, (real *)w->rl[0],
                                                             (real *)w->rl[1], seed);
        GDE_CUDA(cudaGetLastError());
    g.prof.launched();
        k_prep<<<1, 32, 0, p.stream>>>(w->ctl, w->cand[0], w->touched[0], seed);
        g.prof.launched();
    } else {
        k_init_pairs<real><<<grid, kThreads, 0, p.stream>>>(g.n, g.deg, (real *)w->x,
                                                            (RPair<real> *)w->rp, p.eps, seed, p.gbeta);
        GDE_CUDA(cudaGetLastError());
    g.prof.launched();
        k_prep<<<1, 32, 0, p.stream>>>(w->ctl, w->cand[0], nullptr, seed);
        g.prof.launched();
    }
    GDE_CUDA(cudaGetLastError());
    w->seed = seed;
    if (p.kind == GDE_KATZ) {
        k_set_source<<<1, 1, 0, p.stream>>>(w->xsrc);
        GDE_CUDA(cudaGetLastError());
        g.prof.launched();
    }
    w->kind = p.kind;
    w->t = 0;
    w->ncand = 1;
    w->ntouched[0] = layered(p.kind) ? 1 : 0;
    w->ntouched[1] = 0;
    w->last_active = 0;
    w->done = false;
}

void dense_begin(Graph &g, DenseWork *w, const SolveParams &p, int32_t seed) {
    if (p.precision == GDE_FP64) begin_impl<double>(g, w, p, seed);
    else begin_impl<float>(g, w, p, seed);
}

template <typename real, int KIND>
static int64_t round_impl(Graph &g, DenseWork *w, const SolveParams &p, RoundInfo *info) {
    const int64_t t = w->t;
    const int cur = (int)(t & 1), nxt = cur ^ 1;
    const bool last_layer = KIND == GDE_HK && t >= p.hk_N;
    k_prep<<<1, 32, 0, p.stream>>>(w->ctl, nullptr, nullptr, 0);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();

    FrontierArgs<real> fa{};
    fa.off = g.off;
    fa.cand = w->cand[cur];
    fa.ncand = w->ncand;
    fa.x = (real *)w->x;
    fa.rp = (RPair<real> *)w->rp;
    fa.rcur = KIND == GDE_HK ? (real *)w->rl[cur] : nullptr;
    fa.propagate = last_layer ? 0 : 1;
    if (KIND == GDE_PPR) { fa.cx = p.param; fa.coef = 1.0 - p.param; fa.gbeta = p.gbeta; }
    else if (KIND == GDE_KATZ) { fa.cx = 1.0; fa.coef = p.param; fa.xsrc = w->xsrc; fa.seed = w->seed; }
    else {
        fa.cx = 1.0;
        fa.coef = layer_ratio(p, t);
        fa.eps_theta = layer_theta(p, t) * p.eps;
        fa.clear_list = w->touched[nxt];
        fa.nclear = t > 0 ? w->ntouched[nxt] : 0;
        fa.rclear = (real *)w->rl[nxt];
    }
    fa.t1 = w->bins.t1;
    fa.t2 = w->bins.t2;
    for (int b = 0; b < 3; b++) { fa.b_beg[b] = w->b_beg[b]; fa.b_deg[b] = w->b_deg[b]; fa.b_w[b] = (real *)w->b_w[b]; }
    fa.hub_vstart = w->hub_vstart;
    fa.active = w->active;
    fa.ctl = w->ctl;
    if (p.deterministic) {
        ensure_det(w, g);
        fa.wbuf = (real *)w->wbuf;
    }
    fa.cap = (unsigned)(g.n > 0 ? g.n : 1);
    const int64_t fitems = w->ncand > fa.nclear ? (int64_t)w->ncand : (int64_t)fa.nclear;
    const int pf = g.prof.start(kProfDenseFrontier, p.stream);
    k_frontier<real, KIND><<<grid_for(fitems), kThreads, 0, p.stream>>>(fa);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
    g.prof.stop(pf, p.stream);

    if (!last_layer && p.deterministic) {
        // S_t is known only on the device: read its size, then sort, expand, sort, apply
        GDE_CUDA(cudaMemcpyAsync(w->hctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p.stream));
        GDE_CUDA(cudaStreamSynchronize(p.stream));
        GDE_REQUIRE(w->hctl->overflow == 0, GDE_ECUDA, "internal list overflow in a LocalGD round");
        const int64_t na = w->hctl->n_active;
        int key_bits = 1;
        while (((int64_t)1 << key_bits) < g.n) key_bits++;
        if (na > 0) {
            uint32_t *act = (uint32_t *)w->active;
            const int r1 = radix_sort<uint32_t>(act, nullptr, w->sact[0], nullptr, na, key_bits, w->dscratch, p.stream);
            const uint32_t *sorted = r1 ? w->sact[0] : act;
            k_det_degrees<<<grid_for(na), kThreads, 0, p.stream>>>(na, sorted, g.off, w->vdeg);
            GDE_CUDA(cudaGetLastError());
            exclusive_scan_i64(w->vdeg, w->vstart, na, w->dtotal, (int64_t *)w->dscratch, p.stream);
            GDE_CUDA(cudaMemcpyAsync(w->htotal, w->dtotal, sizeof(int64_t), cudaMemcpyDeviceToHost, p.stream));
            GDE_CUDA(cudaStreamSynchronize(p.stream));
            const int64_t np = *w->htotal;
            GDE_REQUIRE(np >= 0 && np <= w->pair_cap, GDE_ECUDA, "deterministic scatter: pair count out of range");
            if (np > 0) {
                k_det_expand<real><<<grid_for(na * 32), kThreads, 0, p.stream>>>(
                    na, sorted, g.off, g.col, w->vstart, (const real *)w->wbuf, w->pkey[0], (real *)w->pval[0]);
                GDE_CUDA(cudaGetLastError());
                const int r2 = radix_sort<real>(w->pkey[0], (real *)w->pval[0], w->pkey[1], (real *)w->pval[1],
                                                np, key_bits, w->dscratch, p.stream);
                const uint32_t *pk = w->pkey[r2];
                const real *pv = (const real *)w->pval[r2];
                double etn = 0.0;
                if (KIND == GDE_HK) etn = layer_theta(p, t + 1) * p.eps;
                k_det_apply<real, KIND><<<grid_for(np), kThreads, 0, p.stream>>>(
                    np, pk, pv, (RPair<real> *)w->rp, KIND == GDE_HK ? (real *)w->rl[nxt] : nullptr, g.deg, etn,
                    w->cand[nxt], KIND == GDE_HK ? w->touched[nxt] : nullptr, w->ctl, (unsigned)(g.n > 0 ? g.n : 1));
                GDE_CUDA(cudaGetLastError());
                g.prof.launched(2 * ((key_bits + 3) / 4) * 5 + 4);
            }
        }
    } else if (!last_layer) {
        PushArgs<real> pa{};
        pa.col = g.col;
        pa.deg = g.deg;
        for (int b = 0; b < 3; b++) { pa.b_beg[b] = w->b_beg[b]; pa.b_deg[b] = w->b_deg[b]; pa.b_w[b] = (const real *)w->b_w[b]; }
        pa.hub_vstart = w->hub_vstart;
        pa.rp = (RPair<real> *)w->rp;
        if (KIND == GDE_HK) {
            pa.rnext = (real *)w->rl[nxt];
            pa.eps_theta_next = layer_theta(p, t + 1) * p.eps;
            pa.touched_out = w->touched[nxt];
        }
        pa.cand_out = w->cand[nxt];
        pa.ctl = w->ctl;
        pa.chunk = w->bins.chunk;
        pa.cap = (unsigned)(g.n > 0 ? g.n : 1);
        // the round's volume is only known on the device: a fixed grid of 4 blocks per SM
        // walks the three bins with grid-stride loops
        const int pp = g.prof.start(kProfDensePush, p.stream);
        k_push<real, KIND><<<kSMs * 4, kThreads, 0, p.stream>>>(pa);
        GDE_CUDA(cudaGetLastError());
    g.prof.launched();
        g.prof.stop(pp, p.stream);
    }
    GDE_CUDA(cudaMemcpyAsync(w->hctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, p.stream));
    GDE_CUDA(cudaStreamSynchronize(p.stream));
    const Ctl &h = *w->hctl;
    GDE_REQUIRE(h.overflow == 0, GDE_ECUDA, "internal list overflow in a LocalGD round");
    if (info) {
        info->n_active = h.n_active;
        info->vol = (int64_t)h.vol;
        info->rS_l1 = h.rS_l1;
        info->scat = h.scat;
        info->retired = h.retired;
    }
    if (g.prof.enabled) {
        g.prof.counters.dense_rounds += 1;
        g.prof.counters.edges += (int64_t)h.vol;
        g.prof.counters.pushes += h.n_active;
    }
    w->last_active = h.n_active;
    w->ncand = last_layer ? 0 : h.cand_out;
    if (KIND == GDE_HK) w->ntouched[nxt] = last_layer ? 0 : h.touched_out;
    w->t = t + 1;
    if (h.n_active == 0) w->done = true;
    return h.n_active;
}

int64_t dense_round(Graph &g, DenseWork *w, const SolveParams &p, RoundInfo *info) {
    if (info) *info = RoundInfo{0, 0, 0.0, 0.0, 0.0};
    if (w->done || w->ncand == 0 || (layered(p.kind) && w->t > p.hk_N)) {
        w->done = true;
        w->last_active = 0;
        return 0;
    }
    if (p.precision == GDE_FP64) {
        if (p.kind == GDE_PPR || p.kind == GDE_GPPR) return round_impl<double, GDE_PPR>(g, w, p, info);
        if (p.kind == GDE_KATZ) return round_impl<double, GDE_KATZ>(g, w, p, info);
        return round_impl<double, GDE_HK>(g, w, p, info);
    }
    if (p.kind == GDE_PPR || p.kind == GDE_GPPR) return round_impl<float, GDE_PPR>(g, w, p, info);
    if (p.kind == GDE_KATZ) return round_impl<float, GDE_KATZ>(g, w, p, info);
    return round_impl<float, GDE_HK>(g, w, p, info);
}

int64_t dense_round_index(const DenseWork *w) { return w->t; }

bool dense_pending(const DenseWork *w) { return !w->done && w->ncand > 0; }

void *dense_x(DenseWork *w) { return w->x; }

void dense_read(Graph &g, DenseWork *w, const SolveParams &p, void *x, void *r, int32_t *active,
                int64_t *n_active, bool device_ptrs) {
    const size_t bytes = w->rsz * (size_t)g.n;
    const cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x && g.n) GDE_CUDA(cudaMemcpyAsync(x, w->x, bytes, k, p.stream));
    if (x && g.n && p.kind == GDE_KATZ && p.katz_minus_source) {
        // x - e_s: the source entry from the FP64 source word
        if (device_ptrs) {
            if (p.precision == GDE_FP64)
                k_patch_source<double><<<1, 1, 0, p.stream>>>((double *)x, w->seed, w->xsrc);
            else
                k_patch_source<float><<<1, 1, 0, p.stream>>>((float *)x, w->seed, w->xsrc);
            GDE_CUDA(cudaGetLastError());
        } else {
            double v = 0.0;
            GDE_CUDA(cudaMemcpyAsync(&v, w->xsrc, sizeof v, cudaMemcpyDeviceToHost, p.stream));
            GDE_CUDA(cudaStreamSynchronize(p.stream));
            if (p.precision == GDE_FP64) ((double *)x)[w->seed] = v;
            else ((float *)x)[w->seed] = (float)v;
        }
    }
    if (r && g.n) {
        if (layered(p.kind)) {
            // after round t-1 the current layer is t
            const int cur = (int)(w->t & 1);
            GDE_CUDA(cudaMemcpyAsync(r, w->rl[cur], bytes, k, p.stream));
        } else {
            void *tmp = dmalloc(bytes, "read buffer");
            try {
                if (p.precision == GDE_FP64)
                    k_read_r_pairs<double><<<grid_for(g.n), kThreads, 0, p.stream>>>(
                        g.n, (const RPair<double> *)w->rp, (double *)tmp, g.deg, p.gbeta);
                else
                    k_read_r_pairs<float><<<grid_for(g.n), kThreads, 0, p.stream>>>(
                        g.n, (const RPair<float> *)w->rp, (float *)tmp, g.deg, p.gbeta);
                GDE_CUDA(cudaGetLastError());
                GDE_CUDA(cudaMemcpyAsync(r, tmp, bytes, k, p.stream));
                GDE_CUDA(cudaStreamSynchronize(p.stream));
            } catch (...) {
                dfree(tmp);
                throw;
            }
            dfree(tmp);
        }
    }
    if (active && w->last_active > 0)
        GDE_CUDA(cudaMemcpyAsync(active, w->active, 4 * (size_t)w->last_active, k, p.stream));
    if (n_active) *n_active = w->last_active;
    GDE_CUDA(cudaStreamSynchronize(p.stream));
}

void dense_output(Graph &g, DenseWork *w, const SolveParams &p, void *dst_dev) {
    const bool apply = layered(p.kind);
    const double scale = p.kind == GDE_SERIES ? p.series[0] : (apply ? std::exp(-p.param) : 1.0);
    if (p.precision == GDE_FP64)
        k_scale_copy<double><<<grid_for(g.n), kThreads, 0, p.stream>>>(g.n, (const double *)w->x,
                                                                       (double *)dst_dev, scale, apply);
    else
        k_scale_copy<float><<<grid_for(g.n), kThreads, 0, p.stream>>>(g.n, (const float *)w->x,
                                                                      (float *)dst_dev, scale, apply);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
    if (p.kind == GDE_KATZ && p.katz_minus_source) {
        if (p.precision == GDE_FP64)
            k_patch_source<double><<<1, 1, 0, p.stream>>>((double *)dst_dev, w->seed, w->xsrc);
        else
            k_patch_source<float><<<1, 1, 0, p.stream>>>((float *)dst_dev, w->seed, w->xsrc);
        GDE_CUDA(cudaGetLastError());
        g.prof.launched();
    }
}

}  // namespace gde
