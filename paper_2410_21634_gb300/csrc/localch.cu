// LocalCH for PPR: Section 3.3's local Chebyshev method (its PPR updates in the appendix on
// implementation details), one seed at a time with dense state.  Chebyshev on
// Q = I - (1-alpha) D^-1/2 A D^-1/2 (eigenvalues in [alpha, 2 - alpha]) in the unit-mass
// variables of LocalGD: delta_1 = 1 - alpha, delta_{t+1} = 1/(2/(1-alpha) - delta_t); round 0
// pushes the seed as LocalGD does; round t >= 1, for u in S_t = { u : r_u != 0, |r_u| >= eps d_u }
// (snapshot rho = r_u before any scatter):
//   xh_u = (2 delta_{t+1}/(1-alpha)) alpha rho_u + delta_t delta_{t+1} (x^t - x^{t-1})_u,
//   x_u += xh_u, r_u = rho_u - xh_u/alpha, r_v += ((1-alpha) xh_u/alpha)/d_u for v in N(u).
// Residuals change sign and a pushed node keeps a residual, so the next round's candidates
// are S_t plus every node whose |r| crossed its threshold in the scatter; a per-node round
// stamp drops repeated candidates.
#include <vector>

#include "common.cuh"

namespace gde {

struct ChCtl {
    unsigned n_active;   // |S_t|
    unsigned n_next;     // candidates of the next round
    unsigned overflow;
    unsigned pad;
    unsigned long long vol;
};

template <typename real>
__global__ void k_ch_init(int64_t n, real *x, real *r, real *dx, real *dxn, int32_t *stamp, int32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = real(0);
        r[i] = i == seed ? real(1) : real(0);
        dx[i] = real(0);
        dxn[i] = real(0);
        stamp[i] = 0;
    }
}

__device__ __forceinline__ void ch_append(unsigned *count, int32_t *list, int32_t v, unsigned cap, unsigned *overflow) {
    const unsigned i = atomicAdd(count, 1u);
    if (i < cap) list[i] = v; else atomicOr(overflow, 1u);
}

struct ChArgs {
    const int64_t *off;
    const int32_t *cand;
    unsigned ncand;
    int32_t *stamp;
    int32_t round_tag;   // t + 1
    double eps, alpha, g1, g2;
    int first;           // round 0: xh = alpha rho
    int32_t *active;     // S_t
    int32_t *next;       // candidates of t + 1
    unsigned cap;
    ChCtl *ctl;
};

template <typename real>
__global__ void __launch_bounds__(kThreads) k_ch_frontier(ChArgs a, real *x, real *r, const real *dx, real *dxn,
                                                          real *w) {
    for (int64_t ci = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ci < a.ncand; ci += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = a.cand[ci];
        if (atomicExch(a.stamp + u, a.round_tag) == a.round_tag) continue;  // listed twice
        const int32_t d = (int32_t)(a.off[u + 1] - a.off[u]);
        const double rho = (double)r[u];
        const double thr = __dmul_rn(a.eps, (double)d);
        if (!(rho != 0.0 && fabs(rho) >= thr)) continue;
        const double xh = a.first ? __dmul_rn(a.alpha, rho)
                                  : __dadd_rn(__dmul_rn(a.g1, __dmul_rn(a.alpha, rho)), __dmul_rn(a.g2, (double)dx[u]));
        x[u] = radd<real>(x[u], from_f64<real>(xh));
        r[u] = from_f64<real>(__dsub_rn(rho, __ddiv_rn(xh, a.alpha)));
        dxn[u] = from_f64<real>(xh);
        const double share = d > 0 ? __ddiv_rn(__dmul_rn(1.0 - a.alpha, __ddiv_rn(xh, a.alpha)), (double)d) : 0.0;
        w[u] = from_f64<real>(share);
        ch_append(&a.ctl->n_active, a.active, u, a.cap, &a.ctl->overflow);
        ch_append(&a.ctl->n_next, a.next, u, a.cap, &a.ctl->overflow);  // its residual may still be active
        atomicAdd(&a.ctl->vol, (unsigned long long)d);
    }
}

// one warp per pushed node; a residual whose |r| crosses its threshold lists its node
template <typename real>
__global__ void __launch_bounds__(kThreads) k_ch_scatter(const int64_t *off, const int32_t *col, const int32_t *active,
                                                         const unsigned *n_active, const real *w, real *r, double eps,
                                                         int32_t *next, unsigned cap, ChCtl *ctl) {
    const unsigned na = *n_active;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < na; i += nw) {
        const int32_t u = active[i];
        const real wu = w[u];
        for (int64_t e = off[u] + lane; e < off[u + 1]; e += 32) {
            const int32_t v = col[e];
            const real old = atomicAdd(r + v, wu);
            const double thr = __dmul_rn(eps, (double)(off[v + 1] - off[v]));
            const double nv = (double)radd<real>(old, wu);
            if (fabs((double)old) < thr && fabs(nv) >= thr) ch_append(&ctl->n_next, next, v, cap, &ctl->overflow);
        }
    }
}

template <typename real>
__global__ void k_ch_clear(const int32_t *list, unsigned n, real *dxn) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dxn[list[i]] = real(0);
}

template <typename real>
static void ch_impl(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st) {
    const int64_t n = g.n;
    cudaStream_t s = p.stream;
    std::vector<void *> tmp;
    auto alloc = [&](size_t bytes, const char *what) {
        void *q = dmalloc(bytes, what);
        tmp.push_back(q);
        return q;
    };
    try {
        const size_t nb = sizeof(real) * (size_t)(n > 0 ? n : 1);
        const unsigned cap = (unsigned)(2 * (n > 0 ? n : 1) + 1024);
        real *x = (real *)alloc(nb, "localch x");
        real *r = (real *)alloc(nb, "localch r");
        real *dx = (real *)alloc(nb, "localch momentum");
        real *dxn = (real *)alloc(nb, "localch momentum");
        real *w = (real *)alloc(nb, "localch shares");
        int32_t *stamp = (int32_t *)alloc(4 * (size_t)(n > 0 ? n : 1), "localch stamps");
        int32_t *cand[2] = {(int32_t *)alloc(4 * (size_t)cap, "localch candidates"),
                            (int32_t *)alloc(4 * (size_t)cap, "localch candidates")};
        int32_t *act[2] = {(int32_t *)alloc(4 * (size_t)cap, "localch active"),
                           (int32_t *)alloc(4 * (size_t)cap, "localch active")};
        ChCtl *ctl = (ChCtl *)alloc(sizeof(ChCtl), "localch control");
        const unsigned grid = kSMs * 8;
        k_ch_init<real><<<grid, kThreads, 0, s>>>(n, x, r, dx, dxn, stamp, seed);
        GDE_CUDA(cudaGetLastError());
        GDE_CUDA(cudaMemcpyAsync(cand[0], &seed, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const double alpha = p.param, c = 1.0 - alpha;
        double delta = c;  // delta_1
        unsigned ncand = 1, prev_active = 0;
        int64_t t = 0, vol = 0, pushes = 0, launched = 1;
        bool converged = false;
        for (; t < p.max_rounds; t++) {
            const int cur = (int)(t & 1);
            ChArgs a{};
            a.off = g.off; a.cand = cand[cur]; a.ncand = ncand; a.stamp = stamp; a.round_tag = (int32_t)(t + 1);
            a.eps = p.eps; a.alpha = alpha; a.first = t == 0 ? 1 : 0;
            double dnext = 0.0;
            if (t > 0) {
                dnext = 1.0 / (2.0 / c - delta);
                a.g1 = (2.0 * dnext) / c;
                a.g2 = delta * dnext;
            }
            a.active = act[cur]; a.next = cand[cur ^ 1]; a.cap = cap; a.ctl = ctl;
            GDE_CUDA(cudaMemsetAsync(ctl, 0, sizeof(ChCtl), s));
            k_ch_frontier<real><<<grid, kThreads, 0, s>>>(a, x, r, dx, dxn, w);
            k_ch_scatter<real><<<grid, kThreads, 0, s>>>(g.off, g.col, act[cur], &ctl->n_active, w, r, p.eps,
                                                         cand[cur ^ 1], cap, ctl);
            GDE_CUDA(cudaGetLastError());
            launched += 2;
            ChCtl h{};
            GDE_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(ChCtl), cudaMemcpyDeviceToHost, s));
            GDE_CUDA(cudaStreamSynchronize(s));
            if (h.overflow) {
                set_error("LocalCH: candidate list capacity exceeded");
                throw Fail{GDE_ENOMEM};
            }
            if (h.n_active == 0) { converged = true; break; }
            vol += (int64_t)h.vol;
            pushes += h.n_active;
            // momentum: dx <- this round's updates (on S_t), the old buffer cleared on S_{t-1}
            std::swap(dx, dxn);
            if (t > 0 && prev_active) {
                k_ch_clear<real><<<grid, kThreads, 0, s>>>(act[cur ^ 1], prev_active, dxn);
                GDE_CUDA(cudaGetLastError());
                launched++;
            }
            prev_active = h.n_active;
            ncand = h.n_next < cap ? h.n_next : cap;
            if (t > 0) delta = dnext;
        }
        g.prof.launched((int)launched);
        const cudaMemcpyKind k = x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        GDE_CUDA(cudaMemcpyAsync(x_out, x, nb, k, s));
        GDE_CUDA(cudaStreamSynchronize(s));
        if (st) {
            *st = gde_stats{};
            st->rounds = t;
            st->active_volume = vol;
            st->pushes = pushes;
            st->resid_l1 = -1.0;
            st->mass_l1 = -1.0;
            st->status = converged ? GDE_OK : GDE_ENOTCONV;
        }
    } catch (...) {
        for (void *q : tmp) dfree(q);
        throw;
    }
    for (void *q : tmp) dfree(q);
}

void localch_solve(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st) {
    GDE_REQUIRE(p.kind == GDE_PPR, GDE_EINVAL, "LocalCH serves PPR");
    if (p.precision == GDE_FP64) ch_impl<double>(g, p, seed, x_out, x_dev, st);
    else ch_impl<float>(g, p, seed, x_out, x_dev, st);
}

}  // namespace gde
