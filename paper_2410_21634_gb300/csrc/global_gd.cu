// Standard (global) gradient descent, the counterpart LocalGD is compared with in Section 5
// (Table 2's operation ratio, Figure 6's running times): every iteration updates every node,
// x <- x + c r and r <- M r (PPR: c = alpha, M = (1-alpha) A D^-1; Katz: c = 1, M = beta A),
// until ||D^-1 r||_inf < eps (degree-0 nodes read as degree 1).  M r is a pull SpMV over the
// whole CSR: the graphs are undirected, so row v lists exactly the u with v in N(u), and
// r_v = sum over row v of the neighbours' shares.  Rows up to kGdBlockRow entries are summed
// by 8-lane groups, longer rows by a whole block.  Each iteration is three launches (the
// max, the update, the SpMV); a done flag set on the device turns the rest of a batch of
// iterations into no-ops, so the host checks for convergence once per batch.
#include <vector>

#include "common.cuh"

namespace gde {

constexpr int kGdBatch = 8;         // iterations queued between convergence checks
constexpr int kGdLanes = 8;         // lanes per row in the SpMV
constexpr int kGdBlockRow = 4096;   // rows longer than this get a block each

struct GdCtl {
    unsigned long long qmax;  // bits of max_u |r_u| / max(d_u, 1) (nonnegative doubles order as integers)
    unsigned done;
    unsigned pad;
    long long iters;
};

template <typename real>
__global__ void k_gd_init(int64_t n, real *x, real *r, int32_t seed, GdCtl *ctl) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = real(0);
        r[i] = i == seed ? real(1) : real(0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->qmax = 0ull;
        ctl->done = 0u;
        ctl->iters = 0;
    }
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k_gd_max(int64_t n, const real *r, const int32_t *deg, GdCtl *ctl) {
    if (ctl->done) return;
    double q = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[i];
        const double v = __ddiv_rn(fabs((double)r[i]), (double)(d > 0 ? d : 1));
        q = v > q ? v : q;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, q, o);
        q = y > q ? y : q;
    }
    __shared__ double s[kThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; w++) q = s[w] > q ? s[w] : q;
        atomicMax(&ctl->qmax, (unsigned long long)__double_as_longlong(q));
    }
}

// stop test, then x += c r and the share w of every node; the max is reset for the next test
template <typename real>
__global__ void k_gd_update(int64_t n, real *x, const real *r, real *w, const int32_t *deg, double cx,
                            double coef, int divide, double eps, GdCtl *ctl) {
    if (ctl->done) return;
    const double qmax = __longlong_as_double((long long)ctl->qmax);
    if (qmax < eps) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->done = 1u;
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double rho = (double)r[i];
        x[i] = radd<real>(x[i], from_f64<real>(__dmul_rn(cx, rho)));
        const int32_t d = deg[i];
        double share = 0.0;
        if (d > 0) share = divide ? __ddiv_rn(__dmul_rn(coef, rho), (double)d) : __dmul_rn(coef, rho);
        w[i] = from_f64<real>(share);
    }
}

// the update reads qmax in every block, so its reset waits for the next launch
__global__ void k_gd_tick(GdCtl *ctl) {
    if (ctl->done) return;
    ctl->qmax = 0ull;
    ctl->iters += 1;
}

// r_next[v] = sum of w over row v: 8-lane groups for short rows (long rows are skipped here)
template <typename real>
__global__ void __launch_bounds__(kThreads) k_gd_spmv(int64_t n, const int64_t *off, const int32_t *col, const real *w,
                                                      real *rn, const GdCtl *ctl) {
    if (ctl->done) return;
    const int lane = threadIdx.x & (kGdLanes - 1);
    const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kGdLanes;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / kGdLanes;
    const unsigned gmask = ((1u << kGdLanes) - 1u) << ((threadIdx.x & 31) & ~(kGdLanes - 1));
    for (int64_t v = g0; v < n; v += ng) {
        const int64_t b = off[v], e = off[v + 1];
        if (e - b > kGdBlockRow) continue;  // a block row
        double acc = 0.0;
        for (int64_t k = b + lane; k < e; k += kGdLanes) acc = __dadd_rn(acc, (double)w[col[k]]);
        for (int o = kGdLanes / 2; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(gmask, acc, o, kGdLanes));
        if (lane == 0) rn[v] = from_f64<real>(acc);
    }
}

// one block per long row
template <typename real>
__global__ void __launch_bounds__(kThreads) k_gd_spmv_long(const int32_t *rows, const int64_t *off, const int32_t *col,
                                                           const real *w, real *rn, const GdCtl *ctl) {
    if (ctl->done) return;
    const int32_t v = rows[blockIdx.x];
    const int64_t b = off[v], e = off[v + 1];
    double acc = 0.0;
    for (int64_t k = b + threadIdx.x; k < e; k += kThreads) acc = __dadd_rn(acc, (double)w[col[k]]);
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, o));
    __shared__ double s[kThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; i++) t = __dadd_rn(t, s[i]);
        rn[v] = from_f64<real>(t);
    }
}

__global__ void k_gd_long_rows(int64_t n, const int32_t *deg, int32_t *rows, unsigned *count) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (deg[v] > kGdBlockRow) rows[atomicAdd(count, 1u)] = (int32_t)v;
}

template <typename real>
static void gd_impl(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st) {
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
        real *x = (real *)alloc(nb, "gd x");
        real *r = (real *)alloc(nb, "gd r");
        real *rn = (real *)alloc(nb, "gd r");
        real *w = (real *)alloc(nb, "gd shares");
        GdCtl *ctl = (GdCtl *)alloc(sizeof(GdCtl), "gd control");
        int32_t *rows = (int32_t *)alloc(4 * (size_t)(n > 0 ? n : 1), "gd long rows");
        unsigned *cnt = (unsigned *)alloc(sizeof(unsigned), "gd long rows");
        GDE_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
        const unsigned grid = kSMs * 8;
        k_gd_long_rows<<<grid, kThreads, 0, s>>>(n, g.deg, rows, cnt);
        GDE_CUDA(cudaGetLastError());
        unsigned nlong = 0;
        GDE_CUDA(cudaMemcpyAsync(&nlong, cnt, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        k_gd_init<real><<<grid, kThreads, 0, s>>>(n, x, r, seed, ctl);
        GDE_CUDA(cudaGetLastError());
        GDE_CUDA(cudaStreamSynchronize(s));
        const bool ppr = p.kind == GDE_PPR;
        const double cx = ppr ? p.param : 1.0, coef = ppr ? 1.0 - p.param : p.param;
        GdCtl h{};
        int64_t launched = 2;
        for (int64_t it = 0; it < p.max_rounds; it += kGdBatch) {
            for (int b = 0; b < kGdBatch && it + b < p.max_rounds; b++) {
                k_gd_max<real><<<grid, kThreads, 0, s>>>(n, r, g.deg, ctl);
                k_gd_update<real><<<grid, kThreads, 0, s>>>(n, x, r, w, g.deg, cx, coef, ppr ? 1 : 0, p.eps, ctl);
                k_gd_tick<<<1, 1, 0, s>>>(ctl);
                k_gd_spmv<real><<<grid, kThreads, 0, s>>>(n, g.off, g.col, w, rn, ctl);
                if (nlong) k_gd_spmv_long<real><<<nlong, kThreads, 0, s>>>(rows, g.off, g.col, w, rn, ctl);
                GDE_CUDA(cudaGetLastError());
                launched += nlong ? 5 : 4;
                std::swap(r, rn);
            }
            GDE_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(GdCtl), cudaMemcpyDeviceToHost, s));
            GDE_CUDA(cudaStreamSynchronize(s));
            if (h.done) break;
        }
        g.prof.launched((int)launched);
        // the converged x; r is not reported (its buffer depends on where the batch stopped)
        const cudaMemcpyKind k = x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        GDE_CUDA(cudaMemcpyAsync(x_out, x, nb, k, s));
        GDE_CUDA(cudaStreamSynchronize(s));
        if (st) {
            *st = gde_stats{};
            st->rounds = h.iters;
            st->active_volume = h.iters * g.nnz;  // the standard algorithm touches every edge
            st->pushes = h.iters * n;
            st->resid_l1 = -1.0;
            st->mass_l1 = -1.0;
            st->status = h.done ? GDE_OK : GDE_ENOTCONV;
        }
    } catch (...) {
        for (void *q : tmp) dfree(q);
        throw;
    }
    for (void *q : tmp) dfree(q);
}

void global_gd_solve(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st) {
    GDE_REQUIRE(p.kind == GDE_PPR || p.kind == GDE_KATZ, GDE_EINVAL, "global GD serves PPR and Katz");
    if (p.precision == GDE_FP64) gd_impl<double>(g, p, seed, x_out, x_dev, st);
    else gd_impl<float>(g, p, seed, x_out, x_dev, st);
}

}  // namespace gde
