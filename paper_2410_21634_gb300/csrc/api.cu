// C ABI entry points (include/gde.h): argument checks, graph store lifetime, the
// single-seed solve loop and the stepping interface.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace gde {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

// Test fault injection (gde_test_fail_alloc): the n-th device allocation from the arming
// fails as cudaMalloc's out-of-memory would (0: disarmed).  Process-wide.
static std::atomic<long long> g_fail_alloc_in{0};

void *dmalloc(size_t bytes, const char *what) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) {
        char buf[256];
        snprintf(buf, sizeof(buf), "cudaMalloc(%zu bytes) for %s failed: injected allocation failure", bytes, what);
        set_error(buf);
        throw Fail{GDE_ENOMEM};
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free allocation error
        char buf[256];
        snprintf(buf, sizeof(buf), "cudaMalloc(%zu bytes) for %s failed: %s", bytes, what,
                 cudaGetErrorString(e));
        set_error(buf);
        throw Fail{e == cudaErrorMemoryAllocation ? GDE_ENOMEM : GDE_ECUDA};
    }
    return p;
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

// -------------------------------------------------------------- profiler --

int Profiler::start(int kind, cudaStream_t s) {
    if (!enabled) return -1;
    cudaEvent_t a, b;
    GDE_CUDA(cudaEventCreate(&a));
    GDE_CUDA(cudaEventCreate(&b));
    GDE_CUDA(cudaEventRecord(a, s));
    marks.push_back({kind, {a, b}});
    return (int)marks.size() - 1;
}

void Profiler::stop(int idx, cudaStream_t s) {
    if (idx < 0) return;
    GDE_CUDA(cudaEventRecord(marks[(size_t)idx].second.second, s));
}

void Profiler::reset() {
    for (auto &m : marks) {
        cudaEventDestroy(m.second.first);
        cudaEventDestroy(m.second.second);
    }
    marks.clear();
    counters = gde_profile{};
}

void Profiler::read(gde_profile *out) {
    gde_profile p = counters;
    for (auto &m : marks) {
        GDE_CUDA(cudaEventSynchronize(m.second.second));
        float ms = 0.0f;
        GDE_CUDA(cudaEventElapsedTime(&ms, m.second.first, m.second.second));
        switch (m.first) {
            case kProfBatchRounds: p.batch_rounds_ms += ms; break;
            case kProfBatchClear: p.batch_clear_ms += ms; break;
            case kProfBatchTopk: p.batch_topk_ms += ms; break;
            case kProfDenseFrontier: p.dense_frontier_ms += ms; break;
            case kProfDensePush: p.dense_push_ms += ms; break;
            default: break;
        }
    }
    *out = p;
}

// ----------------------------------------------------------- heat kernel --

// Smallest N with e^-tau sum_{k>N} tau^k/k! <= tol: the Poisson(tau) tail, summed from its
// small end (terms p_k = e^-tau tau^k/k! by the ratio p_{k+1} = p_k tau/(k+1)).
int64_t hk_terms(double tau, double tol) {
    const int64_t kmax = (int64_t)(10.0 * tau) + 200;
    std::vector<double> p((size_t)kmax + 2);
    p[0] = std::exp(-tau);
    for (int64_t k = 0; k < kmax; k++) p[k + 1] = p[k] * tau / (double)(k + 1);
    double tail = 0.0;
    int64_t best = kmax;
    for (int64_t N = kmax - 1; N >= 0; N--) {
        tail += p[N + 1];
        if (tail <= tol) best = N; else break;
    }
    return best;
}

// theta_t = e^tau / ((N+1) psi_t(tau)), psi_t = sum_{j=0}^{N-t} tau^j t!/(t+j)!  (mode 0);
// 1 (mode 1).  Weighting each layer's leftover residual by psi_t and splitting eps evenly over
// the N+1 layers bounds the error of e^-tau x by eps d_u.
double hk_theta(double tau, int64_t N, int64_t t, int mode) {
    if (mode == 1) return 1.0;
    double psi = 0.0, term = 1.0;
    for (int64_t j = 0; j <= N - t; j++) {
        if (j > 0) term = term * (tau / (double)(t + j));
        psi += term;
    }
    return std::exp(tau) / ((double)(N + 1) * psi);
}

// layered engine: the heat kernel's ratio tau/(t+1) and theta_t, or the series' c_{t+1}/c_t and
// 1/((N+1) c_0 psi_t) with psi_t = sum_{j<=N-t} c_{t+j}/c_t (mode 1: theta_t = 1)
double layer_ratio(const SolveParams &p, int64_t t) {
    if (p.kind != GDE_SERIES) return p.param / (double)(t + 1);
    return t < p.hk_N ? p.series[(size_t)t + 1] / p.series[(size_t)t] : 0.0;
}

double layer_theta(const SolveParams &p, int64_t t) {
    if (p.kind != GDE_SERIES) return hk_theta(p.param, p.hk_N, t, p.hk_mode);
    if (p.hk_mode == 1) return 1.0;
    if (t > p.hk_N) return 1.0;
    double psi = 0.0;
    for (int64_t j = 0; j <= p.hk_N - t; j++) psi += p.series[(size_t)(t + j)] / p.series[(size_t)t];
    return 1.0 / ((double)(p.hk_N + 1) * p.series[0] * psi);
}

// Table bytes of a batched solve: the caller's, else automatic.  Sparse tables probe
// shorter: PPR on R-MAT 24 with 1,024 seeds takes 46.3 ms at 16 GiB (1M slots a seed, load up
// to 0.62) and 41.5 ms at 32 GiB.  Katz from a hub and the first layers of the layered kinds
// touch several times the nodes of a PPR solve, so they get up to 64 GiB.  Half the free
// device memory at most, 16 GiB at least.
static int64_t batch_budget(int64_t requested, gde_kind kind) {
    if (requested > 0) return requested;
    size_t free_b = 0, total_b = 0;
    GDE_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const int64_t want = (layered(kind) || kind == GDE_KATZ) ? ((int64_t)64 << 30) : ((int64_t)32 << 30);
    int64_t b = std::min<int64_t>(want, (int64_t)(free_b / 2));
    if (b < ((int64_t)16 << 30)) b = (int64_t)16 << 30;
    return b;
}

static SolveParams make_params(Graph &g, gde_kind kind, double param, double eps,
                               const gde_solve_opts &o) {
    GDE_REQUIRE(kind == GDE_PPR || kind == GDE_KATZ || kind == GDE_HK || kind == GDE_GPPR ||
                    kind == GDE_SERIES, GDE_EINVAL, "unknown kind");
    GDE_REQUIRE(std::isfinite(param) && std::isfinite(eps), GDE_EINVAL, "param and eps must be finite");
    GDE_REQUIRE(eps > 0.0, GDE_EINVAL, "eps must be > 0");
    if (kind == GDE_PPR || kind == GDE_GPPR)
        GDE_REQUIRE(param > 0.0 && param < 1.0, GDE_EINVAL, "PPR alpha must be in (0,1)");
    if (kind == GDE_GPPR)
        GDE_REQUIRE(o.prop_beta >= 0.0 && o.prop_beta <= 1.0, GDE_EINVAL, "prop_beta must be in [0,1]");
    if (kind == GDE_KATZ) GDE_REQUIRE(param > 0.0, GDE_EINVAL, "Katz beta must be > 0");
    if (kind == GDE_HK) GDE_REQUIRE(param > 0.0 && param < 700.0, GDE_EINVAL, "HK tau must be in (0,700)");
    GDE_REQUIRE(o.precision == GDE_FP64 || o.precision == GDE_FP32, GDE_EINVAL, "bad precision");
    GDE_REQUIRE(o.hk_threshold == 0 || o.hk_threshold == 1, GDE_EINVAL, "bad hk_threshold");
    GDE_REQUIRE(o.max_rounds >= 0, GDE_EINVAL, "max_rounds must be >= 0");
    GDE_REQUIRE(o.topk >= 0, GDE_EINVAL, "topk must be >= 0");
    GDE_REQUIRE(o.hk_tol >= 0.0 && o.hk_tol < 1.0, GDE_EINVAL, "hk_tol must be in [0,1)");
    SolveParams p{};
    p.kind = kind;
    p.param = param;
    p.eps = eps;
    p.precision = o.precision;
    p.hk_mode = o.hk_threshold;
    p.hk_tol = o.hk_tol > 0.0 ? o.hk_tol : 1e-12;
    p.max_rounds = o.max_rounds > 0 ? o.max_rounds : 1000000;
    p.hk_N = kind == GDE_HK ? hk_terms(param, p.hk_tol) : 0;
    if (kind == GDE_SERIES) {
        GDE_REQUIRE(o.series_coef != nullptr && o.series_terms >= 1 && o.series_terms <= 1000000, GDE_EINVAL,
                    "a series needs 1 to 10^6 coefficients");
        p.series.assign(o.series_coef, o.series_coef + o.series_terms);
        for (double c : p.series)
            GDE_REQUIRE(std::isfinite(c) && c > 0.0, GDE_EINVAL, "series coefficients must be finite and > 0");
        p.hk_N = o.series_terms - 1;
    }
    GDE_REQUIRE(o.deterministic == 0 || o.deterministic == 1, GDE_EINVAL, "bad deterministic flag");
    p.deterministic = o.deterministic;
    p.stream = o.cuda_stream ? (cudaStream_t)o.cuda_stream : g.stream;
    p.gbeta = kind == GDE_GPPR ? o.prop_beta : 0.0;
    GDE_REQUIRE(o.katz_minus_source == 0 || (o.katz_minus_source == 1 && kind == GDE_KATZ), GDE_EINVAL,
                "katz_minus_source: 0, or 1 with GDE_KATZ");
    GDE_REQUIRE(!(o.katz_minus_source && (o.global_gd || o.chebyshev)), GDE_EINVAL,
                "katz_minus_source: LocalGD only (not global_gd)");
    p.katz_minus_source = o.katz_minus_source;
    return p;
}

static DenseWork *dense_for(Graph &g, int precision) {
    int k = precision == GDE_FP64 ? 0 : 1;
    if (!g.dense[k]) g.dense[k] = dense_work_create(g, precision);
    return g.dense[k];
}

static void tuning_from_bins(const Bins &b, gde_tuning *t) {
    t->t1 = b.t1;
    t->t2 = b.t2;
    t->chunk = b.chunk;
    t->blocks_per_sm = b.blocks_per_sm;
    t->schedule = b.schedule == 1 ? 1 : (b.schedule == 0 ? 2 : (b.schedule == 2 ? 3 : 4));
    t->hub_degree = b.hub_degree;
}

}  // namespace gde

using namespace gde;

struct gde_session {
    gde_graph *graph = nullptr;
    SolveParams p{};
    DenseWork *w = nullptr;
    uint32_t flags = 0;
};

struct gde_bsession {
    gde_graph *graph = nullptr;
    BatchSession *s = nullptr;
};


extern "C" {

void gde_solve_opts_init(gde_solve_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = GDE_FP64;
}

const char *gde_last_error(void) { return g_last_error.c_str(); }

gde_status gde_graph_create(int64_t n, const int64_t *offsets, const int32_t *cols, uint32_t flags,
                            gde_graph **out) {
    API_BEGIN
    GDE_REQUIRE(out != nullptr, GDE_EINVAL, "out is NULL");
    *out = nullptr;
    GDE_REQUIRE(n >= 0 && n < ((int64_t)1 << 31), GDE_EINVAL, "n must be in [0, 2^31)");
    GDE_REQUIRE(offsets != nullptr, GDE_EINVAL, "offsets is NULL");
    const bool dev = (flags & GDE_DEVICE_PTRS) != 0;
    int64_t nnz = 0;
    if (dev) {
        GDE_CUDA(cudaMemcpy(&nnz, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
        nnz = offsets[n];
    }
    GDE_REQUIRE(nnz >= 0 && nnz < ((int64_t)1 << 40), GDE_EINVAL, "offsets[n] out of range");
    GDE_REQUIRE(nnz == 0 || cols != nullptr, GDE_EINVAL, "cols is NULL");
    gde_graph *h = new gde_graph();
    Graph &g = h->g;
    try {
        g.n = n;
        g.nnz = nnz;
        GDE_CUDA(cudaGetDevice(&g.device));
        GDE_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
        g.off = (int64_t *)dmalloc(sizeof(int64_t) * (size_t)(n + 1), "CSR offsets");
        g.col = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), "CSR columns");
        g.deg = (int32_t *)dmalloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1), "degrees");
        const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GDE_CUDA(cudaMemcpyAsync(g.off, offsets, sizeof(int64_t) * (size_t)(n + 1), k, g.stream));
        if (nnz > 0)
            GDE_CUDA(cudaMemcpyAsync(g.col, cols, sizeof(int32_t) * (size_t)nnz, k, g.stream));
        unsigned bits = 0;
        graph_validate(g, (flags & GDE_CHECK_SYMMETRIC) != 0, &bits);
        if (bits) {
            std::string m = "invalid CSR:";
            if (bits & kBadOffsets) m += " offsets not monotone or not starting at 0;";
            if (bits & kBadColRange) m += " column id out of range;";
            if (bits & kUnsorted) m += " row not strictly increasing (unsorted or duplicate);";
            if (bits & kSelfLoop) m += " self-loop;";
            if (bits & kAsymmetric) m += " not symmetric;";
            set_error(m);
            throw Fail{GDE_EINVAL};
        }
    } catch (...) {
        gde_graph_destroy(h);
        throw;
    }
    *out = h;
    API_END
}

gde_status gde_graph_destroy(gde_graph *h) {
    if (!h) return GDE_OK;
    Graph &g = h->g;
    if (g.stream) cudaStreamSynchronize(g.stream);
    for (int k = 0; k < 2; k++) dense_work_destroy(g.dense[k]);
    batch_work_destroy(g.batch);
    update_scratch_free(g);
    g.prof.reset();
    dfree(g.off);
    dfree(g.col);
    dfree(g.deg);
    dfree(g.colp);
    hubs_free(g);
    for (void *q : g.stage_buf) dfree(q);
    dfree(g.topk_part);
    if (g.stream) cudaStreamDestroy(g.stream);
    delete h;
    return GDE_OK;
}

gde_status gde_graph_info(const gde_graph *h, int64_t *n, int64_t *nnz, int32_t *max_degree) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr, GDE_EINVAL, "graph is NULL");
    if (n) *n = h->g.n;
    if (nnz) *nnz = h->g.nnz;
    if (max_degree) *max_degree = h->g.max_degree;
    API_END
}

gde_status gde_graph_csr(const gde_graph *hc, int64_t *offsets, int32_t *cols, uint32_t flags) {
    API_BEGIN
    GDE_REQUIRE(hc != nullptr, GDE_EINVAL, "graph is NULL");
    gde_graph *h = const_cast<gde_graph *>(hc);
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    const cudaMemcpyKind k = (flags & GDE_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (offsets) GDE_CUDA(cudaMemcpyAsync(offsets, g.off, 8 * (size_t)(g.n + 1), k, g.stream));
    if (cols && g.nnz > 0) GDE_CUDA(cudaMemcpyAsync(cols, g.col, 4 * (size_t)g.nnz, k, g.stream));
    GDE_CUDA(cudaStreamSynchronize(g.stream));
    API_END
}

gde_status gde_update_edges(gde_graph *h, const int32_t *src, const int32_t *dst, int64_t m, uint32_t flags,
                            int64_t *added) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr, GDE_EINVAL, "graph is NULL");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    const int64_t a = graph_insert_edges(g, src, dst, m, (flags & GDE_DEVICE_PTRS) != 0, nullptr);
    if (added) *added = a;
    API_END
}

gde_status gde_solve(gde_graph *h, gde_kind kind, double param, double eps, const int32_t *seeds,
                     int32_t nseeds, const gde_solve_opts *opts, void *out_x, int32_t *out_ids,
                     gde_stats *stats) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr, GDE_EINVAL, "graph is NULL");
    gde_solve_opts o;
    gde_solve_opts_init(&o);
    if (opts) o = *opts;
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    SolveParams p = make_params(g, kind, param, eps, o);
    GDE_REQUIRE(nseeds >= 0, GDE_EINVAL, "nseeds must be >= 0");
    if (nseeds == 0) return GDE_OK;
    GDE_REQUIRE(seeds != nullptr && out_x != nullptr, GDE_EINVAL, "seeds or out_x is NULL");
    GDE_REQUIRE(o.topk == 0 || out_ids != nullptr, GDE_EINVAL, "topk output needs out_ids");
    GDE_REQUIRE(o.topk <= 64, GDE_EINVAL, "topk must be <= 64");
    GDE_REQUIRE(o.topk == 0 || o.precision == GDE_FP32, GDE_EINVAL, "topk output is FP32");
    GDE_REQUIRE(o.batched == 0 || o.batched == 1, GDE_EINVAL, "bad batched flag");
    GDE_REQUIRE(!(o.deterministic && o.batched), GDE_EINVAL,
                "deterministic mode solves one seed at a time (batched must be 0)");
    const bool dev = (o.flags & GDE_DEVICE_PTRS) != 0;
    std::vector<int32_t> hs((size_t)nseeds);
    if (dev) {
        GDE_CUDA(cudaMemcpyAsync(hs.data(), seeds, sizeof(int32_t) * (size_t)nseeds,
                                 cudaMemcpyDeviceToHost, p.stream));
        GDE_CUDA(cudaStreamSynchronize(p.stream));
    } else {
        memcpy(hs.data(), seeds, sizeof(int32_t) * (size_t)nseeds);
    }
    for (int32_t i = 0; i < nseeds; i++)
        GDE_REQUIRE(hs[i] >= 0 && hs[i] < g.n, GDE_EINVAL, "seed id out of range");

    const size_t rsz = p.precision == GDE_FP64 ? 8 : 4;
    const int k = o.topk;
    // device views of the outputs (staging buffers for host pointers, reused across calls:
    // the graph's lock is held, so no other call on g uses them meanwhile)
    size_t nstaged = 0;
    auto stage = [&](size_t bytes, const char *what) {
        const size_t i = nstaged++;
        if (g.stage_buf.size() <= i) {
            g.stage_buf.push_back(nullptr);
            g.stage_cap.push_back(0);
        }
        if (g.stage_cap[i] < bytes) {
            dfree(g.stage_buf[i]);
            g.stage_buf[i] = nullptr;
            g.stage_cap[i] = 0;
            g.stage_buf[i] = dmalloc(bytes, what);
            g.stage_cap[i] = bytes;
        }
        return g.stage_buf[i];
    };
    gde_status worst = GDE_OK;
    {
        std::vector<gde_stats> st((size_t)nseeds);
        std::vector<int32_t> todo;  // seeds solved one at a time with dense x and r
        int32_t *ids_dev = nullptr;
        float *vals_dev = nullptr;
        if (k > 0) {
            ids_dev = dev ? out_ids : (int32_t *)stage(4 * (size_t)nseeds * k, "top-k ids");
            vals_dev = dev ? (float *)out_x : (float *)stage(4 * (size_t)nseeds * k, "top-k values");
        }
        if (o.chebyshev) {
            GDE_REQUIRE(o.chebyshev == 1 && !o.global_gd, GDE_EINVAL, "bad chebyshev flag");
            GDE_REQUIRE(k == 0 && !o.batched && !o.deterministic, GDE_EINVAL,
                        "LocalCH writes dense x (no topk, batched or deterministic mode)");
            for (int32_t i = 0; i < nseeds; i++)
                localch_solve(g, p, hs[i], (char *)out_x + rsz * (size_t)g.n * i, dev, &st[(size_t)i]);
            if (stats) memcpy(stats, st.data(), sizeof(gde_stats) * (size_t)nseeds);
            for (const gde_stats &one : st) if (one.status != GDE_OK) worst = (gde_status)one.status;
        } else if (o.global_gd) {
            // the standard algorithm LocalGD is compared with: dense output, one seed at a time
            GDE_REQUIRE(o.global_gd == 1, GDE_EINVAL, "bad global_gd flag");
            GDE_REQUIRE(k == 0 && !o.batched && !o.deterministic, GDE_EINVAL,
                        "global GD writes dense x (no topk, batched or deterministic mode)");
            for (int32_t i = 0; i < nseeds; i++)
                global_gd_solve(g, p, hs[i], (char *)out_x + rsz * (size_t)g.n * i, dev, &st[(size_t)i]);
            if (stats) memcpy(stats, st.data(), sizeof(gde_stats) * (size_t)nseeds);
            for (const gde_stats &one : st) if (one.status != GDE_OK) worst = (gde_status)one.status;
        } else if (o.batched) {
            GDE_REQUIRE(k > 0, GDE_EINVAL, "batched mode returns top-k lists: set topk");
            const int32_t *seeds_dev = seeds;
            if (!dev) {
                int32_t *sd = (int32_t *)stage(4 * (size_t)nseeds, "seeds");
                GDE_CUDA(cudaMemcpyAsync(sd, hs.data(), 4 * (size_t)nseeds, cudaMemcpyHostToDevice, p.stream));
                seeds_dev = sd;
            }
            std::vector<int32_t> of((size_t)nseeds);
            int32_t nof = 0;
            const int64_t budget = batch_budget(o.mem_budget_bytes, kind);
            batch_solve_rebatch(g, p, seeds_dev, hs.data(), nseeds, k, budget, ids_dev, vals_dev,
                                st.data(), of.data(), &nof);
            for (int32_t i = 0; i < nof; i++) todo.push_back(of[i]);
        } else {
            for (int32_t i = 0; i < nseeds; i++) todo.push_back(i);
        }
        if (!todo.empty()) {
            DenseWork *w = dense_for(g, p.precision);
            void *vec = nullptr;
            if (k > 0 || !dev) vec = stage(rsz * (size_t)(g.n > 0 ? g.n : 1), "output staging");
            for (int32_t i : todo) {
                dense_begin(g, w, p, hs[i]);
                gde_stats one{};
                double rl1 = 1.0, xl1 = 0.0;
                if (kind == GDE_GPPR && p.gbeta != 0.0) {
                    // the scaled system's source mass S_s = max(d_s, 1)^b
                    int32_t ds = 0;
                    GDE_CUDA(cudaMemcpy(&ds, g.deg + hs[i], sizeof(int32_t), cudaMemcpyDeviceToHost));
                    rl1 = std::pow((double)(ds > 0 ? ds : 1), p.gbeta);
                }
                int64_t rounds = 0;
                bool converged = false;
                while (rounds < p.max_rounds) {
                    RoundInfo ri;
                    int64_t na = dense_round(g, w, p, &ri);
                    if (na == 0) { converged = true; break; }
                    rounds++;
                    one.active_volume += ri.vol;
                    one.pushes += ri.n_active;
                    xl1 += (kind == GDE_PPR || kind == GDE_GPPR ? param : 1.0) * ri.rS_l1;
                    rl1 = rl1 - ri.rS_l1 + ri.scat;
                }
                if (!converged && !dense_pending(w)) converged = true;
                one.rounds = rounds;
                one.resid_l1 = rl1;
                one.mass_l1 = xl1;
                one.status = converged ? GDE_OK : GDE_ENOTCONV;
                one.fallback = o.batched ? 1 : 0;  // only overflowed seeds come here in batched mode
                void *dst = vec ? vec : (char *)out_x + rsz * (size_t)g.n * i;
                dense_output(g, w, p, dst);
                if (k > 0) {
                    topk_dense_f32(g, (const float *)vec, g.n, k, ids_dev + (size_t)i * k,
                                   vals_dev + (size_t)i * k, p.stream);
                } else if (!dev && g.n > 0) {
                    GDE_CUDA(cudaMemcpyAsync((char *)out_x + rsz * (size_t)g.n * i, vec, rsz * (size_t)g.n,
                                             cudaMemcpyDeviceToHost, p.stream));
                }
                GDE_CUDA(cudaStreamSynchronize(p.stream));
                st[(size_t)i] = one;
            }
        }
        if (k > 0 && !dev) {
            GDE_CUDA(cudaMemcpyAsync(out_ids, ids_dev, 4 * (size_t)nseeds * k, cudaMemcpyDeviceToHost, p.stream));
            GDE_CUDA(cudaMemcpyAsync(out_x, vals_dev, 4 * (size_t)nseeds * k, cudaMemcpyDeviceToHost, p.stream));
        }
        GDE_CUDA(cudaStreamSynchronize(p.stream));
        for (int32_t i = 0; i < nseeds; i++) {
            if (st[(size_t)i].status != GDE_OK) worst = (gde_status)st[(size_t)i].status;
            if (stats) stats[i] = st[(size_t)i];
        }
    }
    if (worst != GDE_OK) {
        set_error("round cap reached before the active set became empty");
        return worst;
    }
    API_END
}

gde_status gde_profile_enable(gde_graph *h, int enable) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr, GDE_EINVAL, "graph is NULL");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    g.prof.reset();
    g.prof.enabled = enable != 0;
    API_END
}

gde_status gde_profile_read(gde_graph *h, gde_profile *out) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && out != nullptr, GDE_EINVAL, "graph or out is NULL");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    g.prof.read(out);
    API_END
}

gde_status gde_profile_rounds(gde_graph *h, double *out, int64_t cap, int64_t *rounds) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && rounds != nullptr, GDE_EINVAL, "graph or rounds is NULL");
    GDE_REQUIRE(cap >= 0 && (cap == 0 || out != nullptr), GDE_EINVAL, "bad output buffer");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    *rounds = batch_round_log(g, out, cap);
    API_END
}

gde_status gde_set_tuning(gde_graph *h, const gde_tuning *t) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && t != nullptr, GDE_EINVAL, "graph or tuning is NULL");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    Bins b = g.bins;
    if (t->t1 > 0) b.t1 = t->t1;
    if (t->t2 > 0) b.t2 = t->t2;
    if (t->chunk > 0) b.chunk = t->chunk;
    if (t->blocks_per_sm > 0) b.blocks_per_sm = t->blocks_per_sm;
    if (t->schedule > 0) b.schedule = t->schedule == 1 ? 1 : (t->schedule == 2 ? 0 : (t->schedule == 3 ? 2 : 3));
    GDE_REQUIRE(t->schedule <= 4, GDE_EINVAL, "tuning: schedule must be 0..4");
    GDE_REQUIRE(t->hub_degree == 0 || t->hub_degree == -1 || t->hub_degree >= 2, GDE_EINVAL,
                "tuning: hub_degree must be -1 (no slab), 0 (keep) or >= 2");
    if (t->hub_degree != 0) b.hub_degree = t->hub_degree;
    GDE_REQUIRE(b.t1 <= b.t2, GDE_EINVAL, "tuning: t1 must be <= t2");
    GDE_REQUIRE(b.chunk >= 32 && b.chunk <= (1 << 24), GDE_EINVAL, "tuning: chunk must be in [32, 2^24]");
    GDE_REQUIRE(b.blocks_per_sm <= 32, GDE_EINVAL, "tuning: blocks_per_sm must be <= 32");
    g.bins = b;
    for (int k = 0; k < 2; k++)
        if (g.dense[k]) { dense_work_destroy(g.dense[k]); g.dense[k] = nullptr; }
    API_END
}

gde_status gde_get_tuning(const gde_graph *h, gde_tuning *t) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && t != nullptr, GDE_EINVAL, "graph or tuning is NULL");
    tuning_from_bins(h->g.bins, t);
    API_END
}

gde_status gde_autotune(gde_graph *h, gde_kind kind, double param, double eps, const int32_t *seeds,
                        int32_t nseeds, const gde_solve_opts *opts, gde_tuning *best, double *best_ms) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && seeds != nullptr && nseeds > 0, GDE_EINVAL, "graph, seeds or nseeds invalid");
    gde_solve_opts o;
    gde_solve_opts_init(&o);
    if (opts) o = *opts;
    o.batched = 1;
    o.precision = GDE_FP32;
    o.deterministic = 0;
    if (o.topk <= 0) o.topk = 64;
    GDE_REQUIRE(o.topk <= 64, GDE_EINVAL, "topk must be <= 64");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    SolveParams p = make_params(g, kind, param, eps, o);
    GDE_REQUIRE(kind == GDE_PPR || kind == GDE_KATZ || kind == GDE_GPPR || kind == GDE_HK || kind == GDE_SERIES,
                GDE_EINVAL, "unknown kind");
    const bool dev = (o.flags & GDE_DEVICE_PTRS) != 0;
    std::vector<void *> owned;
    auto alloc = [&](size_t bytes, const char *what) {
        void *q = dmalloc(bytes, what);
        owned.push_back(q);
        return q;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const Bins saved = g.bins;
    try {
        int32_t *sd = (int32_t *)alloc(4 * (size_t)nseeds, "autotune seeds");
        GDE_CUDA(cudaMemcpyAsync(sd, seeds, 4 * (size_t)nseeds,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p.stream));
        int32_t *ids = (int32_t *)alloc(4 * (size_t)nseeds * o.topk, "autotune ids");
        float *vals = (float *)alloc(4 * (size_t)nseeds * o.topk, "autotune values");
        std::vector<int32_t> of((size_t)nseeds);
        GDE_CUDA(cudaEventCreate(&e0));
        GDE_CUDA(cudaEventCreate(&e1));
        auto time_bins = [&](const Bins &b) {
            g.bins = b;
            int32_t nof = 0;
            batch_solve(g, p, sd, nseeds, o.topk, batch_budget(o.mem_budget_bytes, kind), ids, vals, nullptr,
                        of.data(), &nof);
            float bestt = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                GDE_CUDA(cudaEventRecord(e0, p.stream));
                batch_solve(g, p, sd, nseeds, o.topk, batch_budget(o.mem_budget_bytes, kind), ids, vals, nullptr,
                        of.data(), &nof);
                GDE_CUDA(cudaEventRecord(e1, p.stream));
                GDE_CUDA(cudaEventSynchronize(e1));
                float ms = 0.0f;
                GDE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < bestt) bestt = ms;
            }
            return (double)bestt;
        };
        Bins cur = saved;
        double cur_ms = time_bins(cur);
        const int t1s[] = {4, 8, 16, 32};
        const int t2s[] = {128, 256, 512, 1024, 2048};
        const int chunks[] = {256, 512, 1024, 2048, 4096};
        const int scheds[] = {0, 1, 2, 3};
        const int bpss[] = {0, 3, 2};
        // hub slab thresholds: all at most 160, so every FP32 table entry keeps its bound of
        // 159 additions per round whichever wins
        const int hubs[] = {64, 128, 160};
        auto sweep = [&](const int *vals_, int nv, int Bins::*field, bool need_order) {
            for (int i = 0; i < nv; i++) {
                Bins b = cur;
                b.*field = vals_[i];
                if (need_order && b.t1 > b.t2) continue;
                if (b.*field == cur.*field) continue;
                const double ms = time_bins(b);
                if (ms < cur_ms) { cur_ms = ms; cur = b; }
            }
        };
        sweep(t1s, 4, &Bins::t1, true);
        sweep(t2s, 5, &Bins::t2, true);
        sweep(chunks, 5, &Bins::chunk, false);
        sweep(scheds, 4, &Bins::schedule, false);
        sweep(bpss, 3, &Bins::blocks_per_sm, false);
        if (cur.hub_degree > 0) sweep(hubs, 3, &Bins::hub_degree, false);
        g.bins = cur;
        for (int k = 0; k < 2; k++)
            if (g.dense[k]) { dense_work_destroy(g.dense[k]); g.dense[k] = nullptr; }
        if (best) tuning_from_bins(cur, best);
        if (best_ms) *best_ms = cur_ms;
    } catch (...) {
        g.bins = saved;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        for (void *q : owned) dfree(q);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (void *q : owned) dfree(q);
    API_END
}

gde_status gde_session_begin(gde_graph *h, gde_kind kind, double param, double eps, int32_t seed,
                             const gde_solve_opts *opts, gde_session **out) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && out != nullptr, GDE_EINVAL, "graph or out is NULL");
    *out = nullptr;
    gde_solve_opts o;
    gde_solve_opts_init(&o);
    if (opts) o = *opts;
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    GDE_REQUIRE(seed >= 0 && seed < g.n, GDE_EINVAL, "seed id out of range");
    gde_session *s = new gde_session();
    try {
        s->graph = h;
        s->p = make_params(g, kind, param, eps, o);
        s->flags = o.flags;
        s->w = dense_work_create(g, s->p.precision);
        dense_begin(g, s->w, s->p, seed);
        GDE_CUDA(cudaStreamSynchronize(s->p.stream));
    } catch (...) {
        dense_work_destroy(s->w);
        delete s;
        throw;
    }
    *out = s;
    API_END
}

gde_status gde_session_step(gde_session *s, int64_t *n_active) {
    API_BEGIN
    GDE_REQUIRE(s != nullptr, GDE_EINVAL, "session is NULL");
    Graph &g = s->graph->g;
    std::lock_guard<std::mutex> lock(g.mu);
    int64_t k = dense_round(g, s->w, s->p, nullptr);
    if (n_active) *n_active = k;
    API_END
}

gde_status gde_session_read(gde_session *s, void *x, void *r, int32_t *active, int64_t *n_active) {
    API_BEGIN
    GDE_REQUIRE(s != nullptr, GDE_EINVAL, "session is NULL");
    Graph &g = s->graph->g;
    std::lock_guard<std::mutex> lock(g.mu);
    dense_read(g, s->w, s->p, x, r, active, n_active, (s->flags & GDE_DEVICE_PTRS) != 0);
    API_END
}

gde_status gde_session_end(gde_session *s) {
    if (!s) return GDE_OK;
    if (s->w) {
        cudaStreamSynchronize(s->p.stream);
        dense_work_destroy(s->w);
    }
    delete s;
    return GDE_OK;
}

gde_status gde_test_fail_alloc(int64_t nth) {
    API_BEGIN
    GDE_REQUIRE(nth >= 0, GDE_EINVAL, "nth must be >= 0");
    g_fail_alloc_in.store((long long)nth);
    API_END
}

gde_status gde_test_barrier_fault(gde_graph *h, int64_t limit_ns, int32_t block, int32_t barrier) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr, GDE_EINVAL, "graph is NULL");
    GDE_REQUIRE(limit_ns >= 0, GDE_EINVAL, "limit_ns must be >= 0");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    g.dbg_bar_limit_ns = (unsigned long long)limit_ns;
    g.dbg_fail_block = block < 0 ? -1 : block;
    g.dbg_fail_barrier = block < 0 ? -1 : barrier;
    API_END
}

gde_status gde_bsession_begin(gde_graph *h, gde_kind kind, double param, double eps, const int32_t *seeds,
                              int32_t nseeds, const gde_solve_opts *opts, gde_bsession **out) {
    API_BEGIN
    GDE_REQUIRE(h != nullptr && out != nullptr, GDE_EINVAL, "graph or out is NULL");
    *out = nullptr;
    gde_solve_opts o;
    gde_solve_opts_init(&o);
    if (opts) o = *opts;
    GDE_REQUIRE((o.flags & GDE_DEVICE_PTRS) == 0, GDE_EINVAL, "batched session: seeds are a host array");
    Graph &g = h->g;
    std::lock_guard<std::mutex> lock(g.mu);
    SolveParams p = make_params(g, kind, param, eps, o);
    gde_bsession *b = new gde_bsession();
    try {
        b->graph = h;
        b->s = bsession_begin(g, p, seeds, nseeds, o.mem_budget_bytes);
    } catch (...) {
        delete b;
        throw;
    }
    *out = b;
    API_END
}

gde_status gde_bsession_step(gde_bsession *b, int64_t *n_candidates) {
    API_BEGIN
    GDE_REQUIRE(b != nullptr, GDE_EINVAL, "session is NULL");
    Graph &g = b->graph->g;
    std::lock_guard<std::mutex> lock(g.mu);
    const int64_t c = bsession_step(b->s);
    if (n_candidates) *n_candidates = c;
    API_END
}

gde_status gde_bsession_read(gde_bsession *b, int32_t seed_index, float *x, double *r, int32_t *pushed,
                             int64_t *n_pushed) {
    API_BEGIN
    GDE_REQUIRE(b != nullptr, GDE_EINVAL, "session is NULL");
    Graph &g = b->graph->g;
    std::lock_guard<std::mutex> lock(g.mu);
    const gde_status st = bsession_read(b->s, seed_index, x, r, pushed, n_pushed);
    if (st != GDE_OK) {
        set_error("batched session: this seed's table overflowed");
        return st;
    }
    API_END
}

gde_status gde_bsession_end(gde_bsession *b) {
    if (!b) return GDE_OK;
    bsession_destroy(b->s);
    delete b;
    return GDE_OK;
}

}  // extern "C"
