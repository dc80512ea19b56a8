// Serving loop over a serving pool (continuous batching of PPR/Katz queries on a changing
// graph, Section 4): queries wait in a FIFO and are admitted between device steps while their
// accumulator tables fit the pool's memory (a table is a power-of-two run of pages; its first
// size comes from what recent queries of the same kind and tolerance needed); a step runs a
// bounded number of LocalGD rounds for every resident query at once, so a query that arrives
// while others are on the GPU joins them at the next step; a query whose slot has no candidate
// left has converged and its top-k is emitted; a query whose table overflowed is started again,
// ahead of the queue, with a table four times larger; edge-insertion batches are applied
// between steps, after which every resident query is corrected (warm start) and runs on from
// its corrected state.  A one-shot query leaves its slot (and pages) at its answer; a standing
// query stays resident, tracking the graph (re-answered as an update after every batch), until
// its slot or memory is needed (oldest answer first).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gde {

double server_clock() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace gde

using namespace gde;

namespace {

enum SlotState { kFree = 0, kRunning = 1, kAnswered = 2 };

struct Query {
    uint64_t qid;
    gde_kind kind;
    double param;
    int32_t cls;
    int32_t seed;
    bool track;
    double t_submit;
    int order = -1;  // table size to start with (2^order pages); -1: the class estimate
};

struct Slot {
    SlotState state = kFree;
    Query q{};
    bool answered_once = false;
    double t_answer = 0.0;
    double t_start = 0.0;  // when the current run (first solve or re-convergence) began
};

struct EdgeChunk {
    std::vector<int32_t> src, dst;
};

}  // namespace

struct gde_server {
    gde_graph *graph = nullptr;
    gde_server_opts opts{};
    ServePool *pool = nullptr;
    std::mutex mu;  // queue, pending edges, results (submit / insert / poll may run on other threads)
    std::deque<Query> queue;
    std::vector<EdgeChunk> edges;
    std::vector<gde_server_result> done;
    std::vector<Slot> slots;
    std::mutex step_mu;  // one step at a time
    int64_t steps = 0;
    int64_t edge_batches = 0;
    double t_phase[5] = {0, 0, 0, 0, 0};  // graph, correct, admit, rounds, results (seconds)
    int32_t peak_resident = 0;
    int64_t peak_pages = 0;
    int64_t readmissions = 0;
    int64_t evictions = 0;
    // Table sizes that recent queries needed, per (kind, tolerance class, seed degree bucket
    // floor(log2(d_s + 1))): the table order holding their keys at an eighth load at most, the last
    // kNeedWindow answered queries (or an overflow) of each bucket.  A new query starts at the
    // largest order of its bucket, else of the nearest lower-degree bucket that has one.
    static constexpr int kBuckets = 32;
    static constexpr size_t kNeedWindow = 16;
    std::deque<int> needed[2][4][kBuckets];
    std::vector<int32_t> deg;  // seed degrees (as of creation: the buckets are a guide only)
};

namespace {

int degree_bucket(const gde_server *S, int32_t seed) {
    int b = 0;
    while (b + 1 < gde_server::kBuckets && ((int64_t)2 << b) <= (int64_t)S->deg[(size_t)seed] + 1) b++;
    return b;
}

int start_order(gde_server *S, const Query &q) {
    if (q.order >= 0) return q.order;
    const int kind = q.kind == GDE_KATZ ? 1 : 0;
    for (int b = degree_bucket(S, q.seed); b >= 0; b--) {
        const std::deque<int> &h = S->needed[kind][q.cls][b];
        if (!h.empty()) return *std::max_element(h.begin(), h.end());
    }
    return 0;
}

void note_needed(gde_server *S, const Query &q, int order) {
    std::deque<int> &h = S->needed[q.kind == GDE_KATZ ? 1 : 0][q.cls][degree_bucket(S, q.seed)];
    h.push_back(order);
    if (h.size() > gde_server::kNeedWindow) h.pop_front();
}

// the smallest table order whose slots hold `keys` at an eighth load (short probes)
int order_for_keys(int64_t keys, int64_t page_slots, int max_order) {
    int o = 0;
    while (o < max_order && (page_slots << o) < 8 * keys) o++;
    return o;
}

}  // namespace

extern "C" {

void gde_server_opts_init(gde_server_opts *o) {
    if (!o) return;
    *o = gde_server_opts{};
    o->slots = 256;
    o->rounds_per_step = 4;
    o->topk = 64;
    o->n_eps = 1;
    o->eps[0] = 1e-6;
    o->mem_budget_bytes = 0;
    o->defer_volume = 0;
}

double gde_server_clock(void) { return server_clock(); }

gde_status gde_server_create(gde_graph *g, const gde_server_opts *o, gde_server **out) {
    API_BEGIN
    GDE_REQUIRE(g != nullptr && out != nullptr, GDE_EINVAL, "graph or out is NULL");
    *out = nullptr;
    gde_server_opts op;
    gde_server_opts_init(&op);
    if (o) op = *o;
    GDE_REQUIRE(op.slots >= 1 && op.slots <= (1 << 20), GDE_EINVAL, "slots must be in [1, 2^20]");
    GDE_REQUIRE(op.rounds_per_step >= 1, GDE_EINVAL, "rounds_per_step must be >= 1");
    GDE_REQUIRE(op.topk >= 1 && op.topk <= 64, GDE_EINVAL, "topk must be in [1, 64]");
    GDE_REQUIRE(op.n_eps >= 1 && op.n_eps <= 4, GDE_EINVAL, "n_eps must be in [1, 4]");
    gde_server *S = new gde_server();
    try {
        Graph &G = g->g;
        std::lock_guard<std::mutex> lock(G.mu);
        S->graph = g;
        S->opts = op;
        S->pool = serve_pool_create(G, op.slots, op.mem_budget_bytes, op.eps, op.n_eps);
        serve_pool_set_defer(S->pool, op.defer_volume == 0 ? ((int64_t)1 << 23) : op.defer_volume);
        S->slots.resize((size_t)op.slots);
        S->deg.resize((size_t)G.n);
        if (G.n > 0) GDE_CUDA(cudaMemcpy(S->deg.data(), G.deg, 4 * (size_t)G.n, cudaMemcpyDeviceToHost));
    } catch (...) {
        if (S->pool) serve_pool_destroy(S->pool);
        delete S;
        throw;
    }
    *out = S;
    API_END
}

gde_status gde_server_destroy(gde_server *S) {
    if (!S) return GDE_OK;
    API_BEGIN
    {
        std::lock_guard<std::mutex> lock(S->graph->g.mu);
        serve_pool_destroy(S->pool);
    }
    delete S;
    API_END
}

gde_status gde_server_submit(gde_server *S, uint64_t qid, gde_kind kind, double param, int32_t eps_class,
                             int32_t seed, uint32_t flags, double t_submit) {
    API_BEGIN
    GDE_REQUIRE(S != nullptr, GDE_EINVAL, "server is NULL");
    GDE_REQUIRE(kind == GDE_PPR || kind == GDE_KATZ, GDE_EINVAL, "a server serves PPR and Katz");
    GDE_REQUIRE(kind != GDE_PPR || (param > 0.0 && param < 1.0), GDE_EINVAL, "PPR alpha must be in (0,1)");
    GDE_REQUIRE(kind != GDE_KATZ || param > 0.0, GDE_EINVAL, "Katz beta must be > 0");
    GDE_REQUIRE(eps_class >= 0 && eps_class < S->opts.n_eps, GDE_EINVAL, "tolerance class out of range");
    GDE_REQUIRE(seed >= 0 && seed < S->graph->g.n, GDE_EINVAL, "seed out of range");
    std::lock_guard<std::mutex> lock(S->mu);
    S->queue.push_back(Query{qid, kind, param, eps_class, seed, (flags & GDE_SERVE_TRACK) != 0,
                             t_submit >= 0.0 ? t_submit : server_clock()});
    API_END
}

gde_status gde_server_insert_edges(gde_server *S, const int32_t *src, const int32_t *dst, int64_t m) {
    API_BEGIN
    GDE_REQUIRE(S != nullptr, GDE_EINVAL, "server is NULL");
    GDE_REQUIRE(m >= 0 && (m == 0 || (src && dst)), GDE_EINVAL, "bad edge arrays");
    const int64_t n = S->graph->g.n;
    for (int64_t i = 0; i < m; i++)
        GDE_REQUIRE(src[i] >= 0 && src[i] < n && dst[i] >= 0 && dst[i] < n, GDE_EINVAL, "edge endpoint out of range");
    EdgeChunk c;
    c.src.assign(src, src + m);
    c.dst.assign(dst, dst + m);
    std::lock_guard<std::mutex> lock(S->mu);
    S->edges.push_back(std::move(c));
    API_END
}

gde_status gde_server_step(gde_server *S, int32_t *running, int32_t *queued) {
    API_BEGIN
    GDE_REQUIRE(S != nullptr, GDE_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> step_lock(S->step_mu);
    Graph &G = S->graph->g;
    std::vector<EdgeChunk> edges;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        edges.swap(S->edges);
    }
    std::lock_guard<std::mutex> glock(G.mu);
    ServePool *P = S->pool;
    const int32_t nslots = S->opts.slots;

    // 1. edge batches: update the graph, then correct every resident query (warm start)
    if (!edges.empty()) {
        EdgeChunk all;
        for (auto &c : edges) {
            all.src.insert(all.src.end(), c.src.begin(), c.src.end());
            all.dst.insert(all.dst.end(), c.dst.begin(), c.dst.end());
        }
        EdgeBatch eb{};
        const double tg = server_clock();
        const int64_t added = graph_insert_edges(G, all.src.data(), all.dst.data(), (int64_t)all.src.size(),
                                                 false, &eb);
        S->t_phase[0] += server_clock() - tg;
        S->edge_batches += (int64_t)edges.size();
        if (added > 0) {
            serve_pool_graph_changed(P);
            std::vector<int32_t> res;
            for (int32_t j = 0; j < nslots; j++)
                if (S->slots[(size_t)j].state != kFree) res.push_back(j);
            try {
                const double tc = server_clock();
                serve_pool_correct(G, P, eb, (int32_t)res.size(), res.data());
                GDE_CUDA(cudaStreamSynchronize(G.stream));
                S->t_phase[1] += server_clock() - tc;
            } catch (...) {
                edge_batch_free(eb);
                throw;
            }
            const double now = server_clock();
            for (int32_t j : res) {
                Slot &sl = S->slots[(size_t)j];
                if (sl.state == kAnswered) {
                    sl.state = kRunning;
                    sl.t_start = now;
                }
            }
        }
        edge_batch_free(eb);
    }

    // 2. admission in arrival order, while a slot and the query's table fit: free slots and
    //    free pages first, then the slots and pages of standing queries answered longest ago
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (!S->queue.empty()) {
            std::vector<int32_t> sl_ids, seeds, cls;
            std::vector<gde_kind> kinds;
            std::vector<double> params;
            const double now = server_clock();
            auto evict_oldest = [&]() -> int32_t {
                int32_t best = -1;
                for (int32_t j = 0; j < nslots; j++) {
                    const Slot &sl = S->slots[(size_t)j];
                    if (sl.state == kAnswered && (best < 0 || sl.t_answer < S->slots[(size_t)best].t_answer)) best = j;
                }
                if (best >= 0) {
                    serve_pool_release(P, best);
                    S->slots[(size_t)best].state = kFree;
                    S->evictions++;
                }
                return best;
            };
            while (!S->queue.empty()) {
                const Query q = S->queue.front();
                int32_t j = -1;
                for (int32_t c = 0; c < nslots && j < 0; c++)
                    if (S->slots[(size_t)c].state == kFree) j = c;
                if (j < 0) j = evict_oldest();
                if (j < 0) break;  // every slot runs a query
                const int ord = std::min(start_order(S, q), serve_pool_max_order(P));
                bool ok = serve_pool_reserve(P, j, ord);
                while (!ok && evict_oldest() >= 0) ok = serve_pool_reserve(P, j, ord);
                if (!ok) break;  // waits until running queries give memory back
                S->queue.pop_front();
                Slot &sl = S->slots[(size_t)j];
                sl.state = kRunning;
                sl.q = q;
                sl.answered_once = false;
                sl.t_start = now;
                sl_ids.push_back(j);
                seeds.push_back(q.seed);
                kinds.push_back(q.kind);
                params.push_back(q.param);
                cls.push_back(q.cls);
            }
            if (!sl_ids.empty()) {
                const double ta = server_clock();
                serve_pool_admit(G, P, (int32_t)sl_ids.size(), sl_ids.data(), seeds.data(), kinds.data(),
                                 params.data(), cls.data());
                GDE_CUDA(cudaStreamSynchronize(G.stream));
                S->t_phase[2] += server_clock() - ta;
            }
        }
    }
    {
        int32_t resident = 0;
        for (const Slot &sl : S->slots) resident += sl.state != kFree;
        S->peak_resident = std::max(S->peak_resident, resident);
        S->peak_pages = std::max(S->peak_pages, serve_pool_pages_used(P));
    }

    // 3. a bounded number of rounds for every resident query
    int32_t nrun = 0;
    for (const Slot &sl : S->slots) nrun += sl.state == kRunning;
    if (nrun > 0) {
        const double tr = server_clock();
        serve_pool_run(G, P, S->opts.rounds_per_step);
        const double tq = server_clock();
        S->t_phase[3] += tq - tr;
        // 4. converged: no candidate left in the slot
        std::vector<unsigned> pend((size_t)nslots);
        serve_pool_pending(G, P, pend.data());
        std::vector<int32_t> fin;
        for (int32_t j = 0; j < nslots; j++)
            if (S->slots[(size_t)j].state == kRunning && pend[(size_t)j] == 0) fin.push_back(j);
        if (!fin.empty()) {
            const int k = S->opts.topk;
            const int32_t nf = (int32_t)fin.size();
            std::vector<int32_t> ids((size_t)nf * k), st((size_t)nf), last((size_t)nf);
            std::vector<float> vals((size_t)nf * k);
            std::vector<int64_t> vol((size_t)nf), support((size_t)nf);
            serve_pool_results(G, P, nf, fin.data(), k, ids.data(), vals.data(), st.data(), vol.data(), last.data(),
                               support.data());
            const double now = server_clock();
            std::lock_guard<std::mutex> lock(S->mu);
            std::vector<Query> again;
            for (int32_t i = 0; i < nf; i++) {
                const int32_t j = fin[(size_t)i];
                Slot &sl = S->slots[(size_t)j];
                const int ord = serve_pool_order(P, j);
                if (st[(size_t)i] != GDE_OK && !sl.answered_once && ord < serve_pool_max_order(P)) {
                    // its table overflowed: start it again with a table four times larger, ahead
                    // of the queue (its latency still counts from its arrival); its bucket learns
                    // that it needed more
                    Query q = sl.q;
                    q.order = std::min(ord + 2, serve_pool_max_order(P));
                    note_needed(S, q, q.order);
                    again.push_back(q);
                    serve_pool_release(P, j);
                    sl.state = kFree;
                    S->readmissions++;
                    continue;
                }
                if (st[(size_t)i] == GDE_OK && !sl.answered_once)
                    note_needed(S, sl.q, order_for_keys(support[(size_t)i], serve_pool_page_slots(P),
                                                        serve_pool_max_order(P)));
                gde_server_result r{};
                r.qid = sl.q.qid;
                r.status = st[(size_t)i];
                r.update = sl.answered_once ? 1 : 0;
                r.k = k;
                r.slot = fin[(size_t)i];
                r.volume = vol[(size_t)i];
                r.t_submit = sl.answered_once ? sl.t_start : sl.q.t_submit;
                r.t_done = now;
                for (int e = 0; e < k; e++) {
                    r.ids[e] = ids[(size_t)i * k + e];
                    r.vals[e] = vals[(size_t)i * k + e];
                }
                S->done.push_back(r);
                if (r.status != GDE_OK || !sl.q.track) {
                    sl.state = kFree;  // answered one-shot (or failed) queries leave their slot
                    serve_pool_release(P, j);
                } else {
                    sl.state = kAnswered;
                    sl.answered_once = true;
                    sl.t_answer = now;
                }
            }
            for (auto it = again.rbegin(); it != again.rend(); ++it) S->queue.push_front(*it);
        }
        S->t_phase[4] += server_clock() - tq;
    }
    S->steps++;
    int32_t nr = 0;
    for (const Slot &sl : S->slots) nr += sl.state == kRunning;
    if (running) *running = nr;
    if (queued) {
        std::lock_guard<std::mutex> lock(S->mu);
        *queued = (int32_t)S->queue.size();
    }
    API_END
}

gde_status gde_server_poll(gde_server *S, gde_server_result *out, int32_t cap, int32_t *n) {
    API_BEGIN
    GDE_REQUIRE(S != nullptr && n != nullptr, GDE_EINVAL, "server or n is NULL");
    GDE_REQUIRE(cap >= 0 && (cap == 0 || out != nullptr), GDE_EINVAL, "bad output buffer");
    std::lock_guard<std::mutex> lock(S->mu);
    const int32_t m = (int32_t)std::min<size_t>((size_t)cap, S->done.size());
    for (int32_t i = 0; i < m; i++) out[i] = S->done[(size_t)i];
    S->done.erase(S->done.begin(), S->done.begin() + m);
    *n = m;
    API_END
}

gde_status gde_server_info(gde_server *S, gde_server_info_t *info) {
    API_BEGIN
    GDE_REQUIRE(S != nullptr && info != nullptr, GDE_EINVAL, "server or info is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    info->slots = S->opts.slots;
    info->running = info->answered = 0;
    for (const Slot &sl : S->slots) {
        info->running += sl.state == kRunning;
        info->answered += sl.state == kAnswered;
    }
    info->queued = (int32_t)S->queue.size();
    info->steps = S->steps;
    info->rounds = serve_pool_round(S->pool);
    info->edge_batches = S->edge_batches;
    info->cap = serve_pool_cap(S->pool);
    info->volume = serve_pool_volume(S->pool);
    info->t_graph = S->t_phase[0];
    info->t_correct = S->t_phase[1];
    info->t_admit = S->t_phase[2];
    info->t_rounds = S->t_phase[3];
    info->t_results = S->t_phase[4];
    info->pool_pages = serve_pool_pages(S->pool);
    info->pages_used = serve_pool_pages_used(S->pool);
    info->page_slots = serve_pool_page_slots(S->pool);
    info->peak_resident = S->peak_resident;
    info->readmissions = S->readmissions;
    info->evictions = S->evictions;
    info->peak_pages = S->peak_pages;
    API_END
}

}  // extern "C"
