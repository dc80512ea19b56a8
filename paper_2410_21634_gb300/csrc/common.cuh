// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "gde.h"

namespace gde {

// ------------------------------------------------------------------ errors --

void set_error(const std::string &msg);
void clear_error();

struct Fail {
    gde_status st;
};

#define GDE_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::gde::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
            throw ::gde::Fail{GDE_ECUDA};                                           \
        }                                                                           \
    } while (0)

#define GDE_REQUIRE(cond, status, msg)                                              \
    do {                                                                            \
        if (!(cond)) {                                                              \
            ::gde::set_error(msg);                                                  \
            throw ::gde::Fail{status};                                              \
        }                                                                           \
    } while (0)

// device allocation that throws GDE_ENOMEM (also when the test injector says this one fails)
void *dmalloc(size_t bytes, const char *what);
void dfree(void *p);

// ---------------------------------------------------------------- constants --

constexpr int kSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kThreads = 256;      // block size of the round kernels
constexpr int kWarps = kThreads / 32;

// degree bins of the push (autotunable; these are the defaults)
struct Bins {
    int32_t t1 = 16;      // d <= t1: thread per node
    int32_t t2 = 512;     // t1 < d <= t2: warp per node; d > t2: hub merge-path chunks
    int32_t chunk = 1024; // hub edges per warp work item
    int32_t blocks_per_sm = 0;  // persistent grid; 0 = occupancy limit
    int32_t schedule = 0;       // batched scatter order: 0 all bins in order, 1 hubs in order, 2 strided
    // batched engine: targets of degree >= hub_degree keep their residual in the per-seed
    // fixed-point hub slab instead of the hash tables (-1: no slab).  At 160 every hash entry
    // receives at most 159 float additions per round: within 159 * 2^-24 < 1e-5 of the exact sum.
    int32_t hub_degree = 160;
};

// ---------------------------------------------------------------- profiler --

enum ProfKind { kProfBatchRounds = 0, kProfBatchClear, kProfBatchTopk, kProfDenseFrontier, kProfDensePush, kProfKinds };

struct Profiler {
    bool enabled = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    gde_profile counters{};
    // record a start event; returns the index to close with stop()
    int start(int kind, cudaStream_t s);
    void stop(int idx, cudaStream_t s);
    void reset();
    void read(gde_profile *out);
    void launched(int n = 1) { if (enabled) counters.launches += n; }
};

// ------------------------------------------------------------------- graph --

struct Graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int32_t max_degree = 0;
    int device = 0;
    int64_t *off = nullptr;   // n+1
    int32_t *col = nullptr;   // nnz
    int32_t *deg = nullptr;   // n
    cudaStream_t stream = nullptr;
    std::mutex mu;
    struct DenseWork *dense[2] = {nullptr, nullptr};     // cached single-seed workspace per precision
    struct BatchWork *batch = nullptr;                   // cached batched workspace
    struct UpdateScratch *upd = nullptr;                 // edge-insertion buffers, kept between batches
    // The batched engines' edge stream: each column with its neighbour's degree code in the
    // bits above the node id (degree_code).  Built on first use (ensure_colp); an insertion
    // batch keeps it current when the graph was verified symmetric, else drops it.
    uint32_t *colp = nullptr;
    int64_t colp_cap = 0;      // entries the packed array can hold
    // device staging for gde_solve calls with host pointers, kept between calls (a call
    // takes its buffers in a fixed order, growing one only when a larger call needs it)
    std::vector<void *> stage_buf;
    std::vector<size_t> stage_cap;
    unsigned long long *topk_part = nullptr;  // dense top-k partial lists, allocated on first use
    // Hubs of the batched engine: the nodes of degree >= hub_min_deg ranked by degree
    // (descending, then id).  colq is the packed column array with each hub's rank in place of
    // its id (the degree code above it says which words name hubs: code >= hub_code).  Built on
    // first use; an insertion batch drops it (graph_changed).
    uint32_t *colq = nullptr;
    int64_t colq_cap = 0;
    int32_t *hub_node = nullptr;   // rank -> node
    int32_t *hub_deg = nullptr;    // rank -> degree
    int32_t *hub_rank = nullptr;   // node -> rank, -1 for other nodes
    int64_t hub_cap = 0;           // entries hub_node / hub_deg can hold
    int64_t hub_n = 0;
    int32_t hub_min_deg = 0;       // the degree threshold the hub data was built for
    uint32_t hub_code = 0;         // degree codes at or above it name hubs
    bool hub_valid = false;
    std::vector<int32_t> hub_node_host;
    int colp_idbits = 0;       // 0: no packing (n too large), thresholds are read per edge
    int colp_exact = 0;
    bool colp_valid = false;   // packed from the current CSR
    bool symmetric = false;    // A = A^T verified at creation (insertions keep it)
    Profiler prof;
    Bins bins;                 // launch shape used by later solves
    // test fault injection of the batched round kernel (gde_test_barrier_fault)
    unsigned long long dbg_bar_limit_ns = 0;  // 0: the default limit
    int32_t dbg_fail_block = -1;
    int32_t dbg_fail_barrier = -1;
};

// row validation result bits
enum : unsigned {
    kBadOffsets = 1u, kBadColRange = 2u, kUnsorted = 4u, kSelfLoop = 8u, kAsymmetric = 16u
};

void graph_validate(Graph &g, bool check_symmetric, unsigned *bits_out);

// Degree code of a neighbour, stored above its id in the packed column array: the exact
// degree when d < code_exact, else code_exact + floor(log2 d).  It brackets the neighbour's
// threshold fl(eps d) (rounded up to float) without reading the per-node threshold array:
// exact for small degrees, within [eps 2^k, eps (2^(k+1)-1)] for the log classes.
__host__ __device__ __forceinline__ uint32_t degree_code(int32_t d, int code_exact) {
    if (d < code_exact) return (uint32_t)d;
    uint32_t k = 0;
    while ((2ll << k) <= (long long)d) k++;
    return (uint32_t)code_exact + k;
}

// Builds g.colp from the CSR if it is not current (no-op when n leaves too few spare bits).
void ensure_colp(Graph &g, cudaStream_t s);
// Builds the hub data (hub_node, hub_deg, hub_rank, colq) for degree threshold min_deg if it is
// not current.  Returns false when the graph has no packed columns (then there is no slab).
bool ensure_hubs(Graph &g, int32_t min_deg, cudaStream_t s);
void hubs_free(Graph &g);

// Directed adjacencies added by one insertion batch (device arrays; sorted by (u, v)), with
// the rows that gained them and those rows' degrees before the batch.
struct EdgeBatch {
    bool owned = true;           // false: the arrays live in the graph's update scratch
    int64_t m = 0;               // adjacencies added
    int32_t *u = nullptr, *v = nullptr;
    int64_t rows = 0;            // rows that gained adjacencies (ascending)
    int32_t *row = nullptr;
    int32_t *row_cnt = nullptr;  // adjacencies gained by each
    int64_t *row_start = nullptr;  // first of them in u / v
    int32_t *old_deg = nullptr;  // degree before the batch
};

// Inserts the undirected edges (src[i], dst[i]) into g (both directions; self-loops and
// present adjacencies skipped) and returns the number of directed adjacencies added.  If out
// is not NULL it receives the batch (free with edge_batch_free; its arrays stay valid until the
// next insertion into g).  Derived per-graph state
// (packed columns, thresholds, cached workspaces) is dropped through graph_changed.
int64_t graph_insert_edges(Graph &g, const int32_t *src, const int32_t *dst, int64_t m, bool dev_ptrs,
                           EdgeBatch *out);
void edge_batch_free(EdgeBatch &b);
void update_scratch_free(Graph &g);
void graph_changed(Graph &g);

// ------------------------------------------------------------------- solve --

struct SolveParams {
    gde_kind kind;
    double param;      // alpha | beta | tau
    double eps;
    int precision;     // GDE_FP64 / GDE_FP32
    int hk_mode;       // 0 error-bound theta, 1 literal
    double hk_tol;
    int64_t max_rounds;
    int64_t hk_N;      // Taylor layers - 1 (HK)
    int deterministic; // sort-based scatter (dense engine)
    cudaStream_t stream;
    double gbeta;      // GDE_GPPR: b of M = D^-b A D^(b-1) (the engines run PPR on y = S r, S = max(d,1)^b)
    std::vector<double> series;  // GDE_SERIES: c_0..c_N (the layered system's coefficients)
    int katz_minus_source;       // Katz: output f_Katz = x - e_s (source entry from an FP64 word)
};

// the heat kernel and the general series share the layered engine
inline bool layered(gde_kind k) { return k == GDE_HK || k == GDE_SERIES; }
// layer-t ratio c_{t+1}/c_t and threshold scale of the layered engine
double layer_ratio(const SolveParams &p, int64_t t);
double layer_theta(const SolveParams &p, int64_t t);

// heat-kernel helpers (host)
int64_t hk_terms(double tau, double tol);
double hk_theta(double tau, int64_t N, int64_t t, int mode);

// dense single-seed engine (dense.cu)
struct DenseWork;
DenseWork *dense_work_create(Graph &g, int precision);
void dense_work_destroy(DenseWork *w);

struct RoundInfo {
    int64_t n_active;
    int64_t vol;
    double rS_l1;
    double scat;     // sum over pushed nodes of d_u w_u (mass scattered)
    double retired;  // HK: residual mass of the finished layer that was cleared
};

// begin a solve from `seed`; afterwards dense_round advances one round
void dense_begin(Graph &g, DenseWork *w, const SolveParams &p, int32_t seed);
// runs round t (w keeps t); returns |S_t| (0 = converged) and fills info
int64_t dense_round(Graph &g, DenseWork *w, const SolveParams &p, RoundInfo *info);
int64_t dense_round_index(const DenseWork *w);
// true while another round may have a non-empty active set
bool dense_pending(const DenseWork *w);
// device pointers of the current state
void *dense_x(DenseWork *w);
void dense_read(Graph &g, DenseWork *w, const SolveParams &p, void *x, void *r, int32_t *active,
                int64_t *n_active, bool device_ptrs);
// write the output vector (HK scaled by e^-tau) into dst (device pointer, n values)
void dense_output(Graph &g, DenseWork *w, const SolveParams &p, void *dst_dev);
// top-k of the current x (scaled for HK) into device buffers ids[k], vals[k]
void dense_topk(Graph &g, DenseWork *w, const SolveParams &p, int k, int32_t *ids_dev,
                void *vals_dev);

// batched engine (batched.cu)
struct BatchWork;
void batch_work_destroy(BatchWork *w);
// per-round log of the last batched solve: rows of {candidates, volume, r_S mass, ns}
int64_t batch_round_log(Graph &g, double *out, int64_t cap);

// round-to-nearest add and FP64 -> storage conversion for FP64 / FP32 state
template <typename real> __device__ __forceinline__ real radd(real a, real b);
template <> __device__ __forceinline__ double radd<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float radd<float>(float a, float b) { return __fadd_rn(a, b); }
template <typename real> __device__ __forceinline__ real from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return __double2float_rn(v); }

// standard global GD (global_gd.cu): x_out n values of p.precision
void global_gd_solve(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st);
// LocalCH for PPR (localch.cu)
void localch_solve(Graph &g, const SolveParams &p, int32_t seed, void *x_out, bool x_dev, gde_stats *st);

// C entry points: exceptions become status codes (the message is kept for gde_last_error)
#define API_BEGIN try { ::gde::clear_error();
#define API_END                                                                 \
    }                                                                           \
    catch (const ::gde::Fail &f) { return f.st; }                               \
    catch (const std::bad_alloc &) { ::gde::set_error("host allocation failed"); return GDE_ENOMEM; } \
    catch (...) { ::gde::set_error("unexpected C++ exception"); return GDE_ECUDA; } \
    return GDE_OK;

double server_clock();

// serving pool (batched.cu): slots whose solves continue across launches
struct ServePool;
ServePool *serve_pool_create(Graph &g, int32_t slots, int64_t budget, const double *eps, int ncls);
// slots whose last launch pushed more than v edges run one round per launch (v < 0: never)
void serve_pool_set_defer(ServePool *P, int64_t v);
void serve_pool_destroy(ServePool *P);
int64_t serve_pool_cap(const ServePool *P);
int64_t serve_pool_round(const ServePool *P);
int64_t serve_pool_volume(const ServePool *P);
void serve_pool_graph_changed(ServePool *P);
void serve_pool_admit(Graph &g, ServePool *P, int32_t n, const int32_t *slots, const int32_t *seeds,
                      const gde_kind *kinds, const double *params, const int32_t *cls);
void serve_pool_correct(Graph &g, ServePool *P, const EdgeBatch &eb, int32_t nres, const int32_t *res);
int64_t serve_pool_run(Graph &g, ServePool *P, int64_t rounds);
void serve_pool_pending(Graph &g, ServePool *P, unsigned *pend_host);
void serve_pool_results(Graph &g, ServePool *P, int32_t n, const int32_t *slots, int k, int32_t *ids,
                        float *vals, int32_t *status, int64_t *volume, int32_t *last_round, int64_t *support);
// the paged pool: a query slot's table is 2^order pages (serve_pool_page_slots() slots each)
// taken by serve_pool_reserve (false: no free block that large) and given back by
// serve_pool_release; order <= serve_pool_max_order()
bool serve_pool_reserve(ServePool *P, int32_t slot, int order);
void serve_pool_release(ServePool *P, int32_t slot);
int serve_pool_max_order(const ServePool *P);
int serve_pool_order(const ServePool *P, int32_t slot);
int64_t serve_pool_page_slots(const ServePool *P);
int64_t serve_pool_pages(const ServePool *P);
int64_t serve_pool_pages_used(const ServePool *P);
void batch_solve(Graph &g, const SolveParams &p, const int32_t *seeds_dev, int32_t nseeds, int k,
                 int64_t mem_budget, int32_t *ids_dev, float *vals_dev, gde_stats *stats_host,
                 int32_t *overflow_seeds_host, int32_t *n_overflow);
// batch_solve, then the seeds whose table overflowed again in smaller batches with tables of
// twice, four times, ... the slots under the same budget; those still overflowing at the
// largest table are left in overflow_seeds_host / *n_overflow.  seeds_host: the same ids.
void batch_solve_rebatch(Graph &g, const SolveParams &p, const int32_t *seeds_dev, const int32_t *seeds_host,
                         int32_t nseeds, int k, int64_t mem_budget, int32_t *ids_dev, float *vals_dev,
                         gde_stats *stats_host, int32_t *overflow_seeds_host, int32_t *n_overflow);
// batched engine stepped one round per launch, with the tables read back between rounds
struct BatchSession;
BatchSession *bsession_begin(Graph &g, const SolveParams &p, const int32_t *seeds_host, int32_t nseeds,
                             int64_t budget);
// runs the next round of every seed; returns the candidates of the round after it (0: done)
int64_t bsession_step(BatchSession *S);
gde_status bsession_read(BatchSession *S, int32_t j, float *x, double *r, int32_t *pushed, int64_t *n_pushed);
int64_t bsession_round(const BatchSession *S);
void bsession_destroy(BatchSession *S);
// top-k (x desc, id asc) of a dense float vector on the device
// (enqueued on s; the partial lists live in g.topk_part, kept between calls)
void topk_dense_f32(Graph &g, const float *x_dev, int64_t n, int k, int32_t *ids_dev, float *vals_dev,
                    cudaStream_t s);
// the two kernels of that top-k: per-block top-64 lists into `partial` (64 keys per block),
// then one block merges gridDim-many lists into the first k entries
__global__ void k_topk_dense_partial(int64_t n, const float *x, unsigned long long *partial);
__global__ void k_topk_dense_final(int64_t nparts, const unsigned long long *partial, int k,
                                   int32_t *ids, float *vals);

}  // namespace gde

struct gde_graph {
    gde::Graph g;
};
