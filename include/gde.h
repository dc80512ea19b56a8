/*
 * gde.h — C ABI of the GB300 local graph-diffusion solver.
 *
 * Computes approximate graph diffusion vectors f = sum_k c_k M^k s (Eq. 1 of
 * "Faster Local Solvers for Graph Diffusion Equations", arXiv 2410.21634) for
 * three equations of Table 1, by the parallel local diffusion process LocalGD
 * (Eq. local-gd, Section 3.3):
 *
 *   GDE_PPR   personalized PageRank, M = A D^-1, c_k = alpha (1-alpha)^k   (Eq. f-ppr)
 *   GDE_KATZ  Katz, (I - beta A) x = e_s; the Katz vector is x - e_s      (Eq. f-katz)
 *   GDE_HK    heat kernel exp(-tau (I - A D^-1)) e_s via its Taylor layers (Section 2)
 *   GDE_GPPR  generalised propagation, M = D^-b A D^(b-1), c_k = alpha (1-alpha)^k: the
 *             InstantGNN push of the appendix (b = opts.prop_beta; b = 1/2 is APPNP's
 *             D^-1/2 A D^-1/2 of Table 1, b = 0 is PPR)
 *   GDE_SERIES a general series f = sum_{k<=N} c_k (A D^-1)^k e_s with c_k > 0 given in
 *             opts.series_coef (e.g. IPR's theta^k/(theta^k+theta^10)^2 of Table 1), on the
 *             heat kernel's layered system with layer ratio c_{t+1}/c_t and threshold scale
 *             theta_t = 1/((N+1) c_0 psi_t), psi_t = sum_{j<=N-t} c_{t+j}/c_t, which bounds
 *             0 <= f_N - c_0 x <= eps d_u; the result is c_0 x
 *
 * Each round t takes the active set S_t = { u : r_u != 0, |r_u| >= theta_t eps d_u }
 * (Definition 3.1; theta_t = 1 for PPR and Katz), moves r_S into x and scatters
 * M r_S back into the residual.  The source has unit mass (r0 = e_s):
 *   PPR : x_u += alpha r_u, r_v += ((1-alpha) r_u)/d_u          (v in N(u))
 *   Katz: x_u += r_u,       r_v += beta r_u
 *   HK  : layer-t node u:  x_u += r_u, r_{t+1,v} += ((tau/(t+1)) r_u)/d_u; the last
 *         Taylor layer N (tail mass <= hk_tol) only moves its residual into x.
 *   GPPR: x_u += alpha r_u, r_v += ((1-alpha) r_u)/(d_u^(1-b) d_v^b), active iff
 *         |r_u| >= eps d_u^(1-b).  The library keeps the scaled residual y = S r with
 *         S = diag(max(d, 1)^b), on which the round is PPR's (the similarity
 *         M = S^-1 (A D^-1) S): |y_u| >= eps d_u, y_v += ((1-alpha) y_u)/d_u,
 *         x_u += (alpha y_u)/S_u, seed y_s = S_s.
 * Degree-0 nodes scatter nothing.  All work runs in this library's CUDA kernels
 * (sm_103a); there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - Return GDE_OK or an error status; gde_last_error() then describes the
 *     failure (thread-local, valid until the thread's next call).
 *   - No output is written on failure, except per-seed stats where stated.
 *   - Pointers are host pointers unless GDE_DEVICE_PTRS is set in the relevant
 *     flags; device pointers must be on the device that was current when the graph
 *     was created.  Inputs are copied; outputs are caller-allocated.
 *   - Calls on one graph are serialised by the library (a per-graph lock); use one
 *     graph per host thread for concurrency.
 */
#ifndef GDE_H
#define GDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gde_graph gde_graph;
typedef struct gde_session gde_session;

typedef enum { GDE_PPR = 0, GDE_KATZ = 1, GDE_HK = 2, GDE_GPPR = 3, GDE_SERIES = 4 } gde_kind;

typedef enum {
    GDE_OK = 0,
    GDE_EINVAL = 1,    /* bad argument or malformed CSR */
    GDE_ENOMEM = 2,    /* device or host allocation failed, or the memory budget is too small */
    GDE_ECUDA = 3,     /* a CUDA runtime error */
    GDE_ENOTCONV = 4,  /* the round cap was reached before S_t became empty */
    GDE_ETIMEOUT = 5   /* a bounded device-side wait gave up */
} gde_status;

enum {
    GDE_DEVICE_PTRS = 0x1u,      /* pointer arguments are device pointers */
    GDE_CHECK_SYMMETRIC = 0x2u   /* gde_graph_create: also verify that A = A^T */
};

enum { GDE_FP64 = 0, GDE_FP32 = 1 };

/* Solve options; gde_solve_opts_init() fills the defaults. */
typedef struct {
    int32_t precision;       /* GDE_FP64 (default) or GDE_FP32: storage and arithmetic of x and r.
                                Threshold tests and all reductions are FP64 in both. */
    int32_t deterministic;   /* 1: scatter by sort + segmented reduce (bitwise reproducible);
                                0 (default): atomic scatter */
    int32_t topk;            /* 0 (default): dense output; k > 0: the k largest x per seed */
    int32_t hk_threshold;    /* HK only.  0 (default): theta_t = e^tau/((N+1) psi_t(tau)) with
                                psi_t = sum_{j<=N-t} tau^j t!/(t+j)!, which bounds
                                0 <= f_N - e^-tau x <= eps d_u; 1: theta_t = 1 */
    int32_t batched;         /* 1: all seeds in one persistent launch with per-seed hash
                                accumulators (FP32, topk > 0; every kind: the layered ones,
                                HK and SERIES, keep one key tag per layer and x in a
                                second table: at most 253 layers up to 2^24 nodes and
                                2^(32-ceil(log2 n)) - 3 above, more is GDE_EINVAL);
                                0 (default): one seed at a time with dense x and r */
    uint32_t flags;          /* GDE_DEVICE_PTRS: seeds and outputs are device pointers */
    int64_t max_rounds;      /* round cap; 0 (default) means 1,000,000 */
    int64_t mem_budget_bytes;/* batched: bytes for the hash accumulators (12 per slot, 18 for
                                the layered kinds); 0 = automatic: up to 32 GiB for PPR and
                                the generalised propagation, up to 64 GiB for Katz and the
                                layered kinds (half the free device memory at most, 16 GiB
                                at least) */
    double hk_tol;           /* HK Taylor tail tolerance; 0 (default) means 1e-12 */
    void *cuda_stream;       /* borrowed cudaStream_t to run on; NULL = the graph's stream */
    double prop_beta;        /* GDE_GPPR: the exponent b in [0, 1] of M = D^-b A D^(b-1) */
    const double *series_coef; /* GDE_SERIES: c_0..c_N (host array, copied; all > 0) */
    int64_t series_terms;    /* GDE_SERIES: N + 1, in [1, 10^6] */
    int32_t global_gd;       /* 1: the standard (global) GD LocalGD is compared with in Section 5:
                                every node every iteration (a full SpMV), until
                                ||D^-1 r||_inf < eps; PPR and Katz on an undirected graph, dense
                                output only; stats: rounds = iterations, active_volume =
                                iterations x nnz (its operation count), resid/mass = -1 */
    int32_t chebyshev;       /* 1: LocalCH, Section 3.3's local Chebyshev method with momentum
                                on S_t, for PPR on an undirected graph (Chebyshev on
                                I - (1-alpha) D^-1/2 A D^-1/2, eigenvalues in [alpha, 2-alpha]);
                                dense output only; residuals change sign, so at exit
                                |f - x| < eps d (two-sided); resid/mass = -1 */
    int32_t katz_minus_source; /* GDE_KATZ: 1 returns the Katz vector f_Katz = x - e_s (Eq. f-katz)
                                instead of x.  The source entry x_s = 1 + (residual returned to
                                s) is kept as x_s - 1 in an FP64 word, so f_Katz,s has full
                                relative precision in FP32 too, where x_s - 1 read from an FP32
                                x_s would keep only about 6e-8 absolute.  Plain and batched
                                LocalGD; GDE_EINVAL with other kinds or methods. */
} gde_solve_opts;

/* Per-seed result statistics (Definition 3.1 and Theorem 3.5). */
typedef struct {
    int64_t rounds;          /* T: number of rounds with a non-empty S_t */
    int64_t active_volume;   /* sum_t vol(S_t): the operation count of the paper */
    int64_t pushes;          /* sum_t |S_t| */
    double resid_l1;         /* ||r^(T)||_1 (HK: summed over all Taylor layers; GPPR: of the
                                scaled residual y, with mass_l1 the matching ||S x||_1) */
    double mass_l1;          /* ||x^(T)||_1 before any output scaling */
    int32_t status;          /* gde_status of this seed */
    int32_t fallback;        /* batched seeds whose hash table overflowed: 2 when re-solved
                                in a smaller batch with larger tables (same memory budget),
                                1 when re-solved by the one-seed engine with dense state
                                (overflow at the largest table); else 0 */
} gde_stats;

void gde_solve_opts_init(gde_solve_opts *opts);

/*
 * Upload an undirected simple graph in CSR form and keep it resident in HBM.
 *   n        number of nodes (0 <= n < 2^31)
 *   offsets  n+1 int64 row offsets, offsets[0] = 0, non-decreasing
 *   cols     offsets[n] int32 column ids, each row strictly increasing, in [0, n),
 *            without self-loops (the paper assumes P_uu = 0)
 *   flags    GDE_DEVICE_PTRS, GDE_CHECK_SYMMETRIC
 * The arrays are copied and validated on the device; a violation returns
 * GDE_EINVAL.  *out receives the handle, to be released with gde_graph_destroy.
 */
gde_status gde_graph_create(int64_t n, const int64_t *offsets, const int32_t *cols,
                            uint32_t flags, gde_graph **out);

gde_status gde_graph_destroy(gde_graph *g);

/* n, number of CSR entries and maximum degree of a graph (any pointer may be NULL). */
gde_status gde_graph_info(const gde_graph *g, int64_t *n, int64_t *nnz, int32_t *max_degree);

/*
 * Copies the current CSR out: offsets (n + 1 int64) and cols (nnz int32), host arrays or,
 * with GDE_DEVICE_PTRS in flags, device arrays, allocated by the caller (sizes from
 * gde_graph_info).  Either pointer may be NULL to skip it.  Synchronous.
 */
gde_status gde_graph_csr(const gde_graph *g, int64_t *offsets, int32_t *cols, uint32_t flags);

/*
 * Edge insertion (the dynamic graphs of Section 4: G_t becomes G_{t+1} through a batch of
 * insertion events).  Inserts the m undirected edges (src[i], dst[i]): both adjacencies
 * src -> dst and dst -> src are added to the CSR, self-loops and adjacencies already present
 * are skipped (the graph stays simple; rows stay sorted), degrees follow.  src and dst are
 * host arrays, or device arrays if flags has GDE_DEVICE_PTRS; the library copies them.
 * *added (may be NULL) receives the number of directed adjacencies added.  Solves issued
 * afterwards see the new graph; solved states of earlier calls are not corrected here (a
 * server, below, corrects its resident queries).  Errors: GDE_EINVAL for m < 0, NULL arrays
 * with m > 0 or an endpoint outside [0, n) (the graph is then unchanged); GDE_ENOMEM if the
 * new arrays cannot be allocated (the graph is then unchanged).  Synchronous: returns after
 * the device CSR has been rebuilt.
 */
gde_status gde_update_edges(gde_graph *g, const int32_t *src, const int32_t *dst, int64_t m, uint32_t flags,
                            int64_t *added);

/*
 * Approximate diffusion vectors for nseeds independent unit sources.
 *   kind, param  GDE_PPR with alpha in (0,1); GDE_KATZ with beta > 0 (LocalGD terminates
 *                when beta lambda_max(A) < 1); GDE_HK with tau > 0; GDE_GPPR with alpha in
 *                (0,1) and opts->prop_beta in [0,1]; GDE_SERIES with opts->series_coef
 *                (param unused); every kind in both the plain and the batched mode
 *   eps          tolerance > 0 of the active-set test
 *   seeds        nseeds source node ids in [0, n)
 *   out_x        topk == 0: nseeds x n values, row-major (double for GDE_FP64, float for
 *                GDE_FP32): x for PPR, x = (I - beta A)^-1 e_s approximately for Katz,
 *                e^-tau x (the heat-kernel vector) for HK, c_0 x for SERIES.
 *                topk == k: nseeds x k values, largest first (ties: lower id first), and
 *                out_ids receives the matching nseeds x k node ids (-1 pads seeds whose
 *                support is smaller than k)
 *   stats        NULL or nseeds gde_stats
 * Returns GDE_ENOTCONV if some seed hit max_rounds (its output is still written).
 */
gde_status gde_solve(gde_graph *g, gde_kind kind, double param, double eps,
                     const int32_t *seeds, int32_t nseeds, const gde_solve_opts *opts,
                     void *out_x, int32_t *out_ids, gde_stats *stats);

/*
 * Kernel timing, for benchmarks.  While enabled on a graph, every solve on it records CUDA
 * events on its stream around the round kernels; gde_profile_read synchronises, sums the
 * elapsed times and the work counters since the last gde_profile_enable, and resets nothing.
 */
typedef struct {
    double batch_rounds_ms;      /* persistent batched round kernel (frontier + scatter) */
    double batch_clear_ms;       /* batched: accumulator pool reset */
    double batch_topk_ms;        /* batched: per-seed top-k */
    double dense_frontier_ms;    /* single-seed frontier kernels */
    double dense_push_ms;        /* single-seed push/scatter kernels */
    int64_t batch_launches;      /* persistent launches timed */
    int64_t dense_rounds;        /* single-seed rounds timed */
    int64_t edges;               /* sum of vol(S_t) over the timed work */
    int64_t pushes;              /* sum of |S_t| over the timed work */
    int64_t support;             /* batched: sum over seeds of |supp(x)| */
    int64_t rounds;              /* batched: rounds of the persistent loop */
    int64_t launches;            /* kernels this library launched */
} gde_profile;

gde_status gde_profile_enable(gde_graph *g, int enable);
gde_status gde_profile_read(gde_graph *g, gde_profile *out);

/*
 * Per-round record of the last batched solve on g (Definition 3.1 per round, all seeds
 * together): out receives up to cap rows of 7 doubles {candidates |C_t|, vol(S_t),
 * ||r_S||_1, device ns from the start of the persistent launch to the end of the round,
 * ns to the end of the round's frontier phase, the scatter phase's warp busy time summed
 * over warps (ns), the longest warp's busy time (ns)}; *rounds receives the number of
 * rounds (may exceed cap).
 */
gde_status gde_profile_rounds(gde_graph *g, double *out, int64_t cap, int64_t *rounds);

/*
 * Launch shape of the push (degree bins): nodes with d <= t1 are pushed by one
 * thread, t1 < d <= t2 by one warp, d > t2 in merge-path chunks of `chunk` edges over the
 * concatenated hub adjacency; blocks_per_sm sets the persistent grid (0 = the occupancy
 * limit); schedule orders the batched scatter: 1 hands hub chunks to warps in bin order (the
 * bins are laid out seed by seed, so the warps in flight share a few seeds' tables in L2), 2
 * additionally orders medium and small entries, 3 strides every bin statically, 4 scatters
 * the bins seed by seed (a seed's table enters L2 once per round, its hub slab streamed in
 * ahead; schedule values are stored minus one; 0 keeps the current setting).  Values <= 0
 * keep the current
 * setting.  Applies to later solves on g.
 */
typedef struct {
    int32_t t1;
    int32_t t2;
    int32_t chunk;
    int32_t blocks_per_sm;
    int32_t schedule;
    int32_t hub_degree;  /* batched PPR / Katz / generalised propagation: targets of degree >=
                            hub_degree keep their residual in a dense per-seed fixed-point slab
                            (one integer atomic add per edge, exact sums) instead of the FP32
                            hash tables; at 160 (the default) no FP32 entry receives more than
                            159 additions per round, so each stays within 159 * 2^-24 < 1e-5
                            relative of its exact sum.  Degrees above the graph's exact degree
                            codes (224 up to 2^24 nodes) round up to a power of two.  -1 turns
                            the slab off; 0 keeps the current setting.  The slab needs
                            nseeds * (table slots + hubs) <= 2^32 and 12 bytes per seed and hub
                            (at most 16 GiB), else the solve runs without it. */
} gde_tuning;

gde_status gde_set_tuning(gde_graph *g, const gde_tuning *t);
gde_status gde_get_tuning(const gde_graph *g, gde_tuning *t);

/*
 * Autotuner of the batched push: one pass of coordinate descent over t1, t2, chunk,
 * schedule, blocks_per_sm and (unless the slab is off) hub_degree in {64, 128, 160} (in that
 * order; each tried over a fixed candidate list with the others held), timing batched solves
 * of `seeds` (any kind the batched engine serves, kind/param/eps/opts as for gde_solve;
 * opts->topk in [1,64], batched forced on, FP32) with CUDA events on the solve stream, the
 * fastest of two timed runs per candidate.  The best tuning is applied to g as by
 * gde_set_tuning and, if best is not NULL, returned; *best_ms (may be NULL) receives its time.
 * Allocates its own device buffers; results of the timed solves are discarded.
 */
gde_status gde_autotune(gde_graph *g, gde_kind kind, double param, double eps, const int32_t *seeds,
                        int32_t nseeds, const gde_solve_opts *opts, gde_tuning *best, double *best_ms);

/*
 * Top-k of a dense float vector that allocates no device memory (no counterpart in the
 * paper: an interface for callers that cannot allocate).  Some callers cannot call
 * cudaMalloc: an application that has already handed all device memory to its own pool
 * allocator, a serving loop that must not take the allocator's device-wide lock or
 * implicit synchronisation between requests, or a host that only lets this library touch
 * memory it was given.  This entry point runs the same two top-k kernels as gde_solve's
 * topk output, with their per-block partial lists kept in a fixed scratch array inside the
 * library (GDE_TOPK_NOALLOC_SCRATCH_BYTES = 256 KiB of device memory per GPU, held from the
 * library's loading until process exit) instead of a buffer from cudaMalloc.
 *   x          device pointer, n floats (n in [1, 2^31 - 1]); only entries > 0 are ranked
 *   k          1 <= k <= 64 (GDE_TOPK_NOALLOC_MAX_K); other values return GDE_EINVAL
 *   out_ids    device pointer, k ids: largest x first, ties by lower id, -1 past the support
 *   out_vals   device pointer, k floats (0 past the support)
 *   cuda_stream  cudaStream_t to launch on (NULL: the legacy default stream); the call does
 *              not synchronise: results are ready when the stream reaches this point
 * The first call on a device looks up that device's scratch address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture.  All calls on a
 * device share the one scratch array: calls whose kernels overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  Every call rewrites the
 * scratch it reads, so nothing carries over from a previous call.
 */
#define GDE_TOPK_NOALLOC_MAX_K 64
#define GDE_TOPK_NOALLOC_SCRATCH_BYTES (512 * 64 * 8)
gde_status gde_topk_f32_noalloc(const float *x, int64_t n, int32_t k, int32_t *out_ids,
                                float *out_vals, void *cuda_stream);

/*
 * Random-access calibration of device memory (no counterpart in the paper: a second
 * roofline denominator for the batched scatter, whose cost is set by random 32-byte accesses,
 * not by streaming bandwidth).  Launches one untimed and `reps` timed kernels in which each
 * access picks a pseudo-random 32-byte sector of buf (splitmix64 of the access index, a
 * different salt per launch) and, by mode:
 *   0  reads the sector (two 16-byte loads that bypass L1, as the scatter's probe does),
 *   1  reads it, then atomically adds 1.0f to an FP32 word in it (the insert-or-add pattern),
 *   2  atomically adds 1.0f to an FP32 value in it without reading it first,
 *   3  the same add with its result unused (a reduction: nothing returns to the SM),
 *   4  atomically adds 1 to its first 64-bit integer (the hub-slab insert), result used,
 *   5  the same 64-bit add with its result unused.
 *   buf        device pointer, 256-byte aligned; its contents are zeroed and then overwritten
 *   bytes      size of buf (>= 64); the probe uses the largest power-of-two number of sectors
 *              that fits, so pass a buffer well above the L2 size to measure device memory
 *   nops       accesses per launch (>= 1)
 *   grid       blocks of 256 threads, 1 .. 65535
 *   reps       timed launches, 1 .. 1000
 *   l2_fetch_bytes  0 leaves the context's L2 fetch-granularity limit
 *              (cudaLimitMaxL2FetchGranularity) alone; 32, 64 or 128 set it for the probe, and
 *              the previous value is restored before returning
 *   cuda_stream  cudaStream_t to launch on (NULL: the legacy default stream)
 *   ms_out     receives the mean duration of one timed launch (CUDA events on cuda_stream)
 * Synchronises cuda_stream.  Other arguments out of range return GDE_EINVAL.
 */
gde_status gde_probe_random_access(void *buf, uint64_t bytes, int64_t nops, int32_t mode, int32_t grid,
                                   int32_t reps, int32_t l2_fetch_bytes, void *cuda_stream, double *ms_out);

/*
 * Fault injection for failure-detection tests (no counterpart in the paper).  Nothing faults,
 * traps or hangs on the device: a failure is injected on the host, or a bounded device-side
 * wait is made to run out, and the call reports a status while the context stays usable.
 *   gde_test_fail_alloc     the nth device allocation of this library from now on (any thread)
 *                           fails as cudaMalloc's out-of-memory would: the call that makes it
 *                           returns GDE_ENOMEM and writes no output; 0 disarms, nth < 0 is
 *                           GDE_EINVAL.  Process-wide; for tests only.
 *   gde_test_barrier_fault  later batched launches on g (solves, stepping sessions, servers)
 *                           wait at most limit_ns at each grid barrier of the persistent round
 *                           kernel (0: the default, 20 s), and block `block` of the launch leaves
 *                           at its barrier number `barrier` (0 = first) without arriving, as a
 *                           block that died would; the others' waits run out and the call
 *                           returns GDE_ETIMEOUT.  block < 0 turns the fault off.
 */
gde_status gde_test_fail_alloc(int64_t nth);
gde_status gde_test_barrier_fault(gde_graph *g, int64_t limit_ns, int32_t block, int32_t barrier);

/* Thread-local description of the last failure of this thread ("" if none). */
const char *gde_last_error(void);

/*
 * Stepping interface (one LocalGD round per call), used to compare the device state
 * with the CPU oracle round by round.  Dense state, one seed, opts->precision honoured.
 *   gde_session_begin   x = 0, r = e_seed (HK: layer 0)
 *   gde_session_step    runs round t; *n_active receives |S_t| (0: converged, nothing done)
 *   gde_session_read    copies x (n values), r (n values: the current residual, for HK the
 *                       current layer) and S_t of the last step (ascending ids, *n_active
 *                       entries; active may hold n ints) into host buffers, or device
 *                       buffers if opts->flags had GDE_DEVICE_PTRS; any pointer may be NULL
 */
gde_status gde_session_begin(gde_graph *g, gde_kind kind, double param, double eps, int32_t seed,
                             const gde_solve_opts *opts, gde_session **out);
gde_status gde_session_step(gde_session *s, int64_t *n_active);
gde_status gde_session_read(gde_session *s, void *x, void *r, int32_t *active, int64_t *n_active);
gde_status gde_session_end(gde_session *s);

/*
 * Batched stepping interface: one round of the batched engine per call, for every seed of a
 * batch at once (Eq. local-gd, Section 3.3, run for all seeds together), with the per-seed
 * hash tables copied to the host between rounds, so that the batched engine can be compared
 * with the CPU oracle round by round.  It launches the persistent round kernel of
 * gde_solve's batched mode with a one-round cap, from the state the previous launch left.
 *   kind, param, eps, opts  as for gde_solve's batched mode: opts->precision must be GDE_FP32;
 *                hk_threshold, hk_tol, prop_beta, series_coef are honoured;
 *                opts->mem_budget_bytes sizes the tables (0: 4 GiB; at most 2n slots a table)
 *   seeds        nseeds >= 1 node ids in [0, n), a host array (GDE_DEVICE_PTRS: GDE_EINVAL)
 *   gde_bsession_begin  x = 0, r = e_s (the heat kernel and series: layer 0) for every seed
 *   gde_bsession_step   runs the next round t of every seed; *n_candidates (may be NULL)
 *                       receives the candidates of round t + 1, all seeds together (0: every
 *                       active set is empty and further steps change nothing)
 *   gde_bsession_read   seed index j in [0, nseeds): x (n floats: the engine's x before any
 *                       output scaling), r (n doubles: the residual, for the heat kernel and
 *                       series the layer the next round reads; FP32 table entries widened
 *                       exactly, hub-slab entries as their fixed-point values) as of the
 *                       last step, and the
 *                       node ids the last step pushed (S_t of seed j, unordered, up to n ints;
 *                       *n_pushed receives how many); host buffers, any pointer may be NULL.
 *                       Returns GDE_ENOMEM when that seed's table overflowed (its state is
 *                       then incomplete).
 * The session owns its device workspace (the graph's cached batched workspace is not
 * touched) and borrows the graph, which must outlive it and must not change while it runs
 * (a step after an edge insertion returns GDE_EINVAL).  Every step synchronises and copies
 * the whole pool (12 bytes per table slot, 18 for the layered kinds) to the host: a testing
 * interface, not a fast path.  gde_bsession_end releases everything (NULL is a no-op).
 */
typedef struct gde_bsession gde_bsession;
gde_status gde_bsession_begin(gde_graph *g, gde_kind kind, double param, double eps, const int32_t *seeds,
                              int32_t nseeds, const gde_solve_opts *opts, gde_bsession **out);
gde_status gde_bsession_step(gde_bsession *s, int64_t *n_candidates);
gde_status gde_bsession_read(gde_bsession *s, int32_t seed_index, float *x, double *r, int32_t *pushed,
                             int64_t *n_pushed);
gde_status gde_bsession_end(gde_bsession *s);

/*
 * Serving (continuous batching of PPR and Katz queries on a graph that receives edge
 * insertions; the dynamic setting of Section 4).  A server owns up to `slots` resident
 * queries, each with a hash table of FP32 x and r in device memory, taken from a pool of
 * mem_budget_bytes (default 16 GB; 20 bytes per table slot: key and residual 8, x 4, x-list 8).
 * The pool is cut into pages of 2^16 table slots (fewer for graphs with n < 2^15); a query's
 * table is a power-of-two run of pages (a buddy allocator), at most 2n slots.  Queries are
 * admitted in arrival order while a slot and their table fit, so the number resident at once
 * follows their memory, not a fixed count.  A new query's table starts at the largest size
 * that the last 16 answered queries of its kind, tolerance class and seed-degree bucket
 * (floor(log2(d_s + 1))) needed to hold their keys at an eighth load (the nearest lower bucket's
 * when its own has none yet; one page at first); a query whose table overflows is started
 * again, ahead of the queue and with its arrival time kept, with a table four times larger (up
 * to the largest), and only overflowing the largest table answers GDE_ENOMEM.
 *   gde_server_submit        queues a query (qid chosen by the caller; kind GDE_PPR with
 *                            param = alpha in (0,1), or GDE_KATZ with param = beta > 0;
 *                            eps_class picks one of the server's tolerances; flags
 *                            GDE_SERVE_TRACK keeps the answered query resident as a standing
 *                            query that is corrected and re-answered after every edge batch
 *                            (until its slot is needed), without it the slot is released at
 *                            the first answer; t_submit is the arrival time on
 *                            gde_server_clock, < 0 for now).  Returns at once.
 *   gde_server_insert_edges  queues an edge-insertion batch (copied); applied at the next step.
 *   gde_server_step          one device step: applies the queued edge batches to the graph
 *                            (as gde_update_edges) and corrects every resident query's state
 *                            for them (the Insert of Algorithm 3: x_u rescaled, r moved along
 *                            the new adjacencies; Katz: r_v += beta x_u), so it resumes from
 *                            there instead of from its seed; admits queued queries into free
 *                            slots (then into the slots of standing queries answered longest
 *                            ago) in arrival order; runs at most rounds_per_step LocalGD rounds of all resident
 *                            queries in one persistent launch; and emits the top-k of every
 *                            query that has no active node left (first answer, or an update
 *                            after an edge batch).  *running and *queued (may be NULL) receive
 *                            the queries still running and still waiting.
 *   gde_server_poll          moves up to cap emitted results into out (oldest first).
 * Results: ids/vals hold the k largest x entries (x desc, id asc; -1 pads), x approximates
 * f_PPR, or (I - beta A)^-1 e_s for Katz, within the eps bound of Corollary 3.6 on the graph
 * as of the step that emitted it; t_done - t_submit is the latency (for an update: from the
 * step that applied the edge batch).  status GDE_ENOMEM: the query's table filled up (its
 * slot is released).  submit / insert_edges / poll / info may be called from other threads
 * while a step runs; steps are serialised; destroy must not overlap any other call on the
 * server.  Errors as elsewhere (GDE_EINVAL for bad arguments; a step
 * that fails leaves the server unusable and reports the failure).
 */
typedef struct gde_server gde_server;

#define GDE_SERVE_TRACK 1u  /* gde_server_submit: keep the query as a standing query */

typedef struct {
    int32_t slots;            /* resident queries at most (default 256) */
    int32_t rounds_per_step;  /* LocalGD rounds per device step (default 4) */
    int32_t topk;             /* entries per result, 1..64 (default 64) */
    int32_t n_eps;            /* tolerance classes, 1..4 (default 1) */
    double eps[4];            /* their tolerances (default eps[0] = 1e-6) */
    int64_t mem_budget_bytes; /* table pool bytes (20 per table slot), 0 = 16 GB */
    int64_t defer_volume;     /* a query whose last step pushed more edges than this runs one
                                 round per step (its rounds are unchanged, only spread out) so
                                 the other queries' rounds in a step are not each held up by
                                 its scatter; 0 = 2^23, < 0 = never */
} gde_server_opts;

typedef struct {
    uint64_t qid;
    int32_t status;           /* GDE_OK or GDE_ENOMEM */
    int32_t update;           /* 0: first answer, 1: refreshed after an edge batch */
    int32_t k;
    int32_t slot;
    int64_t volume;           /* edges pushed for this query so far */
    double t_submit, t_done;  /* gde_server_clock seconds */
    int32_t ids[64];
    float vals[64];
} gde_server_result;

typedef struct {
    int32_t slots, running, answered, queued;
    int64_t steps;            /* device steps so far */
    int64_t rounds;           /* LocalGD rounds run by the pool so far */
    int64_t edge_batches;     /* insertion batches applied */
    int64_t cap;              /* hash slots of the largest query table */
    int64_t volume;           /* edges pushed by the pool so far (all queries, all rounds) */
    double t_graph;           /* seconds spent in steps on: graph updates (CSR rebuild), */
    double t_correct;         /*   warm-start corrections of resident queries, */
    double t_admit;           /*   admissions, */
    double t_rounds;          /*   LocalGD rounds (the persistent launches), */
    double t_results;         /*   convergence checks and top-k of answered queries */
    int64_t pool_pages;       /* pages of the table pool (the memory budget) */
    int64_t pages_used;       /* pages held by resident queries now */
    int64_t page_slots;       /* table slots per page */
    int32_t peak_resident;    /* most queries resident at once so far */
    int32_t pad;
    int64_t readmissions;     /* queries started again with a larger table after an overflow */
    int64_t evictions;        /* standing queries whose slot or pages went to new queries */
    int64_t peak_pages;       /* most pages held by resident queries at once so far */
} gde_server_info_t;

void gde_server_opts_init(gde_server_opts *o);
double gde_server_clock(void);  /* steady clock, seconds */
gde_status gde_server_create(gde_graph *g, const gde_server_opts *opts, gde_server **out);
gde_status gde_server_destroy(gde_server *s);
gde_status gde_server_submit(gde_server *s, uint64_t qid, gde_kind kind, double param, int32_t eps_class,
                             int32_t seed, uint32_t flags, double t_submit);
gde_status gde_server_insert_edges(gde_server *s, const int32_t *src, const int32_t *dst, int64_t m);
gde_status gde_server_step(gde_server *s, int32_t *running, int32_t *queued);
gde_status gde_server_poll(gde_server *s, gde_server_result *out, int32_t cap, int32_t *n);
gde_status gde_server_info(gde_server *s, gde_server_info_t *info);

#ifdef __cplusplus
}
#endif

#endif /* GDE_H */
