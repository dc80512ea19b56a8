// Batched LocalGD: many independent unit sources in one persistent launch (Eq. local-gd,
// Section 3.3, run for every seed at once), FP32 x and r in per-seed open-addressed hash
// tables in HBM, top-k output per seed.
//
// Layout (pool of P = nseeds * cap slots, cap a power of two):
//   kr[slot]  64-bit word {low: key, high: r as float bits}; key and residual share one
//             8-byte word, so a probe and the atomic add on r touch the same 32-byte sector.
//             key = node id | epoch tag << idbits; a slot whose tag is not the current
//             solve's (or 0xFFFFFFFF) is empty, so tables need no reset between solves
//   xs[slot]  float x of that node (zero outside the current solve's x-lists)
//   xlist     per seed, the slots whose x became nonzero (appended on first activation),
//             with each one's node id beside it (xnode); the top-k reads only these and
//             zeroes their x
// seed j owns slots [j*cap, (j+1)*cap); a slot index therefore names its seed (slot >> log2cap).
// thr32[v] = fl(eps d_v) rounded up to float (one array per tolerance class, all seeds).
// The layered kinds (heat kernel, series) give each layer its own key tag and keep x in a
// second per-seed table (xkr / xxs), since a layer's slots are reused by the next layer.
//
// Rounds run inside one cooperative kernel: phase A1 builds S_t for every seed from the
// candidate list (slots whose residual crossed its threshold in the previous round), zeroes
// r on S_t, adds to x and records the pushes; phases S and A2 count, scan and place them by
// degree bin, seed by seed, into lists pooled over all seeds (skipped in small rounds, which
// scatter straight from the records); phase B scatters every push into its seed's table
// (insert-or-add) and appends threshold crossings to the next candidate list.  Grid
// barriers separate the phases; every wait is bounded by a time limit after which the
// kernel records GDE_ETIMEOUT and returns.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace gde {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kTopMax = 64;
constexpr int kBHubVolBits = 40;
constexpr unsigned long long kBHubVolMask = (1ull << kBHubVolBits) - 1;
constexpr unsigned long long kBarrierLimitNs = 20ull * 1000 * 1000 * 1000;  // 20 s

enum : int { kSeedOk = 0, kSeedOverflow = 1 };

constexpr int kMaxCls = 4;  // tolerance classes one launch can mix (per-slot eps)

// Per-slot solve parameters, for launches that mix queries (a server's slots): x += cx rho,
// share = coef rho (divided by d_u when divide != 0), tolerance class cls.
struct SlotParam {
    double cx;
    double coef;
    int32_t divide;
    int32_t cls;
    uint32_t tag;    // the slot's key tag (shifted above the id bits): a server retags a slot
                     // for every query, so the previous query's keys read as free
    uint32_t flags;  // kSlotDefer: the slot runs only the first round of a launch
    uint64_t base;   // the slot's table: slots [base, base + 2^log2cap) of the paged pool, whose
    uint32_t log2cap;  // x-list occupies the same range of the x-list arrays
    uint32_t pad;
};

// A slot whose last launch pushed many edges (a query in its heavy rounds) runs one round
// per launch and passes its candidates on unchanged in the launch's later rounds, so the
// other slots' rounds in that launch are not each held up by its scatter.  Its own rounds
// are unchanged, only spread over more launches.
constexpr uint32_t kSlotDefer = 1u;

struct BCtl {  // per-round counters (one set per round parity)
    unsigned long long hub_packed;
    unsigned int cnt_small;
    unsigned int cnt_med;
    unsigned int cand_out;
    unsigned int n_active;
    unsigned long long vol;
    double rS_l1;
    unsigned int overflow;
    unsigned int pad;
    // scatter work handed out in order (hub chunks, medium entries, small groups), so the
    // warps in flight cover a narrow, seed-local window of the bins
    unsigned long long hub_next;
    unsigned int med_next;
    unsigned int small_next;
    // seed-grouped order: work units of all three bins, group by group
    unsigned long long unit_next;
    unsigned long long units_total;
    unsigned int dmax_push;  // largest degree pushed this round
    unsigned int pad2;
};

// A round with at most kDirectCand candidates, none of degree above kDirectMaxDeg, skips the
// seed-ordered binning (two grid barriers and a one-block scan): each warp scatters whole
// push records straight from the frontier's output.  The tail of a solve is dozens of such
// rounds, where the fixed cost of the binning outweighs its locality.
#ifndef GDE_DIRECT_CAND_LOG2
#define GDE_DIRECT_CAND_LOG2 15
#endif
#ifndef GDE_DIRECT_DEG_LOG2
#define GDE_DIRECT_DEG_LOG2 12
#endif
constexpr unsigned kDirectCand = 1u << GDE_DIRECT_CAND_LOG2;
constexpr unsigned kDirectMaxDeg = 1u << GDE_DIRECT_DEG_LOG2;

#ifndef GDE_SEED_GROUP
#define GDE_SEED_GROUP 1
#endif
constexpr int kSeedGroup = GDE_SEED_GROUP;  // seeds whose bins are scattered together (schedule 3)

struct BGlobal {
    BCtl ctl[2];
    unsigned int bar_count;
    unsigned int bar_gen;
    unsigned int error;       // 0, or a gde_status
    unsigned int rounds;      // rounds executed
    unsigned long long total_vol;
    unsigned long long total_pushes;
};

struct RoundLog {
    unsigned long long n_active;
    unsigned long long vol;
    double rS_l1;
    unsigned long long ncand;
    unsigned long long t_ns;   // device time at the end of the round
    unsigned long long tA_ns;  // device time at the end of phase A (S_t built)
    unsigned long long busy_sum_ns;  // phase B: sum over warps of their busy time
    unsigned long long busy_max_ns;  // phase B: the longest warp
};

constexpr int kLogCap = 4096;

struct BatchWork {
    int64_t nseeds_cap = 0;
    int64_t cap = 0;        // slots per seed
    int log2cap = 0;
    int64_t pool = 0;       // nseeds_cap * cap
    int64_t list_cap = 0;   // candidate / bin capacity
    unsigned long long *kr = nullptr;
    float *xs = nullptr;
    float *thr32 = nullptr;
    int64_t thr_n = 0;
    double thr_eps = -1.0;
    uint32_t *cand[2] = {nullptr, nullptr};
    int64_t *b_beg[3] = {nullptr, nullptr, nullptr};
    int32_t *b_deg[3] = {nullptr, nullptr, nullptr};
    float *b_w[3] = {nullptr, nullptr, nullptr};
    int32_t *b_seed[3] = {nullptr, nullptr, nullptr};
    int64_t *hub_vstart = nullptr;
    uint32_t *hub_cstart = nullptr;  // first hub push of each scatter chunk (kHubChunkTab entries)
    unsigned long long *grp_units = nullptr, *grp_off = nullptr;  // per seed group (schedule 3)
    // per-candidate push record of the round (frontier phase -> placement phase)
    int64_t *tmp_beg = nullptr;
    int32_t *tmp_deg = nullptr;
    float *tmp_w = nullptr;
    uint32_t *tmp_jb = nullptr;      // seed | bin << 30
    // per-(bin, seed) segment counts, offsets and cursors of the seed-ordered bins
    unsigned *seg_cnt = nullptr;     // 3 * nseeds
    unsigned *seg_off = nullptr;     // 3 * nseeds
    unsigned *seg_cur = nullptr;     // 2 * nseeds
    unsigned long long *seg_hvol = nullptr;  // nseeds: hub volume per seed
    unsigned long long *vol_off = nullptr;   // nseeds
    unsigned long long *seg_hcur = nullptr;  // nseeds: packed (count << 40) | volume cursor
    int32_t *seeds = nullptr;        // device copy of the seed ids
    int32_t *status = nullptr;       // per seed
    unsigned *inserts = nullptr;     // per seed
    unsigned long long *svol = nullptr;  // per seed
    unsigned *spushes = nullptr;     // per seed
    int32_t *slast = nullptr;        // per seed: last round with a push
    double *spush = nullptr;         // per seed: sum of pushed residual mass (FP64)
    double *sscat = nullptr;         // per seed: sum of scattered mass d_u w_u (FP64)
    double *smass0 = nullptr;        // per seed: the source's residual (1, or S_s when scaled)
    uint32_t *xlist = nullptr;       // per seed: xcap slots whose x is nonzero
    uint32_t *xnode = nullptr;       // the node of each x-list entry (the top-k reads no key word)
    unsigned *xcnt = nullptr;        // per seed: x-list length (may exceed xcap: overflow)
    int64_t xcap = 0;
    BGlobal *glob = nullptr;
    RoundLog *log = nullptr;
    int grid = 0;    // co-resident blocks of the persistent kernel
    int sms = 0;
    int64_t last_rounds = 0;
    bool need_clear = true;   // reset every table before the next solve
    bool list_overflowed = false;  // the last solve ran out of candidate / bin list entries
    // layered solves: per-seed x tables (keys in the low half of xkr, values in xxs) and the
    // per-round threshold and share coefficients
    unsigned long long *xkr = nullptr;
    float *xxs = nullptr;
    int64_t xt_seeds = 0, xt_cap = 0;
    int xt_log2cap = 0;
    double *layer_eps = nullptr, *layer_coef = nullptr;
    int64_t layer_cap = 0;
    uint32_t epoch = 0;       // tag of the current solve's keys
    // hub slab: per seed, H fixed-point residuals (value = count * 2^qexp) and H float x values
    unsigned long long *slab = nullptr;
    float *slab_x = nullptr;
    int64_t slab_seeds = 0, slab_H = 0;  // capacity: seeds (per bank) and hubs a seed
    int slab_banks = 0;                  // capacity: banks
    bool slab_x_dirty = true;  // slab_x must be zeroed before the next solve
    bool slab_dirty = true;    // slab counts must be zeroed before the next solve
    double *xsrc = nullptr;    // Katz with f_Katz output: per seed x_s - 1 in FP64
    bool slab_on = false;      // the last set-up used the slab
    // the counts of a PPR or Katz solve are dead once its round kernel has finished: they are
    // zeroed on a side stream that overlaps the solve's top-k and read-back, and the next
    // set-up waits for z_done on its own stream
    cudaStream_t zs = nullptr;
    cudaEvent_t z_start = nullptr, z_done = nullptr;
    bool z_pending = false;
    uint32_t slab_base = 0;
    int qexp = 0;
};

// ------------------------------------------------------------- device bits --

__device__ __forceinline__ uint32_t mix32(uint32_t v) {
    // murmur3 finaliser
    v ^= v >> 16;
    v *= 0x85EBCA6Bu;
    v ^= v >> 13;
    v *= 0xC2B2AE35u;
    v ^= v >> 16;
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float *r_of(unsigned long long *kr, uint64_t slot) {
    return reinterpret_cast<float *>(kr + slot) + 1;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Returns false if the
// wait exceeded the time limit (limit_ns) or another block recorded an error; the caller then
// returns.  Fault injection for tests: the block fail_block leaves the kernel at its
// fail_barrier-th barrier (counted from 0 in *nbar) without arriving, as a block that died
// would; the others' bounded waits then run out and the launch reports GDE_ETIMEOUT.
__device__ bool grid_sync(BGlobal *g, unsigned nblocks, unsigned long long limit_ns, int fail_block,
                          int fail_barrier, int *nbar) {
    const int k = (*nbar)++;
    if ((int)blockIdx.x == fail_block && k == fail_barrier) return false;
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(&g->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&g->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&g->bar_count, 0u);
            __threadfence();
            atomicAdd(&g->bar_gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer();
            while (ld_acquire_u32(&g->bar_gen) == gen) {
                if (ld_acquire_u32(&g->error) != 0) { ok = 0; break; }
                if (globaltimer() - t0 > limit_ns) {
                    atomicCAS(&g->error, 0u, (unsigned)GDE_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_acquire_u32(&g->error) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T> __device__ __forceinline__ T bwarp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct BArgs {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *colp;   // packed columns (id | degree code << idbits), or NULL
    int idbits;
    uint32_t idmask;
    int code_exact;         // codes below this are exact degrees; from it on, log2 classes
    double eps;              // tolerance of class 0
    double eps_cls[kMaxCls]; // tolerance of each class
    int ncls;
    const float *thr32;      // ncls arrays of n thresholds, thr_stride apart
    int64_t thr_stride;
    const SlotParam *sparam; // per-slot parameters, or NULL: kind/cx/coef below, class 0
    int64_t t0;              // first round of this launch (a resumed launch continues t)
    uint32_t key_idmask;    // node-id bits of a table key
    uint32_t key_tag;       // this solve's epoch tag, already shifted above the id bits
    uint32_t *xlist;
    uint32_t *xnode;
    unsigned *xcnt;
    unsigned xcap;
    double *spush;
    double *sscat;
    unsigned long long *kr;
    float *xs;
    int log2cap;
    uint32_t mask;
    int32_t nseeds;
    int32_t *status;
    unsigned *inserts;
    unsigned load_limit;
    unsigned long long *svol;
    unsigned *spushes;
    int32_t *slast;
    uint32_t *cand[2];
    unsigned list_cap;
    int64_t *b_beg[3];
    int32_t *b_deg[3];
    float *b_w[3];
    int32_t *b_seed[3];
    int64_t *hub_vstart;
    uint32_t *hub_cstart;
    int64_t *tmp_beg;
    int32_t *tmp_deg;
    float *tmp_w;
    uint32_t *tmp_jb;
    unsigned *seg_cnt;
    unsigned *seg_off;
    unsigned *seg_cur;
    unsigned long long *seg_hvol;
    unsigned long long *vol_off;
    unsigned long long *seg_hcur;
    BGlobal *glob;
    RoundLog *log;
    int kind;
    double cx;    // x += cx * rho
    double coef;  // PPR 1-alpha (share divided by d_u), Katz beta
    double gbeta; // generalised propagation: x += (cx * rho) / max(d_u, 1)^gbeta (0: none)
    int64_t max_rounds;
    int32_t t1, t2, chunk;
    int32_t schedule;   // 0: all bins handed out in order; 1: hubs in order, others strided; 2: all strided;
                        // 3: group by group of kSeedGroup seeds, each group's hubs, medium and small
                        // entries together, so a seed's table is brought into L2 once per round
    unsigned long long *grp_units;  // per seed group: its work units (schedule 3)
    unsigned long long *grp_off;    // their exclusive prefix sums
    unsigned *pend;     // not NULL: receives per seed the candidates left for the next launch
    uint32_t *pushed;   // not NULL (stepping sessions): per candidate of the round, 1 if it was pushed
    // paged pool (a server; NULL otherwise): slot ids name their query through the owner of
    // their page, page_owner[slot >> pg_bits], instead of slot >> log2cap
    const int32_t *page_owner;
    int pg_bits;
    // test fault injection: grid-barrier wait limit (0: kBarrierLimitNs) and a block that leaves
    // at one barrier without arriving (fail_block < 0: none)
    unsigned long long bar_limit_ns;
    int32_t fail_block;
    int32_t fail_barrier;
    // hub slab (non-layered kinds without per-slot parameters; slab == NULL: off).  A column
    // word whose degree code is >= hub_code names a hub by its rank (colq); the hub's residual
    // of seed j is the fixed-point integer slab[j * H + rank] (value = count * 2^qexp: sums of
    // integers are exact and take one atomic add, with no probe), its x slab_x[j * H + rank].
    // Candidate and x-list ids at or above slab_base name slab entries (slab_base + j * H + rank).
    unsigned long long *slab;
    float *slab_x;
    int64_t H;
    uint64_t slab_bank;   // entries per bank (nseeds * H); the layered kinds keep two banks,
                          // round t reading layer t from bank t & 1 and writing bank (t + 1) & 1
    uint32_t slab_base;
    uint32_t hub_code;
    const int32_t *hub_node;
    const int32_t *hub_deg;
    int qexp;
    // Katz with f_Katz output (xsrc not NULL): x_s - 1 of seed j in FP64 in xsrc[j] (starts at -1
    // and gains every residual pushed at the seed s = seed_ids[j])
    double *xsrc;
    const int32_t *seed_ids;
    float wscale;    // 2^-qexp: a float share times it is its count (exact scaling)
    double vscale;   // 2^qexp: a count times it is its value
    double tscale;   // 2^-qexp
    // layered kinds (heat kernel, general series): round t reads layer t and writes layer t+1;
    // the keys of layer t carry key_tag + t * tag_step, so a layer's keys read as free slots
    // once the next layer is written, and x lives in a separate per-seed table keyed by node
    const double *layer_eps;   // theta_t eps of round t, t = 0 .. nlayers
    const double *layer_coef;  // share coefficient of round t (divided by d_u)
    int64_t nlayers;           // rounds t < nlayers scatter; round nlayers only adds to x
    uint32_t tag_step;
    unsigned long long *xkr;   // x table: keys in the low half of each word
    float *xxs;                // x table: values
    int xlog2cap;
    uint32_t xmask;
};

__device__ __forceinline__ void bappend(unsigned *counter, uint32_t *list, uint32_t v, unsigned cap,
                                        unsigned *overflow) {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned)g.size());
    const unsigned i = g.shfl(base, 0) + g.thread_rank();
    if (i < cap) list[i] = v; else atomicOr(overflow, 1u);
}

// a probe run this long means the table is effectively full (at <= 3/4 load a run of 64
// full buckets is vanishingly rare); the seed is then re-solved with dense state
constexpr uint32_t kMaxProbe = 256;
constexpr int kStage = 256;            // staged candidates per warp (shared memory)
constexpr int kMedGrab = 4;            // medium-degree entries a warp takes per grab
constexpr int64_t kHubChunkTab = (int64_t)1 << 22;  // chunks whose first push is tabulated

__device__ __forceinline__ unsigned long long slot_word(uint32_t key, float w) {
    return ((unsigned long long)__float_as_uint(w) << 32) | (unsigned long long)key;
}

// Append a candidate slot to this warp's staging buffer in shared memory (one shared atomic
// per group of lanes).  The global candidate list is only touched when the buffer is
// flushed, so threshold crossings do not all queue on one global counter.
__device__ __forceinline__ void stage_push(uint32_t *buf, unsigned *n, uint32_t slot) {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(n, (unsigned)g.size());
    base = g.shfl(base, 0);
    buf[base + g.thread_rank()] = slot;
}

// Whole warp, converged: move the staged candidates to the global list (one global atomic)
// when forced or when another 32 pushes might not fit.
__device__ __forceinline__ void stage_flush(uint32_t *buf, unsigned *n, bool force, BCtl *ctl,
                                            uint32_t *cand_out, unsigned cap) {
    __syncwarp();
    const unsigned cnt = *(volatile unsigned *)n;
    if (cnt == 0 || (!force && cnt <= (unsigned)(kStage - 32))) return;
    const unsigned lane = threadIdx.x & 31;
    unsigned gbase = 0;
    if (lane == 0) gbase = atomicAdd(&ctl->cand_out, cnt);
    gbase = __shfl_sync(0xffffffffu, gbase, 0);
    for (unsigned i = lane; i < cnt; i += 32) {
        if (gbase + i < cap) cand_out[gbase + i] = buf[i]; else atomicOr(&ctl->overflow, 1u);
    }
    __syncwarp();
    if (lane == 0) *(volatile unsigned *)n = 0;
    __syncwarp();
}

#ifndef GDE_PREFETCH
#define GDE_PREFETCH 1  // stream a seed group's hub slab into L2 ahead of its scatter
#endif
constexpr int kPrefetch = GDE_PREFETCH;
constexpr int64_t kPrefetchAhead = 1;  // groups ahead (2 or 3 crowd L2: slower)
constexpr int kPrefetchShift = 3;      // a seed's slab is streamed when its hub pushes are >= hubs / 8
constexpr uint32_t kPrefetchChunk = 8192;  // bytes a bulk L2 prefetch instruction covers

// Whole warp: stream [p, p + bytes) of global memory into L2 with bulk prefetches (a hint with
// no completion to wait for: lines that arrive before the scatter reaches them save it a random
// miss).  The range is shrunk to 16-byte boundaries inside it, as the bulk copy requires.
__device__ __forceinline__ void l2_prefetch_range(const void *p, uint64_t bytes, int lane) {
    const uint64_t a0 = ((uint64_t)p + 15ull) & ~15ull;
    const uint64_t a1 = ((uint64_t)p + bytes) & ~15ull;
    for (uint64_t q = a0 + (uint64_t)lane * kPrefetchChunk; q < a1; q += 32ull * kPrefetchChunk) {
        const uint32_t n = (uint32_t)(a1 - q < kPrefetchChunk ? a1 - q : kPrefetchChunk);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

struct ThrBounds {
    float lo, hi;  // lo <= thr_v <= hi; lo == hi means exact
};

// the brackets of every degree code, built once per block of the round kernel (the FP64
// products that define them are then not on the per-edge path)
__shared__ float2 s_thr_br[kMaxCls][256];
// the same brackets as slab counts, for the hub codes (>= hub_code)
__shared__ ulonglong2 s_hub_br[256];

// fixed-point helpers of the hub slab (value = count * 2^qexp)
__device__ __forceinline__ unsigned long long slab_count(const BArgs &a, float w) {
    return __float2ull_rn(__fmul_rn(w, a.wscale));
}
__device__ __forceinline__ double slab_value(const BArgs &a, unsigned long long c) {
    return __dmul_rn(__ull2double_rn(c), a.vscale);
}
// the smallest count whose value is >= thr (so count >= it <=> value >= thr, exactly)
__device__ __forceinline__ unsigned long long slab_threshold(const BArgs &a, double thr) {
    return __double2ull_ru(__dmul_rn(thr, a.tscale));
}
constexpr unsigned long long kSlabLimit = 1ull << 62;  // a count this large marks the seed overflowed
constexpr uint64_t kSlabMaxBytes = (uint64_t)16 << 30;    // hub slabs of one batch (12 bytes per entry)

__device__ __forceinline__ ThrBounds thr_bounds(const BArgs &a, double eps, uint32_t code) {
    ThrBounds t;
    if ((int)code < a.code_exact) {
        t.lo = t.hi = __double2float_ru(__dmul_rn(eps, (double)code));
    } else {
        const int k = (int)code - a.code_exact;
        t.lo = __double2float_ru(__dmul_rn(eps, (double)(1ll << k)));
        t.hi = __double2float_ru(__dmul_rn(eps, (double)((2ll << k) - 1)));
    }
    return t;
}

// did a residual going from `old` to `nv` cross v's threshold, |old| < thr <= |nv|?  Reads the
// class's threshold array only when the bracket cannot decide.  (With nonnegative residuals
// this happens once per node and round; when corrections made some residuals negative a node
// can cross more than once, and the frontier phase drops the repeats.)
template <bool LAYERED>
__device__ __forceinline__ bool crossed(const float *thr32c, int32_t v, ThrBounds tb, float old, float nv) {
    const float ao = fabsf(old), an = fabsf(nv);
    if (an < tb.lo || ao >= tb.hi) return false;
    // a layered round has no per-node array (its threshold changes every round): crossing the
    // bracket's lower bound lists the node; residuals only grow there, so a node that reaches
    // its threshold is listed exactly once, and the frontier's exact test drops the others
    const float thr = tb.lo == tb.hi ? tb.lo : (LAYERED ? tb.lo : thr32c[v]);
    return ao < thr && an >= thr;
}

// tolerance class and key tag of seed j's table
struct SlotMeta {
    int cls;
    uint32_t tag;
    uint32_t bank;  // hub slab bank the scatter writes (layered kinds: the next layer's parity)
    uint32_t mask;  // the seed's table: slots [base, base + mask + 1)
    uint64_t base;
};

// the keys round t's scatter writes: the next layer's (layered kinds) or the solve's
template <bool LAYERED>
__device__ __forceinline__ uint32_t write_tag(const BArgs &a, int64_t t) {
    return LAYERED ? a.key_tag + (uint32_t)(t + 1) * a.tag_step : a.key_tag;
}

// PAGED: a server's pool, whose slots carry their own parameters and table (SlotParam) and
// name their query through the page owner table; else the batch layout (seed j's table is
// [j << log2cap, (j + 1) << log2cap), one parameter set for all seeds)
template <bool LAYERED, bool PAGED>
__device__ __forceinline__ SlotMeta slot_meta(const BArgs &a, int32_t j, int64_t t) {
    if (!PAGED) return SlotMeta{0, write_tag<LAYERED>(a, t), LAYERED ? (uint32_t)((t + 1) & 1) : 0u, 0u, 0ull};
    const SlotParam &sp = a.sparam[j];
    return SlotMeta{sp.cls, sp.tag, 0u, (uint32_t)((1ull << sp.log2cap) - 1), sp.base};
}

// Adds count wq to hub `rank` of seed j's slab (one integer atomic: the slab has a fixed
// place for every hub, so there is no probe).  PPR and Katz: a count that crosses the hub's
// threshold (exactly once: counts only grow) is staged as a candidate of the next round.  The
// layered kinds stage every entry on its first touch in the layer (count was 0), so the next
// round's frontier takes each touched entry once and leaves the bank empty for reuse.
template <bool LAYERED>
__device__ __forceinline__ void slab_add(const BArgs &a, int32_t j, uint32_t code, uint32_t rank, uint32_t bank,
                                         unsigned long long wq, uint32_t *sbuf, unsigned *sn) {
    const uint64_t idx = (uint64_t)j * (uint64_t)a.H + rank;
    const unsigned long long old = atomicAdd(a.slab + (uint64_t)bank * a.slab_bank + idx, wq);
    const unsigned long long nv = old + wq;
    if (LAYERED) {
        if (old == 0ull) stage_push(sbuf, sn, a.slab_base + (uint32_t)idx);
    } else {
        const ulonglong2 br = s_hub_br[code];
        if (nv >= br.x && old < br.y) {
            const unsigned long long thr =
                br.x == br.y ? br.x : slab_threshold(a, __dmul_rn(a.eps, (double)__ldg(a.hub_deg + rank)));
            if (old < thr && nv >= thr) stage_push(sbuf, sn, a.slab_base + (uint32_t)idx);
        }
    }
    if (nv >= kSlabLimit) atomicExch(a.status + j, kSeedOverflow);
}

// Insert-or-add w at node v of seed j's table.  The probe starts at a 4-slot bucket (one
// 32-byte sector) chosen by mix32(v) and continues linearly bucket by bucket; slots are
// examined in order, so the first empty slot ends the search (keys are never removed).  A
// residual that crosses its threshold from below (exactly once: contributions are positive)
// is staged as a candidate of the next round.  Returns 1 if v was a new key (a server's pool
// also counts its queries' keys, which sizes the tables of later queries).
template <bool LAYERED, bool PAGED>
__device__ __forceinline__ unsigned bscatter(const BArgs &a, int32_t j, SlotMeta m, uint32_t packed, float w,
                                             unsigned long long wq, uint32_t *sbuf, unsigned *sn) {
    if (!PAGED && a.slab) {
        const uint32_t code = packed >> a.idbits;
        if (code >= a.hub_code) {
            slab_add<LAYERED>(a, j, code, packed & a.idmask, m.bank, wq, sbuf, sn);
            return 0;
        }
    }
    const uint64_t base = PAGED ? m.base : (uint64_t)j << a.log2cap;
    const uint32_t tmask = PAGED ? m.mask : a.mask;
    const int32_t v = (int32_t)(packed & a.idmask);
    const uint32_t kcur = (uint32_t)v | m.tag;
    const int cls = m.cls;
    const float *thr32c = LAYERED ? nullptr : a.thr32 + (int64_t)cls * a.thr_stride;
    ThrBounds tb;
    if (a.colp) {
        const float2 br = s_thr_br[cls][packed >> a.idbits];
        tb.lo = br.x;
        tb.hi = br.y;
    } else {
        tb.lo = tb.hi = thr32c[v];
    }
    const uint32_t sector_mask = tmask >= 3 ? 3u : tmask;
    uint32_t h = mix32((uint32_t)v) & tmask & ~sector_mask;
    for (uint32_t probes = 0; probes <= tmask && probes < kMaxProbe;) {
        unsigned long long w0, w1, w2, w3;
        if (sector_mask == 3u) {
            const ulonglong2 lo = __ldcg(reinterpret_cast<const ulonglong2 *>(a.kr + base + h));
            const ulonglong2 hi = __ldcg(reinterpret_cast<const ulonglong2 *>(a.kr + base + h + 2));
            w0 = lo.x; w1 = lo.y; w2 = hi.x; w3 = hi.y;
        } else {  // tables smaller than one sector
            w0 = ld_relaxed_u64(a.kr + base + h);
            w1 = sector_mask >= 1 ? ld_relaxed_u64(a.kr + base + h + 1) : 0ull;
            w2 = w3 = 0ull;
        }
        for (uint32_t k = 0; k <= sector_mask; k++, probes++) {
            const uint64_t slot = base + h + k;
            unsigned long long wk = k == 0 ? w0 : (k == 1 ? w1 : (k == 2 ? w2 : w3));
            for (;;) {
                const uint32_t key = (uint32_t)(wk & 0xFFFFFFFFull);
                if (key == kcur) {
                    const float old = atomicAdd(r_of(a.kr, slot), w);
                    if (crossed<LAYERED>(thr32c, v, tb, old, __fadd_rn(old, w))) stage_push(sbuf, sn, (uint32_t)slot);
                    return 0;
                }
                // another node of this solve: next slot (empty and stale-tag slots are free)
                if (key != kEmpty && (key & ~a.key_idmask) == m.tag) break;
                const unsigned long long prev = atomicCAS(a.kr + slot, wk, slot_word(kcur, w));
                if (prev == wk) {
                    if (crossed<LAYERED>(thr32c, v, tb, 0.0f, w)) stage_push(sbuf, sn, (uint32_t)slot);
                    if (PAGED) {  // one atomic per group of lanes of the same query
                        const unsigned peers = __match_any_sync(__activemask(), j);
                        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(a.inserts + j, (unsigned)__popc(peers));
                    }
                    return 1;
                }
                wk = prev;  // lost the race: look at what was written into this slot
            }
        }
        h = (h + sector_mask + 1) & tmask;
    }
    atomicExch(a.status + j, kSeedOverflow);  // table full
    return 0;
}

// Insert-or-add inc at node v of seed j's x table (layered solves; keys carry the solve's
// tag, slots are probed linearly).  A node is pushed at most once per round, so its slot's
// value has one writer per round.  Returns 1 if v was new (*slot_out then enters the seed's
// x-list), 0 if it was present, -1 if the probe found no room.
__device__ __forceinline__ int xt_add(const BArgs &a, int32_t j, int32_t v, float inc, uint64_t *slot_out) {
    const uint64_t base = (uint64_t)j << a.xlog2cap;
    const uint32_t kcur = (uint32_t)v | a.key_tag;
    uint32_t h = mix32((uint32_t)v) & a.xmask;
    for (uint32_t probes = 0; probes <= a.xmask && probes < kMaxProbe; probes++) {
        const uint64_t slot = base + h;
        unsigned long long wk = ld_relaxed_u64(a.xkr + slot);
        for (;;) {
            const uint32_t key = (uint32_t)(wk & 0xFFFFFFFFull);
            if (key == kcur) {
                atomicAdd(a.xxs + slot, inc);
                *slot_out = slot;
                return 0;
            }
            if (key != kEmpty && (key & ~a.key_idmask) == a.key_tag) break;  // another node of this solve
            const unsigned long long prev = atomicCAS(a.xkr + slot, wk, (unsigned long long)kcur);
            if (prev == wk) {
                atomicAdd(a.xxs + slot, inc);
                *slot_out = slot;
                return 1;
            }
            wk = prev;
        }
        h = (h + 1) & a.xmask;
    }
    return -1;
}

// columns of the push: packed (id | code) when available, else plain ids
__device__ __forceinline__ uint32_t push_col(const BArgs &a, int64_t e) {
    return a.colp ? a.colp[e] : (uint32_t)a.col[e];
}

#ifndef GDE_COL_PREFETCH
#define GDE_COL_PREFETCH 1
#endif
// One thread: ask L2 for the 128-byte lines holding columns [e, e + n) of the push's column
// array (every line lies inside the array), so the warp's later loads of them hit L2 instead
// of waiting on DRAM one 32-column step at a time (a hub chunk's 512 columns: kernel 31.4 ->
// 30.8 ms on R-MAT 24; the rows of a medium-degree grab, at most 4 steps each, gained nothing).
__device__ __forceinline__ void prefetch_cols(const BArgs &a, int64_t e, int64_t n) {
    if (n <= 0) return;
    const char *p0 = a.colp ? (const char *)(a.colp + e) : (const char *)(a.col + e);
    const uint64_t lo = (uint64_t)p0 & ~127ull;
    const uint64_t hi = ((uint64_t)p0 + 4ull * (uint64_t)n - 1ull) & ~127ull;
    for (uint64_t q = lo; q <= hi; q += 128ull) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

__global__ void k_pack_columns(int64_t nnz, const int32_t *col, const int32_t *deg, uint32_t *colp,
                               int idbits, int code_exact) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = col[e];
        colp[e] = (uint32_t)v | (degree_code(deg[v], code_exact) << idbits);
    }
}

// Exclusive prefix sums of n values (one block): out[i] = sum in[0..i), returns the total.
template <typename T>
__device__ T block_scan(const T *in, T *out, int64_t n, T *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T carry = 0;
    for (int64_t base = 0; base < n; base += kThreads) {
        const int64_t i = base + threadIdx.x;
        const T v = i < n ? __ldcg(in + i) : T(0);
        T x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        if (wid == 0) {
            T s = lane < kWarps ? s_warp[lane] : T(0);
#pragma unroll
            for (int o = 1; o < kWarps; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < kWarps) s_warp[lane] = s;
        }
        __syncthreads();
        const T before = wid > 0 ? s_warp[wid - 1] : T(0);
        if (i < n) out[i] = carry + before + x - v;
        const T block_total = s_warp[kWarps - 1];
        __syncthreads();
        carry += block_total;
    }
    return carry;
}

// Hub pushes are scattered in chunks of consecutive columns of their concatenated adjacency.
// Small rounds get shorter chunks so every warp has a share (a lone warp walking a long
// chunk would set the round's latency): the chunk of a round is ceil(VH / 2 warps), rounded
// up to a warp multiple, within [64, tuned chunk].
__device__ __forceinline__ int64_t hub_chunk(int64_t vh, int64_t nwarps, int64_t tuned) {
    int64_t chunk = (vh + 2 * nwarps - 1) / (2 * nwarps);
    chunk = (chunk + 31) & ~(int64_t)31;
    if (chunk < 64) chunk = 64;
    if (chunk > tuned) chunk = tuned;
    return chunk;
}

#ifndef GDE_ROUNDS_MIN_BLOCKS
#define GDE_ROUNDS_MIN_BLOCKS 6  // 40 registers, 48 warps per SM (the kernel is latency-bound)
#endif
template <bool LAYERED, bool PAGED>
__global__ void __launch_bounds__(kThreads, GDE_ROUNDS_MIN_BLOCKS) k_batch_rounds(BArgs a) {
    const unsigned nblocks = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nw = nthreads >> 5;
    // warp rank, warp-major across blocks: the first k warps sit on k different SMs, so a
    // phase that only needs a few warps still spreads them over the GPU
    const int64_t gw = (int64_t)wid * gridDim.x + blockIdx.x;
    BGlobal *G = a.glob;
    const unsigned long long t_start = globaltimer();
    const unsigned long long bar_limit = a.bar_limit_ns ? a.bar_limit_ns : kBarrierLimitNs;
    int nbar = 0;  // grid barriers passed by this block
    __shared__ uint32_t s_stage[kWarps][kStage];
    __shared__ unsigned s_nstage[kWarps];
    uint32_t *sbuf = s_stage[wid];
    unsigned *sn = &s_nstage[wid];
    if (lane == 0) *sn = 0;
    __syncwarp();
    __shared__ double s_rs[kWarps];
    __shared__ unsigned long long s_vol[kWarps];
    __shared__ unsigned long long s_busy[kWarps];
    if (a.colp) {
        for (int i = threadIdx.x; i < a.ncls * 256; i += kThreads) {
            const int cls = i >> 8, c = i & 255;
            // codes past the last log2 class never occur in the columns
            if (c >= a.code_exact && c - a.code_exact > 32) {
                s_thr_br[cls][c] = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7f800000));
                continue;
            }
            const ThrBounds tb = thr_bounds(a, a.eps_cls[cls], (uint32_t)c);
            s_thr_br[cls][c] = make_float2(tb.lo, tb.hi);
        }
    }
    if (!LAYERED && a.slab) {
        // the hub codes' brackets as slab counts (exact for exact degrees)
        for (int c = threadIdx.x; c < 256; c += kThreads) {
            const unsigned long long never = ~0ull;
            if ((uint32_t)c < a.hub_code || (c >= a.code_exact && c - a.code_exact > 32)) {
                s_hub_br[c] = make_ulonglong2(never, never);
                continue;
            }
            ulonglong2 br;
            if (c < a.code_exact) {
                br.x = br.y = slab_threshold(a, __dmul_rn(a.eps, (double)c));
            } else {
                const int k = c - a.code_exact;
                br.x = slab_threshold(a, __dmul_rn(a.eps, (double)(1ll << k)));
                br.y = slab_threshold(a, __dmul_rn(a.eps, (double)((2ll << k) - 1)));
            }
            s_hub_br[c] = br;
        }
    }
    __syncthreads();

    // per-seed count of the candidates this launch leaves behind (a server's unfinished
    // queries): zeroed here, filled after the last round; every round's grid barriers order
    // the two
    if (a.pend && a.max_rounds > 0)
        for (int64_t j = tid; j < a.nseeds; j += nthreads) a.pend[j] = 0u;
    int last_p = -1;         // parity of the last round run
    unsigned last_next = 0;  // its candidates for the next round
    for (int64_t t = a.t0; t < a.t0 + a.max_rounds; t++) {
        const int64_t lt = t - a.t0;  // round of this launch (log row)
        const int p = (int)(t & 1);
        BCtl *ctl = &G->ctl[p];
        BCtl *prev = &G->ctl[p ^ 1];
        const unsigned ncand = min(__ldcg(&prev->cand_out), a.list_cap);
        const uint32_t *cand = a.cand[p];
        const bool last_layer = LAYERED && t >= a.nlayers;

        // ---------------- phase A1: S_t for every seed ----------------
        // threshold test, r_S -> 0, x_S += c r_S, per-edge share; the push record is kept per
        // candidate and counted per (degree bin, seed)
        double my_rs = 0.0;
        unsigned long long my_vol = 0;
        unsigned my_dmax = 0;
        const int64_t ns = a.nseeds;
        for (int64_t ci = tid; ci < ncand; ci += nthreads) {
            const uint32_t slot = __ldcg(cand + ci);
            // a hub slab entry (slab_base + j * H + rank) or a hash slot (j << log2cap | i)
            const bool hub = a.slab && slot >= a.slab_base;
            const uint64_t hidx = hub ? (uint64_t)(slot - a.slab_base) : 0ull;
            const int32_t j = hub ? (int32_t)(hidx / (uint64_t)a.H)
                                  : (PAGED ? __ldg(a.page_owner + (slot >> a.pg_bits)) : (int32_t)(slot >> a.log2cap));
            if (a.pushed) a.pushed[ci] = 0u;
            if (j < 0 || __ldcg(a.status + j) != kSeedOk) { __stcg(a.tmp_deg + ci, 0); continue; }
            int32_t v;
            float rho = 0.0f;
            if (hub) {
                v = __ldg(a.hub_node + (hidx - (uint64_t)j * (uint64_t)a.H));
            } else {
                const unsigned long long word = __ldcg(a.kr + slot);
                v = (int32_t)((uint32_t)(word & 0xFFFFFFFFull) & a.key_idmask);
                rho = __uint_as_float((uint32_t)(word >> 32));
            }
            double cx = a.cx, coef = a.coef;
            bool divide = a.kind != GDE_KATZ;
            int cls = 0;
            // the seed's x-list: a fixed stretch per seed, or (a server's paged pool) the range of
            // its table, whose x entries cannot outnumber its slots
            uint64_t xlbase = (uint64_t)j * a.xcap;
            unsigned xlcap = a.xcap;
            if (PAGED) {
                const SlotParam sp = a.sparam[j];
                cx = sp.cx; coef = sp.coef; divide = sp.divide != 0; cls = sp.cls;
                xlbase = sp.base;
                xlcap = 1u << sp.log2cap;
                if ((sp.flags & kSlotDefer) && t != a.t0) {
                    // sits this round out: the candidate carries over to the next round
                    bappend(&ctl->cand_out, a.cand[p ^ 1], slot, a.list_cap, &ctl->overflow);
                    __stcg(a.tmp_deg + ci, 0);
                    continue;
                }
            }
            // the threshold fl(eps d_v) rounded up to float (the per-node arrays hold the same
            // values), from the row bounds the push needs anyway
            const int64_t beg = a.off[v];
            const int32_t dvol = (int32_t)(a.off[v + 1] - beg);
            const double eps_t = LAYERED ? a.layer_eps[t < a.nlayers ? t : a.nlayers] : a.eps_cls[cls];
            double rho64;
            if (hub) {
                // the exact test on the fixed-point count: count >= tq <=> value >= fl(eps d)
                const unsigned long long tq = slab_threshold(a, __dmul_rn(eps_t, (double)dvol));
                unsigned long long *cp = a.slab + (LAYERED ? (uint64_t)(t & 1) * a.slab_bank : 0ull) + hidx;
                unsigned long long c;
                if (LAYERED) {
                    // every touched entry of the layer is listed once: take it whether or not it
                    // is pushed (what stays below the threshold is the layer's remainder, left
                    // behind as in the tables), so the bank is empty when round t + 1 writes it
                    c = atomicExch(cp, 0ull);
                } else {
                    c = __ldcg(cp);
                    if (!(c != 0ull && c >= tq)) { __stcg(a.tmp_deg + ci, 0); continue; }
                    c = atomicExch(cp, 0ull);
                }
                if (!(c != 0ull && c >= tq)) { __stcg(a.tmp_deg + ci, 0); continue; }
                rho64 = slab_value(a, c);
            } else {
                const float thr = __double2float_ru(__dmul_rn(eps_t, (double)dvol));
                if (!(rho != 0.0f && fabsf(rho) >= thr)) { __stcg(a.tmp_deg + ci, 0); continue; }
                // take the residual: a slot listed twice (possible once residuals can be
                // negative) is pushed by one taker only
                rho = atomicExch(r_of(a.kr, slot), 0.0f);
                if (!(rho != 0.0f && fabsf(rho) >= thr)) { __stcg(a.tmp_deg + ci, 0); continue; }
                rho64 = (double)rho;
            }
            if (a.pushed) a.pushed[ci] = 1u;
            // vol(S_t) counts d_u; the last layer of a layered kind only adds to x (no scatter)
            const int32_t d = last_layer ? 0 : dvol;
            double xinc = __dmul_rn(cx, rho64);
            if (a.gbeta != 0.0) xinc = __ddiv_rn(xinc, pow((double)(d > 0 ? d : 1), a.gbeta));
            bool xfirst;
            uint64_t xslot = slot;
            if (LAYERED && hub) {
                // a hub's x lives in the slab beside its residual (one writer: a node is pushed
                // once per round)
                float *xp = a.slab_x + hidx;
                const float xold = __ldcg(xp);
                __stcg(xp, __fadd_rn(xold, __double2float_rn(xinc)));
                xfirst = xold == 0.0f;
                coef = a.layer_coef[t < a.nlayers ? t : a.nlayers];
            } else if (LAYERED) {
                const int xr = xt_add(a, j, v, __double2float_rn(xinc), &xslot);
                if (xr < 0) atomicExch(a.status + j, kSeedOverflow);  // x table full
                xfirst = xr == 1;
                coef = a.layer_coef[t < a.nlayers ? t : a.nlayers];
            } else {
                float *xp = hub ? a.slab_x + hidx : a.xs + slot;
                const float xold = __ldcg(xp);
                __stcg(xp, __fadd_rn(xold, __double2float_rn(xinc)));
                xfirst = xold == 0.0f;
            }
            float w = 0.0f;
            if (d > 0) {
                if (divide)
                    w = __double2float_rn(__ddiv_rn(__dmul_rn(coef, rho64), (double)d));
                else
                    w = __double2float_rn(__dmul_rn(coef, rho64));
            }
            if (!LAYERED && a.xsrc && v == __ldg(a.seed_ids + j)) a.xsrc[j] = __dadd_rn(a.xsrc[j], rho64);
            my_rs += fabs(rho64);
            my_vol += (unsigned long long)dvol;
            {
                // per-seed counters and FP64 mass: one atomic per group of lanes with the same seed
                const unsigned am = __activemask();
                const unsigned peers = __match_any_sync(am, j);
                const unsigned dsum = __reduce_add_sync(peers, (unsigned)dvol);
                double psum = rho64, ssum = d > 0 ? __dmul_rn((double)w, (double)d) : 0.0;
                if (peers == 0xffffffffu) {
                    // the whole warp on one seed (the usual case: candidates come seed-grouped)
                    for (int o = 16; o >= 1; o >>= 1) {
                        psum += __shfl_xor_sync(0xffffffffu, psum, o);
                        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
                    }
                } else {
                    const double mp = psum, ms = ssum;
                    psum = 0.0;
                    ssum = 0.0;
                    for (unsigned m = peers; m; m &= m - 1) {
                        const int src = __ffs(m) - 1;
                        psum += __shfl_sync(peers, mp, src);
                        ssum += __shfl_sync(peers, ms, src);
                    }
                }
                if (lane == __ffs(peers) - 1) {
                    atomicAdd(a.svol + j, (unsigned long long)dsum);
                    atomicAdd(a.spushes + j, (unsigned)__popc(peers));
                    atomicMax(a.slast + j, (int)t);
                    atomicAdd(a.spush + j, psum);
                    atomicAdd(a.sscat + j, ssum);
                }
            }
            if (xfirst) {
                // first activation of this node in this solve: remember the slot for the top-k
                const unsigned xpeers = __match_any_sync(__activemask(), j);
                const int xl = __ffs(xpeers) - 1;
                unsigned xb = 0;
                if (lane == xl) xb = atomicAdd(a.xcnt + j, (unsigned)__popc(xpeers));
                xb = __shfl_sync(xpeers, xb, xl) + __popc(xpeers & ((1u << lane) - 1u));
                if (xb < xlcap) {
                    __stcg(a.xlist + xlbase + xb, (uint32_t)xslot);
                    __stcg(a.xnode + xlbase + xb, (uint32_t)v);
                }
            }
            if (d == 0) { __stcg(a.tmp_deg + ci, 0); continue; }
            my_dmax = my_dmax > (unsigned)d ? my_dmax : (unsigned)d;
            const int bin = d <= a.t1 ? 0 : (d <= a.t2 ? 1 : 2);
            __stcg(a.tmp_beg + ci, beg);
            __stcg(a.tmp_deg + ci, d);
            __stcg(a.tmp_w + ci, w);
            __stcg(a.tmp_jb + ci, (uint32_t)j | ((uint32_t)bin << 30));
            const int32_t key = (int32_t)(bin * ns + j);
            const unsigned peers = __match_any_sync(__activemask(), key);
            const bool leader = lane == __ffs(peers) - 1;
            if (bin == 2) {
                const unsigned dsum = __reduce_add_sync(peers, (unsigned)d);
                if (leader) atomicAdd(a.seg_hvol + j, (unsigned long long)dsum);
            }
            if (leader) atomicAdd(a.seg_cnt + key, (unsigned)__popc(peers));
        }
        {
            double rs = bwarp_sum(my_rs);
            unsigned long long vv = bwarp_sum(my_vol);
            unsigned dm = __reduce_max_sync(0xffffffffu, my_dmax);
            if (lane == 0) { s_rs[wid] = rs; s_vol[wid] = vv; s_busy[wid] = dm; }
            __syncthreads();
            if (wid == 0) {
                rs = lane < kWarps ? s_rs[lane] : 0.0;
                vv = lane < kWarps ? s_vol[lane] : 0ull;
                dm = lane < kWarps ? (unsigned)s_busy[lane] : 0u;
                rs = bwarp_sum(rs);
                vv = bwarp_sum(vv);
                dm = __reduce_max_sync(0xffffffffu, dm);
                if (lane == 0 && vv + (rs != 0.0)) {
                    atomicAdd(&ctl->rS_l1, rs);
                    atomicAdd(&ctl->vol, vv);
                }
                if (lane == 0 && dm > 0) atomicMax(&ctl->dmax_push, dm);
            }
        }
        if (!grid_sync(G, nblocks, bar_limit, a.fail_block, a.fail_barrier, &nbar)) return;
        const bool direct = ncand <= kDirectCand && __ldcg(&ctl->dmax_push) <= kDirectMaxDeg;
        if (!direct) {

        // ---------------- phase S: segment offsets (one block) ----------------
        // the degree bins are laid out seed by seed, so the scatter phase sweeps the seeds
        // in order and only a few seeds' tables are in use at any moment
        if (blockIdx.x == 0) {
            __shared__ unsigned s_scan32[kWarps];
            __shared__ unsigned long long s_scan64[kWarps];
            const unsigned n0 = block_scan<unsigned>(a.seg_cnt, a.seg_off, ns, s_scan32);
            const unsigned n1 = block_scan<unsigned>(a.seg_cnt + ns, a.seg_off + ns, ns, s_scan32);
            const unsigned n2 = block_scan<unsigned>(a.seg_cnt + 2 * ns, a.seg_off + 2 * ns, ns, s_scan32);
            const unsigned long long vh = block_scan<unsigned long long>(a.seg_hvol, a.vol_off, ns, s_scan64);
            for (int64_t i = threadIdx.x; i < ns; i += kThreads) {
                a.seg_cnt[i] = 0; a.seg_cnt[ns + i] = 0; a.seg_cnt[2 * ns + i] = 0;
                a.seg_hvol[i] = 0; a.seg_cur[i] = 0; a.seg_cur[ns + i] = 0; a.seg_hcur[i] = 0;
            }
            if (threadIdx.x == 0) {
                ctl->cnt_small = n0;
                ctl->cnt_med = n1;
                ctl->hub_packed = ((unsigned long long)n2 << kBHubVolBits) | vh;
                if ((unsigned long long)n0 + n1 + n2 > a.list_cap) ctl->overflow = 1;
            }
            if (a.schedule == 3) {
                // work units of each seed group: its hub chunks, medium grabs and small groups
                const int64_t chunk = hub_chunk((int64_t)vh, nw, a.chunk);
                const int64_t ngroups = (ns + kSeedGroup - 1) / kSeedGroup;
                __syncthreads();  // seg_off / vol_off of every seed are written
                for (int64_t gi = threadIdx.x; gi < ngroups; gi += kThreads) {
                    const int64_t j0 = gi * kSeedGroup, j1 = j0 + kSeedGroup < ns ? j0 + kSeedGroup : ns;
                    const unsigned long long hv = (j1 < ns ? __ldcg(a.vol_off + j1) : vh) - __ldcg(a.vol_off + j0);
                    const unsigned nm = (j1 < ns ? __ldcg(a.seg_off + ns + j1) : n1) - __ldcg(a.seg_off + ns + j0);
                    const unsigned nsm = (j1 < ns ? __ldcg(a.seg_off + j1) : n0) - __ldcg(a.seg_off + j0);
                    a.grp_units[gi] = (hv + (unsigned long long)chunk - 1) / (unsigned long long)chunk +
                                      (nm + kMedGrab - 1) / kMedGrab + (nsm + 31) / 32;
                }
                __syncthreads();
                const unsigned long long tot = block_scan<unsigned long long>(a.grp_units, a.grp_off, ngroups, s_scan64);
                if (threadIdx.x == 0) ctl->units_total = tot;
            }
        }
        if (!grid_sync(G, nblocks, bar_limit, a.fail_block, a.fail_barrier, &nbar)) return;

        // ---------------- phase A2: place the pushes seed by seed ----------------
        for (int64_t ci = tid; ci < ncand; ci += nthreads) {
            const int32_t d = __ldcg(a.tmp_deg + ci);
            if (d == 0) continue;
            const uint32_t jb = __ldcg(a.tmp_jb + ci);
            const int32_t j = (int32_t)(jb & ((1u << 30) - 1u));
            const int bin = (int)(jb >> 30);
            const int64_t beg = __ldcg(a.tmp_beg + ci);
            const float w = __ldcg(a.tmp_w + ci);
            if (bin < 2) {
                const int32_t key = (int32_t)(bin * ns + j);
                const unsigned peers = __match_any_sync(__activemask(), key);
                const int leader = __ffs(peers) - 1;
                const unsigned rank = __popc(peers & ((1u << lane) - 1u));
                unsigned basepos = 0;
                if (lane == leader) basepos = atomicAdd(a.seg_cur + key, (unsigned)__popc(peers));
                basepos = __shfl_sync(peers, basepos, leader);
                const unsigned pos = __ldcg(a.seg_off + key) + basepos + rank;
                if (pos < a.list_cap) {
                    __stcg(a.b_beg[bin] + pos, beg); __stcg(a.b_deg[bin] + pos, d);
                    __stcg(a.b_w[bin] + pos, w); __stcg(a.b_seed[bin] + pos, j);
                } else {
                    atomicOr(&ctl->overflow, 1u);
                }
            } else {
                const unsigned long long old =
                    atomicAdd(a.seg_hcur + j, (1ull << kBHubVolBits) + (unsigned long long)d);
                const unsigned long long pos = __ldcg(a.seg_off + 2 * ns + j) + (old >> kBHubVolBits);
                if (pos < a.list_cap) {
                    __stcg(a.b_beg[2] + pos, beg); __stcg(a.b_deg[2] + pos, d);
                    __stcg(a.b_w[2] + pos, w); __stcg(a.b_seed[2] + pos, j);
                    const int64_t vs = (int64_t)(__ldcg(a.vol_off + j) + (old & kBHubVolMask));
                    __stcg(a.hub_vstart + pos, vs);
                    // the chunks that start inside this push's columns begin at this push (the
                    // pushes' column ranges tile [0, VH), so each chunk start is written once)
                    const int64_t vh = (int64_t)(__ldcg(&ctl->hub_packed) & kBHubVolMask);
                    const int64_t chunk = hub_chunk(vh, nw, a.chunk);
                    for (int64_t c = (vs + chunk - 1) / chunk; c * chunk < vs + d && c < kHubChunkTab; c++)
                        __stcg(a.hub_cstart + c, (uint32_t)pos);
                } else {
                    atomicOr(&ctl->overflow, 1u);
                }
            }
        }
        if (!grid_sync(G, nblocks, bar_limit, a.fail_block, a.fail_barrier, &nbar)) return;
        }  // !direct
        if (tid == 0 && lt < kLogCap) a.log[lt].tA_ns = globaltimer() - t_start;
        const unsigned long long tb0 = globaltimer();

        // ---------------- phase B: scatter ----------------
        if (LAYERED && a.colp) {
            // the crossings of this scatter are tested against the next layer's threshold
            const double en = a.layer_eps[t + 1 <= a.nlayers ? t + 1 : a.nlayers];
            for (int c = threadIdx.x; c < 256; c += kThreads) {
                if (c >= a.code_exact && c - a.code_exact > 32) {
                    s_thr_br[0][c] = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7f800000));
                    continue;
                }
                const ThrBounds tb = thr_bounds(a, en, (uint32_t)c);
                s_thr_br[0][c] = make_float2(tb.lo, tb.hi);
            }
            __syncthreads();
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // the other parity's counters were last read in phase A of this round
            prev->hub_packed = 0; prev->cnt_small = 0; prev->cnt_med = 0; prev->cand_out = 0;
            prev->n_active = 0; prev->vol = 0; prev->rS_l1 = 0.0; prev->overflow = 0;
            prev->hub_next = 0; prev->med_next = 0; prev->small_next = 0;
            prev->unit_next = 0; prev->units_total = 0; prev->dmax_push = 0;
        }
        uint32_t *cand_out = a.cand[p ^ 1];
        if (__ldcg(&ctl->overflow)) {
            if (tid == 0) atomicCAS(&G->error, 0u, (unsigned)GDE_ENOMEM);
        } else {
            const unsigned long long hp = __ldcg(&ctl->hub_packed);
            const int64_t H = (int64_t)(hp >> kBHubVolBits);
            const int64_t VH = (int64_t)(hp & kBHubVolMask);
            const int64_t chunk = hub_chunk(VH, nw, a.chunk);
            const unsigned nmed = min(__ldcg(&ctl->cnt_med), a.list_cap);
            const unsigned nsm = min(__ldcg(&ctl->cnt_small), a.list_cap);
            // hub columns [e0, e1) of the concatenated hub adjacency, h the push holding e0:
            // consecutive lanes on consecutive columns, walking the pushes forward
            auto hub_range = [&](int64_t e0, int64_t e1, int64_t h) {
                int64_t hs = __ldcg(a.hub_vstart + h);
                int64_t he = hs + __ldcg(a.b_deg[2] + h);
                int64_t hb = __ldcg(a.b_beg[2] + h);
                float hw = __ldcg(a.b_w[2] + h);
                unsigned long long hwq = a.slab ? slab_count(a, hw) : 0ull;
                int32_t hj = __ldcg(a.b_seed[2] + h);
                SlotMeta hm = slot_meta<LAYERED, PAGED>(a, hj, t);
                if (GDE_COL_PREFETCH && lane == 0) {
                    // the chunk's column segments, push by push
                    int64_t ps = hs, pe = he, pb = hb, ph = h, e = e0;
                    while (e < e1) {
                        const int64_t se = pe < e1 ? pe : e1;
                        prefetch_cols(a, pb + (e - ps), se - e);
                        e = se;
                        if (e < e1) {
                            ++ph;
                            ps = __ldcg(a.hub_vstart + ph);
                            pe = ps + __ldcg(a.b_deg[2] + ph);
                            pb = __ldcg(a.b_beg[2] + ph);
                        }
                    }
                }
                for (int64_t eb = e0; eb < e1; eb += 32) {
                    const int64_t e = eb + lane;
                    if (e < e1) {
                        while (e >= he) {
                            ++h;
                            hs = __ldcg(a.hub_vstart + h);
                            he = hs + __ldcg(a.b_deg[2] + h);
                            hb = __ldcg(a.b_beg[2] + h);
                            hw = __ldcg(a.b_w[2] + h);
                            hwq = a.slab ? slab_count(a, hw) : 0ull;
                            hj = __ldcg(a.b_seed[2] + h);
                            hm = slot_meta<LAYERED, PAGED>(a, hj, t);
                        }
                        bscatter<LAYERED, PAGED>(a, hj, hm, push_col(a, hb + (e - hs)), hw, hwq, sbuf, sn);
                    }
                    stage_flush(sbuf, sn, false, ctl, cand_out, a.list_cap);
                }
            };
            // the last hub push in [lo, hi) starting at or before e0
            auto hub_find = [&](int64_t e0, int64_t lo, int64_t hi) {
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (__ldcg(a.hub_vstart + mid) <= e0) lo = mid; else hi = mid;
                }
                return lo;
            };
            // one medium-degree push: the whole warp on its columns
            auto med_entry = [&](int64_t i) {
                const int64_t b = __ldcg(a.b_beg[1] + i);
                const int32_t d = __ldcg(a.b_deg[1] + i);
                const float w = __ldcg(a.b_w[1] + i);
                const unsigned long long wq = a.slab ? slab_count(a, w) : 0ull;
                const int32_t j = __ldcg(a.b_seed[1] + i);
                const SlotMeta m = slot_meta<LAYERED, PAGED>(a, j, t);
                for (int32_t k0 = 0; k0 < d; k0 += 32) {
                    const int32_t k = k0 + lane;
                    if (k < d) bscatter<LAYERED, PAGED>(a, j, m, push_col(a, b + k), w, wq, sbuf, sn);
                    stage_flush(sbuf, sn, false, ctl, cand_out, a.list_cap);
                }
            };
            // small-degree pushes [i0, min(i0 + 32, iend)): one thread each (warp-uniform loops
            // so the warp can flush)
            auto small_group = [&](int64_t i0, int64_t iend) {
                const int64_t i = i0 + lane;
                int64_t b = 0;
                int32_t d = 0, j = 0;
                float w = 0.0f;
                if (i < iend) {
                    b = __ldcg(a.b_beg[0] + i);
                    d = __ldcg(a.b_deg[0] + i);
                    w = __ldcg(a.b_w[0] + i);
                    j = __ldcg(a.b_seed[0] + i);
                }
                const int32_t dmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)d);
                const SlotMeta m = d > 0 ? slot_meta<LAYERED, PAGED>(a, j, t) : SlotMeta{0, write_tag<LAYERED>(a, t), 0u, 0u, 0ull};
                const unsigned long long wq = a.slab && d > 0 ? slab_count(a, w) : 0ull;
                for (int32_t k = 0; k < dmax; k++) {
                    if (k < d) bscatter<LAYERED, PAGED>(a, j, m, push_col(a, b + k), w, wq, sbuf, sn);
                    stage_flush(sbuf, sn, false, ctl, cand_out, a.list_cap);
                }
            };
            if (direct) {
                // the per-(bin, seed) counts of the frontier phase are not scanned this round
                for (int64_t i = tid; i < 3 * ns; i += nthreads) a.seg_cnt[i] = 0;
                for (int64_t i = tid; i < ns; i += nthreads) a.seg_hvol[i] = 0;
                for (int64_t ci = gw; ci < ncand; ci += nw) {
                    const int32_t d = __ldcg(a.tmp_deg + ci);
                    if (d == 0) continue;
                    const int64_t b = __ldcg(a.tmp_beg + ci);
                    const float w = __ldcg(a.tmp_w + ci);
                    const unsigned long long wq = a.slab ? slab_count(a, w) : 0ull;
                    const int32_t j = (int32_t)(__ldcg(a.tmp_jb + ci) & ((1u << 30) - 1u));
                    const SlotMeta m = slot_meta<LAYERED, PAGED>(a, j, t);
                    for (int32_t k0 = 0; k0 < d; k0 += 32) {
                        const int32_t k = k0 + lane;
                        if (k < d) bscatter<LAYERED, PAGED>(a, j, m, push_col(a, b + k), w, wq, sbuf, sn);
                        stage_flush(sbuf, sn, false, ctl, cand_out, a.list_cap);
                    }
                }
            } else if (a.schedule == 3) {
                // group by group of seeds: each group's hub chunks, medium grabs and small
                // groups are consecutive work units, so a seed's table is brought into L2 once
                // per round instead of once per bin
                // (units handed out in order, one at a time: with static striding the warps that
                // drew long hub chunks fell behind and held the round)
                const unsigned long long total = __ldcg(&ctl->units_total);
                const int64_t ngroups = (ns + kSeedGroup - 1) / kSeedGroup;
                for (int64_t it = 0; (unsigned long long)gw < total; it++) {
                    unsigned long long u = 0;
                    if (lane == 0) u = atomicAdd(&ctl->unit_next, 1ull);
                    u = __shfl_sync(0xffffffffu, u, 0);
                    if (u >= total) break;
                    int64_t glo = 0, ghi = ngroups;  // the last group starting at or before u
                    while (ghi - glo > 1) {
                        const int64_t mid = (glo + ghi) >> 1;
                        if (__ldcg(a.grp_off + mid) <= u) glo = mid; else ghi = mid;
                    }
                    const int64_t j0 = glo * kSeedGroup, j1 = j0 + kSeedGroup < ns ? j0 + kSeedGroup : ns;
                    int64_t r = (int64_t)(u - __ldcg(a.grp_off + glo));
                    if (kPrefetch && !PAGED && a.slab && r == 0) {
                        // the first unit of a group: stream the next group's hub slabs into L2
                        // (the first group also its own) while this one is scattered, for the
                        // seeds whose hub pushes this round are at least an eighth as many as
                        // hubs (their scatter touches a large share of the slab's sectors; a
                        // random miss costs several times a streamed sector; streaming every
                        // seed's slab wastes the bandwidth and crowds L2).  Streaming the tables
                        // as well gained nothing: their keys are sparser.
                        for (int64_t gp = glo == 0 ? 0 : glo + kPrefetchAhead; gp <= glo + kPrefetchAhead && gp < ngroups; gp++) {
                            const int64_t q1 = min(gp * kSeedGroup + kSeedGroup, ns);
                            for (int64_t jq = gp * kSeedGroup; jq < q1; jq++) {
                                const int64_t hv = (jq + 1 < ns ? (int64_t)__ldcg(a.vol_off + jq + 1) : VH) -
                                                   (int64_t)__ldcg(a.vol_off + jq);
                                if ((hv << kPrefetchShift) >= (int64_t)a.H) {
                                    const uint64_t bank = LAYERED ? (uint64_t)((t + 1) & 1) : 0ull;
                                    l2_prefetch_range(a.slab + bank * a.slab_bank + (uint64_t)jq * a.H, 8ull * a.H, lane);
                                }
                            }
                        }
                    }
                    const int64_t hv0 = (int64_t)__ldcg(a.vol_off + j0);
                    const int64_t hv1 = j1 < ns ? (int64_t)__ldcg(a.vol_off + j1) : VH;
                    const int64_t nch = (hv1 - hv0 + chunk - 1) / chunk;
                    if (r < nch) {
                        const int64_t e0 = hv0 + r * chunk;
                        const int64_t e1 = min(e0 + chunk, hv1);
                        const int64_t h0 = (int64_t)__ldcg(a.seg_off + 2 * ns + j0);
                        const int64_t h1 = j1 < ns ? (int64_t)__ldcg(a.seg_off + 2 * ns + j1) : H;
                        hub_range(e0, e1, hub_find(e0, h0, h1));
                        continue;
                    }
                    r -= nch;
                    const int64_t m0 = (int64_t)__ldcg(a.seg_off + ns + j0);
                    const int64_t m1 = j1 < ns ? (int64_t)__ldcg(a.seg_off + ns + j1) : (int64_t)nmed;
                    const int64_t nmg = (m1 - m0 + kMedGrab - 1) / kMedGrab;
                    if (r < nmg) {
                        const int64_t gend = min(m0 + (r + 1) * kMedGrab, m1);
                        for (int64_t i = m0 + r * kMedGrab; i < gend; i++) med_entry(i);
                        continue;
                    }
                    r -= nmg;
                    const int64_t s0 = (int64_t)__ldcg(a.seg_off + j0);
                    const int64_t s1 = j1 < ns ? (int64_t)__ldcg(a.seg_off + j1) : (int64_t)nsm;
                    small_group(s0 + r * 32, s1);
                }
            } else {
                // hubs: merge-path chunks of the concatenated hub adjacency, one warp per chunk
                if (VH > 0) {
                    const int64_t nchunks = (VH + chunk - 1) / chunk;
                    // warps beyond the chunk count would only find the work gone: they stay out,
                    // so small rounds do not queue every warp on the hand-out counter
                    for (int64_t it = 0; gw < nchunks; it++) {
                        int64_t c;
                        if (a.schedule <= 1) {
                            unsigned long long cg_ = 0;
                            if (lane == 0) cg_ = atomicAdd(&ctl->hub_next, 1ull);
                            c = (int64_t)__shfl_sync(0xffffffffu, cg_, 0);
                        } else {
                            c = gw + it * nw;
                        }
                        if (c >= nchunks) break;
                        const int64_t e0 = c * chunk;
                        const int64_t e1 = min(e0 + chunk, VH);
                        // past the table: the last push starting at or before e0
                        const int64_t h = c < kHubChunkTab ? (int64_t)__ldcg(a.hub_cstart + c) : hub_find(e0, 0, H);
                        hub_range(e0, e1, h);
                    }
                }
                // medium degrees: one warp per node; descending: the hub sweep ends at the last
                // seeds, the medium sweep starts there
                for (int64_t it = 0; gw * kMedGrab < (int64_t)nmed; it++) {
                    unsigned got = 0;
                    if (a.schedule == 0) {
                        if (lane == 0) got = atomicAdd(&ctl->med_next, (unsigned)kMedGrab);
                        got = __shfl_sync(0xffffffffu, got, 0);
                    } else {
                        const int64_t g0 = (gw + it * nw) * kMedGrab;
                        got = g0 < nmed ? (unsigned)g0 : nmed;
                    }
                    if (got >= nmed) break;
                    const unsigned gend = min(got + (unsigned)kMedGrab, nmed);
                    for (unsigned ii = got; ii < gend; ii++) med_entry((int64_t)nmed - 1 - ii);
                }
                // small degrees: one thread per node
                for (int64_t it = 0; gw * 32 < (int64_t)nsm; it++) {
                    int64_t i0;
                    if (a.schedule == 0) {
                        unsigned got = 0;
                        if (lane == 0) got = atomicAdd(&ctl->small_next, 32u);
                        i0 = (int64_t)__shfl_sync(0xffffffffu, got, 0);
                    } else {
                        i0 = (gw + it * nw) * 32;
                    }
                    if (i0 >= nsm) break;
                    small_group(i0, nsm);
                }
            }
        }
        stage_flush(sbuf, sn, true, ctl, cand_out, a.list_cap);
        if (lt < kLogCap) {
            // phase-B busy time of the warps (for the load-balance record), summed per block
            // first so the record costs two global atomics per block
            const unsigned long long busy = globaltimer() - tb0;
            if (lane == 0) s_busy[wid] = busy;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long bs = 0, bm = 0;
                for (int w2 = 0; w2 < kWarps; w2++) { bs += s_busy[w2]; bm = bm > s_busy[w2] ? bm : s_busy[w2]; }
                atomicAdd(&a.log[lt].busy_sum_ns, bs);
                atomicMax(&a.log[lt].busy_max_ns, bm);
            }
        }
        if (!grid_sync(G, nblocks, bar_limit, a.fail_block, a.fail_barrier, &nbar)) return;
        const unsigned next = __ldcg(&ctl->cand_out);
        const unsigned ovf = __ldcg(&ctl->overflow);
        if (tid == 0) {
            G->rounds = (unsigned)(t + 1);
            const unsigned long long rv = __ldcg(&ctl->vol);
            G->total_vol += rv;
            if (lt < kLogCap) {
                a.log[lt].vol = rv;
                a.log[lt].rS_l1 = __ldcg(&ctl->rS_l1);
                a.log[lt].ncand = ncand;
                a.log[lt].n_active = next;
                a.log[lt].t_ns = globaltimer() - t_start;
            }
            if (ovf || next > a.list_cap) atomicCAS(&G->error, 0u, (unsigned)GDE_ENOMEM);
        }
        last_p = p;
        last_next = next <= a.list_cap ? next : a.list_cap;
        if (next == 0 || next > a.list_cap || ovf) break;
    }
    if (a.pend && last_p >= 0) {
        const uint32_t *left = a.cand[last_p ^ 1];
        for (int64_t i = tid; i < (int64_t)last_next; i += nthreads) {
            const uint32_t slot = __ldcg(left + i);
            const int32_t j = PAGED ? a.page_owner[slot >> a.pg_bits] : (int32_t)(slot >> a.log2cap);
            if (j >= 0) atomicAdd(a.pend + j, 1u);
        }
    }
}

// clear the pool and fill the per-node thresholds
__global__ void k_batch_clear(int64_t pool, unsigned long long *kr, float *xs) {
    const unsigned long long empty = (unsigned long long)kEmpty;  // r = 0.0f in the high half
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pool;
         i += (int64_t)gridDim.x * blockDim.x) {
        kr[i] = empty;
        xs[i] = 0.0f;
    }
}

__global__ void k_batch_thr(int64_t n, const int32_t *deg, float *thr32, double eps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        thr32[i] = __double2float_ru(__dmul_rn(eps, (double)deg[i]));
}

// Seeds the hub slab instead of the hash table when the seed is a hub (slab not NULL and
// hub_rank[s] >= 0), so that all of a node's residual lives in one place.
struct SeedSlab {
    unsigned long long *slab;
    const int32_t *hub_rank;
    int64_t H;
    uint32_t slab_base;
    double tscale;  // 2^-qexp
};

__global__ void k_batch_seed(int32_t nseeds, const int32_t *seeds, unsigned long long *kr,
                             uint32_t *cand0, int log2cap, uint32_t mask, BGlobal *G,
                             int32_t *status, unsigned *inserts, unsigned long long *svol,
                             unsigned *spushes, int32_t *slast, uint32_t key_tag, unsigned *xcnt,
                             double *spush, double *sscat, const int32_t *deg, double gbeta, double *smass0,
                             SeedSlab sl, double *xsrc) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j == 0) {
        memset(G, 0, sizeof(BGlobal));
        G->ctl[1].cand_out = (unsigned)nseeds;
    }
    if (j >= nseeds) return;
    const int32_t s = seeds[j];
    // the first slot of the seed's probe bucket, where bscatter's search for s begins
    const uint32_t sector_mask = mask >= 3 ? 3u : mask;
    const uint64_t slot = ((uint64_t)j << log2cap) + (mix32((uint32_t)s) & mask & ~sector_mask);
    // unit source; the generalised propagation keeps it scaled, y_s = max(d_s, 1)^gbeta
    const double m0 = gbeta != 0.0 ? pow((double)(deg[s] > 0 ? deg[s] : 1), gbeta) : 1.0;
    const int32_t rank = sl.slab ? sl.hub_rank[s] : -1;
    if (rank >= 0) {
        const uint64_t idx = (uint64_t)j * (uint64_t)sl.H + (uint64_t)rank;
        const unsigned long long c = __double2ull_rn(__dmul_rn((double)(float)m0, sl.tscale));
        sl.slab[idx] = c;
        cand0[j] = sl.slab_base + (uint32_t)idx;
    } else {
        kr[slot] = ((unsigned long long)__float_as_uint((float)m0) << 32) | (unsigned long long)((uint32_t)s | key_tag);
        cand0[j] = (uint32_t)slot;
    }
    smass0[j] = (double)(float)m0;
    if (xsrc) xsrc[j] = -1.0;
    status[j] = kSeedOk;
    inserts[j] = 1;
    xcnt[j] = 0;
    spush[j] = 0.0;
    sscat[j] = 0.0;
    svol[j] = 0;
    spushes[j] = 0;
    slast[j] = -1;
}

// ------------------------------------------------------------------- top-k --

// bitonic helpers on 64-bit keys, one key per lane, descending order
__device__ __forceinline__ unsigned long long cmpx(unsigned long long v, int partner_mask, bool keep_max) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, partner_mask);
    return keep_max ? (v > o ? v : o) : (v < o ? v : o);
}

// sort 32 keys (one per lane) descending
__device__ __forceinline__ unsigned long long sort32_desc(unsigned long long v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const bool up = ((lane & k) == 0);       // this block sorted descending
            const bool lower = ((lane & j) == 0);
            v = cmpx(v, j, up == lower);
        }
    }
    return v;
}

// bitonic sequence of 32 (one per lane) -> descending
__device__ __forceinline__ unsigned long long merge32_desc(unsigned long long v, int lane) {
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) v = cmpx(v, j, (lane & j) == 0);
    return v;
}

// top-64 list held as a (positions 0..31) and b (32..63), both descending across lanes.
// Insert a batch of 32 candidates c (one per lane, any order).
__device__ __forceinline__ void top64_insert(unsigned long long &a, unsigned long long &b,
                                             unsigned long long c, int lane) {
    const unsigned long long lmin = __shfl_sync(0xffffffffu, b, 31);
    if (!__any_sync(0xffffffffu, c > lmin)) return;
    c = sort32_desc(c, lane);
    // top 32 of (b U c): elementwise max of b and reversed c, then sort
    const unsigned long long crev = __shfl_sync(0xffffffffu, c, 31 - lane);
    unsigned long long m = b > crev ? b : crev;
    m = merge32_desc(m, lane);
    // merge a (desc) and m (desc): a followed by reversed m is bitonic
    const unsigned long long mrev = __shfl_sync(0xffffffffu, m, 31 - lane);
    const unsigned long long hi = a > mrev ? a : mrev;
    const unsigned long long lo = a > mrev ? mrev : a;
    a = merge32_desc(hi, lane);
    b = merge32_desc(lo, lane);
}

constexpr int kTopkThreads = 512;
constexpr int kTopkWarps = kTopkThreads / 32;

struct TopkArgs {
    const unsigned long long *kr;
    float *xs;                  // read, then zeroed for the next solve
    int log2cap;
    int64_t cap;
    uint32_t key_idmask;
    const uint32_t *xlist;
    const uint32_t *xnode;      // node of each x-list entry
    const unsigned *xcnt;
    unsigned xcap;
    int k;
    int32_t *out_ids;
    float *out_vals;
    unsigned *ssupport;         // |supp(x)| per seed
    const int32_t *slots;       // block b reads seed slots[b] (NULL: seed b); output row b
    int keep;                   // nonzero: leave x in place (a server's resident queries)
    float scale;                // output values are x * scale (0 reads as 1)
    // Katz with f_Katz output (xsrc not NULL): the seed's entry is xsrc[j] = x_s - 1 (FP64)
    const double *xsrc;
    const int32_t *seed_ids;
    // hub slab (slab_x NULL: none): x-list ids at or above slab_base are slab entries
    float *slab_x;
    uint32_t slab_base;
    int64_t H;
    const int32_t *hub_node;
};

// One block per seed: the top-k of (x desc, id asc) over the slots of the seed's x-list (every
// node with nonzero x), which are zeroed for the next solve.  If the list overflowed, the whole
// table is scanned instead.
// one block of kTopkThreads per seed: the seeds with the longest x-lists set the kernel's time, so
// wide blocks (512 threads: 0.94 ms for the benchmark's batch, 1.02 ms at 256, 1.14 ms at 128)
__global__ void __launch_bounds__(kTopkThreads, 2) k_batch_topk(TopkArgs a) {
    const int j = a.slots ? a.slots[blockIdx.x] : (int)blockIdx.x;
    const int64_t orow = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)j << a.log2cap;
    unsigned long long ta = 0, tb = 0;
    const unsigned nx = a.xcnt[j];
    const bool use_list = nx <= a.xcap;
    const int64_t n = use_list ? (int64_t)nx : a.cap + (a.slab_x ? a.H : 0);
    unsigned support = 0;
    // x-list entries 4 a lane at a time: the four x loads (random) are in flight together
    constexpr int kU = 4;
    const int64_t nl = use_list ? n : 0;
    for (int64_t i0 = (int64_t)wid * 32 * kU; i0 < nl; i0 += kTopkThreads * kU) {
        float *xp[kU];
        uint32_t v[kU];
        float x[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const int64_t i = i0 + u * 32 + lane;
            xp[u] = nullptr;
            v[u] = 0u;
            if (i < nl) {
                const uint64_t li = (uint64_t)j * a.xcap + i;
                const uint32_t id = a.xlist[li];
                xp[u] = a.slab_x && id >= a.slab_base ? a.slab_x + (id - a.slab_base) : a.xs + id;
                v[u] = a.xnode[li];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) x[u] = xp[u] ? *xp[u] : 0.0f;
#pragma unroll
        for (int u = 0; u < kU; u++) {
            unsigned long long key = 0;
            if (x[u] > 0.0f) {
                if (!a.keep) *xp[u] = 0.0f;
                support++;
                float xv = x[u];
                if (a.xsrc && (int32_t)v[u] == a.seed_ids[j]) xv = __double2float_rn(a.xsrc[j]);
                if (xv > 0.0f)
                    key = ((unsigned long long)__float_as_uint(xv) << 32) | (unsigned long long)(0xFFFFFFFFu - v[u]);
            }
            top64_insert(ta, tb, key, lane);
        }
    }
    // an overflowed x-list: the whole table, then the seed's slab entries
    for (int64_t i0 = (int64_t)wid * 32; i0 < n && !use_list; i0 += kTopkThreads) {
        const int64_t i = i0 + lane;
        unsigned long long key = 0;
        if (i < n) {
            float *xp;
            uint32_t v;
            if (i < a.cap) {
                xp = a.xs + base + (uint64_t)i;
                v = (uint32_t)(a.kr[base + (uint64_t)i] & 0xFFFFFFFFull) & a.key_idmask;
            } else {
                xp = a.slab_x + (uint64_t)j * (uint64_t)a.H + (uint64_t)(i - a.cap);
                v = (uint32_t)a.hub_node[i - a.cap];
            }
            float x = *xp;
            if (x > 0.0f) {
                if (!a.keep) *xp = 0.0f;
                support++;
                if (a.xsrc && (int32_t)v == a.seed_ids[j]) x = __double2float_rn(a.xsrc[j]);
                if (x > 0.0f)
                    key = ((unsigned long long)__float_as_uint(x) << 32) | (unsigned long long)(0xFFFFFFFFu - v);
            }
        }
        top64_insert(ta, tb, key, lane);
    }
    __shared__ unsigned long long s_a[kTopkWarps][32], s_b[kTopkWarps][32];
    __shared__ unsigned s_k[kTopkWarps];
    s_a[wid][lane] = ta;
    s_b[wid][lane] = tb;
    support = bwarp_sum(support);
    if (lane == 0) s_k[wid] = support;
    __syncthreads();
    if (wid == 0) {
        for (int ww = 1; ww < kTopkWarps; ww++) {
            top64_insert(ta, tb, s_a[ww][lane], lane);
            top64_insert(ta, tb, s_b[ww][lane], lane);
        }
        unsigned kk = lane < kTopkWarps ? s_k[lane] : 0u;
        kk = bwarp_sum(kk);
        if (lane == 0) a.ssupport[j] = kk;
        const int k = a.k;
        for (int half = 0; half < 2; half++) {
            const int pos = half * 32 + lane;
            const unsigned long long key = half ? tb : ta;
            if (pos < k) {
                const bool valid = key != 0;
                a.out_ids[orow * k + pos] = valid ? (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)) : -1;
                const float sc = a.scale != 0.0f ? a.scale : 1.0f;
                a.out_vals[orow * k + pos] = valid ? __fmul_rn(__uint_as_float((uint32_t)(key >> 32)), sc) : 0.0f;
            }
        }
    }
}

// dense top-k over x[0..n) (float): partial top-64 per block, then one block merges
__global__ void __launch_bounds__(kThreads) k_topk_dense_partial(int64_t n, const float *x,
                                                                 unsigned long long *partial) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long ta = 0, tb = 0;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(lo + per, n);
    for (int64_t i0 = lo + (int64_t)wid * 32; i0 < hi; i0 += kThreads) {
        const int64_t i = i0 + lane;
        unsigned long long key = 0;
        if (i < hi) {
            const float v = x[i];
            if (v > 0.0f) key = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
        }
        top64_insert(ta, tb, key, lane);
    }
    __shared__ unsigned long long s_a[kWarps][32], s_b[kWarps][32];
    s_a[wid][lane] = ta;
    s_b[wid][lane] = tb;
    __syncthreads();
    if (wid == 0) {
        for (int w = 1; w < kWarps; w++) {
            top64_insert(ta, tb, s_a[w][lane], lane);
            top64_insert(ta, tb, s_b[w][lane], lane);
        }
        partial[(int64_t)blockIdx.x * 64 + lane] = ta;
        partial[(int64_t)blockIdx.x * 64 + 32 + lane] = tb;
    }
}

__global__ void __launch_bounds__(kThreads) k_topk_dense_final(int64_t nparts, const unsigned long long *partial,
                                                               int k, int32_t *ids, float *vals) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long ta = 0, tb = 0;
    for (int64_t i0 = (int64_t)wid * 32; i0 < nparts * 64; i0 += kThreads) {
        const int64_t i = i0 + lane;
        top64_insert(ta, tb, i < nparts * 64 ? partial[i] : 0ull, lane);
    }
    __shared__ unsigned long long s_a[kWarps][32], s_b[kWarps][32];
    s_a[wid][lane] = ta;
    s_b[wid][lane] = tb;
    __syncthreads();
    if (wid == 0) {
        for (int w = 1; w < kWarps; w++) {
            top64_insert(ta, tb, s_a[w][lane], lane);
            top64_insert(ta, tb, s_b[w][lane], lane);
        }
        for (int half = 0; half < 2; half++) {
            const int pos = half * 32 + lane;
            const unsigned long long key = half ? tb : ta;
            if (pos < k) {
                const bool valid = key != 0;
                ids[pos] = valid ? (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)) : -1;
                vals[pos] = valid ? __uint_as_float((uint32_t)(key >> 32)) : 0.0f;
            }
        }
    }
}

void topk_dense_f32(Graph &g, const float *x_dev, int64_t n, int k, int32_t *ids_dev, float *vals_dev,
                    cudaStream_t s) {
    GDE_REQUIRE(k >= 1 && k <= kTopMax, GDE_EINVAL, "topk must be in [1, 64]");
    const int parts = kSMs * 2;
    if (!g.topk_part) g.topk_part = (unsigned long long *)dmalloc(8 * 64 * (size_t)parts, "top-k partials");
    k_topk_dense_partial<<<parts, kThreads, 0, s>>>(n, x_dev, g.topk_part);
    GDE_CUDA(cudaGetLastError());
    k_topk_dense_final<<<1, kThreads, 0, s>>>(parts, g.topk_part, k, ids_dev, vals_dev);
    GDE_CUDA(cudaGetLastError());
}

// =============================================================== host ====

static void batch_free(BatchWork *w) {
    if (!w) return;
    dfree(w->kr); dfree(w->xs); dfree(w->thr32);
    for (int k = 0; k < 2; k++) dfree(w->cand[k]);
    for (int b = 0; b < 3; b++) { dfree(w->b_beg[b]); dfree(w->b_deg[b]); dfree(w->b_w[b]); dfree(w->b_seed[b]); }
    dfree(w->hub_vstart); dfree(w->hub_cstart); dfree(w->grp_units); dfree(w->grp_off); dfree(w->tmp_beg); dfree(w->tmp_deg); dfree(w->tmp_w); dfree(w->tmp_jb);
    dfree(w->seg_cnt); dfree(w->seg_off); dfree(w->seg_cur); dfree(w->seg_hvol); dfree(w->vol_off);
    dfree(w->seg_hcur); dfree(w->seeds); dfree(w->status); dfree(w->inserts); dfree(w->svol);
    dfree(w->spushes); dfree(w->slast); dfree(w->spush); dfree(w->sscat); dfree(w->smass0); dfree(w->xlist); dfree(w->xnode); dfree(w->xcnt); dfree(w->glob); dfree(w->log);
    dfree(w->xkr); dfree(w->xxs); dfree(w->layer_eps); dfree(w->layer_coef);
    if (w->zs) cudaStreamSynchronize(w->zs);
    dfree(w->slab); dfree(w->slab_x); dfree(w->xsrc);
    if (w->z_start) cudaEventDestroy(w->z_start);
    if (w->z_done) cudaEventDestroy(w->z_done);
    if (w->zs) cudaStreamDestroy(w->zs);
    delete w;
}

void batch_work_destroy(BatchWork *w) { batch_free(w); }

// the CSR changed (edge insertions): columns, degrees and offsets moved, so the packed
// columns and thresholds are rebuilt on the next solve and the dense workspaces dropped
void graph_changed(Graph &g) {
    for (int k = 0; k < 2; k++) {
        dense_work_destroy(g.dense[k]);
        g.dense[k] = nullptr;
    }
    if (BatchWork *w = g.batch) {
        w->thr_eps = -1.0;
        w->thr_n = -1;
    }
    g.hub_valid = false;  // degrees moved: the hub ranks and colq are rebuilt on next use
}

static BatchWork *batch_work_alloc(int64_t nseeds, int64_t cap, int64_t list_cap, int64_t xcap_max = (int64_t)1 << 16) {
    BatchWork *w = new BatchWork();
    try {
        w->nseeds_cap = nseeds;
        w->cap = cap;
        w->log2cap = 0;
        while (((int64_t)1 << w->log2cap) < cap) w->log2cap++;
        w->pool = nseeds * cap;
        w->list_cap = list_cap;
        w->kr = (unsigned long long *)dmalloc(8 * (size_t)w->pool, "hash keys/residuals");
        w->xs = (float *)dmalloc(4 * (size_t)w->pool, "hash x");
        for (int k = 0; k < 2; k++) w->cand[k] = (uint32_t *)dmalloc(4 * (size_t)list_cap, "candidates");
        for (int b = 0; b < 3; b++) {
            w->b_beg[b] = (int64_t *)dmalloc(8 * (size_t)list_cap, "bins");
            w->b_deg[b] = (int32_t *)dmalloc(4 * (size_t)list_cap, "bins");
            w->b_w[b] = (float *)dmalloc(4 * (size_t)list_cap, "bins");
            w->b_seed[b] = (int32_t *)dmalloc(4 * (size_t)list_cap, "bins");
        }
        w->hub_vstart = (int64_t *)dmalloc(8 * (size_t)list_cap, "hub offsets");
        w->hub_cstart = (uint32_t *)dmalloc(4 * (size_t)kHubChunkTab, "hub chunk starts");
        const size_t ngroups = (size_t)(nseeds + kSeedGroup - 1) / kSeedGroup + 1;
        w->grp_units = (unsigned long long *)dmalloc(8 * ngroups, "seed group units");
        w->grp_off = (unsigned long long *)dmalloc(8 * ngroups, "seed group units");
        w->tmp_beg = (int64_t *)dmalloc(8 * (size_t)list_cap, "push records");
        w->tmp_deg = (int32_t *)dmalloc(4 * (size_t)list_cap, "push records");
        w->tmp_w = (float *)dmalloc(4 * (size_t)list_cap, "push records");
        w->tmp_jb = (uint32_t *)dmalloc(4 * (size_t)list_cap, "push records");
        w->seg_cnt = (unsigned *)dmalloc(4 * 3 * (size_t)nseeds, "segments");
        w->seg_off = (unsigned *)dmalloc(4 * 3 * (size_t)nseeds, "segments");
        w->seg_cur = (unsigned *)dmalloc(4 * 2 * (size_t)nseeds, "segments");
        w->seg_hvol = (unsigned long long *)dmalloc(8 * (size_t)nseeds, "segments");
        w->vol_off = (unsigned long long *)dmalloc(8 * (size_t)nseeds, "segments");
        w->seg_hcur = (unsigned long long *)dmalloc(8 * (size_t)nseeds, "segments");
        w->seeds = (int32_t *)dmalloc(4 * (size_t)nseeds, "seeds");
        w->status = (int32_t *)dmalloc(4 * (size_t)nseeds, "seed status");
        w->inserts = (unsigned *)dmalloc(4 * (size_t)nseeds, "seed inserts");
        w->svol = (unsigned long long *)dmalloc(8 * (size_t)nseeds, "seed volume");
        w->spushes = (unsigned *)dmalloc(4 * (size_t)nseeds, "seed pushes");
        w->slast = (int32_t *)dmalloc(4 * (size_t)nseeds, "seed rounds");
        w->spush = (double *)dmalloc(8 * (size_t)nseeds, "seed pushed mass");
        w->sscat = (double *)dmalloc(8 * (size_t)nseeds, "seed scattered mass");
        w->smass0 = (double *)dmalloc(8 * (size_t)nseeds, "seed source mass");
        w->xsrc = (double *)dmalloc(8 * (size_t)nseeds, "seed source entries");
        w->xcap = cap < xcap_max ? cap : xcap_max;
        w->xlist = (uint32_t *)dmalloc(4 * (size_t)nseeds * (size_t)w->xcap, "x lists");
        w->xnode = (uint32_t *)dmalloc(4 * (size_t)nseeds * (size_t)w->xcap, "x lists");
        w->xcnt = (unsigned *)dmalloc(4 * (size_t)nseeds, "x list lengths");
        w->glob = (BGlobal *)dmalloc(sizeof(BGlobal), "batch control");
        w->log = (RoundLog *)dmalloc(sizeof(RoundLog) * kLogCap, "round log");
        int per_sm = 0;
        GDE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_rounds<false, false>, kThreads, 0));
        int per_sm_layered = 0, per_sm_paged = 0;
        GDE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_layered, k_batch_rounds<true, false>, kThreads, 0));
        GDE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_paged, k_batch_rounds<false, true>, kThreads, 0));
        per_sm = std::min(per_sm, std::min(per_sm_layered, per_sm_paged));  // one grid serves all
        int dev = 0, sms = 0;
        GDE_CUDA(cudaGetDevice(&dev));
        GDE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        GDE_REQUIRE(per_sm > 0, GDE_ECUDA, "batched kernel cannot be resident");
        w->grid = sms * per_sm;
        w->sms = sms;
    } catch (...) {
        batch_free(w);
        throw;
    }
    return w;
}

static BatchWork *batch_work_get(Graph &g, int64_t nseeds, int64_t cap, int64_t list_cap) {
    BatchWork *w = g.batch;
    if (w && w->nseeds_cap >= nseeds && w->cap == cap && w->list_cap >= list_cap) return w;
    if (w) { batch_free(w); g.batch = nullptr; }
    g.batch = batch_work_alloc(nseeds, cap, list_cap);
    return g.batch;
}

// packed columns (id | degree code) of the current CSR, built on first use
void ensure_colp(Graph &g, cudaStream_t s) {
    if ((g.colp && g.colp_valid) || g.nnz <= 0) return;
    int idbits = 1;
    while (((int64_t)1 << idbits) < g.n) idbits++;
    const int spare = 32 - idbits;
    if (spare < 5) return;
    const int codes = spare >= 8 ? 256 : (1 << spare);
    if (g.colp_cap < g.nnz) {
        // after edge insertions the graph has grown: leave room for more
        const int64_t cap = g.colp_cap ? g.nnz + g.nnz / 4 + 1024 : g.nnz;
        dfree(g.colp);
        g.colp = nullptr;
        g.colp_cap = 0;
        g.colp = (uint32_t *)dmalloc(4 * (size_t)cap, "packed columns");
        g.colp_cap = cap;
    }
    g.colp_valid = true;
    g.colp_idbits = idbits;
    g.colp_exact = codes - 32;
    k_pack_columns<<<kSMs * 8, kThreads, 0, s>>>(g.nnz, g.col, g.deg, g.colp, idbits, g.colp_exact);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
}

__global__ void k_hub_ranks(int64_t H, const int32_t *hub_node, int32_t *hub_rank) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < H; r += (int64_t)gridDim.x * blockDim.x)
        hub_rank[hub_node[r]] = (int32_t)r;
}

// colq: colp with each hub's rank in place of its id (the degree code is unchanged)
__global__ void k_pack_hub_columns(int64_t nnz, const uint32_t *colp, const int32_t *hub_rank, uint32_t *colq,
                                   int idbits, uint32_t idmask, uint32_t hub_code) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = colp[e];
        const uint32_t code = w >> idbits;
        colq[e] = code >= hub_code ? ((uint32_t)hub_rank[w & idmask] | (code << idbits)) : w;
    }
}

void hubs_free(Graph &g) {
    dfree(g.colq); g.colq = nullptr; g.colq_cap = 0;
    dfree(g.hub_node); g.hub_node = nullptr;
    dfree(g.hub_deg); g.hub_deg = nullptr;
    dfree(g.hub_rank); g.hub_rank = nullptr;
    g.hub_cap = 0;
    g.hub_n = 0;
    g.hub_valid = false;
    g.hub_node_host.clear();
}

// The degree code that marks hubs of degree >= min_deg: the degree itself below code_exact,
// else the log2 class (min_deg is then rounded up to a power of two, the classes' bounds).
static uint32_t hub_code_of(int32_t *min_deg, int code_exact) {
    if (*min_deg <= code_exact) return (uint32_t)*min_deg;
    int k = 0;
    while ((1ll << k) < (long long)*min_deg) k++;
    *min_deg = (int32_t)(1ll << k);
    return (uint32_t)(code_exact + k);
}

bool ensure_hubs(Graph &g, int32_t min_deg, cudaStream_t s) {
    ensure_colp(g, s);
    if (!g.colp_valid || g.colp_idbits <= 0 || min_deg < 2) return false;
    const uint32_t code = hub_code_of(&min_deg, g.colp_exact);
    if (g.hub_valid && g.hub_min_deg == min_deg) return true;
    // rank the hubs by degree (descending, then id): the hottest ones share sectors
    std::vector<int32_t> deg((size_t)g.n);
    if (g.n > 0) GDE_CUDA(cudaMemcpyAsync(deg.data(), g.deg, 4 * (size_t)g.n, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> hubs;
    for (int64_t v = 0; v < g.n; v++)
        if (deg[(size_t)v] >= min_deg) hubs.push_back((int32_t)v);
    std::stable_sort(hubs.begin(), hubs.end(), [&](int32_t x, int32_t y) { return deg[(size_t)x] > deg[(size_t)y]; });
    const int64_t H = (int64_t)hubs.size();
    std::vector<int32_t> hdeg((size_t)H);
    for (int64_t r = 0; r < H; r++) hdeg[(size_t)r] = deg[(size_t)hubs[(size_t)r]];
    g.hub_valid = false;
    if (g.hub_cap < H || !g.hub_node) {
        dfree(g.hub_node); g.hub_node = nullptr;
        dfree(g.hub_deg); g.hub_deg = nullptr;
        g.hub_cap = 0;
        g.hub_node = (int32_t *)dmalloc(4 * (size_t)(H > 0 ? H : 1), "hub ranks");
        g.hub_deg = (int32_t *)dmalloc(4 * (size_t)(H > 0 ? H : 1), "hub degrees");
        g.hub_cap = H;
    }
    if (!g.hub_rank) g.hub_rank = (int32_t *)dmalloc(4 * (size_t)(g.n > 0 ? g.n : 1), "hub rank of each node");
    if (g.colq_cap < g.nnz || !g.colq) {
        dfree(g.colq); g.colq = nullptr; g.colq_cap = 0;
        g.colq = (uint32_t *)dmalloc(4 * (size_t)(g.colp_cap > 0 ? g.colp_cap : 1), "hub packed columns");
        g.colq_cap = g.colp_cap;
    }
    if (H > 0) {
        GDE_CUDA(cudaMemcpyAsync(g.hub_node, hubs.data(), 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        GDE_CUDA(cudaMemcpyAsync(g.hub_deg, hdeg.data(), 4 * (size_t)H, cudaMemcpyHostToDevice, s));
    }
    GDE_CUDA(cudaMemsetAsync(g.hub_rank, 0xFF, 4 * (size_t)(g.n > 0 ? g.n : 1), s));
    if (H > 0) {
        k_hub_ranks<<<kSMs * 4, kThreads, 0, s>>>(H, g.hub_node, g.hub_rank);
        GDE_CUDA(cudaGetLastError());
    }
    const uint32_t idmask = (uint32_t)(((uint64_t)1 << g.colp_idbits) - 1);
    k_pack_hub_columns<<<kSMs * 8, kThreads, 0, s>>>(g.nnz, g.colp, g.hub_rank, g.colq, g.colp_idbits, idmask, code);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched(H > 0 ? 2 : 1);
    GDE_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    g.hub_node_host.swap(hubs);
    g.hub_n = H;
    g.hub_min_deg = min_deg;
    g.hub_code = code;
    g.hub_valid = true;
    return true;
}

// the fields of the round kernel's arguments that come from the graph and the workspace
static BArgs bargs_base(Graph &g, BatchWork *w, int64_t cap, int64_t list_cap, int32_t nseeds,
                        uint32_t key_tag, uint32_t key_idmask) {
    BArgs a{};
    a.off = g.off; a.col = g.col; a.thr32 = w->thr32; a.kr = w->kr; a.xs = w->xs;
    a.colp = g.colp_valid ? g.colp : nullptr; a.idbits = g.colp_idbits;
    a.idmask = a.colp ? (uint32_t)(((uint64_t)1 << g.colp_idbits) - 1) : 0xFFFFFFFFu;
    a.code_exact = g.colp_exact;
    a.thr_stride = g.n;
    a.key_idmask = key_idmask; a.key_tag = key_tag;
    a.xlist = w->xlist; a.xnode = w->xnode; a.xcnt = w->xcnt; a.xcap = (unsigned)w->xcap;
    a.spush = w->spush; a.sscat = w->sscat;
    a.log2cap = w->log2cap; a.mask = (uint32_t)(cap - 1); a.nseeds = nseeds;
    a.status = w->status; a.inserts = w->inserts;
    a.load_limit = (unsigned)(cap * 3 / 4);
    a.svol = w->svol; a.spushes = w->spushes; a.slast = w->slast;
    a.cand[0] = w->cand[0]; a.cand[1] = w->cand[1];
    a.list_cap = (unsigned)list_cap;
    for (int b = 0; b < 3; b++) { a.b_beg[b] = w->b_beg[b]; a.b_deg[b] = w->b_deg[b]; a.b_w[b] = w->b_w[b]; a.b_seed[b] = w->b_seed[b]; }
    a.hub_vstart = w->hub_vstart; a.hub_cstart = w->hub_cstart;
    a.grp_units = w->grp_units; a.grp_off = w->grp_off;
    a.tmp_beg = w->tmp_beg; a.tmp_deg = w->tmp_deg; a.tmp_w = w->tmp_w; a.tmp_jb = w->tmp_jb;
    a.seg_cnt = w->seg_cnt; a.seg_off = w->seg_off; a.seg_cur = w->seg_cur;
    a.seg_hvol = w->seg_hvol; a.vol_off = w->vol_off; a.seg_hcur = w->seg_hcur;
    a.glob = w->glob; a.log = w->log;
    const Bins &bins = g.bins;
    a.t1 = bins.t1; a.t2 = bins.t2; a.chunk = bins.chunk; a.schedule = bins.schedule;
    a.bar_limit_ns = g.dbg_bar_limit_ns;
    a.fail_block = g.dbg_fail_block;
    a.fail_barrier = g.dbg_fail_barrier;
    return a;
}

// cooperative launch of the round kernel on the persistent grid (tuning's blocks_per_sm)
static void launch_rounds(Graph &g, BatchWork *w, const BArgs &a, cudaStream_t s) {
    int grid = w->grid;
    if (g.bins.blocks_per_sm > 0 && g.bins.blocks_per_sm * w->sms < grid) grid = g.bins.blocks_per_sm * w->sms;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int pr = g.prof.start(kProfBatchRounds, s);
    if (a.layer_eps) GDE_CUDA(cudaLaunchKernelEx(&cfg, k_batch_rounds<true, false>, a));
    else if (a.page_owner) GDE_CUDA(cudaLaunchKernelEx(&cfg, k_batch_rounds<false, true>, a));
    else GDE_CUDA(cudaLaunchKernelEx(&cfg, k_batch_rounds<false, false>, a));
    g.prof.launched();
    g.prof.stop(pr, s);
}

static inline int64_t floor_pow2(int64_t v) {
    int64_t p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

static inline int64_t ceil_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p *= 2;
    return p;
}

// Hubs of the slab a batched solve of nseeds seeds with tables of cap slots gets (0: no slab):
// the tuning asks for one, the graph has packed columns and hubs, the slab ids fit 32 bits
// after the pool's slot ids, and the slabs (two residual banks for the layered kinds) fit
// kSlabMaxBytes.  Builds the hub data if needed.
static int64_t slab_hubs(Graph &g, const SolveParams &p, int64_t nseeds, int64_t cap, cudaStream_t s) {
    if (g.bins.hub_degree <= 0 || !ensure_hubs(g, g.bins.hub_degree, s) || g.hub_n <= 0) return 0;
    const uint64_t entry_bytes = layered(p.kind) ? 20ull : 12ull;
    if ((uint64_t)nseeds * (uint64_t)(cap + g.hub_n) > ((uint64_t)1 << 32)) return 0;
    if ((uint64_t)nseeds * (uint64_t)g.hub_n * entry_bytes > kSlabMaxBytes) return 0;
    return g.hub_n;
}

// Prepares a batched solve of nseeds seeds on workspace w (tables of cap slots, candidate and
// bin lists of list_cap entries): copies the seed ids, builds the packed columns, takes the
// solve's epoch tag (clearing the pool on first use, after a failure or when the tag wraps),
// the layered kinds' x tables and per-round constants or the per-node thresholds, and seeds
// every table.  Returns the round kernel's arguments for round 0.
static BArgs batch_setup(Graph &g, const SolveParams &p, BatchWork *w, const int32_t *seeds_dev, int32_t nseeds,
                         int64_t cap, int64_t list_cap, uint32_t *key_tag_out, uint32_t *key_idmask_out) {
    const bool lay = layered(p.kind);
    cudaStream_t s = p.stream;
    GDE_CUDA(cudaMemcpyAsync(w->seeds, seeds_dev, 4 * (size_t)nseeds, cudaMemcpyDeviceToDevice, s));
    ensure_colp(g, s);
    // epoch tags: keys carry the solve's tag above their id bits, so the previous solve's keys
    // read as empty; the tables are only reset on first use, after a failure, or when the tag
    // wraps (x is zeroed by the previous top-k through the x-lists)
    int key_idbits = 1;
    while (((int64_t)1 << key_idbits) < g.n) key_idbits++;
    const int tag_bits = 32 - key_idbits < 8 ? 32 - key_idbits : 8;
    const uint32_t max_tag = tag_bits >= 2 ? (1u << tag_bits) - 2u : 0u;  // never all ones
    // a layered solve gives every layer its own tag: nlayers + 1 layers, and the keys the last
    // layer's (empty) scatter would write
    const int64_t nlayers = lay ? p.hk_N : 0;
    const uint32_t tags = lay ? (uint32_t)(nlayers + 2) : 1u;
    GDE_REQUIRE(!lay || (nlayers + 2 <= (int64_t)max_tag), GDE_EINVAL,
                "batched layered solve: more layers than this graph's key tags can tell apart");
    bool fresh_x = false;
    if (lay && (w->xt_seeds != (int64_t)nseeds || w->xt_cap != cap / 2)) {
        dfree(w->xkr); w->xkr = nullptr;
        dfree(w->xxs); w->xxs = nullptr;
        w->xt_seeds = w->xt_cap = 0;
        const int64_t xcap = cap / 2;
        w->xkr = (unsigned long long *)dmalloc(8 * (size_t)nseeds * (size_t)xcap, "x tables");
        w->xxs = (float *)dmalloc(4 * (size_t)nseeds * (size_t)xcap, "x tables");
        w->xt_seeds = nseeds;
        w->xt_cap = xcap;
        w->xt_log2cap = 0;
        while (((int64_t)1 << w->xt_log2cap) < xcap) w->xt_log2cap++;
        fresh_x = true;
    }
    w->epoch = w->epoch + 1;
    if (w->need_clear || w->epoch + tags - 1 > max_tag || fresh_x) {
        const int pc = g.prof.start(kProfBatchClear, s);
        k_batch_clear<<<kSMs * 8, kThreads, 0, s>>>(w->pool, w->kr, w->xs);
        GDE_CUDA(cudaGetLastError());
        g.prof.launched();
        if (w->xkr) {
            k_batch_clear<<<kSMs * 8, kThreads, 0, s>>>(w->xt_seeds * w->xt_cap, w->xkr, w->xxs);
            GDE_CUDA(cudaGetLastError());
            g.prof.launched();
        }
        g.prof.stop(pc, s);
        w->epoch = max_tag >= 1 ? 1u : 0u;
    }
    w->need_clear = true;  // until this solve completes
    const uint32_t key_tag = w->epoch << key_idbits;
    w->epoch += tags - 1;  // the last tag this solve uses
    const uint32_t key_idmask = (uint32_t)(((uint64_t)1 << key_idbits) - 1);
    if (lay) {
        // per-round constants: theta_t eps and the share coefficient of round t
        GDE_REQUIRE(g.colp_valid && g.colp_idbits > 0, GDE_EINVAL,
                    "batched layered solve: graph too large for packed columns");
        const int64_t nl1 = nlayers + 1;
        if (w->layer_cap < nl1) {
            dfree(w->layer_eps); w->layer_eps = nullptr;
            dfree(w->layer_coef); w->layer_coef = nullptr;
            w->layer_cap = 0;
            w->layer_eps = (double *)dmalloc(8 * (size_t)nl1, "layer constants");
            w->layer_coef = (double *)dmalloc(8 * (size_t)nl1, "layer constants");
            w->layer_cap = nl1;
        }
        std::vector<double> le((size_t)nl1), lc((size_t)nl1);
        for (int64_t t = 0; t < nl1; t++) {
            le[(size_t)t] = layer_theta(p, t) * p.eps;
            lc[(size_t)t] = layer_ratio(p, t);
        }
        GDE_CUDA(cudaMemcpyAsync(w->layer_eps, le.data(), 8 * (size_t)nl1, cudaMemcpyHostToDevice, s));
        GDE_CUDA(cudaMemcpyAsync(w->layer_coef, lc.data(), 8 * (size_t)nl1, cudaMemcpyHostToDevice, s));
        GDE_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    } else if (w->thr_eps != p.eps || w->thr_n != g.n || !w->thr32) {
        if (!w->thr32) w->thr32 = (float *)dmalloc(4 * (size_t)(g.n > 0 ? g.n : 1), "thresholds");
        k_batch_thr<<<kSMs * 8, kThreads, 0, s>>>(g.n, g.deg, w->thr32, p.eps);
        GDE_CUDA(cudaGetLastError());
        g.prof.launched();
        w->thr_eps = p.eps;
        w->thr_n = g.n;
    }
    // hub slab: the residuals of nodes of degree >= the tuning's hub_degree live in a dense
    // fixed-point array per seed (two banks, one per layer parity, for the layered kinds); ids of
    // slab entries follow the pool's slot ids, so both must fit 32 bits; at most kSlabMaxBytes
    const bool katz_f = p.kind == GDE_KATZ && p.katz_minus_source;
    w->slab_on = false;
    SeedSlab sl{};
    const int banks = lay ? 2 : 1;
    if (w->z_pending) {
        // the last solve's slab zeroing (side stream) completes before this solve touches it
        GDE_CUDA(cudaStreamWaitEvent(s, w->z_done, 0));
        w->z_pending = false;
    }
    if (slab_hubs(g, p, nseeds, cap, s) > 0) {
        const int64_t H = g.hub_n;
        if (!w->slab || w->slab_seeds < (int64_t)nseeds || w->slab_banks < banks || w->slab_H != H) {
            // grow to cover both this solve and the last allocation (PPR and the layered kinds
            // alternate without reallocating when H is unchanged)
            int64_t cs = w->slab && w->slab_H == H ? std::max<int64_t>(w->slab_seeds, nseeds) : nseeds;
            int cb = w->slab && w->slab_H == H ? std::max(w->slab_banks, banks) : banks;
            if ((uint64_t)cs * (uint64_t)H * (8ull * (uint64_t)cb + 4ull) > kSlabMaxBytes) {
                cs = nseeds;
                cb = banks;
            }
            if (w->z_done) GDE_CUDA(cudaEventSynchronize(w->z_done));
            dfree(w->slab); w->slab = nullptr;
            dfree(w->slab_x); w->slab_x = nullptr;
            w->slab_seeds = w->slab_H = 0;
            w->slab_banks = 0;
            w->slab = (unsigned long long *)dmalloc(8 * (size_t)cs * (size_t)H * (size_t)cb, "hub slab");
            w->slab_x = (float *)dmalloc(4 * (size_t)cs * (size_t)H, "hub slab x");
            w->slab_seeds = cs;
            w->slab_banks = cb;
            w->slab_H = H;
            w->slab_x_dirty = true;
            w->slab_dirty = true;
        }
        // residual counts start at zero: PPR and Katz leave the remainders of touched hubs behind
        // (one memset per solve), while a completed layered solve leaves every bank empty (its
        // frontier takes every entry it lists), so only a new slab or a failed, capped or
        // overflowed layered solve needs one; x is zeroed by the top-k through the x-lists.  A
        // dirty array is zeroed whole: a solve may use more seeds or banks than the one before
        const size_t cap_entries = (size_t)w->slab_seeds * (size_t)H;
        if (w->slab_dirty) GDE_CUDA(cudaMemsetAsync(w->slab, 0, 8 * cap_entries * (size_t)w->slab_banks, s));
        if (w->slab_x_dirty) GDE_CUDA(cudaMemsetAsync(w->slab_x, 0, 4 * cap_entries, s));
        w->slab_x_dirty = true;  // until this solve's top-k has run
        w->slab_dirty = true;    // until this solve has completed
        // fixed-point scale 2^qexp: the finest whose counts (below the 2^62 overflow mark) hold
        // 64 times the largest residual the solve can reach: the source mass for PPR and Katz
        // (the generalised propagation's source is d_s^b), the largest layer mass
        // prod_{s<t} c_{s+1}/c_s for the layered kinds
        double m_max = 1.0;
        if (p.gbeta != 0.0) m_max = std::pow((double)(g.max_degree > 1 ? g.max_degree : 1), p.gbeta);
        if (lay) {
            double prod = 1.0;
            for (int64_t t = 0; t < nlayers; t++) {
                prod *= layer_ratio(p, t);
                if (prod > m_max) m_max = prod;
            }
        }
        const int qexp = (int)std::ceil(std::log2(64.0 * m_max)) - 62;
        w->slab_on = true;
        w->slab_base = (uint32_t)((int64_t)nseeds * cap);
        w->qexp = qexp;
        sl.slab = w->slab;
        sl.hub_rank = g.hub_rank;
        sl.H = H;
        sl.slab_base = w->slab_base;
        sl.tscale = std::ldexp(1.0, -qexp);
    }
    GDE_CUDA(cudaMemsetAsync(w->log, 0, sizeof(RoundLog) * kLogCap, s));
    k_batch_seed<<<(nseeds + kThreads - 1) / kThreads, kThreads, 0, s>>>(
        nseeds, w->seeds, w->kr, w->cand[0], w->log2cap, (uint32_t)(cap - 1), w->glob, w->status,
        w->inserts, w->svol, w->spushes, w->slast, key_tag, w->xcnt, w->spush, w->sscat, g.deg, p.gbeta,
        w->smass0, sl, katz_f ? w->xsrc : nullptr);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();

    BArgs a = bargs_base(g, w, cap, list_cap, nseeds, key_tag, key_idmask);
    if (katz_f) {
        a.xsrc = w->xsrc;
        a.seed_ids = w->seeds;
    }
    if (w->slab_on) {
        a.colp = g.colq;  // hub words carry the hub's rank
        a.slab = w->slab;
        a.slab_x = w->slab_x;
        a.H = g.hub_n;
        a.slab_bank = (uint64_t)nseeds * (uint64_t)g.hub_n;
        a.slab_base = w->slab_base;
        a.hub_code = g.hub_code;
        a.hub_node = g.hub_node;
        a.hub_deg = g.hub_deg;
        a.qexp = w->qexp;
        a.wscale = std::ldexp(1.0f, -w->qexp);
        a.vscale = std::ldexp(1.0, w->qexp);
        a.tscale = std::ldexp(1.0, -w->qexp);
    }
    a.eps = p.eps;
    a.eps_cls[0] = p.eps; a.ncls = 1; a.sparam = nullptr; a.t0 = 0;
    GDE_CUDA(cudaMemsetAsync(w->seg_cnt, 0, 4 * 3 * (size_t)nseeds, s));
    GDE_CUDA(cudaMemsetAsync(w->seg_hvol, 0, 8 * (size_t)nseeds, s));
    a.kind = p.kind == GDE_GPPR ? GDE_PPR : p.kind;
    a.cx = a.kind == GDE_PPR ? p.param : 1.0;
    a.coef = a.kind == GDE_PPR ? 1.0 - p.param : p.param;
    a.gbeta = p.gbeta;
    a.max_rounds = p.max_rounds;
    if (lay) {
        a.kind = GDE_HK;  // shares divided by d_u, x += r_u
        a.cx = 1.0;
        a.coef = 0.0;
        a.gbeta = 0.0;
        a.layer_eps = w->layer_eps;
        a.layer_coef = w->layer_coef;
        a.nlayers = nlayers;
        a.tag_step = 1u << key_idbits;
        a.xkr = w->xkr;
        a.xxs = w->xxs;
        a.xlog2cap = w->xt_log2cap;
        a.xmask = (uint32_t)(w->xt_cap - 1);
    }
    *key_tag_out = key_tag;
    *key_idmask_out = key_idmask;
    return a;
}

// Runs a batched PPR/Katz solve.  seeds_dev: device seed ids.  Outputs (device): ids[nseeds*k],
// vals[nseeds*k] (float).  stats_host may be NULL.  Seeds whose table overflowed are reported
// with status GDE_ENOMEM in stats and in *n_overflow; their outputs are not valid.
static void batch_solve_once(Graph &g, const SolveParams &p, const int32_t *seeds_dev, int32_t nseeds, int k,
                             int64_t mem_budget, int32_t *ids_dev, float *vals_dev, gde_stats *stats_host,
                             int32_t *overflow_seeds_host, int32_t *n_overflow, int list_scale,
                             bool *list_full) {
    GDE_REQUIRE(k >= 1 && k <= kTopMax, GDE_EINVAL, "batched mode needs 1 <= topk <= 64");
    GDE_REQUIRE(p.kind == GDE_PPR || p.kind == GDE_KATZ || p.kind == GDE_GPPR || layered(p.kind), GDE_EINVAL,
                "batched mode supports PPR, Katz, the generalised propagation, the heat kernel and series");
    GDE_REQUIRE(p.precision == GDE_FP32, GDE_EINVAL, "batched mode stores x and r in FP32");
    GDE_REQUIRE(g.n < ((int64_t)1 << 31) - 1, GDE_EINVAL, "graph too large for 32-bit keys");
    const bool lay = layered(p.kind);
    const int64_t budget = mem_budget > 0 ? mem_budget : ((int64_t)16 << 30);
    // layered kinds add an x table of half the residual table's slots (12 + 6 bytes per slot)
    int64_t cap = floor_pow2(budget / ((lay ? 18 : 12) * (int64_t)nseeds));
    // a table of 2n slots never exceeds half load (at most n keys)
    // (at most 2^31 slots per table: slot indices are 32-bit and carry the seed above log2(cap))
    const int64_t cap_max = std::min<int64_t>(ceil_pow2(2 * (g.n > 0 ? g.n : 1)), (int64_t)1 << 31);
    if (cap > cap_max) cap = cap_max;
    GDE_REQUIRE(cap >= 64 || cap == cap_max, GDE_ENOMEM, "memory budget too small for the batch");
    GDE_REQUIRE((int64_t)nseeds * cap <= ((int64_t)1 << 32), GDE_EINVAL, "batch pool exceeds 2^32 slots");
    // candidate and bin lists: every slot (and hub slab entry) can enter a list at most once
    // per round, but the per-round frontier of all seeds together is far smaller than the pool;
    // past this capacity the solve reports GDE_ENOMEM
    const int64_t entries = (int64_t)nseeds * (cap + slab_hubs(g, p, nseeds, cap, p.stream));
    int64_t list_cap = entries;
    int64_t list_max = (int64_t)nseeds << 14;
    if (list_max < ((int64_t)1 << 22)) list_max = (int64_t)1 << 22;
    if (list_max > ((int64_t)1 << 24)) list_max = (int64_t)1 << 24;
    list_max <<= 2 * list_scale;  // a retry after an overflow: four times larger
    if (list_cap > list_max) list_cap = list_max;
    GDE_REQUIRE(nseeds <= list_cap, GDE_EINVAL, "too many seeds for one batch");
    *list_full = list_cap == entries;
    BatchWork *w = batch_work_get(g, nseeds, cap, list_cap);
    if (w->list_cap > list_cap) {
        // a workspace that an earlier solve left larger keeps its longer lists
        list_cap = std::min<int64_t>(w->list_cap, std::min<int64_t>(entries, 0xFFFFFFFFll));
        *list_full = list_cap == entries;
    }
    cudaStream_t s = p.stream;
    uint32_t key_tag = 0, key_idmask = 0;
    BArgs a = batch_setup(g, p, w, seeds_dev, nseeds, cap, list_cap, &key_tag, &key_idmask);
    (void)key_tag;
    launch_rounds(g, w, a, s);
    if (w->slab_on && !lay) {
        // PPR and Katz leave residual counts behind; nothing reads them after the round
        // kernel, so they are zeroed now, beside the top-k, instead of before the next solve
        if (!w->zs) {
            GDE_CUDA(cudaStreamCreateWithFlags(&w->zs, cudaStreamNonBlocking));
            GDE_CUDA(cudaEventCreateWithFlags(&w->z_start, cudaEventDisableTiming));
            GDE_CUDA(cudaEventCreateWithFlags(&w->z_done, cudaEventDisableTiming));
        }
        GDE_CUDA(cudaEventRecord(w->z_start, s));
        GDE_CUDA(cudaStreamWaitEvent(w->zs, w->z_start, 0));
        GDE_CUDA(cudaMemsetAsync(w->slab, 0, 8 * (size_t)w->slab_seeds * (size_t)w->slab_H * (size_t)w->slab_banks,
                                 w->zs));
        GDE_CUDA(cudaEventRecord(w->z_done, w->zs));
        w->z_pending = true;
        w->slab_dirty = false;
    }

    TopkArgs ta{};
    ta.kr = w->kr; ta.xs = w->xs; ta.log2cap = w->log2cap; ta.cap = cap; ta.k = k;
    ta.key_idmask = key_idmask; ta.xlist = w->xlist; ta.xnode = w->xnode; ta.xcnt = w->xcnt;
    ta.xcap = (unsigned)w->xcap;
    ta.out_ids = ids_dev; ta.out_vals = vals_dev; ta.ssupport = w->inserts;
    if (lay) {
        // x lives in the x tables; the output is e^-tau x (heat kernel) or c_0 x (series)
        ta.kr = w->xkr; ta.xs = w->xxs; ta.log2cap = w->xt_log2cap; ta.cap = w->xt_cap;
        ta.scale = (float)(p.kind == GDE_SERIES ? p.series[0] : std::exp(-p.param));
    }
    if (w->slab_on) {
        ta.slab_x = w->slab_x; ta.slab_base = w->slab_base; ta.H = g.hub_n; ta.hub_node = g.hub_node;
    }
    if (p.kind == GDE_KATZ && p.katz_minus_source) {
        ta.xsrc = w->xsrc; ta.seed_ids = w->seeds;
    }
    const int pt = g.prof.start(kProfBatchTopk, s);
    k_batch_topk<<<nseeds, kTopkThreads, 0, s>>>(ta);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
    g.prof.stop(pt, s);

    // per-seed results
    BGlobal hg;
    GDE_CUDA(cudaMemcpyAsync(&hg, w->glob, sizeof(BGlobal), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> st(nseeds), last(nseeds);
    std::vector<unsigned long long> vol(nseeds);
    std::vector<unsigned> pushes(nseeds);
    std::vector<double> pushed(nseeds), scat(nseeds), m0(nseeds);
    std::vector<unsigned> ins(nseeds);
    GDE_CUDA(cudaMemcpyAsync(st.data(), w->status, 4 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
    if (g.prof.enabled)
        GDE_CUDA(cudaMemcpyAsync(ins.data(), w->inserts, 4 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
    if (stats_host || g.prof.enabled) {
        GDE_CUDA(cudaMemcpyAsync(last.data(), w->slast, 4 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(vol.data(), w->svol, 8 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(pushes.data(), w->spushes, 4 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(pushed.data(), w->spush, 8 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(scat.data(), w->sscat, 8 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(m0.data(), w->smass0, 8 * (size_t)nseeds, cudaMemcpyDeviceToHost, s));
    }
    GDE_CUDA(cudaStreamSynchronize(s));
    w->need_clear = false;  // the top-k zeroed x on every x-list (or table) it read
    if (w->slab_on) w->slab_x_dirty = false;
    if (hg.error == GDE_ETIMEOUT) {
        set_error("batched solve: a grid barrier wait timed out");
        throw Fail{GDE_ETIMEOUT};
    }
    if (hg.error != 0) {
        set_error("batched solve: candidate or bin list capacity exceeded");
        w->list_overflowed = hg.error == GDE_ENOMEM;
        throw Fail{(gde_status)hg.error};
    }
    w->last_rounds = hg.rounds;
    if (g.prof.enabled) {
        g.prof.counters.batch_launches += 1;
        g.prof.counters.rounds += hg.rounds;
        for (int32_t j = 0; j < nseeds; j++) {
            g.prof.counters.edges += (int64_t)vol[j];
            g.prof.counters.pushes += pushes[j];
            g.prof.counters.support += ins[j];
        }
    }
    const bool capped = (int64_t)hg.rounds >= p.max_rounds;
    int32_t nof = 0;
    for (int32_t j = 0; j < nseeds; j++) {
        const bool of = st[j] != kSeedOk;
        if (of && overflow_seeds_host) overflow_seeds_host[nof] = j;
        if (of) nof++;
        if (stats_host) {
            gde_stats &o = stats_host[j];
            o.rounds = last[j] + 1;
            o.active_volume = (int64_t)vol[j];
            o.pushes = pushes[j];
            // unit source: ||r||_1 = 1 - pushed + scattered; ||x||_1 = c_x * pushed (layered
            // kinds leave each layer's remainder behind: not reported)
            o.resid_l1 = lay ? -1.0 : m0[j] - pushed[j] + scat[j];
            o.mass_l1 = lay ? -1.0 : (p.kind == GDE_KATZ ? 1.0 : p.param) * pushed[j];
            o.status = of ? GDE_ENOMEM : ((capped && last[j] + 1 >= (int64_t)hg.rounds) ? GDE_ENOTCONV : GDE_OK);
            o.fallback = 0;
        }
    }
    if (n_overflow) *n_overflow = nof;
    // a layered solve's frontier took every slab entry it listed, unless a seed overflowed (its
    // candidates are skipped) or the round cap stopped the solve with entries still listed
    if (w->slab_on && lay && nof == 0 && !capped) w->slab_dirty = false;
}

// ============================================================ serving pool ====
// A long-lived batch whose solves continue across launches (continuous batching): a query is
// admitted into a free slot (table cleared, unit residual at its seed, the slot listed as a
// candidate of the next round), resident queries are corrected after edge insertions (the
// Insert of Algorithm 3, Section 4, applied to every slot whose x touches a changed row), and
// each launch runs at most R rounds of all slots together, resuming the round counter, the
// candidate list and every table where the previous launch stopped.  Slots carry their own
// kind, coefficient and tolerance class.

// Memory: the pool is a paged array of table slots (12 bytes each, plus 8 bytes of x-list) of
// the server's memory budget.  A query's table is a power-of-two run of 2^order pages taken
// from a buddy allocator, so queries are admitted while their tables fit rather than by a
// fixed slot count, and a query that outgrows its table is started again with a larger one.
// Its x-list occupies the same range of the x-list arrays (a table cannot hold more x entries
// than slots).  A slot id names its query through the owner of its page.

struct ServePool {
    BatchWork *w = nullptr;
    int32_t slots = 0;           // query slots (concurrent queries at most)
    int64_t list_cap = 0;
    int pg_bits = 16;            // table slots per page: 2^pg_bits
    int64_t pages = 0;           // a power of two
    int max_order = 0;           // largest table: 2^max_order pages
    int64_t pages_used = 0;
    std::vector<std::set<int64_t>> free_blocks;  // per order: first pages of free blocks
    std::vector<int32_t> h_owner;  // per page: its query slot, or -1
    int32_t *d_owner = nullptr;
    bool owner_dirty = true;
    std::vector<int> order;        // per slot: its table's order, or -1 (no table)
    int ncls = 0;
    double eps[kMaxCls] = {};
    float *thr = nullptr;        // ncls arrays of n thresholds
    int64_t thr_n = -1;          // rebuilt when the graph changed
    SlotParam *d_param = nullptr;
    std::vector<SlotParam> h_param;
    uint32_t key_idmask = 0;
    uint32_t tag = 0;            // key tag of every table (tables are cleared at admission)
    int64_t T = 0;               // the next round to run
    int64_t volume = 0;          // edges pushed so far
    unsigned *pend = nullptr;    // per-slot candidates of the next round
    int32_t *d_list = nullptr;   // slot-list scratch
    int32_t *d_seeds = nullptr;
    int32_t *d_ids = nullptr;
    float *d_vals = nullptr;
    unsigned long long *d_partial = nullptr;  // top-k parts
    cudaStream_t s = nullptr;
    // slots whose last launch pushed more than defer_vol edges run one round per launch
    int64_t defer_vol = (int64_t)1 << 23;
    std::vector<unsigned long long> last_vol;  // per slot: its pushed volume after the last launch
    std::vector<uint8_t> heavy;
    std::vector<unsigned> h_pend;  // per slot: candidates the last launch left (when pend_valid)
    bool pend_valid = false;       // cleared by anything that changes the candidate list
};

// device view of the pool's tables, shared by the admission and correction kernels
struct SlotTable {
    unsigned long long *kr;
    float *xs;
    uint32_t key_idmask;
};

// slot of node v in the table [base, base + mask + 1), or -1 (the probe stops at the first
// free slot)
__device__ int64_t slot_find(const SlotTable &t, uint64_t base, uint32_t mask, uint32_t tag, uint32_t v) {
    const uint32_t kcur = v | tag;
    const uint32_t sector_mask = mask >= 3 ? 3u : mask;
    uint32_t h = mix32(v) & mask & ~sector_mask;
    for (uint32_t probes = 0; probes <= mask && probes < kMaxProbe; probes++) {
        const uint32_t key = (uint32_t)(ld_relaxed_u64(t.kr + base + h) & 0xFFFFFFFFull);
        if (key == kcur) return (int64_t)(base + h);
        if (key == kEmpty || (key & ~t.key_idmask) != tag) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// insert-or-add w at node v of the table [base, base + mask + 1); returns the slot (and the
// residual after the add in *nv), or -1 if the table is full
__device__ int64_t slot_add(const SlotTable &t, uint64_t base, uint32_t mask, uint32_t tag, uint32_t v, float w,
                            float *nv) {
    const uint32_t kcur = v | tag;
    const uint32_t sector_mask = mask >= 3 ? 3u : mask;
    uint32_t h = mix32(v) & mask & ~sector_mask;
    for (uint32_t probes = 0; probes <= mask && probes < kMaxProbe; probes++) {
        const uint64_t slot = base + h;
        unsigned long long wk = ld_relaxed_u64(t.kr + slot);
        for (;;) {
            const uint32_t key = (uint32_t)(wk & 0xFFFFFFFFull);
            if (key == kcur) {
                *nv = __fadd_rn(atomicAdd(r_of(t.kr, slot), w), w);
                return (int64_t)slot;
            }
            if (key != kEmpty && (key & ~t.key_idmask) == tag) break;
            const unsigned long long prev = atomicCAS(t.kr + slot, wk, slot_word(kcur, w));
            if (prev == wk) {
                *nv = w;
                return (int64_t)slot;
            }
            wk = prev;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ void list_append(uint32_t *cand, unsigned *count, unsigned cap, unsigned *error,
                                            uint32_t slot) {
    const unsigned pos = atomicAdd(count, 1u);
    if (pos < cap) cand[pos] = slot; else atomicCAS(error, 0u, (unsigned)GDE_ENOMEM);
}

// blockIdx.y: the i-th admitted slot; its table [base, base + 2^log2cap) is emptied (keys free,
// x zero) by gridDim.x blocks
__global__ void k_serve_clear(const int32_t *slots, const SlotParam *sparam, unsigned long long *kr, float *xs) {
    const SlotParam sp = sparam[slots[blockIdx.y]];
    const int64_t cap = (int64_t)1 << sp.log2cap;
    const unsigned long long empty = (unsigned long long)kEmpty;  // r = 0.0f in the high half
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x) {
        kr[sp.base + (uint64_t)i] = empty;
        xs[sp.base + (uint64_t)i] = 0.0f;
    }
}

struct AdmitArgs {
    SlotTable t;
    const SlotParam *sparam;
    int32_t n;
    const int32_t *slots;
    const int32_t *seeds;
    uint32_t tag;
    uint32_t *cand;
    unsigned *count;
    unsigned list_cap;
    unsigned *error;
    int32_t *status;
    unsigned *inserts;
    unsigned long long *svol;
    unsigned *spushes;
    int32_t *slast;
    unsigned *xcnt;
    double *spush;
    double *sscat;
};

// unit residual at the seed of each admitted slot (its table was just emptied, so the seed
// takes the first slot of its probe), per-slot counters reset, the seed's slot listed for the
// next round
__global__ void k_serve_seed(AdmitArgs a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int32_t j = a.slots[i];
    const SlotParam sp = a.sparam[j];
    const uint32_t mask = (uint32_t)((1ull << sp.log2cap) - 1);
    const uint32_t s = (uint32_t)a.seeds[i];
    const uint32_t sector_mask = mask >= 3 ? 3u : mask;
    const uint64_t slot = sp.base + (mix32(s) & mask & ~sector_mask);
    a.t.kr[slot] = ((unsigned long long)__float_as_uint(1.0f) << 32) | (unsigned long long)(s | a.tag);
    a.status[j] = kSeedOk;
    a.inserts[j] = 1;
    a.xcnt[j] = 0;
    a.spush[j] = 0.0;
    a.sscat[j] = 0.0;
    a.svol[j] = 0;
    a.spushes[j] = 0;
    a.slast[j] = -1;
    list_append(a.cand, a.count, a.list_cap, a.error, (uint32_t)slot);
}

struct CorrectArgs {
    SlotTable t;
    const SlotParam *sparam;
    const float *thr;
    int64_t thr_stride;
    const int32_t *res;       // resident slots
    int32_t nres;
    const int32_t *row;       // rows that gained adjacencies (EdgeBatch)
    const int32_t *row_cnt;
    const int64_t *row_start;
    const int32_t *old_deg;
    const int32_t *added;     // the gained columns, row by row
    int64_t rows;
    uint32_t *cand;
    unsigned *count;
    unsigned list_cap;
    unsigned *error;
    int32_t *status;
};

// One thread per (resident slot, changed row u).  PPR (unit mass, d the degree before the
// batch, k the adjacencies u gained, x_u / d unchanged by each single insertion):
//   x_u <- x_u (d + k) / d,  r_u -= k x_u / (alpha d),  r_v += (1 - alpha) x_u / (alpha d) for
//   each gained v; a row of degree 0 scatters nothing before its first adjacency, so there
//   x_u <- k x_u, r_u -= (k - 1) x_u / alpha, r_v += (1 - alpha) x_u / alpha.
// Katz: r_v += beta x_u for each gained v.  (x and d before the batch: the per-insertion
// updates of a batch commute, so the batch is applied at once.)  Every residual that ends at
// or above its threshold is listed for the next round.
__global__ void k_serve_correct(CorrectArgs a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)a.nres * a.rows) return;
    const int32_t j = a.res[i / a.rows];
    const int64_t ri = i % a.rows;
    const int32_t u = a.row[ri];
    const SlotParam sp = a.sparam[j];
    const uint32_t mask = (uint32_t)((1ull << sp.log2cap) - 1);
    const int64_t su = slot_find(a.t, sp.base, mask, sp.tag, (uint32_t)u);
    if (su < 0) return;
    const float x = a.t.xs[su];
    if (x == 0.0f) return;
    const float *thr = a.thr + (int64_t)sp.cls * a.thr_stride;
    const int32_t k = a.row_cnt[ri];
    const int32_t d0 = a.old_deg[ri];
    const int64_t st = a.row_start[ri];
    float give;
    if (sp.divide) {
        const double alpha = sp.cx;
        const double denom = d0 > 0 ? (double)d0 : 1.0;
        const double share = (double)x / (alpha * denom);
        a.t.xs[su] = (float)(((double)x * (double)(d0 + k)) / denom);
        const double take = (double)(d0 > 0 ? k : k - 1) * share;
        if (take != 0.0) {
            const float tf = (float)take;
            const float old = atomicAdd(r_of(a.t.kr, (uint64_t)su), -tf);
            if (fabsf(__fadd_rn(old, -tf)) >= thr[u])
                list_append(a.cand, a.count, a.list_cap, a.error, (uint32_t)su);
        }
        give = (float)((1.0 - alpha) * share);
    } else {
        give = (float)(sp.coef * (double)x);
    }
    for (int32_t e = 0; e < k; e++) {
        const int32_t v = a.added[st + e];
        float nv = 0.0f;
        const int64_t sv = slot_add(a.t, sp.base, mask, sp.tag, (uint32_t)v, give, &nv);
        if (sv < 0) {
            atomicExch(a.status + j, kSeedOverflow);
            continue;
        }
        if (fabsf(nv) >= thr[v]) list_append(a.cand, a.count, a.list_cap, a.error, (uint32_t)sv);
    }
}

__global__ void k_serve_pending(const unsigned *count, unsigned list_cap, const uint32_t *cand,
                                const int32_t *page_owner, int pg_bits, unsigned *pend) {
    const unsigned n = min(*count, list_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t j = page_owner[cand[i] >> pg_bits];
        if (j >= 0) atomicAdd(pend + j, 1u);
    }
}

static unsigned *next_count(ServePool *P) {
    // candidates of round T sit in cand[T & 1], counted by the other parity's cand_out
    BCtl *ctl = &P->w->glob->ctl[(P->T & 1) ^ 1];
    return &ctl->cand_out;
}

static SlotTable slot_table(ServePool *P) {
    SlotTable t;
    t.kr = P->w->kr; t.xs = P->w->xs;
    t.key_idmask = P->key_idmask;
    return t;
}

static void serve_sync_owner(ServePool *P) {
    if (!P->owner_dirty) return;
    GDE_CUDA(cudaMemcpyAsync(P->d_owner, P->h_owner.data(), 4 * (size_t)P->pages, cudaMemcpyHostToDevice, P->s));
    GDE_CUDA(cudaStreamSynchronize(P->s));  // the host table may change before the next launch
    P->owner_dirty = false;
}

static void serve_check_error(ServePool *P) {
    unsigned err = 0;
    GDE_CUDA(cudaMemcpyAsync(&err, &P->w->glob->error, sizeof(unsigned), cudaMemcpyDeviceToHost, P->s));
    GDE_CUDA(cudaStreamSynchronize(P->s));
    if (err == GDE_ETIMEOUT) {
        set_error("serving pool: a grid barrier wait timed out");
        throw Fail{GDE_ETIMEOUT};
    }
    if (err != 0) {
        set_error("serving pool: candidate or bin list capacity exceeded");
        throw Fail{(gde_status)err};
    }
}

// Top-k of served queries in two passes, so a query with a large support is ranked by many
// blocks: block (i, c) ranks part c of query i's x-list into a partial top-64, then one block
// per query merges its parts.
constexpr int kServeTopkParts = 16;

__global__ void __launch_bounds__(kThreads) k_serve_topk_partial(TopkArgs a, const SlotParam *sparam,
                                                                 unsigned long long *partial) {
    const int qi = blockIdx.x / kServeTopkParts, part = blockIdx.x % kServeTopkParts;
    const int j = a.slots[qi];
    const SlotParam sp = sparam[j];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t cap = (int64_t)1 << sp.log2cap;
    const unsigned nx = a.xcnt[j];
    // the x-list has room for every slot of the table; a count past it would scan the table
    const bool use_list = (int64_t)nx <= cap;
    const int64_t n = use_list ? (int64_t)nx : cap;
    const int64_t per = (n + kServeTopkParts - 1) / kServeTopkParts;
    const int64_t lo = (int64_t)part * per, hi = min(lo + per, n);
    unsigned long long ta = 0, tb = 0;
    for (int64_t i0 = lo + (int64_t)wid * 32; i0 < hi; i0 += kThreads) {
        const int64_t i = i0 + lane;
        unsigned long long key = 0;
        if (i < hi) {
            const uint64_t li = sp.base + (uint64_t)i;
            const uint64_t slot = use_list ? (uint64_t)a.xlist[li] : sp.base + (uint64_t)i;
            const float x = a.xs[slot];
            if (x > 0.0f) {
                const uint32_t v = use_list ? a.xnode[li] : (uint32_t)(a.kr[slot] & 0xFFFFFFFFull) & a.key_idmask;
                key = ((unsigned long long)__float_as_uint(x) << 32) | (unsigned long long)(0xFFFFFFFFu - v);
            }
        }
        top64_insert(ta, tb, key, lane);
    }
    __shared__ unsigned long long s_a[kWarps][32], s_b[kWarps][32];
    s_a[wid][lane] = ta;
    s_b[wid][lane] = tb;
    __syncthreads();
    if (wid == 0) {
        for (int w = 1; w < kWarps; w++) {
            top64_insert(ta, tb, s_a[w][lane], lane);
            top64_insert(ta, tb, s_b[w][lane], lane);
        }
        partial[(int64_t)blockIdx.x * 64 + lane] = ta;
        partial[(int64_t)blockIdx.x * 64 + 32 + lane] = tb;
    }
}

__global__ void __launch_bounds__(kThreads) k_serve_topk_final(int k, const unsigned long long *partial,
                                                               int32_t *out_ids, float *out_vals) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long *pp = partial + (int64_t)blockIdx.x * kServeTopkParts * 64;
    unsigned long long ta = 0, tb = 0;
    for (int i0 = wid * 32; i0 < kServeTopkParts * 64; i0 += kThreads) top64_insert(ta, tb, pp[i0 + lane], lane);
    __shared__ unsigned long long s_a[kWarps][32], s_b[kWarps][32];
    s_a[wid][lane] = ta;
    s_b[wid][lane] = tb;
    __syncthreads();
    if (wid == 0) {
        for (int w = 1; w < kWarps; w++) {
            top64_insert(ta, tb, s_a[w][lane], lane);
            top64_insert(ta, tb, s_b[w][lane], lane);
        }
        for (int half = 0; half < 2; half++) {
            const int pos = half * 32 + lane;
            const unsigned long long key = half ? tb : ta;
            if (pos < k) {
                const bool valid = key != 0;
                out_ids[(int64_t)blockIdx.x * k + pos] = valid ? (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)) : -1;
                out_vals[(int64_t)blockIdx.x * k + pos] = valid ? __uint_as_float((uint32_t)(key >> 32)) : 0.0f;
            }
        }
    }
}

ServePool *serve_pool_create(Graph &g, int32_t slots, int64_t budget, const double *eps, int ncls) {
    GDE_REQUIRE(slots >= 1, GDE_EINVAL, "a server needs at least one slot");
    GDE_REQUIRE(ncls >= 1 && ncls <= kMaxCls, GDE_EINVAL, "1 to 4 tolerance classes");
    for (int c = 0; c < ncls; c++) GDE_REQUIRE(eps[c] > 0.0, GDE_EINVAL, "tolerances must be > 0");
    GDE_REQUIRE(g.n < ((int64_t)1 << 31) - 1, GDE_EINVAL, "graph too large for 32-bit keys");
    if (budget <= 0) budget = (int64_t)16 << 30;
    // a table never needs more than 2n slots (at most n keys: half load); pages of 2^16 slots,
    // smaller for small graphs so that one page is not already larger than that
    const int64_t cap_max = std::min<int64_t>(ceil_pow2(2 * (g.n > 0 ? g.n : 1)), (int64_t)1 << 31);
    int pg = 16;
    while (pg > 6 && ((int64_t)1 << pg) > cap_max) pg--;
    const int64_t page_bytes = ((int64_t)1 << pg) * 20;  // kr 8 + x 4 + x-list 8 per table slot
    // the budget, but no more than `slots` queries with the largest tables could hold
    const int64_t pages_need = ceil_pow2((int64_t)slots * (cap_max >> pg));
    int64_t pages = std::min<int64_t>(floor_pow2(std::max<int64_t>(budget / page_bytes, 1)), pages_need);
    // slot ids are 32-bit: pages * 2^pg <= 2^32
    while ((pages << pg) > ((int64_t)1 << 32)) pages >>= 1;
    int max_order = 0;
    while (((int64_t)1 << (max_order + 1)) <= pages && ((int64_t)1 << (pg + max_order + 1)) <= cap_max) max_order++;
    // a served stream mixes queries whose rounds touch millions of nodes, and a resumed state
    // cannot be re-run after an overflow: the lists get room for 2^26 candidates up front
    int64_t list_cap = std::min<int64_t>((int64_t)1 << 26, pages << pg);
    ServePool *P = new ServePool();
    try {
        P->slots = slots;
        P->list_cap = list_cap;
        P->pg_bits = pg;
        P->pages = pages;
        P->max_order = max_order;
        int lp = 0;
        while (((int64_t)1 << lp) < pages) lp++;
        P->free_blocks.assign((size_t)lp + 1, std::set<int64_t>());
        P->free_blocks[(size_t)lp].insert(0);
        P->h_owner.assign((size_t)pages, -1);
        P->order.assign((size_t)slots, -1);
        P->ncls = ncls;
        for (int c = 0; c < ncls; c++) P->eps[c] = eps[c];
        P->s = g.stream;
        // per-slot arrays and the candidate / bin lists come from a batch workspace; the tables
        // and x-lists are the paged pool's own
        P->w = batch_work_alloc(slots, 1, list_cap, 1);
        const size_t total = (size_t)pages << pg;
        dfree(P->w->kr); P->w->kr = nullptr;
        dfree(P->w->xs); P->w->xs = nullptr;
        dfree(P->w->xlist); P->w->xlist = nullptr;
        dfree(P->w->xnode); P->w->xnode = nullptr;
        P->w->kr = (unsigned long long *)dmalloc(8 * total, "served tables");
        P->w->xs = (float *)dmalloc(4 * total, "served tables");
        P->w->xlist = (uint32_t *)dmalloc(4 * total, "served x-lists");
        P->w->xnode = (uint32_t *)dmalloc(4 * total, "served x-lists");
        P->w->pool = (int64_t)total;
        P->d_owner = (int32_t *)dmalloc(4 * (size_t)pages, "page owners");
        P->thr = (float *)dmalloc(4 * (size_t)ncls * (size_t)(g.n > 0 ? g.n : 1), "class thresholds");
        P->d_param = (SlotParam *)dmalloc(sizeof(SlotParam) * (size_t)slots, "slot parameters");
        P->h_param.assign((size_t)slots, SlotParam{0.15, 0.85, 1, 0});
        P->last_vol.assign((size_t)slots, 0ull);
        P->heavy.assign((size_t)slots, 0);
        P->pend = (unsigned *)dmalloc(4 * (size_t)slots, "pending counts");
        P->d_list = (int32_t *)dmalloc(4 * (size_t)slots, "slot list");
        P->d_seeds = (int32_t *)dmalloc(4 * (size_t)slots, "slot seeds");
        P->d_ids = (int32_t *)dmalloc(4 * 64 * (size_t)slots, "slot top-k");
        P->d_vals = (float *)dmalloc(4 * 64 * (size_t)slots, "slot top-k");
        P->d_partial = (unsigned long long *)dmalloc(8 * 64 * (size_t)kServeTopkParts * (size_t)slots, "top-k parts");
        int key_idbits = 1;
        while (((int64_t)1 << key_idbits) < g.n) key_idbits++;
        P->key_idmask = (uint32_t)(((uint64_t)1 << key_idbits) - 1);
        P->tag = key_idbits < 32 ? (1u << key_idbits) : 0u;
        cudaStream_t s = P->s;
        GDE_CUDA(cudaMemsetAsync(P->w->glob, 0, sizeof(BGlobal), s));
        GDE_CUDA(cudaMemsetAsync(P->w->seg_cnt, 0, 4 * 3 * (size_t)slots, s));
        GDE_CUDA(cudaMemsetAsync(P->w->seg_hvol, 0, 8 * (size_t)slots, s));
        GDE_CUDA(cudaMemsetAsync(P->w->status, 0, 4 * (size_t)slots, s));
        GDE_CUDA(cudaMemsetAsync(P->w->xcnt, 0, 4 * (size_t)slots, s));
        GDE_CUDA(cudaStreamSynchronize(s));
        serve_sync_owner(P);
    } catch (...) {
        serve_pool_destroy(P);
        throw;
    }
    return P;
}

void serve_pool_destroy(ServePool *P) {
    if (!P) return;
    if (P->s) cudaStreamSynchronize(P->s);
    batch_free(P->w);
    dfree(P->thr); dfree(P->d_param); dfree(P->pend); dfree(P->d_list); dfree(P->d_seeds); dfree(P->d_owner);
    dfree(P->d_ids); dfree(P->d_vals); dfree(P->d_partial);
    delete P;
}

int64_t serve_pool_cap(const ServePool *P) { return (int64_t)1 << (P->pg_bits + P->max_order); }
int serve_pool_max_order(const ServePool *P) { return P->max_order; }
int64_t serve_pool_page_slots(const ServePool *P) { return (int64_t)1 << P->pg_bits; }
int64_t serve_pool_pages(const ServePool *P) { return P->pages; }
int64_t serve_pool_pages_used(const ServePool *P) { return P->pages_used; }
int serve_pool_order(const ServePool *P, int32_t slot) { return P->order[(size_t)slot]; }

// Buddy allocation of 2^ord pages for query slot j (host bookkeeping; the device owner table
// follows before the next launch).  Returns false when no block of that size is free.
bool serve_pool_reserve(ServePool *P, int32_t j, int ord) {
    GDE_REQUIRE(j >= 0 && j < P->slots && P->order[(size_t)j] < 0, GDE_EINVAL, "slot busy or out of range");
    GDE_REQUIRE(ord >= 0 && ord <= P->max_order, GDE_EINVAL, "table order out of range");
    int o = ord;
    while (o < (int)P->free_blocks.size() && P->free_blocks[(size_t)o].empty()) o++;
    if (o >= (int)P->free_blocks.size()) return false;
    int64_t page = *P->free_blocks[(size_t)o].begin();
    P->free_blocks[(size_t)o].erase(P->free_blocks[(size_t)o].begin());
    while (o > ord) {  // split: keep the lower half, free the upper
        o--;
        P->free_blocks[(size_t)o].insert(page + ((int64_t)1 << o));
    }
    for (int64_t q = page; q < page + ((int64_t)1 << ord); q++) P->h_owner[(size_t)q] = j;
    P->owner_dirty = true;
    P->pages_used += (int64_t)1 << ord;
    P->order[(size_t)j] = ord;
    SlotParam &sp = P->h_param[(size_t)j];
    sp.base = (uint64_t)page << P->pg_bits;
    sp.log2cap = (uint32_t)(P->pg_bits + ord);
    return true;
}

void serve_pool_release(ServePool *P, int32_t j) {
    const int ord = P->order[(size_t)j];
    if (ord < 0) return;
    int64_t page = (int64_t)(P->h_param[(size_t)j].base >> P->pg_bits);
    for (int64_t q = page; q < page + ((int64_t)1 << ord); q++) P->h_owner[(size_t)q] = -1;
    P->owner_dirty = true;
    P->pages_used -= (int64_t)1 << ord;
    P->order[(size_t)j] = -1;
    int o = ord;
    while (o + 1 < (int)P->free_blocks.size()) {  // merge with the free buddy
        const int64_t buddy = page ^ ((int64_t)1 << o);
        auto it = P->free_blocks[(size_t)o].find(buddy);
        if (it == P->free_blocks[(size_t)o].end()) break;
        P->free_blocks[(size_t)o].erase(it);
        page = std::min(page, buddy);
        o++;
    }
    P->free_blocks[(size_t)o].insert(page);
}

void serve_pool_set_defer(ServePool *P, int64_t v) { P->defer_vol = v; }

void serve_pool_graph_changed(ServePool *P) {
    P->thr_n = -1;
}

static void serve_ensure_graph_state(Graph &g, ServePool *P) {
    ensure_colp(g, P->s);
    if (P->thr_n != g.n) {
        for (int c = 0; c < P->ncls; c++) {
            k_batch_thr<<<kSMs * 8, kThreads, 0, P->s>>>(g.n, g.deg, P->thr + (int64_t)c * g.n, P->eps[c]);
            GDE_CUDA(cudaGetLastError());
        }
        P->thr_n = g.n;
    }
}

void serve_pool_admit(Graph &g, ServePool *P, int32_t n, const int32_t *slots, const int32_t *seeds,
                      const gde_kind *kinds, const double *params, const int32_t *cls) {
    if (n <= 0) return;
    P->pend_valid = false;
    cudaStream_t s = P->s;
    for (int32_t i = 0; i < n; i++) {
        GDE_REQUIRE(slots[i] >= 0 && slots[i] < P->slots, GDE_EINVAL, "slot out of range");
        GDE_REQUIRE(P->order[(size_t)slots[i]] >= 0, GDE_EINVAL, "slot has no table reserved");
        GDE_REQUIRE(seeds[i] >= 0 && seeds[i] < g.n, GDE_EINVAL, "seed out of range");
        GDE_REQUIRE(cls[i] >= 0 && cls[i] < P->ncls, GDE_EINVAL, "tolerance class out of range");
        SlotParam &sp = P->h_param[(size_t)slots[i]];
        if (kinds[i] == GDE_PPR) {
            GDE_REQUIRE(params[i] > 0.0 && params[i] < 1.0, GDE_EINVAL, "PPR alpha must be in (0,1)");
            sp.cx = params[i]; sp.coef = 1.0 - params[i]; sp.divide = 1;
        } else {
            GDE_REQUIRE(kinds[i] == GDE_KATZ && params[i] > 0.0, GDE_EINVAL, "a server serves PPR and Katz");
            sp.cx = 1.0; sp.coef = params[i]; sp.divide = 0;
        }
        sp.cls = cls[i];
        sp.tag = P->tag;
        sp.flags = 0;
        P->last_vol[(size_t)slots[i]] = 0;
        P->heavy[(size_t)slots[i]] = 0;
    }
    serve_sync_owner(P);
    GDE_CUDA(cudaMemcpyAsync(P->d_param, P->h_param.data(), sizeof(SlotParam) * (size_t)P->slots,
                             cudaMemcpyHostToDevice, s));
    GDE_CUDA(cudaMemcpyAsync(P->d_list, slots, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    GDE_CUDA(cudaMemcpyAsync(P->d_seeds, seeds, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    // empty the admitted tables (a page may have belonged to any earlier query), then seed them
    int bx = 1;
    for (int32_t i = 0; i < n; i++) {
        const int64_t cap = (int64_t)1 << P->h_param[(size_t)slots[i]].log2cap;
        const int64_t want = (cap + (int64_t)kThreads * 16 - 1) / ((int64_t)kThreads * 16);
        if (want > bx) bx = (int)std::min<int64_t>(want, 1024);
    }
    for (int32_t i0 = 0; i0 < n; i0 += 32768) {  // gridDim.y stays below its limit of 65535
        const int32_t m = std::min<int32_t>(32768, n - i0);
        k_serve_clear<<<dim3((unsigned)bx, (unsigned)m), kThreads, 0, s>>>(P->d_list + i0, P->d_param, P->w->kr,
                                                                            P->w->xs);
        GDE_CUDA(cudaGetLastError());
    }
    AdmitArgs a{};
    a.t = slot_table(P);
    a.sparam = P->d_param;
    a.n = n; a.slots = P->d_list; a.seeds = P->d_seeds; a.tag = P->tag;
    a.cand = P->w->cand[P->T & 1]; a.count = next_count(P); a.list_cap = (unsigned)P->list_cap;
    a.error = &P->w->glob->error;
    a.status = P->w->status; a.inserts = P->w->inserts; a.svol = P->w->svol; a.spushes = P->w->spushes;
    a.slast = P->w->slast; a.xcnt = P->w->xcnt; a.spush = P->w->spush; a.sscat = P->w->sscat;
    k_serve_seed<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched(2);
}

void serve_pool_correct(Graph &g, ServePool *P, const EdgeBatch &eb, int32_t nres, const int32_t *res) {
    if (nres <= 0 || eb.rows <= 0) return;
    P->pend_valid = false;
    serve_ensure_graph_state(g, P);
    GDE_CUDA(cudaMemcpyAsync(P->d_list, res, 4 * (size_t)nres, cudaMemcpyHostToDevice, P->s));
    CorrectArgs a{};
    a.t = slot_table(P);
    a.sparam = P->d_param; a.thr = P->thr; a.thr_stride = g.n;
    a.res = P->d_list; a.nres = nres;
    a.row = eb.row; a.row_cnt = eb.row_cnt; a.row_start = eb.row_start; a.old_deg = eb.old_deg;
    a.added = eb.v; a.rows = eb.rows;
    a.cand = P->w->cand[P->T & 1]; a.count = next_count(P); a.list_cap = (unsigned)P->list_cap;
    a.error = &P->w->glob->error; a.status = P->w->status;
    const int64_t total = (int64_t)nres * eb.rows;
    k_serve_correct<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, P->s>>>(a);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
}

int64_t serve_pool_run(Graph &g, ServePool *P, int64_t rounds) {
    P->pend_valid = false;
    serve_ensure_graph_state(g, P);
    serve_sync_owner(P);
    BatchWork *w = P->w;
    // heavy slots (by their volume in the last launch) run one round of this launch
    bool changed = false;
    for (int32_t j = 0; j < P->slots; j++) {
        const uint32_t want = (rounds > 1 && P->heavy[(size_t)j]) ? kSlotDefer : 0u;
        if ((P->h_param[(size_t)j].flags & kSlotDefer) != want) {
            P->h_param[(size_t)j].flags = (P->h_param[(size_t)j].flags & ~kSlotDefer) | want;
            changed = true;
        }
    }
    if (changed)
        GDE_CUDA(cudaMemcpyAsync(P->d_param, P->h_param.data(), sizeof(SlotParam) * (size_t)P->slots,
                                 cudaMemcpyHostToDevice, P->s));
    BArgs a = bargs_base(g, w, 1, P->list_cap, P->slots, P->tag, P->key_idmask);
    a.page_owner = P->d_owner;
    a.pg_bits = P->pg_bits;
    a.thr32 = P->thr;
    a.thr_stride = g.n;
    a.eps = P->eps[0];
    for (int c = 0; c < kMaxCls; c++) a.eps_cls[c] = c < P->ncls ? P->eps[c] : P->eps[0];
    a.ncls = P->ncls;
    a.sparam = P->d_param;
    a.t0 = P->T;
    a.max_rounds = rounds;
    a.pend = P->pend;
    a.kind = GDE_PPR;
    a.cx = 0.0;
    a.coef = 0.0;
    launch_rounds(g, w, a, P->s);
    BGlobal hg;
    GDE_CUDA(cudaMemcpyAsync(&hg, w->glob, sizeof(BGlobal), cudaMemcpyDeviceToHost, P->s));
    std::vector<unsigned long long> vol((size_t)P->slots);
    GDE_CUDA(cudaMemcpyAsync(vol.data(), w->svol, 8 * (size_t)P->slots, cudaMemcpyDeviceToHost, P->s));
    P->h_pend.resize((size_t)P->slots);
    GDE_CUDA(cudaMemcpyAsync(P->h_pend.data(), P->pend, 4 * (size_t)P->slots, cudaMemcpyDeviceToHost, P->s));
    GDE_CUDA(cudaStreamSynchronize(P->s));
    P->pend_valid = true;
    for (int32_t j = 0; j < P->slots; j++) {
        const unsigned long long prev = P->last_vol[(size_t)j], now = vol[(size_t)j];
        const unsigned long long delta = now >= prev ? now - prev : now;  // re-admitted: counted anew
        P->heavy[(size_t)j] = P->defer_vol >= 0 && delta > (unsigned long long)P->defer_vol ? 1 : 0;
        P->last_vol[(size_t)j] = now;
    }
    if (hg.error != 0) serve_check_error(P);
    const int64_t ran = (int64_t)hg.rounds - P->T;
    P->T = hg.rounds;
    P->volume = (int64_t)hg.total_vol;
    return ran;
}

int64_t serve_pool_volume(const ServePool *P) { return P->volume; }

void serve_pool_pending(Graph &g, ServePool *P, unsigned *pend_host) {
    if (P->pend_valid) {  // counted by the launch that just ran
        std::copy(P->h_pend.begin(), P->h_pend.end(), pend_host);
        return;
    }
    serve_sync_owner(P);
    GDE_CUDA(cudaMemsetAsync(P->pend, 0, 4 * (size_t)P->slots, P->s));
    k_serve_pending<<<kSMs * 2, kThreads, 0, P->s>>>(next_count(P), (unsigned)P->list_cap, P->w->cand[P->T & 1],
                                                      P->d_owner, P->pg_bits, P->pend);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched();
    GDE_CUDA(cudaMemcpyAsync(pend_host, P->pend, 4 * (size_t)P->slots, cudaMemcpyDeviceToHost, P->s));
    GDE_CUDA(cudaStreamSynchronize(P->s));
}

void serve_pool_results(Graph &g, ServePool *P, int32_t n, const int32_t *slots, int k, int32_t *ids,
                        float *vals, int32_t *status, int64_t *volume, int32_t *last_round, int64_t *support) {
    if (n <= 0) return;
    GDE_REQUIRE(k >= 1 && k <= kTopMax, GDE_EINVAL, "topk must be in [1, 64]");
    cudaStream_t s = P->s;
    GDE_CUDA(cudaMemcpyAsync(P->d_list, slots, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    TopkArgs ta{};
    ta.kr = P->w->kr; ta.xs = P->w->xs; ta.k = k;
    ta.key_idmask = P->key_idmask; ta.xlist = P->w->xlist; ta.xnode = P->w->xnode; ta.xcnt = P->w->xcnt;
    ta.out_ids = P->d_ids; ta.out_vals = P->d_vals; ta.ssupport = P->w->inserts;
    ta.slots = P->d_list; ta.keep = 1;
    k_serve_topk_partial<<<(unsigned)(n * kServeTopkParts), kThreads, 0, s>>>(ta, P->d_param, P->d_partial);
    GDE_CUDA(cudaGetLastError());
    k_serve_topk_final<<<(unsigned)n, kThreads, 0, s>>>(k, P->d_partial, P->d_ids, P->d_vals);
    GDE_CUDA(cudaGetLastError());
    g.prof.launched(2);
    GDE_CUDA(cudaMemcpyAsync(ids, P->d_ids, 4 * (size_t)n * k, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(vals, P->d_vals, 4 * (size_t)n * k, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> st((size_t)P->slots), last((size_t)P->slots);
    std::vector<unsigned long long> vol((size_t)P->slots);
    std::vector<unsigned> keys((size_t)P->slots);
    GDE_CUDA(cudaMemcpyAsync(st.data(), P->w->status, 4 * (size_t)P->slots, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(last.data(), P->w->slast, 4 * (size_t)P->slots, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(vol.data(), P->w->svol, 8 * (size_t)P->slots, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(keys.data(), P->w->inserts, 4 * (size_t)P->slots, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaStreamSynchronize(s));
    for (int32_t i = 0; i < n; i++) {
        const size_t j = (size_t)slots[i];
        status[i] = st[j] == kSeedOk ? GDE_OK : GDE_ENOMEM;
        volume[i] = (int64_t)vol[j];
        last_round[i] = last[j];
        if (support) support[i] = (int64_t)keys[j];  // keys its table holds
    }
}

int64_t serve_pool_round(const ServePool *P) { return P->T; }


// A round's candidates of all seeds must fit the candidate and bin lists, sized from the
// batch; a solve that overflows them (GDE_ENOMEM from the kernel, the pool marked for a reset)
// is run again with lists four times larger, up to one entry per pool slot.
void batch_solve(Graph &g, const SolveParams &p, const int32_t *seeds_dev, int32_t nseeds, int k,
                 int64_t mem_budget, int32_t *ids_dev, float *vals_dev, gde_stats *stats_host,
                 int32_t *overflow_seeds_host, int32_t *n_overflow) {
    for (int scale = 0;; scale++) {
        bool full = false;
        try {
            batch_solve_once(g, p, seeds_dev, nseeds, k, mem_budget, ids_dev, vals_dev, stats_host,
                             overflow_seeds_host, n_overflow, scale, &full);
            return;
        } catch (const Fail &f) {
            if (f.st != GDE_ENOMEM || full || !g.batch || !g.batch->list_overflowed) throw;
            g.batch->list_overflowed = false;
        }
    }
}

// rows[i] of the output receives row i of the chunk's output
__global__ void k_put_rows(int32_t m, int k, const int32_t *rows, const int32_t *src_ids, const float *src_vals,
                           int32_t *dst_ids, float *dst_vals) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)m * k) return;
    const int64_t r = i / k, c = i % k;
    dst_ids[(int64_t)rows[r] * k + c] = src_ids[i];
    dst_vals[(int64_t)rows[r] * k + c] = src_vals[i];
}

void batch_solve_rebatch(Graph &g, const SolveParams &p, const int32_t *seeds_dev, const int32_t *seeds_host,
                         int32_t nseeds, int k, int64_t mem_budget, int32_t *ids_dev, float *vals_dev,
                         gde_stats *stats_host, int32_t *overflow_seeds_host, int32_t *n_overflow) {
    batch_solve(g, p, seeds_dev, nseeds, k, mem_budget, ids_dev, vals_dev, stats_host, overflow_seeds_host,
                n_overflow);
    if (*n_overflow == 0) return;
    const int64_t budget = mem_budget > 0 ? mem_budget : ((int64_t)16 << 30);
    const int64_t per_slot = layered(p.kind) ? 18 : 12;
    const int64_t cap_max = std::min<int64_t>(ceil_pow2(2 * (g.n > 0 ? g.n : 1)), (int64_t)1 << 31);
    int64_t cap = floor_pow2(budget / (per_slot * (int64_t)nseeds));
    std::vector<int32_t> pending(overflow_seeds_host, overflow_seeds_host + *n_overflow);
    std::vector<void *> tmp;
    auto alloc = [&](size_t bytes, const char *what) {
        void *q = dmalloc(bytes, what);
        tmp.push_back(q);
        return q;
    };
    try {
        cudaStream_t s = p.stream;
        while (!pending.empty() && cap < cap_max) {
            cap *= 2;
            const int64_t chunk = budget / (per_slot * cap);  // seeds per batch at this table size
            if (chunk < 1) break;
            const int32_t m0 = (int32_t)std::min<int64_t>(chunk, (int64_t)pending.size());
            if (tmp.empty()) {
                alloc(4 * (size_t)pending.size(), "re-batched seeds");
                alloc(4 * (size_t)pending.size(), "re-batched rows");
                alloc(4 * (size_t)pending.size() * (size_t)k, "re-batched ids");
                alloc(4 * (size_t)pending.size() * (size_t)k, "re-batched values");
            }
            int32_t *d_seeds = (int32_t *)tmp[0], *d_rows = (int32_t *)tmp[1];
            int32_t *d_ids = (int32_t *)tmp[2];
            float *d_vals = (float *)tmp[3];
            std::vector<int32_t> next;
            std::vector<gde_stats> cst((size_t)m0);
            std::vector<int32_t> cof((size_t)m0);
            for (size_t c0 = 0; c0 < pending.size(); c0 += (size_t)m0) {
                const int32_t m = (int32_t)std::min<size_t>((size_t)m0, pending.size() - c0);
                std::vector<int32_t> hseeds((size_t)m), hrows((size_t)m);
                for (int32_t i = 0; i < m; i++) {
                    hrows[(size_t)i] = pending[c0 + (size_t)i];
                    hseeds[(size_t)i] = seeds_host[hrows[(size_t)i]];
                }
                GDE_CUDA(cudaMemcpyAsync(d_seeds, hseeds.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, s));
                GDE_CUDA(cudaMemcpyAsync(d_rows, hrows.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, s));
                int32_t cn = 0;
                // the same budget over m seeds gives tables of at least `cap` slots
                batch_solve(g, p, d_seeds, m, k, budget, d_ids, d_vals, cst.data(), cof.data(), &cn);
                const int64_t items = (int64_t)m * k;
                k_put_rows<<<(unsigned)((items + kThreads - 1) / kThreads), kThreads, 0, s>>>(
                    m, k, d_rows, d_ids, d_vals, ids_dev, vals_dev);
                GDE_CUDA(cudaGetLastError());
                g.prof.launched();
                GDE_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
                std::vector<bool> of((size_t)m, false);
                for (int32_t i = 0; i < cn; i++) of[(size_t)cof[(size_t)i]] = true;
                for (int32_t i = 0; i < m; i++) {
                    if (of[(size_t)i]) next.push_back(hrows[(size_t)i]);
                    if (stats_host) {
                        gde_stats one = cst[(size_t)i];
                        one.fallback = of[(size_t)i] ? 0 : 2;
                        stats_host[hrows[(size_t)i]] = one;
                    }
                }
            }
            pending.swap(next);
        }
    } catch (...) {
        for (void *q : tmp) dfree(q);
        throw;
    }
    for (void *q : tmp) dfree(q);
    for (size_t i = 0; i < pending.size(); i++) overflow_seeds_host[i] = pending[i];
    *n_overflow = (int32_t)pending.size();
}

int64_t batch_round_log(Graph &g, double *out, int64_t cap) {
    BatchWork *w = g.batch;
    if (!w) return 0;
    const int64_t r = w->last_rounds;
    const int64_t m = std::min<int64_t>(std::min<int64_t>(r, cap), kLogCap);
    if (m > 0) {
        std::vector<RoundLog> h((size_t)m);
        GDE_CUDA(cudaMemcpy(h.data(), w->log, sizeof(RoundLog) * (size_t)m, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m; i++) {
            out[7 * i + 0] = (double)h[(size_t)i].ncand;
            out[7 * i + 1] = (double)h[(size_t)i].vol;
            out[7 * i + 2] = h[(size_t)i].rS_l1;
            out[7 * i + 3] = (double)h[(size_t)i].t_ns;
            out[7 * i + 4] = (double)h[(size_t)i].tA_ns;
            out[7 * i + 5] = (double)h[(size_t)i].busy_sum_ns;
            out[7 * i + 6] = (double)h[(size_t)i].busy_max_ns;
        }
    }
    return r;
}


// ======================================================= stepping session ====
// The batched engine run one round per launch, with every seed's table read back between
// rounds, so that its rounds (Eq. local-gd for all seeds of a batch at once) can be compared
// with the oracle's from exactly the same state.  The round kernel, its arguments and the
// set-up are the batched solve's; only max_rounds = 1 and the per-candidate push flags differ.
// The session owns its workspace (the graph's cached one is untouched); the graph must not
// change while it runs.

struct BatchSession {
    Graph *g = nullptr;
    SolveParams p;
    BatchWork *w = nullptr;
    int32_t nseeds = 0;
    int64_t cap = 0, list_cap = 0;
    uint32_t key_tag = 0, key_idmask = 0, tag_step = 0;
    BArgs a{};
    int64_t T = 0;                       // the next round
    int32_t *d_seeds = nullptr;
    uint32_t *d_pushed = nullptr;        // per candidate of the last round: pushed or not
    const int64_t *off0 = nullptr;       // the CSR as of begin (an insertion swaps the arrays)
    const int32_t *col0 = nullptr;
    int64_t nnz0 = 0;
    std::vector<unsigned long long> h_kr, h_xkr, h_slab;  // host copies of the tables after the last step
    std::vector<float> h_xs, h_xxs, h_slab_x;
    std::vector<int32_t> h_status;
    std::vector<double> h_xsrc;
    std::vector<std::vector<int32_t>> pushed;     // per seed: the nodes pushed in the last round
    std::vector<int32_t> seeds_host;
};

static float host_bits_to_float(uint32_t b) {
    float f;
    std::memcpy(&f, &b, sizeof f);
    return f;
}

static void bsession_mirror(BatchSession *S) {
    BatchWork *w = S->w;
    cudaStream_t s = S->p.stream;
    const size_t pool = (size_t)S->nseeds * (size_t)S->cap;
    S->h_kr.resize(pool);
    S->h_xs.resize(pool);
    S->h_status.resize((size_t)S->nseeds);
    GDE_CUDA(cudaMemcpyAsync(S->h_kr.data(), w->kr, 8 * pool, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(S->h_xs.data(), w->xs, 4 * pool, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(S->h_status.data(), w->status, 4 * (size_t)S->nseeds, cudaMemcpyDeviceToHost, s));
    if (S->p.kind == GDE_KATZ && S->p.katz_minus_source) {
        S->h_xsrc.resize((size_t)S->nseeds);
        GDE_CUDA(cudaMemcpyAsync(S->h_xsrc.data(), w->xsrc, 8 * (size_t)S->nseeds, cudaMemcpyDeviceToHost, s));
    }
    if (w->slab_on) {
        // the bank the next round reads (the layered kinds keep two)
        const size_t sp = (size_t)S->nseeds * (size_t)w->slab_H;
        const size_t bank = layered(S->p.kind) ? (size_t)(S->T & 1) : 0;
        S->h_slab.resize(sp);
        S->h_slab_x.resize(sp);
        GDE_CUDA(cudaMemcpyAsync(S->h_slab.data(), w->slab + bank * sp, 8 * sp, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(S->h_slab_x.data(), w->slab_x, 4 * sp, cudaMemcpyDeviceToHost, s));
    }
    if (layered(S->p.kind)) {
        const size_t xp = (size_t)w->xt_seeds * (size_t)w->xt_cap;
        S->h_xkr.resize(xp);
        S->h_xxs.resize(xp);
        GDE_CUDA(cudaMemcpyAsync(S->h_xkr.data(), w->xkr, 8 * xp, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaMemcpyAsync(S->h_xxs.data(), w->xxs, 4 * xp, cudaMemcpyDeviceToHost, s));
    }
    GDE_CUDA(cudaStreamSynchronize(s));
}

static void bsession_free(BatchSession *S) {
    if (!S) return;
    if (S->p.stream) cudaStreamSynchronize(S->p.stream);
    batch_free(S->w);
    dfree(S->d_seeds);
    dfree(S->d_pushed);
    delete S;
}

void bsession_destroy(BatchSession *S) { bsession_free(S); }

BatchSession *bsession_begin(Graph &g, const SolveParams &p, const int32_t *seeds_host, int32_t nseeds,
                             int64_t budget) {
    GDE_REQUIRE(p.kind == GDE_PPR || p.kind == GDE_KATZ || p.kind == GDE_GPPR || layered(p.kind), GDE_EINVAL,
                "batched session: PPR, Katz, the generalised propagation, the heat kernel or a series");
    GDE_REQUIRE(p.precision == GDE_FP32, GDE_EINVAL, "batched session: the batched engine stores x and r in FP32");
    GDE_REQUIRE(nseeds >= 1 && seeds_host != nullptr, GDE_EINVAL, "batched session: needs at least one seed");
    GDE_REQUIRE(g.n >= 1 && g.n < ((int64_t)1 << 31) - 1, GDE_EINVAL, "batched session: graph size out of range");
    for (int32_t i = 0; i < nseeds; i++)
        GDE_REQUIRE(seeds_host[i] >= 0 && seeds_host[i] < g.n, GDE_EINVAL, "seed id out of range");
    const bool lay = layered(p.kind);
    if (budget <= 0) budget = (int64_t)4 << 30;
    int64_t cap = floor_pow2(budget / ((lay ? 18 : 12) * (int64_t)nseeds));
    const int64_t cap_max = std::min<int64_t>(ceil_pow2(2 * g.n), (int64_t)1 << 31);
    if (cap > cap_max) cap = cap_max;
    GDE_REQUIRE(cap >= 64 || cap == cap_max, GDE_ENOMEM, "batched session: memory budget too small");
    GDE_REQUIRE((int64_t)nseeds * cap <= ((int64_t)1 << 32), GDE_EINVAL, "batched session: pool exceeds 2^32 slots");
    int64_t list_cap = std::min<int64_t>((int64_t)nseeds * (cap + slab_hubs(g, p, nseeds, cap, p.stream)),
                                         (int64_t)1 << 24);
    GDE_REQUIRE(nseeds <= list_cap, GDE_EINVAL, "batched session: too many seeds");
    BatchSession *S = new BatchSession();
    try {
        S->g = &g;
        S->p = p;
        S->nseeds = nseeds;
        S->cap = cap;
        S->list_cap = list_cap;
        S->w = batch_work_alloc(nseeds, cap, list_cap);
        S->d_seeds = (int32_t *)dmalloc(4 * (size_t)nseeds, "session seeds");
        S->d_pushed = (uint32_t *)dmalloc(4 * (size_t)list_cap, "session push flags");
        cudaStream_t s = p.stream;
        GDE_CUDA(cudaMemcpyAsync(S->d_seeds, seeds_host, 4 * (size_t)nseeds, cudaMemcpyHostToDevice, s));
        S->a = batch_setup(g, p, S->w, S->d_seeds, nseeds, cap, list_cap, &S->key_tag, &S->key_idmask);
        S->a.max_rounds = 1;
        S->a.pushed = S->d_pushed;
        S->tag_step = S->a.tag_step;
        S->off0 = g.off;
        S->col0 = g.col;
        S->nnz0 = g.nnz;
        S->pushed.assign((size_t)nseeds, std::vector<int32_t>());
        S->seeds_host.assign(seeds_host, seeds_host + nseeds);
        bsession_mirror(S);
    } catch (...) {
        bsession_free(S);
        throw;
    }
    return S;
}

// candidates of round T: in cand[T & 1], counted by the other parity's cand_out
static unsigned bsession_ncand(BatchSession *S) {
    unsigned c = 0;
    GDE_CUDA(cudaMemcpyAsync(&c, &S->w->glob->ctl[(S->T & 1) ^ 1].cand_out, sizeof(unsigned),
                             cudaMemcpyDeviceToHost, S->p.stream));
    GDE_CUDA(cudaStreamSynchronize(S->p.stream));
    return c;
}

int64_t bsession_step(BatchSession *S) {
    Graph &g = *S->g;
    GDE_REQUIRE(g.off == S->off0 && g.col == S->col0 && g.nnz == S->nnz0, GDE_EINVAL,
                "batched session: the graph changed since the session began");
    for (auto &v : S->pushed) v.clear();
    unsigned ncand = bsession_ncand(S);
    if (ncand == 0) return 0;
    GDE_REQUIRE(ncand <= (unsigned)S->list_cap, GDE_ENOMEM, "batched session: candidate list overflowed");
    cudaStream_t s = S->p.stream;
    std::vector<uint32_t> cand(ncand), flag(ncand);
    GDE_CUDA(cudaMemcpyAsync(cand.data(), S->w->cand[S->T & 1], 4 * (size_t)ncand, cudaMemcpyDeviceToHost, s));
    S->a.t0 = S->T;
    launch_rounds(g, S->w, S->a, s);
    BGlobal hg;
    GDE_CUDA(cudaMemcpyAsync(&hg, S->w->glob, sizeof(BGlobal), cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaMemcpyAsync(flag.data(), S->d_pushed, 4 * (size_t)ncand, cudaMemcpyDeviceToHost, s));
    GDE_CUDA(cudaStreamSynchronize(s));
    if (hg.error == GDE_ETIMEOUT) {
        set_error("batched session: a grid barrier wait timed out");
        throw Fail{GDE_ETIMEOUT};
    }
    GDE_REQUIRE(hg.error == 0, (gde_status)hg.error, "batched session: candidate or bin list capacity exceeded");
    // the pushed candidates' nodes, decoded from the tables as they were before the round
    for (unsigned i = 0; i < ncand; i++) {
        if (!flag[i]) continue;
        const uint32_t slot = cand[i];
        if (S->w->slab_on && slot >= S->w->slab_base) {
            const uint64_t idx = slot - S->w->slab_base;
            const int64_t j = (int64_t)(idx / (uint64_t)S->w->slab_H);
            S->pushed[(size_t)j].push_back(g.hub_node_host[(size_t)(idx - (uint64_t)j * S->w->slab_H)]);
            continue;
        }
        const int32_t j = (int32_t)(slot >> S->w->log2cap);
        const uint32_t key = (uint32_t)(S->h_kr[slot] & 0xFFFFFFFFull);
        S->pushed[(size_t)j].push_back((int32_t)(key & S->key_idmask));
    }
    S->T = S->T + 1;
    bsession_mirror(S);
    return (int64_t)bsession_ncand(S);
}

// x (n floats: the unscaled x of the engine), r (n doubles: the residual, for the layered kinds
// the current layer) of seed j after the last step, and the nodes pushed in that step
gde_status bsession_read(BatchSession *S, int32_t j, float *x, double *r, int32_t *pushed, int64_t *n_pushed) {
    GDE_REQUIRE(j >= 0 && j < S->nseeds, GDE_EINVAL, "batched session: seed index out of range");
    const int64_t n = S->g->n;
    const uint64_t base = (uint64_t)j << S->w->log2cap;
    const bool lay = layered(S->p.kind);
    const uint32_t rtag = lay ? S->key_tag + (uint32_t)S->T * S->tag_step : S->key_tag;
    if (x) std::fill(x, x + n, 0.0f);
    if (r) std::fill(r, r + n, 0.0);
    for (int64_t i = 0; i < S->cap; i++) {
        const unsigned long long word = S->h_kr[base + (uint64_t)i];
        const uint32_t key = (uint32_t)(word & 0xFFFFFFFFull);
        if (key == kEmpty || (key & ~S->key_idmask) != rtag) continue;
        const uint32_t v = key & S->key_idmask;
        if (r) r[v] = (double)host_bits_to_float((uint32_t)(word >> 32));
        if (x && !lay) x[v] = S->h_xs[base + (uint64_t)i];
    }
    if (S->w->slab_on) {
        // hubs: fixed-point counts (value = count * 2^qexp) and their x
        const int64_t H = S->w->slab_H;
        const Graph &g = *S->g;
        for (int64_t rk = 0; rk < H; rk++) {
            const size_t idx = (size_t)j * (size_t)H + (size_t)rk;
            const int32_t v = g.hub_node_host[(size_t)rk];
            if (r) r[v] = std::ldexp((double)S->h_slab[idx], S->w->qexp);
            if (x) x[v] = S->h_slab_x[idx];
        }
    }
    if (x && lay) {
        const uint64_t xb = (uint64_t)j << S->w->xt_log2cap;
        for (int64_t i = 0; i < S->w->xt_cap; i++) {
            const uint32_t key = (uint32_t)(S->h_xkr[xb + (uint64_t)i] & 0xFFFFFFFFull);
            if (key == kEmpty || (key & ~S->key_idmask) != S->key_tag) continue;
            x[key & S->key_idmask] = S->h_xxs[xb + (uint64_t)i];
        }
    }
    if (x && S->p.kind == GDE_KATZ && S->p.katz_minus_source) x[S->seeds_host[(size_t)j]] = (float)S->h_xsrc[(size_t)j];
    const std::vector<int32_t> &pl = S->pushed[(size_t)j];
    if (pushed) std::copy(pl.begin(), pl.end(), pushed);
    if (n_pushed) *n_pushed = (int64_t)pl.size();
    return S->h_status[(size_t)j] == kSeedOk ? GDE_OK : GDE_ENOMEM;
}

int64_t bsession_round(const BatchSession *S) { return S->T; }

}  // namespace gde
