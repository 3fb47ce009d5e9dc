// C ABI of the SOP-model Langevin library: context life cycle, schedules,
// CUDA-graph replay, host I/O and checkpoints. Declared in include/sop.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sop_internal.h"

using namespace sop;

namespace {

thread_local std::string g_create_error;

constexpr int kObsChunk = kObsChunkBeads;   // beads per FP64 observable partial (FP64 is slow per SM: spread it)
// Largest system the batched schedule takes: its state lives in shared memory, one CTA per
// system up to about 3,400 beads (rows in global memory beyond 512), and the cluster form,
// which keeps a copy of all positions in every CTA of the cluster, up to 4,096.
constexpr int kBatchedMaxBeads = 4096;
// Largest system the automatic choice sends to the batched schedule (the one-CTA forms fit).
constexpr int kBatchedAutoBeads = 3200;
constexpr int64_t kBatchedChunk = 4096;  // steps per batched launch

// k_B in kcal/(mol K): molar gas constant 8.314462618 J/(mol K) / 4184 J/kcal.
constexpr double kBoltzmannKcal = 8.314462618 / 4184.0;

}  // namespace

void sop::set_global_error(const std::string &msg) { g_create_error = msg; }

struct sop_ctx {
    // sizes
    int32_t n = 0, n_chains = 0, n_sys = 0, R = 0, n_seg = 0;
    sop_params prm{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    // host topology
    std::vector<int32_t> chain_off, sys_lo, chain_of, sys_of, sys_ree_last;
    std::vector<uint8_t> flags;
    std::vector<uint8_t> fixed_by_mask;   // [n] fixed through the topology's fixed_mask (never cleared)
    std::vector<std::pair<int32_t, int32_t>> xlinks;   // cross-links (i < j) of the topology
    std::vector<int32_t> h_nat_row, h_nat_col;
    std::vector<double> h_nat_r0;
    std::vector<int32_t> h_seg_bead_lo, h_seg_cell_base, h_seg_chunk_lo, h_brute_cta_lo;
    // device memory
    std::vector<void *> allocs;
    int32_t *d_chain = nullptr, *d_sys = nullptr, *d_sys_lo = nullptr, *d_sys_ree_last = nullptr,
            *d_sys_nat_pairs = nullptr;
    uint8_t *d_flags = nullptr;
    uint4 *d_taus = nullptr;   // Hybrid Taus state per bead (SOP_RNG_HYBRID_TAUS)
    float4 *d_vel = nullptr;   // stored velocity per bead (SOP_INTEGRATOR_BAOAB)
    float *d_bond_r0 = nullptr;
    double *d_bond_r0d = nullptr;
    const int32_t *d_xb_row = nullptr, *d_xb_col = nullptr;   // cross-links (NULL: none)
    const float *d_xb_r0 = nullptr;
    const double *d_xb_r0d = nullptr;
    int32_t *d_nat_row = nullptr, *d_nat_col = nullptr;
    float *d_nat_r0sq = nullptr;
    uint2 *d_nat_ent = nullptr;
    double *d_nat_r0 = nullptr;
    int64_t nat_nnz = 0;
    // batched natives (ELL)
    int32_t *d_nat_ell_off = nullptr, *d_nat_ell_cnt = nullptr;
    uint16_t *d_nat_ell_col = nullptr;
    float *d_nat_ell_r0sq = nullptr;
    uint16_t *d_nat_slot_bead = nullptr, *d_nat_slot_cnt = nullptr;
    uint2 *d_nat_slot_ent = nullptr;
    // pair form: native pairs split between the rows of their two beads (own / reverse tables)
    int32_t *d_nat_own_off = nullptr, *d_nat_own_cnt = nullptr, *d_nat_rev_off = nullptr, *d_nat_rev_cnt = nullptr;
    uint16_t *d_nat_own_col = nullptr, *d_nat_rev_col = nullptr, *d_nat_rev_k = nullptr;
    float *d_nat_own_r0sq = nullptr;
    std::vector<int32_t> h_nat_own_cnt, h_nat_rev_cnt;   // per bead
    // static exclusion masks of the batched rebuild scan (systems of at most 256 beads)
    int32_t *d_excl_off = nullptr;
    uint32_t *d_excl = nullptr;
    // state
    float4 *d_pos[2] = {nullptr, nullptr};
    float4 *d_comp = nullptr, *d_snap = nullptr, *d_force = nullptr;
    int cur = 0;
    int64_t step = 0, list_step = -1, events = 0, consumed = 0;
    int64_t *d_step = nullptr, *d_events = nullptr;
    int32_t *d_rep_status = nullptr, *d_halt = nullptr;
    double *d_energy = nullptr;
    int32_t *h_abort = nullptr;      // host-mapped
    int32_t *d_abort = nullptr;
    // streamed list and cells
    DevPairList pl, pl2;
    // pair-based form: tables of the run's list (pt) and of the forces-only list (pt2)
    bool pairs = false;
    DevPairTables pt, pt2;
    // streamed chunks of small launches: the K steps in one cooperative launch
    bool coop = false;
    unsigned *d_bar = nullptr;   // its grid barrier (count, generation)
    DevCells cells;
    int64_t pl_cap = 0;
    int ppb = 64;
    // dumps of the batched list
    int32_t *d_dump_start = nullptr, *d_dump_len = nullptr, *d_dump_col = nullptr;
    // observables
    DevObs obs;
    // external forces (host mirrors)
    std::vector<int32_t> pull_of_sys, pull_anchor, pull_bead, pull_sys;
    std::vector<double> pull_ks, pull_v, pull_dir, pull_n0, pull_tip0;
    int32_t *d_pull_of_sys = nullptr, *d_pull_anchor = nullptr, *d_pull_bead = nullptr;
    double *d_pull_ks = nullptr, *d_pull_v = nullptr, *d_pull_dir = nullptr, *d_pull_n0 = nullptr,
           *d_pull_tip0 = nullptr;
    size_t pull_alloc = 0;
    bool has_ind = false;
    double ind_c0[3] = {0, 0, 0}, ind_dir[3] = {0, 0, 0}, ind_radius = 0, ind_v = 0, ind_n0 = 0;
    // kernel arguments
    StepArgs sa;
    // batched schedule: work items (system, replica) grouped into size buckets, each with
    // its own tuned configuration and stream
    struct Bucket {
        int max_n = 0;          // largest system of the bucket
        int cap = 0;            // Verlet capacity per row
        int row_width = 0;      // natives + cap
        int pair_pool = 0;      // pair form: shared-memory pool bytes per item (0: the form does not fit)
        int32_t item_off = 0;   // first item in the item arrays
        int32_t n_items = 0;
        BatchedConfig cfg;
        uint16_t *rows = nullptr;   // rows in global memory (when cfg.rows_global)
        // tuning: the configuration holding the least SM time (cfg: the fastest alone), the
        // cache key, and whether this bucket was timed (not taken from the cache or default)
        BatchedConfig alt;
        std::string key;
        float span_ms = 0.f;
        bool timed = false;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    int schedule = SOP_SCHED_STREAMED;
    // batched forms the tuner may choose: 0 both (timed), 1 the particle-based gather only,
    // 2 the pair form wherever it fits (the gather elsewhere)
    int batched_form = 0;
    std::vector<Bucket> buckets;
    cudaEvent_t fork_ev = nullptr;
    int batched_cap = 64;   // largest Verlet capacity over the buckets
    int max_sys = 0;
    int32_t n_items = 0;
    int32_t *d_item_rep = nullptr, *d_item_sys = nullptr;
    // graphs: [start buffer] for the streamed K-step chunk, one for the batched chunk
    // streamed K-step chunk graphs by [start buffer][chunk ends at an observation step]
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t gexec_launches[2][2] = {{0, 0}, {0, 0}};   // kernels in each streamed chunk graph
    cudaGraphExec_t bexec = nullptr;
    // in-flight limiter: at most kInFlight chunks queued ahead of the device, so that
    // sop_abort takes effect within a few chunks and the step counter stays exact
    cudaEvent_t chunk_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t chunk_no = 0;
    bool graphs_enabled = true;
    int lanes = 8;
    sop_stats st{};
    std::string err;
};

namespace {

sop_status fail(sop_ctx *c, sop_status code, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

#define CUDA_OR_RETURN(ctx, expr)                                                                      \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? SOP_ERR_OOM : SOP_ERR_CUDA,           \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

template <typename T>
cudaError_t dalloc(sop_ctx *c, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(T));
    if (e == cudaSuccess) {
        c->allocs.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

template <typename T>
cudaError_t upload(sop_ctx *c, T **p, const std::vector<T> &v) {
    cudaError_t e = dalloc(c, p, v.size());
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

constexpr int kInFlight = 3;

// Wait until no more than kInFlight chunks are queued, then record this chunk's slot.
sop_status throttle_before_chunk(sop_ctx *c) {
    if (!c->chunk_ev[0])
        for (auto &e : c->chunk_ev) CUDA_OR_RETURN(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (c->chunk_no >= kInFlight) CUDA_OR_RETURN(c, cudaEventSynchronize(c->chunk_ev[(c->chunk_no - kInFlight) % 4]));
    return SOP_OK;
}

sop_status record_chunk(sop_ctx *c) {
    CUDA_OR_RETURN(c, cudaEventRecord(c->chunk_ev[c->chunk_no % 4], c->stream));
    c->chunk_no++;
    return SOP_OK;
}

void destroy_graphs(sop_ctx *c) {
    for (auto &row : c->gexec)
        for (auto &g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (c->bexec) { cudaGraphExecDestroy(c->bexec); c->bexec = nullptr; }
}

SegRange full_range(const sop_ctx *c) {
    SegRange r;
    r.g_lo = 0;
    r.g_hi = c->n_seg;
    r.b_lo = c->h_seg_bead_lo[0];
    r.b_hi = c->h_seg_bead_lo[c->n_seg];
    r.c_lo = c->h_seg_cell_base[0];
    r.c_hi = c->h_seg_cell_base[c->n_seg];
    r.max_seg = c->max_sys;
    r.k_lo = c->h_brute_cta_lo[0];
    r.k_hi = c->h_brute_cta_lo[c->n_seg];
    return r;
}

SegRange seg_range(const sop_ctx *c, int g_lo, int g_hi) {
    SegRange r;
    r.g_lo = g_lo;
    r.g_hi = g_hi;
    r.b_lo = c->h_seg_bead_lo[g_lo];
    r.b_hi = c->h_seg_bead_lo[g_hi];
    r.c_lo = c->h_seg_cell_base[g_lo];
    r.c_hi = c->h_seg_cell_base[g_hi];
    r.max_seg = c->max_sys;
    r.k_lo = c->h_brute_cta_lo[g_lo];
    r.k_hi = c->h_brute_cta_lo[g_hi];
    return r;
}

// Rebuild of the run's Verlet list (and, in the pair-based form, its half list).
void rebuild_list(sop_ctx *c, const float4 *pos, float4 *snap, const SegRange &rg, int64_t *launches) {
    launch_rebuild(c->sa, c->cells, c->pl, pos, snap, rg, c->stream, launches);
    if (c->pairs) launch_pair_index(c->sa, c->pl, c->pt, rg, c->stream, launches);
}

// One step of the beads of rg from layer `in` to layer `out`, particle- or pair-based.
void step_range(sop_ctx *c, const float4 *in, float4 *out, const SegRange &rg, int32_t k_off, int64_t *launches) {
    if (c->pairs)
        launch_pairs_step(c->sa, c->pl, c->pt, in, out, c->d_comp, rg, k_off, c->lanes, c->stream, launches);
    else
        launch_step(c->sa, c->pl, in, out, c->d_comp, rg.b_lo, rg.b_hi, k_off, c->lanes, c->stream, launches);
}

// Refresh the pulling / indenter part of the kernel arguments.
void sync_external(sop_ctx *c) {
    DevExternal &e = c->sa.ext;
    e.pull_of_sys = c->d_pull_of_sys;
    e.pull_anchor = c->d_pull_anchor;
    e.pull_bead = c->d_pull_bead;
    e.pull_ks = c->d_pull_ks;
    e.pull_v = c->d_pull_v;
    e.pull_dir = c->d_pull_dir;
    e.pull_n0 = c->d_pull_n0;
    e.pull_tip0 = c->d_pull_tip0;
    e.n_pull = (int32_t)c->pull_bead.size();
    e.has_indenter = c->has_ind ? 1 : 0;
    for (int k = 0; k < 3; ++k) { e.ind_c0[k] = c->ind_c0[k]; e.ind_dir[k] = c->ind_dir[k]; }
    e.ind_radius = c->ind_radius;
    e.ind_v = c->ind_v;
    e.ind_n0 = c->ind_n0;
}

sop_status rebuild_streamed(sop_ctx *c) {
    rebuild_list(c, c->d_pos[c->cur], c->d_snap, full_range(c), &c->st.kernel_launches);
    c->list_step = c->step;
    c->st.rebuilds++;
    CUDA_OR_RETURN(c, cudaGetLastError());
    return SOP_OK;
}

BatchedArgs batched_args(sop_ctx *c, const sop_ctx::Bucket &bk) {
    BatchedArgs a;
    a.sa = c->sa;
    a.n_items = bk.n_items;
    a.item_rep = c->d_item_rep + bk.item_off;
    a.item_sys = c->d_item_sys + bk.item_off;
    a.nat_ell_off = c->d_nat_ell_off;
    a.nat_ell_cnt = c->d_nat_ell_cnt;
    a.nat_ell_col = c->d_nat_ell_col;
    a.nat_ell_r0sq = c->d_nat_ell_r0sq;
    a.nat_slot_bead = c->d_nat_slot_bead;
    a.nat_slot_cnt = c->d_nat_slot_cnt;
    a.nat_slot_ent = c->d_nat_slot_ent;
    a.nat_own_off = c->d_nat_own_off;
    a.nat_own_cnt = c->d_nat_own_cnt;
    a.nat_own_col = c->d_nat_own_col;
    a.nat_own_r0sq = c->d_nat_own_r0sq;
    a.nat_rev_off = c->d_nat_rev_off;
    a.nat_rev_cnt = c->d_nat_rev_cnt;
    a.nat_rev_col = c->d_nat_rev_col;
    a.nat_rev_k = c->d_nat_rev_k;
    a.pair_pool = bk.pair_pool;
    a.excl_off = c->d_excl_off;
    a.excl = c->d_excl;
    a.pos = c->d_pos[0];
    a.comp = c->d_comp;
    a.snap = c->d_snap;
    a.d_step = c->d_step;
    a.d_events = c->d_events;
    a.K = c->prm.rebuild_every;
    a.cap = bk.cap;
    a.max_n = bk.max_n;
    a.row_global = bk.rows;
    a.row_width = bk.row_width;
    a.obs = c->obs;
    a.obs_every = c->prm.obs_every;
    a.n_seg = c->n_seg;
    return a;
}

// Launch the batched kernel for every bucket. `patch` adjusts each bucket's arguments
// (steps, forces mode, buffers). With several buckets they run concurrently on their own
// streams, forked from and joined back into the context's stream (also under capture).
template <class Patch>
sop_status launch_buckets(sop_ctx *c, Patch patch, int64_t *launches) {
    if (c->buckets.size() == 1) {
        BatchedArgs a = batched_args(c, c->buckets[0]);
        patch(a);
        cudaError_t e = launch_batched(a, c->buckets[0].cfg, c->stream, launches);
        if (e != cudaSuccess) return fail(c, SOP_ERR_CUDA, std::string("batched launch: ") + cudaGetErrorString(e));
        return SOP_OK;
    }
    CUDA_OR_RETURN(c, cudaEventRecord(c->fork_ev, c->stream));
    for (auto &bk : c->buckets) {
        CUDA_OR_RETURN(c, cudaStreamWaitEvent(bk.stream, c->fork_ev, 0));
        BatchedArgs a = batched_args(c, bk);
        patch(a);
        cudaError_t e = launch_batched(a, bk.cfg, bk.stream, launches);
        if (e != cudaSuccess) return fail(c, SOP_ERR_CUDA, std::string("batched launch: ") + cudaGetErrorString(e));
        CUDA_OR_RETURN(c, cudaEventRecord(bk.done, bk.stream));
    }
    for (auto &bk : c->buckets) CUDA_OR_RETURN(c, cudaStreamWaitEvent(c->stream, bk.done, 0));
    return SOP_OK;
}

int64_t events_in(int64_t s0, int64_t s1, int32_t every) {   // multiples of every in (s0, s1]
    if (every <= 0) return 0;
    auto fl = [every](int64_t x) { return x >= 0 ? x / every : -((-x + every - 1) / every); };
    return fl(s1) - fl(s0);
}

void note_events(sop_ctx *c, int64_t s0, int64_t s1) { c->events += events_in(s0, s1, c->prm.obs_every); }

// ---- streamed schedule --------------------------------------------------------------
// One K-step chunk from an aligned step whose list is current: K fused steps, the
// rebuild for the next chunk, the observables of the chunk's last step when it is an
// observation step (with_obs; also gated on the device), and the step counter advance.
void enqueue_streamed_chunk(sop_ctx *c, int start_buf, bool with_obs, int64_t *launches) {
    const int K = c->prm.rebuild_every;
    const SegRange all = full_range(c);
    int b = start_buf;
    if (c->coop) {
        launch_step_coop(c->sa, c->pl, c->d_pos[b], c->d_pos[b ^ 1], c->d_comp, all.b_lo, all.b_hi, 0, K, c->lanes,
                         c->d_bar, c->stream, launches);
        if (K & 1) b ^= 1;
    } else {
        for (int k = 0; k < K; ++k) {
            step_range(c, c->d_pos[b], c->d_pos[b ^ 1], all, k, launches);
            b ^= 1;
        }
    }
    // the list of step + K is built from the positions of step + K (the next chunk's first step)
    rebuild_list(c, c->d_pos[b], c->d_snap, all, launches);
    if (c->prm.obs_every > 0 && with_obs)
        launch_observables(c->sa, c->pl, c->obs, c->d_pos[b], c->n_seg, K, c->prm.obs_every, c->stream, launches);
    launch_tick(c->d_step, K, c->d_events, c->prm.obs_every > 0 ? c->prm.obs_every : 0, 0, c->stream, launches);
}

sop_status build_streamed_graph(sop_ctx *c, int start_buf, bool with_obs) {
    cudaGraph_t g = nullptr;
    int64_t launches = 0;
    CUDA_OR_RETURN(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_streamed_chunk(c, start_buf, with_obs, &launches);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&c->gexec[start_buf][with_obs], g, 0);
        cudaGraphDestroy(g);
        g = nullptr;
    }
    if (e != cudaSuccess && c->coop) {   // no cooperative node in the graph: fall back to one launch per step
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        c->coop = false;
        return build_streamed_graph(c, start_buf, with_obs);
    }
    c->gexec_launches[start_buf][with_obs] = launches;
    if (e != cudaSuccess) return fail(c, SOP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return SOP_OK;
}

sop_status step_streamed(sop_ctx *c, int64_t n_steps) {
    const int K = c->prm.rebuild_every;
    const int32_t every = c->prm.obs_every;
    const bool aligned_obs = every <= 0 || every % K == 0;
    const SegRange all = full_range(c);
    int64_t left = n_steps;
    while (left > 0) {
        if (*(volatile int32_t *)c->h_abort) break;
        if (c->step % K == 0 && left >= K && aligned_obs && c->graphs_enabled) {
            if (c->list_step != c->step) {
                sop_status s = rebuild_streamed(c);
                if (s != SOP_OK) return s;
            }
            const int wo = every > 0 && (c->step + K) % every == 0 ? 1 : 0;
            if (!c->gexec[c->cur][wo]) {
                sop_status s = build_streamed_graph(c, c->cur, wo != 0);
                if (s != SOP_OK) return s;
            }
            sop_status th = throttle_before_chunk(c);
            if (th != SOP_OK) return th;
            CUDA_OR_RETURN(c, cudaGraphLaunch(c->gexec[c->cur][wo], c->stream));
            th = record_chunk(c);
            if (th != SOP_OK) return th;
            c->st.graph_launches++;
            c->st.kernel_launches += c->gexec_launches[c->cur][wo];
            c->st.rebuilds++;
            if (K & 1) c->cur ^= 1;
            note_events(c, c->step, c->step + K);
            c->step += K;
            c->list_step = c->step;
            left -= K;
            continue;
        }
        // single step
        if (c->step % K == 0 && c->list_step != c->step) {
            sop_status s = rebuild_streamed(c);
            if (s != SOP_OK) return s;
        }
        step_range(c, c->d_pos[c->cur], c->d_pos[c->cur ^ 1], all, 0, &c->st.kernel_launches);
        c->cur ^= 1;
        const int64_t s1 = c->step + 1;
        if (every > 0 && s1 % every == 0) {
            if (s1 % K == 0) {
                rebuild_list(c, c->d_pos[c->cur], c->d_snap, all, &c->st.kernel_launches);
                c->st.rebuilds++;
                c->list_step = s1;
            }
            launch_observables(c->sa, c->pl, c->obs, c->d_pos[c->cur], c->n_seg, 1, 0, c->stream,
                               &c->st.kernel_launches);
        }
        launch_tick(c->d_step, 1, c->d_events, 0, (every > 0 && s1 % every == 0) ? 1 : 0, c->stream,
                    &c->st.kernel_launches);
        note_events(c, c->step, s1);
        c->step = s1;
        --left;
    }
    CUDA_OR_RETURN(c, cudaGetLastError());
    return SOP_OK;
}

// ---- plain schedule: one system after another, per-step launches, no graph ---------------
sop_status step_plain(sop_ctx *c, int64_t n_steps) {
    const int K = c->prm.rebuild_every;
    const int32_t every = c->prm.obs_every;
    const int64_t s0 = c->step;
    for (int g = 0; g < c->n_seg; ++g) {
        if (*(volatile int32_t *)c->h_abort) break;
        const SegRange rg = seg_range(c, g, g + 1);
        int b = c->cur;
        bool built = false;   // the list of the current step was built for the observables
        for (int64_t k = 0; k < n_steps; ++k) {
            const int64_t s = s0 + k;
            if (s % K == 0 && !(k == 0 && c->list_step == s) && !built)
                launch_rebuild(c->sa, c->cells, c->pl, c->d_pos[b], c->d_snap, rg, c->stream, &c->st.kernel_launches);
            built = false;
            launch_step(c->sa, c->pl, c->d_pos[b], c->d_pos[b ^ 1], c->d_comp, rg.b_lo, rg.b_hi, (int32_t)k, c->lanes,
                        c->stream, &c->st.kernel_launches);
            b ^= 1;
            if (every > 0 && (s + 1) % every == 0) {   // this segment's record of step s + 1
                if ((s + 1) % K == 0) {
                    launch_rebuild(c->sa, c->cells, c->pl, c->d_pos[b], c->d_snap, rg, c->stream,
                                   &c->st.kernel_launches);
                    built = true;
                }
                launch_observables_seg(c->sa, c->pl, c->obs, c->d_pos[b], g, c->n_seg, c->h_seg_chunk_lo[g],
                                       c->h_seg_chunk_lo[g + 1], (int32_t)(k + 1), events_in(s0, s + 1, every) - 1,
                                       c->stream, &c->st.kernel_launches);
            }
        }
    }
    launch_tick(c->d_step, n_steps, c->d_events, 0, events_in(s0, s0 + n_steps, every), c->stream,
                &c->st.kernel_launches);
    note_events(c, s0, s0 + n_steps);
    if (n_steps & 1) c->cur ^= 1;
    c->step = s0 + n_steps;
    // the list in use is the one built at the last multiple of K inside this call, if any
    if (n_steps > 0) {
        const int64_t last = ((c->step - 1) / K) * K;
        if (last >= s0) c->list_step = last;
    }
    CUDA_OR_RETURN(c, cudaGetLastError());
    return SOP_OK;
}

// ---- batched schedule -----------------------------------------------------------------
sop_status step_batched(sop_ctx *c, int64_t n_steps) {
    // The batched kernel reads and writes layer 0; bring the state there first.
    if (c->cur != 0) {
        CUDA_OR_RETURN(c, cudaMemcpyAsync(c->d_pos[0], c->d_pos[1], sizeof(float4) * (size_t)c->R * c->n,
                                          cudaMemcpyDeviceToDevice, c->stream));
        c->cur = 0;
    }
    int64_t left = n_steps;
    while (left > 0) {
        if (*(volatile int32_t *)c->h_abort) break;
        const int64_t chunk = std::min<int64_t>(left, kBatchedChunk);
        const int64_t nev = events_in(c->step, c->step + chunk, c->prm.obs_every);
        sop_status th = throttle_before_chunk(c);
        if (th != SOP_OK) return th;
        auto set_steps = [chunk](BatchedArgs &a) { a.n_steps = (int32_t)chunk; };
        // a full chunk whose cadence divides it always holds the same number of records:
        // replay it from a graph; anything else is launched directly
        const bool regular = c->prm.obs_every <= 0 || kBatchedChunk % c->prm.obs_every == 0;
        if (c->graphs_enabled && chunk == kBatchedChunk && regular) {
            if (!c->bexec) {
                cudaGraph_t g = nullptr;
                CUDA_OR_RETURN(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                int64_t dummy = 0;
                sop_status s1 = launch_buckets(c, set_steps, &dummy);
                launch_tick(c->d_step, chunk, c->d_events, 0, nev, c->stream, &dummy);
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
                if (s1 != SOP_OK) {
                    if (g) cudaGraphDestroy(g);
                    return s1;
                }
                if (e2 != cudaSuccess)
                    return fail(c, SOP_ERR_CUDA, std::string("batched graph capture: ") + cudaGetErrorString(e2));
                cudaError_t e3 = cudaGraphInstantiate(&c->bexec, g, 0);
                cudaGraphDestroy(g);
                if (e3 != cudaSuccess)
                    return fail(c, SOP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
            }
            CUDA_OR_RETURN(c, cudaGraphLaunch(c->bexec, c->stream));
            c->st.graph_launches++;
            c->st.kernel_launches += (int64_t)c->buckets.size() + 1;
        } else {
            sop_status s1 = launch_buckets(c, set_steps, &c->st.kernel_launches);
            if (s1 != SOP_OK) return s1;
            launch_tick(c->d_step, chunk, c->d_events, 0, nev, c->stream, &c->st.kernel_launches);
        }
        th = record_chunk(c);
        if (th != SOP_OK) return th;
        c->st.rebuilds += events_in(c->step - 1, c->step + chunk - 1, c->prm.rebuild_every);
        note_events(c, c->step, c->step + chunk);
        c->step += chunk;
        c->list_step = (c->step / c->prm.rebuild_every) * c->prm.rebuild_every;
        left -= chunk;
    }
    CUDA_OR_RETURN(c, cudaGetLastError());
    return SOP_OK;
}

// Validate and normalise inputs; fill the host topology tables.
sop_status build_host_topology(sop_ctx *c, const sop_topology *t) {
    if (!t || t->n_beads < 1 || t->n_chains < 1 || !t->chain_offsets)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: n_beads >= 1, n_chains >= 1 and chain_offsets required");
    if (t->n_beads > (1 << 26)) return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: too many beads per replica");
    c->n = t->n_beads;
    c->n_chains = t->n_chains;
    c->chain_off.assign(t->chain_offsets, t->chain_offsets + t->n_chains + 1);
    if (c->chain_off[0] != 0 || c->chain_off[t->n_chains] != t->n_beads)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: chain_offsets must start at 0 and end at n_beads");
    for (int k = 0; k < t->n_chains; ++k)
        if (c->chain_off[k + 1] <= c->chain_off[k])
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: chain_offsets must be strictly increasing");
    std::vector<int32_t> sys_chain;   // [n_sys+1] in chains
    if (t->n_systems == 0) {
        sys_chain.resize(t->n_chains + 1);
        for (int k = 0; k <= t->n_chains; ++k) sys_chain[k] = k;
    } else {
        if (t->n_systems < 0 || !t->system_offsets)
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: system_offsets required when n_systems > 0");
        sys_chain.assign(t->system_offsets, t->system_offsets + t->n_systems + 1);
        if (sys_chain[0] != 0 || sys_chain[t->n_systems] != t->n_chains)
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: system_offsets must start at 0 and end at n_chains");
        for (int k = 0; k < t->n_systems; ++k)
            if (sys_chain[k + 1] <= sys_chain[k])
                return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: system_offsets must be strictly increasing");
    }
    c->n_sys = (int32_t)sys_chain.size() - 1;
    c->sys_lo.resize(c->n_sys + 1);
    for (int s = 0; s <= c->n_sys; ++s) c->sys_lo[s] = c->chain_off[sys_chain[s]];
    c->chain_of.resize(c->n);
    c->sys_of.resize(c->n);
    for (int k = 0; k < c->n_chains; ++k)
        for (int i = c->chain_off[k]; i < c->chain_off[k + 1]; ++i) c->chain_of[i] = k;
    for (int s = 0; s < c->n_sys; ++s)
        for (int i = c->sys_lo[s]; i < c->sys_lo[s + 1]; ++i) c->sys_of[i] = s;
    c->flags.assign(c->n, 0);
    c->fixed_by_mask.assign(c->n, 0);
    if (t->fixed_mask)
        for (int i = 0; i < c->n; ++i) {
            c->fixed_by_mask[i] = t->fixed_mask[i] ? 1 : 0;
            c->flags[i] = t->fixed_mask[i] ? kFlagFixed : 0;
        }
    c->sys_ree_last.resize(c->n_sys);
    for (int s = 0; s < c->n_sys; ++s) {
        const int first = c->sys_lo[s];
        c->flags[first] |= kFlagFirstOfSystem;
        c->sys_ree_last[s] = c->chain_off[c->chain_of[first] + 1] - 1;
        c->max_sys = std::max(c->max_sys, c->sys_lo[s + 1] - c->sys_lo[s]);
    }
    if (t->n_extra_bonds < 0 || (t->n_extra_bonds > 0 && !t->extra_bonds))
        return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: n_extra_bonds >= 0 and extra_bonds required");
    for (int k = 0; k < t->n_extra_bonds; ++k) {
        int32_t i = t->extra_bonds[2 * k], j = t->extra_bonds[2 * k + 1];
        if (i < 0 || j < 0 || i >= c->n || j >= c->n || i == j)
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: an extra bond names a bead out of range, or one twice");
        if (i > j) std::swap(i, j);
        if (c->sys_of[i] != c->sys_of[j])
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: an extra bond joins two systems");
        if (j == i + 1 && c->chain_of[i] == c->chain_of[j])
            return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: an extra bond repeats a chain bond (i, i+1)");
        c->xlinks.emplace_back(i, j);
    }
    std::sort(c->xlinks.begin(), c->xlinks.end());
    if (std::adjacent_find(c->xlinks.begin(), c->xlinks.end()) != c->xlinks.end())
        return fail(nullptr, SOP_ERR_INVALID_ARG, "topology: an extra bond is listed twice");
    return SOP_OK;
}

sop_status validate_params(const sop_params *p) {
    if (!p) return fail(nullptr, SOP_ERR_INVALID_ARG, "params is NULL");
    const double pos[] = {p->k_fene, p->R0, p->native_cut, p->sigma, p->zeta, p->dt, p->pair_cut};
    for (double v : pos)
        if (!finite_pos(v)) return fail(nullptr, SOP_ERR_INVALID_ARG, "params: k_fene, R0, native_cut, sigma, zeta, dt, pair_cut must be finite and > 0");
    if (!std::isfinite(p->eps_h) || !std::isfinite(p->eps_l) || p->eps_h < 0 || p->eps_l < 0)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: eps_h, eps_l must be finite and >= 0");
    if (!std::isfinite(p->T) || p->T < 0) return fail(nullptr, SOP_ERR_INVALID_ARG, "params: T must be finite and >= 0");
    if (p->rebuild_every < 1) return fail(nullptr, SOP_ERR_INVALID_ARG, "params: rebuild_every >= 1");
    if (p->n_replicas < 1) return fail(nullptr, SOP_ERR_INVALID_ARG, "params: n_replicas >= 1");
    if (p->obs_every < 0 || p->obs_capacity < 0 || p->pairs_per_bead < 0)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: obs_every, obs_capacity, pairs_per_bead >= 0");
    if (p->obs_every_q < 0 || (p->obs_every_q > 0 && (p->obs_every <= 0 || p->obs_every_q % p->obs_every != 0)))
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: obs_every_q must be 0 or a multiple of obs_every > 0");
    if (p->schedule < SOP_SCHED_AUTO || p->schedule > SOP_SCHED_BATCHED_PAIRS)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: unknown schedule");
    if (p->rng != SOP_RNG_PHILOX && p->rng != SOP_RNG_HYBRID_TAUS)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: unknown rng");
    if (p->integrator != SOP_INTEGRATOR_OVERDAMPED && p->integrator != SOP_INTEGRATOR_BAOAB)
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: unknown integrator");
    if (p->integrator == SOP_INTEGRATOR_BAOAB && !(std::isfinite(p->mass) && p->mass > 0))
        return fail(nullptr, SOP_ERR_INVALID_ARG, "params: the underdamped integrator needs a finite mass > 0");
    return SOP_OK;
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA'14): advance the Weyl state, mix the result.
uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial Hybrid Taus state of bead i of replica r (see sop_get_rng_state).
void taus_seed(uint64_t seed, int r, int i, uint32_t out[4]) {
    uint64_t x = ((seed + (uint64_t)r) << 32) + (uint64_t)(uint32_t)i;
    const uint64_t a = splitmix64(x), b = splitmix64(x);
    out[0] = (uint32_t)a;
    out[1] = (uint32_t)(a >> 32);
    out[2] = (uint32_t)b;
    out[3] = (uint32_t)(b >> 32);
    if (out[0] < 2u) out[0] += 2u;
    if (out[1] < 8u) out[1] += 8u;
    if (out[2] < 16u) out[2] += 16u;
}

sop_status alloc_pull_arrays(sop_ctx *c, size_t n_pull) {
    if (n_pull <= c->pull_alloc && c->d_pull_anchor) return SOP_OK;
    const size_t m = std::max<size_t>(1, n_pull);
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_anchor, m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_bead, m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_ks, m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_v, m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_dir, 3 * m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_n0, m));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_pull_tip0, 3 * m * (size_t)c->R));
    c->pull_alloc = m;
    return SOP_OK;
}

// A complete set of pulling records, assembled and checked before it replaces the
// context's records (so that a failing call leaves the context as it was).
struct PullSet {
    std::vector<int32_t> sys, anchor, bead;
    std::vector<double> ks, v, n0, dir, tip0;
    void resize(size_t np, int R) {
        sys.resize(np); anchor.resize(np); bead.resize(np);
        ks.resize(np); v.resize(np); n0.resize(np); dir.resize(3 * np); tip0.resize(3 * np * (size_t)R);
    }
};

// Replace the pulling records. The flags of the old records are cleared first: the
// pulled mark always, the fixed mark only where the topology's fixed_mask did not set it.
void install_pulls(sop_ctx *c, PullSet &&ps) {
    for (size_t k = 0; k < c->pull_bead.size(); ++k) {
        c->flags[c->pull_bead[k]] &= (uint8_t)~kFlagPulled;
        const int a = c->pull_anchor[k];
        if (!c->fixed_by_mask[a]) c->flags[a] &= (uint8_t)~kFlagFixed;
    }
    c->pull_sys = std::move(ps.sys);
    c->pull_anchor = std::move(ps.anchor);
    c->pull_bead = std::move(ps.bead);
    c->pull_ks = std::move(ps.ks);
    c->pull_v = std::move(ps.v);
    c->pull_n0 = std::move(ps.n0);
    c->pull_dir = std::move(ps.dir);
    c->pull_tip0 = std::move(ps.tip0);
    c->pull_of_sys.assign(c->n_sys, -1);
    for (size_t k = 0; k < c->pull_bead.size(); ++k) {
        c->pull_of_sys[c->pull_sys[k]] = (int32_t)k;
        c->flags[c->pull_bead[k]] |= kFlagPulled;
        c->flags[c->pull_anchor[k]] |= kFlagFixed;
    }
}

sop_status upload_pulls(sop_ctx *c) {
    const size_t np = c->pull_bead.size();
    sop_status s = alloc_pull_arrays(c, np);
    if (s != SOP_OK) return s;
    CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_of_sys, c->pull_of_sys.data(), sizeof(int32_t) * c->n_sys, cudaMemcpyHostToDevice));
    if (np) {
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_anchor, c->pull_anchor.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_bead, c->pull_bead.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_ks, c->pull_ks.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_v, c->pull_v.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_dir, c->pull_dir.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_n0, c->pull_n0.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pull_tip0, c->pull_tip0.data(), sizeof(double) * 3 * np * c->R,
                                     cudaMemcpyHostToDevice));
    }
    CUDA_OR_RETURN(c, cudaMemcpy(c->d_flags, c->flags.data(), c->n, cudaMemcpyHostToDevice));
    sync_external(c);
    destroy_graphs(c);   // kernel arguments changed
    return SOP_OK;
}

// Copy positions of every replica to the host as float4.
sop_status positions_f4(sop_ctx *c, std::vector<float4> &h) {
    h.resize((size_t)c->R * c->n);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(h.data(), c->d_pos[c->cur], sizeof(float4) * h.size(), cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

sop_status read_status(sop_ctx *c, bool aborted) {
    std::vector<int32_t> st(c->R);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(st.data(), c->d_rep_status, sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    for (int r = 0; r < c->R; ++r)
        if (st[r] != 0 && st[r] != SOP_ERR_ABORTED) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "replica %d stopped with status %d (first failing replica)", r, st[r]);
            return fail(c, (sop_status)st[r], buf);
        }
    if (aborted) return fail(c, SOP_ERR_ABORTED, "aborted by sop_abort");
    return SOP_OK;
}

// Balanced orientation of the native pairs for the pair form: each pair goes to the row of
// one of its two beads, and every bead owns half of its native pairs (rounded either way).
// All pairs are walked as closed trails after the odd-degree beads have been joined in pairs
// by extra edges (so that every degree is even and a trail can only end where it began);
// each pair belongs to the bead the trail leaves it from. A closed trail enters and leaves a
// bead equally often, so a bead's own pairs differ from half its degree by at most the one
// extra edge. Returns, per CSR entry q of (row i, col j), whether i owns the pair.
std::vector<uint8_t> orient_natives(int n, const std::vector<int32_t> &row, const std::vector<int32_t> &col) {
    std::vector<int32_t> eu, ev;   // edges: real pairs (i < j) first, then the extra ones
    std::vector<int32_t> q_of;     // CSR entry (i -> j) of each real edge
    for (int i = 0; i < n; ++i)
        for (int q = row[i]; q < row[i + 1]; ++q)
            if (col[q] > i) { eu.push_back(i); ev.push_back(col[q]); q_of.push_back(q); }
    const int n_real = (int)eu.size();
    int pending = -1;
    for (int i = 0; i < n; ++i)
        if ((row[i + 1] - row[i]) & 1) {
            if (pending < 0) pending = i;
            else { eu.push_back(pending); ev.push_back(i); pending = -1; }
        }
    const int m = (int)eu.size();
    std::vector<int32_t> adj_off(n + 1, 0), adj;
    for (int e = 0; e < m; ++e) { ++adj_off[eu[e] + 1]; ++adj_off[ev[e] + 1]; }
    for (int i = 0; i < n; ++i) adj_off[i + 1] += adj_off[i];
    adj.resize(adj_off[n]);
    std::vector<int32_t> fill(adj_off.begin(), adj_off.end() - 1);
    for (int e = 0; e < m; ++e) { adj[fill[eu[e]]++] = e; adj[fill[ev[e]]++] = e; }
    std::vector<uint8_t> used(m, 0), tail_is_u(m, 0);
    std::vector<int32_t> next(adj_off.begin(), adj_off.end() - 1);
    for (int v0 = 0; v0 < n; ++v0) {
        for (;;) {
            int v = v0;
            bool moved = false;
            for (;;) {
                while (next[v] < adj_off[v + 1] && used[adj[next[v]]]) ++next[v];
                if (next[v] == adj_off[v + 1]) break;
                const int e = adj[next[v]];
                used[e] = 1;
                tail_is_u[e] = (eu[e] == v) ? 1 : 0;
                v = (eu[e] == v) ? ev[e] : eu[e];
                moved = true;
            }
            if (!moved) break;
        }
    }
    std::vector<uint8_t> owner_is_row(col.size(), 0);
    for (int e = 0; e < n_real; ++e) {
        const int q = q_of[e];   // entry (eu -> ev)
        owner_is_row[q] = tail_is_u[e];
        // the mirrored entry (ev -> eu)
        const int j = ev[e];
        for (int r = row[j]; r < row[j + 1]; ++r)
            if (col[r] == eu[e]) { owner_is_row[r] = tail_is_u[e] ? 0 : 1; break; }
    }
    return owner_is_row;
}

// The pair form's native tables: per system, column-major ELL by bead of the own pairs
// (partner, r0^2) and of the reverse pairs (partner, index of the bead among the partner's
// own pairs), partners ascending.
sop_status build_pair_tables(sop_ctx *c, const std::vector<float> &h_r0sq) {
    const std::vector<uint8_t> own = orient_natives(c->n, c->h_nat_row, c->h_nat_col);
    std::vector<int32_t> own_cnt(c->n, 0), rev_cnt(c->n, 0), own_off(c->n_sys), rev_off(c->n_sys);
    for (int i = 0; i < c->n; ++i)
        for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q) (own[q] ? own_cnt[i] : rev_cnt[i])++;
    size_t to = 0, tr = 0;
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        int wo = 0, wr = 0;
        for (int i = lo; i < hi; ++i) { wo = std::max(wo, own_cnt[i]); wr = std::max(wr, rev_cnt[i]); }
        own_off[s] = (int32_t)to;
        rev_off[s] = (int32_t)tr;
        to += (size_t)wo * ns;
        tr += (size_t)wr * ns;
    }
    if (to > (size_t)INT32_MAX || tr > (size_t)INT32_MAX) return fail(c, SOP_ERR_UNSUPPORTED, "pair-form native tables too large");
    std::vector<uint16_t> ocol(std::max<size_t>(1, to), 0), rcol(std::max<size_t>(1, tr), 0), rk(std::max<size_t>(1, tr), 0);
    std::vector<float> or0(std::max<size_t>(1, to), 0.f);
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        for (int i = lo; i < hi; ++i) {
            int ko = 0, kr = 0;
            for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q) {
                const int j = c->h_nat_col[q];
                if (own[q]) {
                    const size_t e = (size_t)own_off[s] + (size_t)ko++ * ns + (i - lo);
                    ocol[e] = (uint16_t)(j - lo);
                    or0[e] = h_r0sq[q];
                } else {
                    // the index of i among j's own pairs (ascending partners)
                    int kj = 0;
                    for (int r = c->h_nat_row[j]; r < c->h_nat_row[j + 1] && c->h_nat_col[r] < i; ++r) kj += own[r];
                    const size_t e = (size_t)rev_off[s] + (size_t)kr++ * ns + (i - lo);
                    rcol[e] = (uint16_t)(j - lo);
                    rk[e] = (uint16_t)kj;
                }
            }
        }
    }
    c->h_nat_own_cnt = own_cnt;
    c->h_nat_rev_cnt = rev_cnt;
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_own_off, own_off));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_own_cnt, own_cnt));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_own_col, ocol));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_own_r0sq, or0));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_rev_off, rev_off));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_rev_cnt, rev_cnt));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_rev_col, rcol));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_rev_k, rk));
    return SOP_OK;
}

// Static exclusions of the batched rebuild scan for systems of at most 256 beads: for bead b
// and candidate block blk (beads 32 blk .. 32 blk + 31 of the system), the bits of the bead
// itself, its bonded neighbours (bond length > 0, as the kernels test it) and its native
// partners. Larger systems (offset -1) exclude on the fly.
sop_status build_exclusions(sop_ctx *c) {
    std::vector<float> r0(c->n);
    CUDA_OR_RETURN(c, cudaMemcpy(r0.data(), c->d_bond_r0, sizeof(float) * c->n, cudaMemcpyDeviceToHost));
    std::vector<int32_t> off(c->n_sys, -1);
    std::vector<uint32_t> ex;
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], ns = c->sys_lo[s + 1] - lo;
        if (ns > 256) continue;
        const int nblk = (ns + 31) / 32;
        off[s] = (int32_t)ex.size();
        ex.resize(ex.size() + (size_t)nblk * ns, 0u);
        uint32_t *e = ex.data() + off[s];
        auto mark = [&](int b, int j) { e[(j >> 5) * ns + b] |= 1u << (j & 31); };
        for (int b = 0; b < ns; ++b) {
            const int i = lo + b;
            mark(b, b);
            if (b > 0 && r0[i - 1] > 0.f) mark(b, b - 1);
            if (b + 1 < ns && r0[i] > 0.f) mark(b, b + 1);
            for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q) mark(b, c->h_nat_col[q] - lo);
        }
    }
    if (ex.empty()) ex.push_back(0u);
    CUDA_OR_RETURN(c, upload(c, &c->d_excl_off, off));
    CUDA_OR_RETURN(c, upload(c, &c->d_excl, ex));
    return SOP_OK;
}

// Batched natives: per system, column-major ELL of system-local partner indices.
sop_status build_batched_tables(sop_ctx *c) {
    std::vector<int32_t> off(c->n_sys), cnt(c->n);
    std::vector<uint16_t> col;
    std::vector<float> r0sq;
    std::vector<float> h_r0sq(c->nat_nnz);
    if (c->nat_nnz) {
        CUDA_OR_RETURN(c, cudaMemcpy(h_r0sq.data(), c->d_nat_r0sq, sizeof(float) * c->nat_nnz, cudaMemcpyDeviceToHost));
    }
    size_t total = 0;
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        int w = 0;
        for (int i = lo; i < hi; ++i) {
            cnt[i] = c->h_nat_row[i + 1] - c->h_nat_row[i];
            w = std::max(w, cnt[i]);
        }
        off[s] = (int32_t)total;
        total += (size_t)w * ns;
    }
    if (total > (size_t)INT32_MAX) return fail(c, SOP_ERR_UNSUPPORTED, "batched native table too large");
    col.assign(std::max<size_t>(1, total), 0);
    r0sq.assign(std::max<size_t>(1, total), 0.f);
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        for (int i = lo; i < hi; ++i)
            for (int k = 0; k < cnt[i]; ++k) {
                const int p = c->h_nat_row[i] + k;
                const size_t e = (size_t)off[s] + (size_t)k * ns + (i - lo);
                col[e] = (uint16_t)(c->h_nat_col[p] - lo);
                r0sq[e] = h_r0sq[p];
            }
    }
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_ell_off, off));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_ell_cnt, cnt));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_ell_col, col));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_ell_r0sq, r0sq));
    // the same entries in native-slot order (beads by native count, descending, stable)
    std::vector<uint16_t> sbead(c->n), scnt(c->n);
    std::vector<uint2> sent(col.size(), make_uint2(0u, 0u));
    for (int s = 0; s < c->n_sys; ++s) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        std::vector<int> ord(ns);
        for (int t = 0; t < ns; ++t) ord[t] = t;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cnt[lo + x] > cnt[lo + y]; });
        for (int t = 0; t < ns; ++t) {
            const int b = ord[t];
            sbead[lo + t] = (uint16_t)b;
            scnt[lo + t] = (uint16_t)cnt[lo + b];
            for (int k = 0; k < cnt[lo + b]; ++k) {
                const size_t src = (size_t)off[s] + (size_t)k * ns + b;
                uint32_t bits;
                std::memcpy(&bits, &r0sq[src], sizeof bits);
                sent[(size_t)off[s] + (size_t)k * ns + t] = make_uint2(col[src], bits);
            }
        }
    }
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_slot_bead, sbead));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_slot_cnt, scnt));
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_slot_ent, sent));
    sop_status se = build_exclusions(c);
    if (se != SOP_OK) return se;
    return build_pair_tables(c, h_r0sq);
}

// Size buckets of the batched schedule: systems of up to 32, 64, 96, 128, 192, 256, 384, 512,
// 768, 1024, 1536, 2048, 4096 and 8192 beads. Each bucket gets its work items (system,
// replica; heaviest system first), a Verlet capacity from the first list of its systems and
// the width of its merged rows.
// Pool bytes of the pair form for the systems `sys` (all at most kPairMaxBeads beads), from
// their first Verlet list (replica 0): own and reverse entries per bead under the ownership
// rules of the kernel, slots grouped by 32 in the kernel's order (decreasing 2 own + rev),
// each group as wide as its widest row, plus a margin of a fifth and one entry per row.
int pair_pool_for(const sop_ctx *c, const std::vector<int32_t> &sys, const std::vector<int32_t> &first_start,
                  const std::vector<int32_t> &first_len, const std::vector<int32_t> &first_col) {
    size_t pool = 0;
    for (int s : sys) {
        const int lo = c->sys_lo[s], hi = c->sys_lo[s + 1], ns = hi - lo;
        std::vector<int> own(ns), rev(ns), key(ns), ord(ns);
        for (int b = 0; b < ns; ++b) { own[b] = c->h_nat_own_cnt[lo + b]; rev[b] = c->h_nat_rev_cnt[lo + b]; }
        for (int b = 0; b < ns; ++b)
            for (int q = 0; q < first_len[lo + b]; ++q) {
                const int j = first_col[first_start[lo + b] + q] - lo;
                const bool mine = ((b + j) & 1) ? j > b : j < b;
                (mine ? own[b] : rev[b])++;
            }
        for (int b = 0; b < ns; ++b) { key[b] = 2 * own[b] + rev[b]; ord[b] = b; }
        std::stable_sort(ord.begin(), ord.end(), [&key](int x, int y) { return key[x] > key[y]; });
        int so = 0, sr = 0;
        const int G = (ns + 31) / 32;
        for (int g = 0; g < G; ++g) {
            int wo = 0, wr = 0;
            for (int p = 32 * g; p < std::min(ns, 32 * g + 32); ++p) { wo = std::max(wo, own[ord[p]]); wr = std::max(wr, rev[ord[p]]); }
            so += 32 * wo;
            sr += 32 * wr;
        }
        so += so / 5 + 32 * G;
        sr += sr / 5 + 32 * G;
        pool = std::max(pool, pair_pool_bytes(so, sr, ns));
    }
    return (int)pool;
}

sop_status build_buckets(sop_ctx *c, const std::vector<int32_t> &first_start, const std::vector<int32_t> &first_len,
                         const std::vector<int32_t> &first_col) {
    static const int bounds[] = {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 4096, 8192};
    std::vector<int32_t> ir, is;
    int lo = 0;
    for (int hi : bounds) {
        std::vector<int32_t> sys;
        for (int s = 0; s < c->n_sys; ++s) {
            const int ns = c->sys_lo[s + 1] - c->sys_lo[s];
            if (ns > lo && ns <= hi) sys.push_back(s);
        }
        lo = hi;
        if (sys.empty()) continue;
        std::stable_sort(sys.begin(), sys.end(), [c](int a, int b) {
            return c->sys_lo[a + 1] - c->sys_lo[a] > c->sys_lo[b + 1] - c->sys_lo[b];
        });
        sop_ctx::Bucket bk;
        int maxnat = 0, mrow = 0;
        for (int s : sys) {
            bk.max_n = std::max(bk.max_n, c->sys_lo[s + 1] - c->sys_lo[s]);
            for (int i = c->sys_lo[s]; i < c->sys_lo[s + 1]; ++i) {
                maxnat = std::max(maxnat, c->h_nat_row[i + 1] - c->h_nat_row[i]);
                mrow = std::max(mrow, first_len[i]);
            }
        }
        bk.cap = std::min(128, std::max(32, ((mrow * 3) / 2 + 8 + 7) / 8 * 8));
        bk.row_width = maxnat + bk.cap;
        if (bk.row_width > 256) return fail(c, SOP_ERR_UNSUPPORTED, "batched rows wider than 256 entries");
        if (bk.max_n <= kPairMaxBeads && c->batched_form != 1)
            bk.pair_pool = pair_pool_for(c, sys, first_start, first_len, first_col);
        bk.item_off = (int32_t)ir.size();
        for (int s : sys)
            for (int r = 0; r < c->R; ++r) { ir.push_back(r); is.push_back(s); }
        bk.n_items = (int32_t)ir.size() - bk.item_off;
        c->batched_cap = std::max(c->batched_cap, bk.cap);
        c->buckets.push_back(bk);
    }
    if (lo < c->max_sys) return fail(c, SOP_ERR_UNSUPPORTED, "system too large for the batched schedule");
    c->n_items = (int32_t)ir.size();
    CUDA_OR_RETURN(c, upload(c, &c->d_item_rep, ir));
    CUDA_OR_RETURN(c, upload(c, &c->d_item_sys, is));
    if (c->buckets.size() > 1) {
        CUDA_OR_RETURN(c, cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        for (auto &bk : c->buckets) {
            CUDA_OR_RETURN(c, cudaStreamCreateWithFlags(&bk.stream, cudaStreamNonBlocking));
            CUDA_OR_RETURN(c, cudaEventCreateWithFlags(&bk.done, cudaEventDisableTiming));
        }
    }
    return SOP_OK;
}

// Autotuner of one size bucket. Candidates are (threads per CTA, beads per thread, register
// cap, rows in shared or global memory); each is timed on a 20-step trial of the bucket's
// first items (up to 16 CTAs per SM) on scratch copies of the state (the run's state,
// records and statuses are untouched) and the fastest is kept (with several buckets, the
// one holding the least SM time, as the buckets fill each other's last waves). Results are cached in the
// file named by SOP_TUNE_CACHE, keyed by the bucket's size, row width and trial size;
// SOP_TUNE=0 skips the trial and takes the default.
sop_status tune_bucket(sop_ctx *c, sop_ctx::Bucket &bk) {
    std::vector<BatchedConfig> cands;
    const int need = 32 * ((bk.max_n + 31) / 32);
    // the pair form (each pair evaluated once) where it fits; alone when it was asked for
    std::vector<BatchedConfig> pairs;
    if (bk.pair_pool > 0 && c->batched_form != 1)
        for (int threads : {64, 128, 256})
            for (int minb : {2, 3, 4}) {
                BatchedConfig cfg;
                if (threads > need && threads > 64) continue;
                if (pair_config(bk.max_n, bk.pair_pool, threads, minb, &cfg)) pairs.push_back(cfg);
            }
    const bool pairs_only = c->batched_form == 2 && !pairs.empty();
    for (int threads : {64, 128, 256})
        for (int minb : {2, 3, 4}) {
            BatchedConfig cfg;
            if (pairs_only || (threads > need && threads > 64)) continue;   // idle threads only
            if (batched_config(bk.max_n, bk.row_width, threads, false, minb, &cfg)) cands.push_back(cfg);
        }
    for (int threads : {128, 256, 512, 1024}) {
        BatchedConfig cfg;
        if (pairs_only || (threads > need && threads > 128)) continue;
        if (batched_config(bk.max_n, bk.row_width, threads, true, 1, &cfg)) cands.push_back(cfg);
    }
    cands.insert(cands.end(), pairs.begin(), pairs.end());
    // the cluster form for larger systems: one system over 2..16 CTAs of 2^sh beads each,
    // served by 1, 2 or 4 lanes per bead. SOP_FORCE_CLUSTER=sh keeps only the cluster
    // configurations of 2^sh beads per CTA (sh 5 to 9, when the bucket has one), and
    // SOP_CLUSTER_LANES=l only those of l lanes per bead: tuning overrides that make the form
    // testable at any size (one lane per bead sums in the one-CTA form's order)
    const char *fc = std::getenv("SOP_FORCE_CLUSTER");
    const int force_sh = fc ? std::atoi(fc) : 0;
    const char *fl = std::getenv("SOP_CLUSTER_LANES");
    const int force_ln = fl ? std::atoi(fl) : 0;
    if ((bk.max_n > 256 || force_sh > 0) && !pairs_only) {
        std::vector<BatchedConfig> clusters;
        for (int sh = 5; sh <= 9; ++sh) {
            if (force_sh > 0 ? sh != force_sh : sh < 7) continue;
            for (int ln : {1, 2, 4}) {
                if (force_ln > 0 && ln != force_ln) continue;
                for (int threads : {ln << sh, (ln << sh) / 2}) {
                    BatchedConfig cfg;
                    if (threads < (force_sh > 0 ? 32 : 64) || threads > 1024) continue;
                    if (cluster_config(bk.max_n, bk.row_width, threads, sh, ln, &cfg) && cluster_capacity(cfg) > 0)
                        clusters.push_back(cfg);
                }
            }
        }
        if (force_sh > 0 && !clusters.empty()) cands = clusters;
        else cands.insert(cands.end(), clusters.begin(), clusters.end());
    }
    if (cands.empty()) return fail(c, SOP_ERR_UNSUPPORTED, "no batched configuration fits the bucket");
    // default without a trial: shared-memory rows, the largest CTA at 64 registers (the pair
    // form when it was asked for); else global rows
    bk.cfg = cands[0];
    for (const auto &cf : cands)
        if (!cf.rows_global && cf.min_blocks == 4 && cf.threads >= bk.cfg.threads && cf.pair_form == pairs_only)
            bk.cfg = cf;
    const char *env = std::getenv("SOP_TUNE");
    // the whole bucket up to 64 items per SM: a trial on a few waves can rank configurations
    // whose last waves fill to different fractions otherwise than the full run does
    const int trial_items = std::min<int>(bk.n_items, 152 * 64);
    if (!(env && std::string(env) == "0") && cands.size() > 1) {
        char key[128];
        std::snprintf(key, sizeof key, "batched %d %d %d %d %d", bk.max_n, bk.row_width, bk.pair_pool, trial_items,
                      c->batched_form);
        bool cached = false;
        const char *cache = std::getenv("SOP_TUNE_CACHE");
        if (cache) {
            if (FILE *f = std::fopen(cache, "r")) {
                char line[256];
                while (!cached && std::fgets(line, sizeof line, f)) {
                    int t = 0, bpt = 0, mb = 0, rg = 0, cs = 0, sh = 0, pf = 0, lns = 0;
                    if (std::strncmp(line, key, std::strlen(key)) == 0 &&
                        std::sscanf(line + std::strlen(key), " -> %d %d %d %d %d %d %d %d", &t, &bpt, &mb, &rg, &cs, &sh,
                                    &pf, &lns) == 8) {
                        for (const auto &cf : cands)
                            if (cf.threads == t && cf.beads_per_thread == bpt && cf.min_blocks == mb &&
                                (int)cf.rows_global == rg && cf.cluster == cs && cf.m_shift == sh &&
                                (int)cf.pair_form == pf && cf.lanes == lns) {
                                bk.cfg = cf;
                                cached = true;
                            }
                    }
                }
                std::fclose(f);
            }
        }
        if (!cached) {
            const size_t RN = (size_t)c->R * c->n;
            float4 *sp = nullptr, *sc = nullptr, *ss = nullptr;
            int32_t *sst = nullptr;
            uint16_t *srows = nullptr;
            CUDA_OR_RETURN(c, cudaMalloc(&sp, sizeof(float4) * RN));
            CUDA_OR_RETURN(c, cudaMalloc(&sc, sizeof(float4) * RN));
            CUDA_OR_RETURN(c, cudaMalloc(&ss, sizeof(float4) * RN));
            CUDA_OR_RETURN(c, cudaMalloc(&sst, sizeof(int32_t) * c->R));
            CUDA_OR_RETURN(c, cudaMalloc(&srows, sizeof(uint16_t) * (size_t)trial_items * bk.row_width * bk.max_n));
            cudaEvent_t e0, e1;
            CUDA_OR_RETURN(c, cudaEventCreate(&e0));
            CUDA_OR_RETURN(c, cudaEventCreate(&e1));
            float best_ms = 1e30f, best_cost = 1e30f;
            sop_status status = SOP_OK;
            for (const auto &cf : cands) {
                BatchedArgs a = batched_args(c, bk);
                a.pos = sp;
                a.comp = sc;
                a.snap = ss;
                a.sa.rep_status = sst;
                a.sa.taus = nullptr;   // trials draw Philox noise: the run's Taus state is untouched
                a.sa.vel = nullptr;    // and take the overdamped update: the run's velocities are untouched
                a.obs_every = 0;
                a.n_items = trial_items;
                a.n_steps = 20;
                a.row_global = srows;
                float ms = 0.f;
                for (int rep = 0; rep < 3 && status == SOP_OK; ++rep) {
                    cudaMemcpyAsync(sp, c->d_pos[0], sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                    cudaMemcpyAsync(sc, c->d_comp, sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                    cudaMemcpyAsync(ss, c->d_snap, sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                    cudaMemsetAsync(sst, 0, sizeof(int32_t) * c->R, c->stream);
                    cudaEventRecord(e0, c->stream);
                    cudaError_t e = launch_batched(a, cf, c->stream, nullptr);
                    cudaEventRecord(e1, c->stream);
                    if (e != cudaSuccess) {   // a configuration this device cannot launch: not a candidate
                        cudaGetLastError();
                        ms = 1e30f;
                        break;
                    }
                    const cudaError_t es = cudaEventSynchronize(e1);
                    if (es != cudaSuccess) {
                        status = fail(c, SOP_ERR_CUDA, std::string("autotune trial: ") + cudaGetErrorString(es));
                        break;
                    }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms = rep == 1 ? t : std::min(ms, t);
                }
                if (status != SOP_OK) break;
                // Several buckets run side by side, and the partly filled last wave of one is
                // taken up by the others' CTAs; so beside the fastest alone, keep the one that
                // holds the least SM time (the time scaled by the filled fraction of its waves).
                // tune_joint times the two sets together.
                float cost = ms;
                if (ms < 1e29f) {
                    const int slots = batched_resident_ctas(cf);
                    if (slots > 0) {
                        const double waves = (double)trial_items * std::max(1, cf.cluster) / slots;
                        cost = (float)(ms * waves / std::ceil(waves));
                    }
                }
                if (ms < best_ms) { best_ms = ms; bk.cfg = cf; }
                if (cost < best_cost) { best_cost = cost; bk.alt = cf; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaFree(sp);
            cudaFree(sc);
            cudaFree(ss);
            cudaFree(sst);
            cudaFree(srows);
            if (status != SOP_OK) return status;
            c->st.tune_ms += best_ms;
            bk.key = key;
            bk.span_ms = best_ms;
            bk.timed = true;
        }
    }
    return SOP_OK;
}

bool same_config(const BatchedConfig &x, const BatchedConfig &y) {
    return x.threads == y.threads && x.beads_per_thread == y.beads_per_thread && x.min_blocks == y.min_blocks &&
           x.rows_global == y.rows_global && x.cluster == y.cluster && x.m_shift == y.m_shift &&
           x.pair_form == y.pair_form && x.lanes == y.lanes;
}

// Buckets run side by side, so the configurations fastest on their own need not be the
// fastest together. With several buckets, all of them run at once for 100 steps on scratch
// copies of the state, with every timed bucket on its fastest-alone configuration and then
// on its least-SM-time one, and the faster set is kept. Then the choices are cached
// (SOP_TUNE_CACHE) and the global-memory rows are allocated.
sop_status tune_joint(sop_ctx *c) {
    bool differ = false;
    for (const auto &bk : c->buckets) differ |= bk.timed && !same_config(bk.cfg, bk.alt);
    if (c->buckets.size() > 1 && differ) {
        const size_t RN = (size_t)c->R * c->n;
        std::vector<void *> scratch;
        auto grab = [&](size_t bytes, void **p) {
            const cudaError_t e = cudaMalloc(p, bytes);
            if (e == cudaSuccess) scratch.push_back(*p);
            return e;
        };
        auto release = [&]() {
            for (void *q : scratch) cudaFree(q);
            for (auto &bk : c->buckets) bk.rows = nullptr;
        };
        float4 *sp = nullptr, *sc = nullptr, *ss = nullptr;
        int32_t *sst = nullptr;
        cudaError_t e = grab(sizeof(float4) * RN, (void **)&sp);
        if (e == cudaSuccess) e = grab(sizeof(float4) * RN, (void **)&sc);
        if (e == cudaSuccess) e = grab(sizeof(float4) * RN, (void **)&ss);
        if (e == cudaSuccess) e = grab(sizeof(int32_t) * c->R, (void **)&sst);
        for (auto &bk : c->buckets)
            if (e == cudaSuccess && (bk.cfg.rows_global || (bk.timed && bk.alt.rows_global)))
                e = grab(sizeof(uint16_t) * (size_t)bk.n_items * bk.row_width * bk.max_n, (void **)&bk.rows);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        std::vector<BatchedConfig> fast(c->buckets.size());
        for (size_t k = 0; k < c->buckets.size(); ++k) fast[k] = c->buckets[k].cfg;
        sop_status status = SOP_OK;
        // all buckets at once for 100 steps on the scratch state: the best of two runs after a warm-up
        auto time_all = [&]() {
            float best = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess && status == SOP_OK; ++rep) {
                cudaMemcpyAsync(sp, c->d_pos[0], sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                cudaMemcpyAsync(sc, c->d_comp, sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                cudaMemcpyAsync(ss, c->d_snap, sizeof(float4) * RN, cudaMemcpyDeviceToDevice, c->stream);
                cudaMemsetAsync(sst, 0, sizeof(int32_t) * c->R, c->stream);
                cudaEventRecord(e0, c->stream);
                status = launch_buckets(
                    c,
                    [&](BatchedArgs &a) {
                        a.pos = sp;
                        a.comp = sc;
                        a.snap = ss;
                        a.sa.rep_status = sst;
                        a.sa.taus = nullptr;
                        a.sa.vel = nullptr;
                        a.obs_every = 0;
                        a.n_steps = 100;
                    },
                    nullptr);
                cudaEventRecord(e1, c->stream);
                e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess && status == SOP_OK) {
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) best = std::min(best, ms);
                }
            }
            return best;
        };
        // the two sets; the faster is kept (per-bucket swaps judged on short joint trials
        // did not carry over to full launches)
        std::vector<bool> use_alt(c->buckets.size(), false);
        auto apply = [&]() {
            for (size_t k = 0; k < c->buckets.size(); ++k)
                if (c->buckets[k].timed) c->buckets[k].cfg = use_alt[k] ? c->buckets[k].alt : fast[k];
        };
        float t_fast = 1e30f, t_alt = 1e30f;
        if (e == cudaSuccess) {
            apply();
            t_fast = time_all();
            std::fill(use_alt.begin(), use_alt.end(), true);
            apply();
            t_alt = time_all();
            std::fill(use_alt.begin(), use_alt.end(), t_alt < t_fast);
            apply();
        }
        const float t_best = std::min(t_fast, t_alt);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        release();
        if (status != SOP_OK) return status;
        if (e != cudaSuccess) return fail(c, SOP_ERR_CUDA, std::string("joint tuning: ") + cudaGetErrorString(e));
        c->st.tune_ms += t_best;
    }
    const char *cache = std::getenv("SOP_TUNE_CACHE");
    for (auto &bk : c->buckets) {
        if (cache && bk.timed)
            if (FILE *f = std::fopen(cache, "a")) {
                std::fprintf(f, "%s -> %d %d %d %d %d %d %d %d %.4f\n", bk.key.c_str(), bk.cfg.threads,
                             bk.cfg.beads_per_thread, bk.cfg.min_blocks, (int)bk.cfg.rows_global, bk.cfg.cluster,
                             bk.cfg.m_shift, (int)bk.cfg.pair_form, bk.cfg.lanes, bk.span_ms);
                std::fclose(f);
            }
        if (bk.cfg.rows_global)
            CUDA_OR_RETURN(c, dalloc(c, &bk.rows, (size_t)bk.n_items * bk.row_width * bk.max_n));
    }
    return SOP_OK;
}

// Tables of the pair-based form: the static native half list with each entry's row and
// reverse entry (from the host copy of the native map), the force slots, and the Verlet
// half-list buffers of the run's list (pt) or of the forces-only list (pt2, which shares
// the native lists and the force slots: every slot a gathering reads is rewritten by the
// pair kernel of the same step).
sop_status alloc_pair_tables(sop_ctx *c, DevPairTables &t) {
    if (t.vpair) return SOP_OK;
    const size_t RN = (size_t)c->R * c->n;
    if (!c->pt.fb) {
        std::vector<int32_t> half, owner(c->nat_nnz), mirror(c->nat_nnz);
        const int32_t *col = c->h_nat_col.data();
        for (int i = 0; i < c->n; ++i)
            for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q) {
                const int j = col[q];
                owner[q] = i;
                if (j > i) half.push_back(q);
                const int32_t *b = col + c->h_nat_row[j], *e = col + c->h_nat_row[j + 1];
                const int32_t *it = std::lower_bound(b, e, i);
                if (it == e || *it != i) return fail(c, SOP_ERR_CUDA, "native map is not symmetric");
                mirror[q] = (int32_t)(it - col);
            }
        int32_t *d_half = nullptr, *d_owner = nullptr, *d_mirror = nullptr;
        CUDA_OR_RETURN(c, upload(c, &d_half, half));
        CUDA_OR_RETURN(c, upload(c, &d_owner, owner));
        CUDA_OR_RETURN(c, upload(c, &d_mirror, mirror));
        c->pt.nat_half = d_half;
        c->pt.nat_owner = d_owner;
        c->pt.nat_mirror = d_mirror;
        c->pt.n_nat_half = (int32_t)half.size();
        c->pt.nnz = c->nat_nnz;
        CUDA_OR_RETURN(c, dalloc(c, &c->pt.fb, 2 * RN + 2));
        CUDA_OR_RETURN(c, cudaMemset(c->pt.fb, 0, sizeof(float4) * (2 * RN + 2)));   // absent bonds read 0
        CUDA_OR_RETURN(c, dalloc(c, &c->pt.fn, (size_t)c->R * c->nat_nnz));
        CUDA_OR_RETURN(c, dalloc(c, &c->pt.fv, c->pl_cap));
    }
    if (&t != &c->pt) {
        t.nat_half = c->pt.nat_half;
        t.nat_owner = c->pt.nat_owner;
        t.nat_mirror = c->pt.nat_mirror;
        t.n_nat_half = c->pt.n_nat_half;
        t.nnz = c->pt.nnz;
        t.fb = c->pt.fb;
        t.fn = c->pt.fn;
        t.fv = c->pt.fv;
    }
    // a symmetric list has half as many upper entries as entries
    t.vcap = c->pl_cap / 2 + 1024;
    CUDA_OR_RETURN(c, dalloc(c, &t.vpair, (size_t)t.vcap));
    CUDA_OR_RETURN(c, dalloc(c, &t.vcount, RN));
    CUDA_OR_RETURN(c, dalloc(c, &t.voff, RN + 1));
    CUDA_OR_RETURN(c, dalloc(c, &t.scan_tmp, scan_tmp_elems((int64_t)RN)));
    return SOP_OK;
}

// The streamed schedule's choice between the particle-based gather (Algorithm 2) with 4,
// 8 or 16 lanes per bead and the pair-based form (Algorithms 4, 5): the force evaluations
// are timed on the current positions and list (forces only; the run's state is untouched)
// and the fastest is kept. SOP_TUNE=0 keeps the particle-based form with 8 lanes per bead.
sop_status tune_streamed_form(sop_ctx *c) {
    const char *env = std::getenv("SOP_TUNE");
    if (env && std::string(env) == "0") return SOP_OK;
    sop_status s = alloc_pair_tables(c, c->pt);
    if (s != SOP_OK) return s;
    const SegRange all = full_range(c);
    launch_pair_index(c->sa, c->pl, c->pt, all, c->stream, nullptr);
    cudaEvent_t e0, e1;
    CUDA_OR_RETURN(c, cudaEventCreate(&e0));
    CUDA_OR_RETURN(c, cudaEventCreate(&e1));
    // the particle-based gather with 4, 8, 16 and 32 lanes per bead, and the pair-based form
    constexpr int kGather = 4;
    const int gather_lanes[kGather] = {8, 4, 16, 32};
    float ms[kGather + 1] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int reps = 20;
    for (int form = 0; form <= kGather; ++form) {
        // the gather kernels index their threads (beads x lanes) with 32-bit integers
        if (form < kGather && (int64_t)c->R * c->n * gather_lanes[form] > ((int64_t)1 << 31)) {
            ms[form] = 1e30f;
            continue;
        }
        for (int rep = 0; rep <= reps; ++rep) {
            if (rep == 1) cudaEventRecord(e0, c->stream);   // the first launch is a warm-up
            if (form < kGather)
                launch_forces(c->sa, c->pl, c->d_pos[c->cur], c->d_force, all.b_lo, all.b_hi, c->step, c->stream,
                              nullptr, gather_lanes[form]);
            else
                launch_pairs_forces(c->sa, c->pl, c->pt, c->d_pos[c->cur], c->d_force, all, c->step, c->stream,
                                    nullptr);
        }
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(c, SOP_ERR_CUDA, std::string("streamed form trial: ") + cudaGetErrorString(e));
        }
        cudaEventElapsedTime(&ms[form], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = 0;
    for (int form = 1; form < kGather; ++form)
        if (ms[form] < ms[best]) best = form;
    c->pairs = ms[kGather] < ms[best];
    c->lanes = c->pairs ? 8 : gather_lanes[best];   // the pair-based trial gathers with 8
    c->st.tune_ms = (c->pairs ? ms[kGather] : ms[best]) / reps;
    return SOP_OK;
}

// Largest Verlet row of replica 0 after the initial build.
sop_status max_row(sop_ctx *c, int *out) {
    std::vector<int32_t> len(c->n);
    CUDA_OR_RETURN(c, cudaMemcpy(len.data(), c->pl.len, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost));
    int m = 0;
    int64_t tot = 0;
    for (int v : len) { m = std::max(m, v); tot += v; }
    c->st.pairlist_entries = tot;
    *out = m;
    return SOP_OK;
}

// Cross-links: drop the linked pairs from the native map (a covalent link is not a
// non-covalent native contact) and upload the links as a CSR over beads, both directions,
// ascending, with their FP64 native lengths ((dx*dx + dy*dy) + dz*dz, rounded square root)
// and those rounded to FP32.
sop_status apply_xlinks(sop_ctx *c, const double *xyz) {
    const int n = c->n;
    auto linked = [c](int32_t i, int32_t j) {
        return std::binary_search(c->xlinks.begin(), c->xlinks.end(), std::make_pair(std::min(i, j), std::max(i, j)));
    };
    std::vector<int32_t> row(n + 1, 0), col;
    std::vector<double> r0;
    col.reserve(c->h_nat_col.size());
    r0.reserve(c->h_nat_col.size());
    for (int i = 0; i < n; ++i) {
        for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q)
            if (!linked(i, c->h_nat_col[q])) {
                col.push_back(c->h_nat_col[q]);
                r0.push_back(c->h_nat_r0[q]);
            }
        row[i + 1] = (int32_t)col.size();
    }
    if ((int64_t)col.size() != c->nat_nnz) {   // some links were native contacts: new map
        std::vector<float> r0sq(r0.size());
        for (size_t q = 0; q < r0.size(); ++q) r0sq[q] = (float)(r0[q] * r0[q]);
        c->h_nat_row = row;
        c->h_nat_col = col;
        c->h_nat_r0 = r0;
        c->nat_nnz = (int64_t)col.size();
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_nat_row, row.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
        if (c->nat_nnz) {
            CUDA_OR_RETURN(c, cudaMemcpy(c->d_nat_col, col.data(), sizeof(int32_t) * c->nat_nnz, cudaMemcpyHostToDevice));
            CUDA_OR_RETURN(c, cudaMemcpy(c->d_nat_r0, r0.data(), sizeof(double) * c->nat_nnz, cudaMemcpyHostToDevice));
            CUDA_OR_RETURN(c, cudaMemcpy(c->d_nat_r0sq, r0sq.data(), sizeof(float) * c->nat_nnz, cudaMemcpyHostToDevice));
        }
    }
    std::vector<std::vector<int32_t>> adj(n);
    for (const auto &e : c->xlinks) {
        adj[e.first].push_back(e.second);
        adj[e.second].push_back(e.first);
    }
    std::vector<int32_t> xrow(n + 1, 0), xcol;
    std::vector<double> xr0;
    for (int i = 0; i < n; ++i) {
        std::sort(adj[i].begin(), adj[i].end());
        for (int32_t j : adj[i]) {
            const double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1];
            const double dz = xyz[3 * i + 2] - xyz[3 * j + 2];
            xcol.push_back(j);
            xr0.push_back(std::sqrt((dx * dx + dy * dy) + dz * dz));
        }
        xrow[i + 1] = (int32_t)xcol.size();
    }
    std::vector<float> xr0f(xr0.begin(), xr0.end());
    int32_t *d_row = nullptr, *d_col = nullptr;
    float *d_r0 = nullptr;
    double *d_r0d = nullptr;
    CUDA_OR_RETURN(c, upload(c, &d_row, xrow));
    CUDA_OR_RETURN(c, upload(c, &d_col, xcol));
    CUDA_OR_RETURN(c, upload(c, &d_r0, xr0f));
    CUDA_OR_RETURN(c, upload(c, &d_r0d, xr0));
    c->d_xb_row = d_row;
    c->d_xb_col = d_col;
    c->d_xb_r0 = d_r0;
    c->d_xb_r0d = d_r0d;
    return SOP_OK;
}

sop_status create_impl(sop_ctx *c, const sop_topology *topo, const double *xyz, const sop_params *p) {
    sop_status s = validate_params(p);
    if (s != SOP_OK) return s;
    if (!xyz) return fail(nullptr, SOP_ERR_INVALID_ARG, "native_xyz is NULL");
    s = build_host_topology(c, topo);
    if (s != SOP_OK) return s;
    for (int64_t k = 0; k < 3 * (int64_t)c->n; ++k)
        if (!std::isfinite(xyz[k])) return fail(nullptr, SOP_ERR_INVALID_ARG, "native_xyz holds a non-finite value");
    c->prm = *p;
    c->R = p->n_replicas;
    if ((int64_t)c->R * c->n > (1LL << 28)) return fail(nullptr, SOP_ERR_INVALID_ARG, "n_replicas * n_beads too large");
    c->n_seg = c->R * c->n_sys;
    if (p->obs_capacity == 0) c->prm.obs_capacity = 4096;
    c->ppb = p->pairs_per_bead > 0 ? p->pairs_per_bead : 64;
    CUDA_OR_RETURN(c, cudaGetDevice(&c->device));
    if (p->cuda_stream) {
        c->stream = static_cast<cudaStream_t>(p->cuda_stream);
    } else {
        CUDA_OR_RETURN(c, cudaStreamCreate(&c->stream));
        c->own_stream = true;
    }
    const int n = c->n, R = c->R;
    // ---- topology on the device
    CUDA_OR_RETURN(c, upload(c, &c->d_chain, c->chain_of));
    CUDA_OR_RETURN(c, upload(c, &c->d_sys, c->sys_of));
    CUDA_OR_RETURN(c, upload(c, &c->d_sys_lo, c->sys_lo));
    CUDA_OR_RETURN(c, upload(c, &c->d_sys_ree_last, c->sys_ree_last));
    CUDA_OR_RETURN(c, upload(c, &c->d_flags, c->flags));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_bond_r0, n));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_bond_r0d, n));
    double *d_xyz = nullptr;
    CUDA_OR_RETURN(c, dalloc(c, &d_xyz, 3 * (size_t)n));
    CUDA_OR_RETURN(c, cudaMemcpy(d_xyz, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    launch_setup_bonds(d_xyz, c->d_chain, c->d_bond_r0, c->d_bond_r0d, n, c->stream);
    CUDA_OR_RETURN(c, cudaGetLastError());
    // ---- native map: count, host prefix sum, fill (FP64 decisions on the GPU)
    int32_t *d_cnt = nullptr;
    CUDA_OR_RETURN(c, dalloc(c, &d_cnt, n));
    launch_native_count(d_xyz, c->d_chain, c->d_sys, c->d_sys_lo, n, p->native_cut, d_cnt, c->stream);
    std::vector<int32_t> cnt(n);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    c->h_nat_row.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) c->h_nat_row[i + 1] = c->h_nat_row[i] + cnt[i];
    c->nat_nnz = c->h_nat_row[n];
    CUDA_OR_RETURN(c, upload(c, &c->d_nat_row, c->h_nat_row));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_nat_col, c->nat_nnz));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_nat_r0, c->nat_nnz));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_nat_r0sq, c->nat_nnz));
    launch_native_fill(d_xyz, c->d_chain, c->d_sys, c->d_sys_lo, n, p->native_cut, c->d_nat_row, c->d_nat_col,
                       c->d_nat_r0, c->d_nat_r0sq, c->stream);
    CUDA_OR_RETURN(c, cudaGetLastError());
    c->h_nat_col.resize(c->nat_nnz);
    c->h_nat_r0.resize(c->nat_nnz);
    if (c->nat_nnz) {
        CUDA_OR_RETURN(c, cudaMemcpyAsync(c->h_nat_col.data(), c->d_nat_col, sizeof(int32_t) * c->nat_nnz,
                                          cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaMemcpyAsync(c->h_nat_r0.data(), c->d_nat_r0, sizeof(double) * c->nat_nnz,
                                          cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    if (!c->xlinks.empty()) {
        s = apply_xlinks(c, xyz);
        if (s != SOP_OK) return s;
    }
    c->st.native_entries = c->nat_nnz / 2;
    {   // packed (partner, r0^2) entries for the streamed gather
        std::vector<float> r0sq(c->nat_nnz);
        if (c->nat_nnz)
            CUDA_OR_RETURN(c, cudaMemcpy(r0sq.data(), c->d_nat_r0sq, sizeof(float) * c->nat_nnz, cudaMemcpyDeviceToHost));
        std::vector<uint2> ent(std::max<int64_t>(1, c->nat_nnz), make_uint2(0u, 0u));
        for (int64_t q = 0; q < c->nat_nnz; ++q) {
            uint32_t bits;
            std::memcpy(&bits, &r0sq[q], sizeof bits);
            ent[q] = make_uint2((uint32_t)c->h_nat_col[q], bits);
        }
        CUDA_OR_RETURN(c, upload(c, &c->d_nat_ent, ent));
    }
    std::vector<int32_t> sys_np(c->n_sys, 0);
    for (int i = 0; i < n; ++i)
        for (int q = c->h_nat_row[i]; q < c->h_nat_row[i + 1]; ++q)
            if (c->h_nat_col[q] > i) sys_np[c->sys_of[i]]++;
    CUDA_OR_RETURN(c, upload(c, &c->d_sys_nat_pairs, sys_np));
    // ---- state: every replica starts at the native coordinates (FP32)
    std::vector<float4> p4((size_t)R * n);
    for (int i = 0; i < n; ++i) {
        const float4 v = make_float4((float)xyz[3 * i], (float)xyz[3 * i + 1], (float)xyz[3 * i + 2], 0.f);
        for (int r = 0; r < R; ++r) p4[(size_t)r * n + i] = v;
    }
    for (int b = 0; b < 2; ++b) CUDA_OR_RETURN(c, dalloc(c, &c->d_pos[b], (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_comp, (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_snap, (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_force, (size_t)R * n));
    CUDA_OR_RETURN(c, cudaMemcpy(c->d_pos[0], p4.data(), sizeof(float4) * p4.size(), cudaMemcpyHostToDevice));
    CUDA_OR_RETURN(c, cudaMemcpy(c->d_pos[1], p4.data(), sizeof(float4) * p4.size(), cudaMemcpyHostToDevice));
    CUDA_OR_RETURN(c, cudaMemset(c->d_comp, 0, sizeof(float4) * p4.size()));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_step, 1));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_events, 1));
    CUDA_OR_RETURN(c, cudaMemset(c->d_step, 0, sizeof(int64_t)));
    CUDA_OR_RETURN(c, cudaMemset(c->d_events, 0, sizeof(int64_t)));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_rep_status, R));
    CUDA_OR_RETURN(c, cudaMemset(c->d_rep_status, 0, sizeof(int32_t) * R));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_halt, 1));
    CUDA_OR_RETURN(c, cudaMemset(c->d_halt, 0, sizeof(int32_t)));
    CUDA_OR_RETURN(c, dalloc(c, &c->d_energy, 1));
    CUDA_OR_RETURN(c, cudaHostAlloc((void **)&c->h_abort, sizeof(int32_t), cudaHostAllocMapped));
    *c->h_abort = 0;
    CUDA_OR_RETURN(c, cudaHostGetDevicePointer((void **)&c->d_abort, c->h_abort, 0));
    // ---- segments: (replica, system), cells and Verlet-list ranges
    c->h_seg_bead_lo.resize(c->n_seg + 1);
    c->h_seg_cell_base.resize(c->n_seg + 1);
    std::vector<int64_t> pl_base(c->n_seg), pl_end(c->n_seg);
    int64_t cells = 0, cols = 0;
    for (int r = 0; r < R; ++r)
        for (int s2 = 0; s2 < c->n_sys; ++s2) {
            const int g = r * c->n_sys + s2;
            const int ng = c->sys_lo[s2 + 1] - c->sys_lo[s2];
            c->h_seg_bead_lo[g] = r * n + c->sys_lo[s2];
            c->h_seg_cell_base[g] = (int32_t)cells;
            cells += 2 * (int64_t)ng + 8;
            pl_base[g] = cols;
            cols += (int64_t)c->ppb * ng;
            pl_end[g] = cols;
        }
    c->h_seg_bead_lo[c->n_seg] = R * n;
    if (cells > INT32_MAX || cols > INT32_MAX) return fail(c, SOP_ERR_UNSUPPORTED, "too many cells or list entries");
    c->h_seg_cell_base[c->n_seg] = (int32_t)cells;
    int32_t *d_sbl = nullptr, *d_scb = nullptr;
    CUDA_OR_RETURN(c, upload(c, &d_sbl, c->h_seg_bead_lo));
    CUDA_OR_RETURN(c, upload(c, &d_scb, c->h_seg_cell_base));
    c->cells.n_seg = c->n_seg;
    c->cells.seg_bead_lo = d_sbl;
    c->cells.seg_cell_base = d_scb;
    c->cells.n_cells = cells;
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.seg_lo, c->n_seg));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.seg_dims, c->n_seg));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.cell_of, (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.cell_cnt, cells));
    CUDA_OR_RETURN(c, cudaMemset(c->cells.cell_cnt, 0, sizeof(int32_t) * cells));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.cell_start, cells + 1));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.sorted, (size_t)R * n));   // float4 per bead
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.scan_tmp, scan_tmp_elems(cells)));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.seg_box, 8 * (size_t)c->n_seg));
    launch_seg_box_init(c->cells.seg_box, c->n_seg, c->stream);
    int64_t *d_plb = nullptr, *d_ple = nullptr;
    CUDA_OR_RETURN(c, upload(c, &d_plb, pl_base));
    CUDA_OR_RETURN(c, upload(c, &d_ple, pl_end));
    c->pl_cap = cols;
    for (DevPairList *L : {&c->pl, &c->pl2}) {
        L->seg_base = d_plb;
        L->seg_end = d_ple;
        L->cap = cols;
    }
    CUDA_OR_RETURN(c, dalloc(c, &c->pl.start, (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->pl.len, (size_t)R * n));
    CUDA_OR_RETURN(c, dalloc(c, &c->pl.col, cols));
    CUDA_OR_RETURN(c, dalloc(c, &c->pl.cursor, c->n_seg));
    // the all-pairs build of small segments expects each cursor at its first column
    std::vector<int32_t> cur0(c->n_seg);
    for (int g = 0; g < c->n_seg; ++g) cur0[g] = (int32_t)pl_base[g];
    CUDA_OR_RETURN(c, cudaMemcpy(c->pl.cursor, cur0.data(), sizeof(int32_t) * c->n_seg, cudaMemcpyHostToDevice));
    c->h_brute_cta_lo.assign(c->n_seg + 1, 0);
    for (int g = 0; g < c->n_seg; ++g) {
        const int ng = c->h_seg_bead_lo[g + 1] - c->h_seg_bead_lo[g];
        c->h_brute_cta_lo[g + 1] = c->h_brute_cta_lo[g] + (ng + kBruteSliceBeads - 1) / kBruteSliceBeads;
    }
    {
        int32_t *d_bcl = nullptr;
        CUDA_OR_RETURN(c, upload(c, &d_bcl, c->h_brute_cta_lo));
        c->cells.brute_cta_lo = d_bcl;
    }
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.brute_done, c->n_seg));
    CUDA_OR_RETURN(c, cudaMemset(c->cells.brute_done, 0, sizeof(int32_t) * c->n_seg));
    CUDA_OR_RETURN(c, dalloc(c, &c->cells.brute_used, c->n_seg));
    CUDA_OR_RETURN(c, cudaMemset(c->cells.brute_used, 0, sizeof(int32_t) * c->n_seg));
    // ---- observables: chunks of at most kObsChunk beads per segment
    std::vector<int32_t> ch_seg, ch_lo, ch_hi;
    c->h_seg_chunk_lo.assign(c->n_seg + 1, 0);
    for (int g = 0; g < c->n_seg; ++g) {
        c->h_seg_chunk_lo[g] = (int32_t)ch_seg.size();
        for (int b = c->h_seg_bead_lo[g]; b < c->h_seg_bead_lo[g + 1]; b += kObsChunk) {
            ch_seg.push_back(g);
            ch_lo.push_back(b);
            ch_hi.push_back(std::min(b + kObsChunk, c->h_seg_bead_lo[g + 1]));
        }
    }
    c->h_seg_chunk_lo[c->n_seg] = (int32_t)ch_seg.size();
    int32_t *d_cs = nullptr, *d_cl = nullptr, *d_chh = nullptr, *d_scl = nullptr;
    CUDA_OR_RETURN(c, upload(c, &d_cs, ch_seg));
    CUDA_OR_RETURN(c, upload(c, &d_cl, ch_lo));
    CUDA_OR_RETURN(c, upload(c, &d_chh, ch_hi));
    CUDA_OR_RETURN(c, upload(c, &d_scl, c->h_seg_chunk_lo));
    c->obs.n_chunks = (int32_t)ch_seg.size();
    c->obs.chunk_seg = d_cs;
    c->obs.chunk_lo = d_cl;
    c->obs.chunk_hi = d_chh;
    c->obs.seg_chunk_lo = d_scl;
    c->obs.max_seg_chunks = 0;
    for (int g = 0; g < c->n_seg; ++g)
        c->obs.max_seg_chunks = std::max(c->obs.max_seg_chunks, c->h_seg_chunk_lo[g + 1] - c->h_seg_chunk_lo[g]);
    CUDA_OR_RETURN(c, dalloc(c, &c->obs.partial, 8 * (size_t)c->obs.n_chunks));
    c->obs.cap = std::max<int64_t>(c->prm.obs_capacity, c->n_seg);
    CUDA_OR_RETURN(c, dalloc(c, &c->obs.ring, c->obs.cap));
    c->obs.events = c->d_events;
    c->obs.obs_every = c->prm.obs_every;
    c->obs.q_every = c->prm.obs_every_q;
    // ---- externals (none yet)
    c->pull_of_sys.assign(c->n_sys, -1);
    CUDA_OR_RETURN(c, upload(c, &c->d_pull_of_sys, c->pull_of_sys));
    s = alloc_pull_arrays(c, 0);
    if (s != SOP_OK) return s;
    // ---- kernel arguments
    StepArgs &a = c->sa;
    a.topo.n = n;
    a.topo.n_sys = c->n_sys;
    a.topo.chain = c->d_chain;
    a.topo.sys = c->d_sys;
    a.topo.flags = c->d_flags;
    a.topo.bond_r0 = c->d_bond_r0;
    a.topo.bond_r0d = c->d_bond_r0d;
    a.topo.nat_row = c->d_nat_row;
    a.topo.nat_col = c->d_nat_col;
    a.topo.nat_r0sq = c->d_nat_r0sq;
    a.topo.nat_r0 = c->d_nat_r0;
    a.topo.nat_ent = c->d_nat_ent;
    a.topo.sys_lo = c->d_sys_lo;
    a.topo.sys_ree_last = c->d_sys_ree_last;
    a.topo.sys_nat_pairs = c->d_sys_nat_pairs;
    a.topo.xb_row = c->d_xb_row;
    a.topo.xb_col = c->d_xb_col;
    a.topo.xb_r0 = c->d_xb_r0;
    a.topo.xb_r0d = c->d_xb_r0d;
    const double kT = kBoltzmannKcal * p->T;
    a.fp.k_fene = (float)p->k_fene;
    a.fp.inv_R02 = (float)(1.0 / (p->R0 * p->R0));
    a.fp.eps12_h = (float)(12.0 * p->eps_h);
    a.fp.eps6_l = (float)(6.0 * p->eps_l);
    a.fp.rep_k = (float)(6.0 * p->eps_l * std::pow(p->sigma, 6));
    a.fp.sigma2 = (float)(p->sigma * p->sigma);
    a.fp.mob = (float)(p->dt / p->zeta);
    a.fp.amp = (float)std::sqrt(2.0 * kT * p->dt / p->zeta);
    a.cut2_d = p->pair_cut * p->pair_cut;
    a.cut2_f = (float)a.cut2_d;
    a.k_fene = p->k_fene;
    a.R0 = p->R0;
    a.eps_h = p->eps_h;
    a.eps_l = p->eps_l;
    a.sigma = p->sigma;
    a.seed = p->seed;
    a.R = R;
    a.d_step = c->d_step;
    a.rep_status = c->d_rep_status;
    a.halt = c->d_halt;
    if (p->rng == SOP_RNG_HYBRID_TAUS) {
        std::vector<uint4> st((size_t)R * n);
        for (int r = 0; r < R; ++r)
            for (int i = 0; i < n; ++i) {
                uint32_t w[4];
                taus_seed(p->seed, r, i, w);
                st[(size_t)r * n + i] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        CUDA_OR_RETURN(c, upload(c, &c->d_taus, st));
    }
    a.taus = c->d_taus;
    if (p->integrator == SOP_INTEGRATOR_BAOAB) {
        CUDA_OR_RETURN(c, dalloc(c, &c->d_vel, (size_t)R * n));
        CUDA_OR_RETURN(c, cudaMemset(c->d_vel, 0, sizeof(float4) * (size_t)R * n));
        const double c1 = std::exp(-p->zeta * p->dt / p->mass);
        a.h_m = (float)(p->dt / p->mass);
        a.half_h = (float)(0.5 * p->dt);
        a.c1 = (float)c1;
        a.c2 = (float)std::sqrt(kT * (1.0 - c1 * c1) / p->mass);
    }
    a.vel = c->d_vel;
    sync_external(c);
    // ---- the first Verlet list (streamed builder; also fills the snapshot)
    s = rebuild_streamed(c);
    if (s != SOP_OK) return s;
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    int mrow = 0;
    s = max_row(c, &mrow);
    if (s != SOP_OK) return s;
    // ---- schedule: batched for small systems or many of them, streamed for a few large ones
    int sched = p->schedule;
    if (sched == SOP_SCHED_BATCHED_PAIRS) {
        sched = SOP_SCHED_BATCHED;
        c->batched_form = 2;
    } else if (sched == SOP_SCHED_BATCHED) {
        c->batched_form = 1;
    }
    const bool batched_ok = c->max_sys <= kBatchedMaxBeads;
    if (sched == SOP_SCHED_AUTO) {
        const int64_t items = (int64_t)c->R * c->n_sys;
        sched = c->max_sys <= kBatchedAutoBeads && (c->max_sys <= 512 || items >= 152) && c->xlinks.empty()
                    ? SOP_SCHED_BATCHED
                    : SOP_SCHED_STREAMED;
    }
    if (sched == SOP_SCHED_BATCHED && !c->xlinks.empty())
        return fail(c, SOP_ERR_UNSUPPORTED, "the batched schedules take no extra bonds (use a streamed one)");
    if (sched == SOP_SCHED_BATCHED && !batched_ok)
        return fail(c, SOP_ERR_UNSUPPORTED, "the batched schedule takes systems of at most 4096 beads");
    if (sched == SOP_SCHED_PAIRS) {
        s = alloc_pair_tables(c, c->pt);
        if (s != SOP_OK) return s;
        c->pairs = true;
        launch_pair_index(c->sa, c->pl, c->pt, full_range(c), c->stream, &c->st.kernel_launches);
    } else if (sched == SOP_SCHED_STREAMED && p->schedule == SOP_SCHED_AUTO) {
        s = tune_streamed_form(c);
        if (s != SOP_OK) return s;
        if (c->pairs) sched = SOP_SCHED_PAIRS;
    }
    // SOP_COOP=1 runs each K-step chunk of a streamed launch of at most this many beads as one
    // cooperative launch with a grid barrier between steps. Off by default: on GB300 it was
    // slower than the graph of per-step launches at every size from 512 to 32,768 beads.
    if ((sched == SOP_SCHED_STREAMED) && (int64_t)c->R * c->n <= 38912) {
        const char *env = std::getenv("SOP_COOP");
        if (env && std::string(env) == "1") {
            CUDA_OR_RETURN(c, dalloc(c, &c->d_bar, 2));
            CUDA_OR_RETURN(c, cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned)));
            c->coop = true;
        }
    }
    c->schedule = sched;
    c->st.schedule = sched;
    c->st.block_threads = 256;
    c->st.pairs_per_bead = c->ppb;
    if (sched == SOP_SCHED_BATCHED) {
        // the first list of replica 0 sizes the rows of every bucket
        std::vector<int32_t> first_start(n), first_len(n), first_col;
        CUDA_OR_RETURN(c, cudaMemcpy(first_start.data(), c->pl.start, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        CUDA_OR_RETURN(c, cudaMemcpy(first_len.data(), c->pl.len, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        int32_t clo = INT32_MAX, chi = 0;
        for (int i = 0; i < n; ++i)
            if (first_len[i] > 0) { clo = std::min(clo, first_start[i]); chi = std::max(chi, first_start[i] + first_len[i]); }
        if (chi > clo) {
            first_col.resize(chi - clo);
            CUDA_OR_RETURN(c, cudaMemcpy(first_col.data(), c->pl.col + clo, sizeof(int32_t) * (chi - clo),
                                         cudaMemcpyDeviceToHost));
            for (int i = 0; i < n; ++i) first_start[i] = first_len[i] > 0 ? first_start[i] - clo : 0;
        }
        s = build_batched_tables(c);
        if (s != SOP_OK) return s;
        s = build_buckets(c, first_start, first_len, first_col);
        if (s != SOP_OK) return s;
        size_t main_bucket = 0;
        for (size_t k = 0; k < c->buckets.size(); ++k) {
            s = tune_bucket(c, c->buckets[k]);
            if (s != SOP_OK) return s;
            if (c->buckets[k].n_items > c->buckets[main_bucket].n_items) main_bucket = k;
        }
        s = tune_joint(c);
        if (s != SOP_OK) return s;
        const BatchedConfig &cfg = c->buckets[main_bucket].cfg;
        c->st.block_threads = cfg.threads;
        c->st.pairs_per_bead = c->batched_cap;
        c->st.beads_per_thread = cfg.beads_per_thread;
        c->st.min_blocks = cfg.rows_global ? 0 : cfg.min_blocks;
        c->st.buckets = (int32_t)c->buckets.size();
        c->st.cluster_size = cfg.cluster;
        c->st.cluster_buckets = 0;
        c->st.pair_buckets = 0;
        for (const auto &bk : c->buckets) {
            c->st.cluster_buckets += bk.cfg.cluster > 0 ? 1 : 0;
            c->st.pair_buckets += bk.cfg.pair_form ? 1 : 0;
        }
    }
    (void)mrow;
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

void free_all(sop_ctx *c) {
    destroy_graphs(c);
    for (auto &bk : c->buckets) {
        if (bk.stream) cudaStreamDestroy(bk.stream);
        if (bk.done) cudaEventDestroy(bk.done);
        bk.stream = nullptr;
        bk.done = nullptr;
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    c->fork_ev = nullptr;
    for (auto &e : c->chunk_ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (void *q : c->allocs) cudaFree(q);
    c->allocs.clear();
    if (c->h_abort) cudaFreeHost(c->h_abort);
    c->h_abort = nullptr;
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->stream = nullptr;
}

// Canonical CSR (rows ascending, both directions) from per-bead rows.
void to_csr(int n, const std::vector<int32_t> &start, const std::vector<int32_t> &len, const std::vector<int32_t> &col,
            int32_t base_index, std::vector<int32_t> &row_ptr, std::vector<int32_t> &out) {
    row_ptr.assign(n + 1, 0);
    out.clear();
    for (int i = 0; i < n; ++i) {
        if (len[i] <= 0 || start[i] < 0 || (size_t)start[i] + (size_t)len[i] > col.size()) {
            row_ptr[i + 1] = (int32_t)out.size();
            continue;
        }
        std::vector<int32_t> row(col.begin() + start[i], col.begin() + start[i] + len[i]);
        for (auto &v : row) v -= base_index;
        std::sort(row.begin(), row.end());
        out.insert(out.end(), row.begin(), row.end());
        row_ptr[i + 1] = (int32_t)out.size();
    }
}

}  // namespace

// =====================================================================================
// Entry points
// =====================================================================================
extern "C" {

sop_status sop_create(const sop_topology *topo, const double *native_xyz, const sop_params *params, sop_ctx **out) {
    if (!out) return fail(nullptr, SOP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sop_ctx *c = new (std::nothrow) sop_ctx();
    if (!c) return fail(nullptr, SOP_ERR_OOM, "host allocation failed");
    sop_status s;
    try {
        s = create_impl(c, topo, native_xyz, params);
    } catch (const std::exception &e) {
        s = fail(c, SOP_ERR_OOM, std::string("host exception: ") + e.what());
    }
    if (s != SOP_OK) {
        if (!c->err.empty()) g_create_error = c->err;
        free_all(c);
        delete c;
        return s;
    }
    *out = c;
    return SOP_OK;
}

sop_status sop_step(sop_ctx *c, int64_t n_steps) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (n_steps < 0) return fail(c, SOP_ERR_INVALID_ARG, "n_steps < 0");
    try {
        *c->h_abort = 0;
        sop_status s = SOP_OK;
        if (n_steps > 0) {
            switch (c->schedule) {
            case SOP_SCHED_BATCHED: s = step_batched(c, n_steps); break;
            case SOP_SCHED_PLAIN: s = step_plain(c, n_steps); break;
            case SOP_SCHED_PAIRS: s = step_streamed(c, n_steps); break;
            default: s = step_streamed(c, n_steps); break;
            }
        }
        if (s != SOP_OK) return s;
        c->st.steps = c->step;
        const bool aborted = *(volatile int32_t *)c->h_abort != 0;
        return read_status(c, aborted);
    } catch (const std::exception &e) {
        return fail(c, SOP_ERR_OOM, std::string("host exception: ") + e.what());
    }
}

sop_status sop_forces(sop_ctx *c, int32_t replica, double *out_f, double *out_energy) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (replica < 0 || replica >= c->R) return fail(c, SOP_ERR_INVALID_ARG, "replica out of range");
    try {
        // a list for these positions, in separate buffers so the run's list is untouched
        if (!c->pl2.col) {
            CUDA_OR_RETURN(c, dalloc(c, &c->pl2.start, (size_t)c->R * c->n));
            CUDA_OR_RETURN(c, dalloc(c, &c->pl2.len, (size_t)c->R * c->n));
            CUDA_OR_RETURN(c, dalloc(c, &c->pl2.col, c->pl_cap));
            CUDA_OR_RETURN(c, dalloc(c, &c->pl2.cursor, c->n_seg));
            CUDA_OR_RETURN(c, cudaMemcpy(c->pl2.cursor, c->pl.cursor, sizeof(int32_t) * c->n_seg,
                                         cudaMemcpyDeviceToDevice));
            // rows of replicas not rebuilt here must read as empty, never as garbage
            CUDA_OR_RETURN(c, cudaMemset(c->pl2.start, 0, sizeof(int32_t) * (size_t)c->R * c->n));
            CUDA_OR_RETURN(c, cudaMemset(c->pl2.len, 0, sizeof(int32_t) * (size_t)c->R * c->n));
        }
        const int g_lo = replica * c->n_sys, g_hi = g_lo + c->n_sys;
        const SegRange rg = seg_range(c, g_lo, g_hi);
        launch_rebuild(c->sa, c->cells, c->pl2, c->d_pos[c->cur], nullptr, rg, c->stream, &c->st.kernel_launches);
        if (c->schedule == SOP_SCHED_BATCHED) {
            // forces mode of the batched kernel for every item (cheap next to the transfer)
            float4 *pos = c->d_pos[c->cur], *force = c->d_force;
            sop_status sb = launch_buckets(c, [pos, force](BatchedArgs &a) {
                a.pos = pos;
                a.n_steps = 0;
                a.force_out = force;
            }, &c->st.kernel_launches);
            if (sb != SOP_OK) return sb;
        } else if (c->pairs) {
            sop_status sp = alloc_pair_tables(c, c->pt2);
            if (sp != SOP_OK) return sp;
            launch_pair_index(c->sa, c->pl2, c->pt2, rg, c->stream, &c->st.kernel_launches);
            launch_pairs_forces(c->sa, c->pl2, c->pt2, c->d_pos[c->cur], c->d_force, rg, c->step, c->stream,
                                &c->st.kernel_launches);
        } else {
            int64_t step_now = c->step;
            launch_forces(c->sa, c->pl2, c->d_pos[c->cur], c->d_force, rg.b_lo, rg.b_hi, step_now, c->stream,
                          &c->st.kernel_launches);
        }
        // energy: the observable partials of this replica's segments at the current step
        launch_energy(c->sa, c->pl2, c->obs, c->d_pos[c->cur], g_lo, g_hi, c->h_seg_chunk_lo[g_lo],
                      c->h_seg_chunk_lo[g_hi], c->d_energy, c->stream,
                      &c->st.kernel_launches);
        CUDA_OR_RETURN(c, cudaGetLastError());
        std::vector<float4> f(c->n);
        CUDA_OR_RETURN(c, cudaMemcpyAsync(f.data(), c->d_force + (size_t)replica * c->n, sizeof(float4) * c->n,
                                          cudaMemcpyDeviceToHost, c->stream));
        double e = 0.0;
        CUDA_OR_RETURN(c, cudaMemcpyAsync(&e, c->d_energy, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
        bool bad = false;
        if (out_f)
            for (int i = 0; i < c->n; ++i) {
                out_f[3 * i] = f[i].x;
                out_f[3 * i + 1] = f[i].y;
                out_f[3 * i + 2] = f[i].z;
                bad |= f[i].w != 0.f;
            }
        if (out_energy) *out_energy = e;
        if (bad) return fail(c, SOP_ERR_FENE_BREAK, "a bond is broken or a bead is inside the indenter");
        return SOP_OK;
    } catch (const std::exception &e) {
        return fail(c, SOP_ERR_OOM, std::string("host exception: ") + e.what());
    }
}

sop_status sop_pairlist_rebuild(sop_ctx *c) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    sop_status s = rebuild_streamed(c);
    if (s != SOP_OK) return s;
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

sop_status sop_pull(sop_ctx *c, int32_t n, const sop_pull_params *pulls) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !pulls)) return fail(c, SOP_ERR_INVALID_ARG, "pulls");
    try {
        std::vector<int> seen(c->n_sys, 0);
        for (int k = 0; k < n; ++k) {
            const sop_pull_params &q = pulls[k];
            if (q.system < 0 || q.system >= c->n_sys || seen[q.system]++)
                return fail(c, SOP_ERR_INVALID_ARG, "pull: system out of range or repeated");
            const int lo = c->sys_lo[q.system], hi = c->sys_lo[q.system + 1];
            if (q.anchor < lo || q.anchor >= hi || q.pulled < lo || q.pulled >= hi || q.anchor == q.pulled)
                return fail(c, SOP_ERR_INVALID_ARG, "pull: anchor and pulled must be distinct beads of the system");
            if (!std::isfinite(q.k_s) || q.k_s < 0 || !std::isfinite(q.v))
                return fail(c, SOP_ERR_INVALID_ARG, "pull: k_s >= 0 and finite v required");
        }
        std::vector<float4> h;
        sop_status s = positions_f4(c, h);
        if (s != SOP_OK) return s;
        // every new record is built (and checked) before the context changes
        PullSet ps;
        ps.resize(n, c->R);
        for (int k = 0; k < n; ++k) {
            const sop_pull_params &q = pulls[k];
            ps.sys[k] = q.system;
            ps.anchor[k] = q.anchor;
            ps.bead[k] = q.pulled;
            ps.ks[k] = q.k_s;
            ps.v[k] = q.v;
            ps.n0[k] = (double)c->step;
            // direction anchor -> pulled at the start, from replica 0 (all replicas share it)
            const float4 a = h[q.anchor], b = h[q.pulled];
            const double d[3] = {(double)b.x - (double)a.x, (double)b.y - (double)a.y, (double)b.z - (double)a.z};
            const double len = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            if (!(len > 0) || !std::isfinite(len)) return fail(c, SOP_ERR_INVALID_ARG, "pull: anchor and pulled coincide");
            for (int m = 0; m < 3; ++m) ps.dir[3 * k + m] = d[m] / len;
        }
        for (int r = 0; r < c->R; ++r)
            for (int k = 0; k < n; ++k) {
                const float4 b = h[(size_t)r * c->n + ps.bead[k]];
                double *t = &ps.tip0[((size_t)r * n + k) * 3];
                t[0] = b.x; t[1] = b.y; t[2] = b.z;
            }
        install_pulls(c, std::move(ps));
        return upload_pulls(c);
    } catch (const std::exception &e) {
        return fail(c, SOP_ERR_OOM, std::string("host exception: ") + e.what());
    }
}

sop_status sop_indenter(sop_ctx *c, const double center[3], const double direction[3], double radius, double v) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!(radius > 0)) {
        c->has_ind = false;
    } else {
        if (!center || !direction || !std::isfinite(v)) return fail(c, SOP_ERR_INVALID_ARG, "indenter");
        const double len = std::sqrt((direction[0] * direction[0] + direction[1] * direction[1]) + direction[2] * direction[2]);
        if (!(len > 0) || !std::isfinite(len)) return fail(c, SOP_ERR_INVALID_ARG, "indenter: direction");
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(center[k])) return fail(c, SOP_ERR_INVALID_ARG, "indenter: centre");
            c->ind_c0[k] = center[k];
            c->ind_dir[k] = direction[k] / len;
        }
        c->has_ind = true;
        c->ind_radius = radius;
        c->ind_v = v;
        c->ind_n0 = (double)c->step;
    }
    sync_external(c);
    destroy_graphs(c);
    return SOP_OK;
}

sop_status sop_get_positions(sop_ctx *c, int32_t replica, double *out) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!out || replica < -1 || replica >= c->R) return fail(c, SOP_ERR_INVALID_ARG, "replica or out");
    const size_t cnt = replica < 0 ? (size_t)c->R * c->n : (size_t)c->n;
    const size_t off = replica < 0 ? 0 : (size_t)replica * c->n;
    std::vector<float4> h(cnt);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(h.data(), c->d_pos[c->cur] + off, sizeof(float4) * cnt, cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < cnt; ++i) {
        out[3 * i] = h[i].x;
        out[3 * i + 1] = h[i].y;
        out[3 * i + 2] = h[i].z;
    }
    return SOP_OK;
}

sop_status sop_set_positions(sop_ctx *c, int32_t replica, const double *xyz) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!xyz || replica < -1 || replica >= c->R) return fail(c, SOP_ERR_INVALID_ARG, "replica or xyz");
    const size_t cnt = replica < 0 ? (size_t)c->R * c->n : (size_t)c->n;
    const size_t off = replica < 0 ? 0 : (size_t)replica * c->n;
    std::vector<float4> h(cnt);
    for (size_t i = 0; i < cnt; ++i) {
        if (!std::isfinite(xyz[3 * i]) || !std::isfinite(xyz[3 * i + 1]) || !std::isfinite(xyz[3 * i + 2]))
            return fail(c, SOP_ERR_INVALID_ARG, "positions hold a non-finite value");
        h[i] = make_float4((float)xyz[3 * i], (float)xyz[3 * i + 1], (float)xyz[3 * i + 2], 0.f);
    }
    CUDA_OR_RETURN(c, cudaMemcpyAsync(c->d_pos[c->cur] + off, h.data(), sizeof(float4) * cnt, cudaMemcpyHostToDevice,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaMemsetAsync(c->d_comp + off, 0, sizeof(float4) * cnt, c->stream));
    // the list follows the new positions: they become the snapshot of the last rebuild
    if (c->schedule == SOP_SCHED_BATCHED) {
        CUDA_OR_RETURN(c, cudaMemcpyAsync(c->d_snap + off, c->d_pos[c->cur] + off, sizeof(float4) * cnt,
                                          cudaMemcpyDeviceToDevice, c->stream));
    } else {
        rebuild_list(c, c->d_pos[c->cur], c->d_snap, full_range(c), &c->st.kernel_launches);
        c->list_step = c->step;
        c->st.rebuilds++;
    }
    CUDA_OR_RETURN(c, cudaGetLastError());
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

sop_status sop_get_velocities(sop_ctx *c, int32_t replica, double *out) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d_vel) return fail(c, SOP_ERR_UNSUPPORTED, "the overdamped integrator has no velocities");
    if (!out || replica < -1 || replica >= c->R) return fail(c, SOP_ERR_INVALID_ARG, "replica or out");
    const size_t cnt = replica < 0 ? (size_t)c->R * c->n : (size_t)c->n;
    const size_t off = replica < 0 ? 0 : (size_t)replica * c->n;
    std::vector<float4> h(cnt);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(h.data(), c->d_vel + off, sizeof(float4) * cnt, cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < cnt; ++i) {
        out[3 * i] = h[i].x;
        out[3 * i + 1] = h[i].y;
        out[3 * i + 2] = h[i].z;
    }
    return SOP_OK;
}

sop_status sop_set_velocities(sop_ctx *c, int32_t replica, const double *v) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d_vel) return fail(c, SOP_ERR_UNSUPPORTED, "the overdamped integrator has no velocities");
    if (!v || replica < -1 || replica >= c->R) return fail(c, SOP_ERR_INVALID_ARG, "replica or v");
    const size_t cnt = replica < 0 ? (size_t)c->R * c->n : (size_t)c->n;
    const size_t off = replica < 0 ? 0 : (size_t)replica * c->n;
    std::vector<float4> h(cnt);
    for (size_t i = 0; i < cnt; ++i) {
        if (!std::isfinite(v[3 * i]) || !std::isfinite(v[3 * i + 1]) || !std::isfinite(v[3 * i + 2]))
            return fail(c, SOP_ERR_INVALID_ARG, "velocities hold a non-finite value");
        h[i] = make_float4((float)v[3 * i], (float)v[3 * i + 1], (float)v[3 * i + 2], 0.f);
    }
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    CUDA_OR_RETURN(c, cudaMemcpyAsync(c->d_vel + off, h.data(), sizeof(float4) * cnt, cudaMemcpyHostToDevice,
                                      c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

sop_status sop_get_pairlist(sop_ctx *c, int32_t replica, int32_t *row_ptr, int32_t *col, int64_t cap, int64_t *nnz) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (replica < 0 || replica >= c->R || !row_ptr || !nnz) return fail(c, SOP_ERR_INVALID_ARG, "replica or outputs");
    const int n = c->n;
    std::vector<int32_t> start(n), len(n), cols;
    int32_t base_index = 0;
    if (c->schedule == SOP_SCHED_BATCHED) {
        // the batched kernel builds its list in shared memory; rebuild it from the snapshot
        // (the positions of the last rebuild) in forces mode and dump it
        const int stride = c->batched_cap;
        if (!c->d_dump_col) {
            CUDA_OR_RETURN(c, dalloc(c, &c->d_dump_start, (size_t)c->R * n));
            CUDA_OR_RETURN(c, dalloc(c, &c->d_dump_len, (size_t)c->R * n));
            CUDA_OR_RETURN(c, dalloc(c, &c->d_dump_col, (size_t)c->R * n * stride));
            CUDA_OR_RETURN(c, cudaMemset(c->d_dump_len, 0, sizeof(int32_t) * (size_t)c->R * n));
        }
        sop_ctx *cc = c;
        sop_status sb = launch_buckets(c, [cc, stride](BatchedArgs &a) {
            a.pos = cc->d_snap;
            a.n_steps = 0;
            a.force_out = cc->d_force;
            a.pl_dump_start = cc->d_dump_start;
            a.pl_dump_len = cc->d_dump_len;
            a.pl_dump_col = cc->d_dump_col;
            a.pl_dump_stride = stride;
        }, &c->st.kernel_launches);
        if (sb != SOP_OK) return sb;
        cols.resize((size_t)n * stride);
        CUDA_OR_RETURN(c, cudaMemcpyAsync(len.data(), c->d_dump_len + (size_t)replica * n, sizeof(int32_t) * n,
                                          cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaMemcpyAsync(cols.data(), c->d_dump_col + (size_t)replica * n * stride,
                                          sizeof(int32_t) * cols.size(), cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
        for (int i = 0; i < n; ++i) {
            if (len[i] > stride) return fail(c, SOP_ERR_PAIRLIST_OVERFLOW, "a Verlet row is longer than the dump stride");
            start[i] = i * stride;
        }
    } else {
        CUDA_OR_RETURN(c, cudaMemcpyAsync(start.data(), c->pl.start + (size_t)replica * n, sizeof(int32_t) * n,
                                          cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaMemcpyAsync(len.data(), c->pl.len + (size_t)replica * n, sizeof(int32_t) * n,
                                          cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
        int32_t lo = INT32_MAX, hi = 0;
        for (int i = 0; i < n; ++i)
            if (len[i] > 0) { lo = std::min(lo, start[i]); hi = std::max(hi, start[i] + len[i]); }
        if (hi > lo) {
            cols.resize(hi - lo);
            CUDA_OR_RETURN(c, cudaMemcpyAsync(cols.data(), c->pl.col + lo, sizeof(int32_t) * (hi - lo),
                                              cudaMemcpyDeviceToHost, c->stream));
            for (int i = 0; i < n; ++i) start[i] = len[i] > 0 ? start[i] - lo : 0;
        }
    }
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> rp, out;
    to_csr(n, start, len, cols, base_index, rp, out);
    *nnz = (int64_t)out.size();
    std::memcpy(row_ptr, rp.data(), sizeof(int32_t) * (n + 1));
    if (!col || cap < (int64_t)out.size()) return fail(c, SOP_ERR_CAPACITY, "col capacity below nnz");
    std::memcpy(col, out.data(), sizeof(int32_t) * out.size());
    return SOP_OK;
}

sop_status sop_get_native_map(sop_ctx *c, int32_t *row_ptr, int32_t *col, double *r0, int64_t cap, int64_t *nnz) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!row_ptr || !nnz) return fail(c, SOP_ERR_INVALID_ARG, "outputs");
    *nnz = c->nat_nnz;
    std::memcpy(row_ptr, c->h_nat_row.data(), sizeof(int32_t) * (c->n + 1));
    if (!col || !r0 || cap < c->nat_nnz) return fail(c, SOP_ERR_CAPACITY, "capacity below nnz");
    std::memcpy(col, c->h_nat_col.data(), sizeof(int32_t) * c->nat_nnz);
    std::memcpy(r0, c->h_nat_r0.data(), sizeof(double) * c->nat_nnz);
    return SOP_OK;
}

sop_status sop_get_observables(sop_ctx *c, sop_record *out, int64_t cap, int64_t *n_records, int64_t *n_lost) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!n_records) return fail(c, SOP_ERR_INVALID_ARG, "n_records is NULL");
    const int64_t per = c->n_seg;
    const int64_t ring_events = c->obs.cap / per;
    int64_t first = c->consumed;
    int64_t lost = 0;
    if (c->events - first > ring_events) {
        lost = (c->events - ring_events - first) * per;
        first = c->events - ring_events;
    }
    const int64_t n_ev = c->events - first;
    *n_records = n_ev * per;
    if (n_lost) *n_lost = lost;
    if (n_ev == 0) return SOP_OK;
    if (!out || cap < n_ev * per) return fail(c, SOP_ERR_CAPACITY, "out capacity below the pending records");
    std::vector<sop_record> ring(c->obs.cap);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(ring.data(), c->obs.ring, sizeof(sop_record) * c->obs.cap,
                                      cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    int64_t w = 0;
    for (int64_t e = first; e < c->events; ++e)
        for (int64_t g = 0; g < per; ++g) out[w++] = ring[(e * per + g) % c->obs.cap];
    c->consumed = c->events;
    return SOP_OK;
}

// Checkpoint layout: header of int64 fields, then arrays.
sop_status sop_get_state(sop_ctx *c, void *buf, int64_t cap, int64_t *size) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!size) return fail(c, SOP_ERR_INVALID_ARG, "size is NULL");
    const size_t RN = (size_t)c->R * c->n;
    const size_t np = c->pull_bead.size();
    const size_t need = 16 * sizeof(int64_t) + 3 * RN * sizeof(float4) + c->R * sizeof(int32_t) +
                        np * (3 * sizeof(int32_t) + 6 * sizeof(double)) + 3 * np * c->R * sizeof(double) +
                        9 * sizeof(double) + (c->d_taus ? RN * sizeof(uint4) : 0) +
                        (c->d_vel ? RN * sizeof(float4) : 0);
    *size = (int64_t)need;
    if (!buf) return SOP_OK;
    if (cap < (int64_t)need) return fail(c, SOP_ERR_CAPACITY, "buffer too small");
    char *p = static_cast<char *>(buf);
    int64_t hdr[16] = {0x534f5031, SOP_ABI_VERSION, c->n, c->R, c->step, c->list_step, (int64_t)np,
                       c->has_ind ? 1 : 0, c->events, c->consumed, c->d_taus ? 1 : 0, c->d_vel ? 1 : 0, 0, 0, 0, 0};
    std::memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    CUDA_OR_RETURN(c, cudaMemcpyAsync(p, c->d_pos[c->cur], RN * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
    p += RN * sizeof(float4);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(p, c->d_comp, RN * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
    p += RN * sizeof(float4);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(p, c->d_snap, RN * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
    p += RN * sizeof(float4);
    CUDA_OR_RETURN(c, cudaMemcpyAsync(p, c->d_rep_status, c->R * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    p += c->R * sizeof(int32_t);
    // optional parts at the end of the buffer: the Taus state, then the velocities
    const size_t tail_vel = c->d_vel ? RN * sizeof(float4) : 0;
    if (c->d_taus)
        CUDA_OR_RETURN(c, cudaMemcpyAsync(static_cast<char *>(buf) + need - tail_vel - RN * sizeof(uint4), c->d_taus,
                                          RN * sizeof(uint4), cudaMemcpyDeviceToHost, c->stream));
    if (c->d_vel)
        CUDA_OR_RETURN(c, cudaMemcpyAsync(static_cast<char *>(buf) + need - tail_vel, c->d_vel, tail_vel,
                                          cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    auto put = [&p](const void *src, size_t bytes) { if (bytes) std::memcpy(p, src, bytes); p += bytes; };
    put(c->pull_sys.data(), np * sizeof(int32_t));
    put(c->pull_anchor.data(), np * sizeof(int32_t));
    put(c->pull_bead.data(), np * sizeof(int32_t));
    put(c->pull_ks.data(), np * sizeof(double));
    put(c->pull_v.data(), np * sizeof(double));
    put(c->pull_n0.data(), np * sizeof(double));
    put(c->pull_dir.data(), 3 * np * sizeof(double));
    put(c->pull_tip0.data(), 3 * np * c->R * sizeof(double));
    double ind[9] = {c->ind_c0[0], c->ind_c0[1], c->ind_c0[2], c->ind_dir[0], c->ind_dir[1], c->ind_dir[2],
                     c->ind_radius, c->ind_v, c->ind_n0};
    put(ind, sizeof ind);
    return SOP_OK;
}

sop_status sop_set_state(sop_ctx *c, const void *buf, int64_t size) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!buf || size < (int64_t)(16 * sizeof(int64_t))) return fail(c, SOP_ERR_INVALID_ARG, "state buffer");
    try {
        // Everything in the buffer is read and checked before the context changes.
        const char *base = static_cast<const char *>(buf);
        int64_t hdr[16];
        std::memcpy(hdr, base, sizeof hdr);
        if (hdr[0] != 0x534f5031 || hdr[1] != SOP_ABI_VERSION || hdr[2] != c->n || hdr[3] != c->R)
            return fail(c, SOP_ERR_INVALID_ARG, "state does not match this context");
        if (hdr[6] < 0 || hdr[6] > c->n_sys)
            return fail(c, SOP_ERR_INVALID_ARG, "state: pulling record count out of range");
        if (hdr[4] < 0 || hdr[5] < -1 || hdr[5] > hdr[4] || hdr[8] < 0 || hdr[9] < 0 || hdr[9] > hdr[8] ||
            (hdr[7] != 0 && hdr[7] != 1))
            return fail(c, SOP_ERR_INVALID_ARG, "state: step, list step or record counters out of range");
        if ((hdr[10] != 0) != (c->d_taus != nullptr))
            return fail(c, SOP_ERR_INVALID_ARG, "state: noise source differs from this context");
        if ((hdr[11] != 0) != (c->d_vel != nullptr))
            return fail(c, SOP_ERR_INVALID_ARG, "state: integrator differs from this context");
        const size_t RN = (size_t)c->R * c->n;
        const size_t np = (size_t)hdr[6];
        const size_t tail_vel = c->d_vel ? RN * sizeof(float4) : 0;
        const size_t tail_taus = c->d_taus ? RN * sizeof(uint4) : 0;
        const size_t need = 16 * sizeof(int64_t) + 3 * RN * sizeof(float4) + c->R * sizeof(int32_t) +
                            np * (3 * sizeof(int32_t) + 6 * sizeof(double)) + 3 * np * c->R * sizeof(double) +
                            9 * sizeof(double) + tail_taus + tail_vel;
        if ((uint64_t)size < need) return fail(c, SOP_ERR_INVALID_ARG, "state buffer truncated");
        const char *p_pos = base + sizeof hdr;
        const char *p_status = p_pos + 3 * RN * sizeof(float4);
        const char *p = p_status + c->R * sizeof(int32_t);
        std::vector<int32_t> status(c->R);
        std::memcpy(status.data(), p_status, c->R * sizeof(int32_t));
        for (int32_t v : status)
            if (v < SOP_OK || v > SOP_ERR_INDENTER_OVERLAP)
                return fail(c, SOP_ERR_INVALID_ARG, "state: replica status out of range");
        auto get = [&p](void *dst, size_t bytes) { if (bytes) std::memcpy(dst, p, bytes); p += bytes; };
        PullSet ps;
        ps.resize(np, c->R);
        get(ps.sys.data(), np * sizeof(int32_t));
        get(ps.anchor.data(), np * sizeof(int32_t));
        get(ps.bead.data(), np * sizeof(int32_t));
        get(ps.ks.data(), np * sizeof(double));
        get(ps.v.data(), np * sizeof(double));
        get(ps.n0.data(), np * sizeof(double));
        get(ps.dir.data(), 3 * np * sizeof(double));
        get(ps.tip0.data(), 3 * np * c->R * sizeof(double));
        std::vector<int> seen(c->n_sys, 0);
        for (size_t k = 0; k < np; ++k) {
            const int sy = ps.sys[k];
            if (sy < 0 || sy >= c->n_sys || seen[sy]++)
                return fail(c, SOP_ERR_INVALID_ARG, "state: pull system out of range or repeated");
            const int lo = c->sys_lo[sy], hi = c->sys_lo[sy + 1];
            if (ps.anchor[k] < lo || ps.anchor[k] >= hi || ps.bead[k] < lo || ps.bead[k] >= hi ||
                ps.anchor[k] == ps.bead[k])
                return fail(c, SOP_ERR_INVALID_ARG, "state: pull beads out of range");
            const double *d = &ps.dir[3 * k];
            const double len2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!std::isfinite(ps.ks[k]) || ps.ks[k] < 0 || !std::isfinite(ps.v[k]) || !std::isfinite(ps.n0[k]) ||
                !(std::fabs(len2 - 1.0) < 1e-9))
                return fail(c, SOP_ERR_INVALID_ARG, "state: pull spring, speed, start or direction invalid");
        }
        double ind[9];
        get(ind, sizeof ind);
        for (double v : ind)
            if (!std::isfinite(v)) return fail(c, SOP_ERR_INVALID_ARG, "state: indenter record not finite");
        if (hdr[7] != 0 && !(ind[6] > 0)) return fail(c, SOP_ERR_INVALID_ARG, "state: indenter radius");
        const uint32_t *taus = c->d_taus
            ? reinterpret_cast<const uint32_t *>(base + need - tail_vel - tail_taus) : nullptr;
        if (taus) {
            for (size_t k = 0; k < RN; ++k) {
                uint32_t w[3];
                std::memcpy(w, taus + 4 * k, sizeof w);
                if (w[0] < 2u || w[1] < 8u || w[2] < 16u)
                    return fail(c, SOP_ERR_INVALID_ARG, "state: Hybrid Taus state needs y1 >= 2, y2 >= 8, y3 >= 16");
            }
        }
        // checked: now replace the context's state
        CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));   // no queued work may still use the state
        if (taus) CUDA_OR_RETURN(c, cudaMemcpy(c->d_taus, taus, tail_taus, cudaMemcpyHostToDevice));
        if (c->d_vel)
            CUDA_OR_RETURN(c, cudaMemcpy(c->d_vel, base + need - tail_vel, tail_vel, cudaMemcpyHostToDevice));
        c->cur = 0;
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_pos[0], p_pos, RN * sizeof(float4), cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_comp, p_pos + RN * sizeof(float4), RN * sizeof(float4), cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_snap, p_pos + 2 * RN * sizeof(float4), RN * sizeof(float4),
                                     cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_rep_status, status.data(), c->R * sizeof(int32_t), cudaMemcpyHostToDevice));
        install_pulls(c, std::move(ps));
        c->has_ind = hdr[7] != 0;
        for (int k = 0; k < 3; ++k) { c->ind_c0[k] = ind[k]; c->ind_dir[k] = ind[3 + k]; }
        c->ind_radius = ind[6];
        c->ind_v = ind[7];
        c->ind_n0 = ind[8];
        c->step = hdr[4];
        c->events = hdr[8];
        c->consumed = hdr[9];
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_step, &c->step, sizeof(int64_t), cudaMemcpyHostToDevice));
        CUDA_OR_RETURN(c, cudaMemcpy(c->d_events, &c->events, sizeof(int64_t), cudaMemcpyHostToDevice));
        sop_status s = upload_pulls(c);
        if (s != SOP_OK) return s;
        // the list in use is the one built from the snapshot
        rebuild_list(c, c->d_snap, nullptr, full_range(c), &c->st.kernel_launches);
        c->list_step = hdr[5];
        CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
        return SOP_OK;
    } catch (const std::exception &e) {
        return fail(c, SOP_ERR_OOM, std::string("host exception: ") + e.what());
    }
}

sop_status sop_get_rng_state(sop_ctx *c, uint32_t *state, int64_t n_words) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d_taus) return fail(c, SOP_ERR_UNSUPPORTED, "the context draws its noise from Philox (no state)");
    const size_t RN = (size_t)c->R * c->n;
    if (!state) return fail(c, SOP_ERR_INVALID_ARG, "state is NULL");
    if (n_words < (int64_t)(4 * RN)) return fail(c, SOP_ERR_CAPACITY, "state buffer too small");
    CUDA_OR_RETURN(c, cudaMemcpyAsync(state, c->d_taus, RN * sizeof(uint4), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

sop_status sop_set_rng_state(sop_ctx *c, const uint32_t *state, int64_t n_words) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->d_taus) return fail(c, SOP_ERR_UNSUPPORTED, "the context draws its noise from Philox (no state)");
    const size_t RN = (size_t)c->R * c->n;
    if (!state) return fail(c, SOP_ERR_INVALID_ARG, "state is NULL");
    if (n_words < (int64_t)(4 * RN)) return fail(c, SOP_ERR_CAPACITY, "state buffer too small");
    for (size_t k = 0; k < RN; ++k)
        if (state[4 * k] < 2u || state[4 * k + 1] < 8u || state[4 * k + 2] < 16u)
            return fail(c, SOP_ERR_INVALID_ARG, "Hybrid Taus state needs y1 >= 2, y2 >= 8, y3 >= 16");
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    CUDA_OR_RETURN(c, cudaMemcpy(c->d_taus, state, RN * sizeof(uint4), cudaMemcpyHostToDevice));
    return SOP_OK;
}

sop_status sop_replica_status(sop_ctx *c, int32_t *out) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(c, SOP_ERR_INVALID_ARG, "out is NULL");
    CUDA_OR_RETURN(c, cudaMemcpyAsync(out, c->d_rep_status, sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_RETURN(c, cudaStreamSynchronize(c->stream));
    return SOP_OK;
}

void sop_abort(sop_ctx *c) {
    if (c && c->h_abort) *(volatile int32_t *)c->h_abort = 1;
}

sop_status sop_get_stats(sop_ctx *c, sop_stats *out) {
    if (!c) return fail(nullptr, SOP_ERR_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(c, SOP_ERR_INVALID_ARG, "out is NULL");
    c->st.steps = c->step;
    *out = c->st;
    return SOP_OK;
}

const char *sop_last_error(const sop_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void sop_destroy(sop_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
