// Internal interfaces between the C-ABI layer (sop_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sop.h"
#include "sop_device.cuh"

namespace sop {

// Bead flag bits (per bead of a replica, shared by all replicas).
enum : uint8_t { kFlagFixed = 1, kFlagPulled = 2, kFlagFirstOfSystem = 4 };

// Shared topology on the device. Bead indices are replica-local (0..n-1).
struct DevTopo {
    int32_t n = 0;                 // beads per replica
    int32_t n_sys = 0;             // systems per replica
    const int32_t *chain = nullptr;      // [n] chain id
    const int32_t *sys = nullptr;        // [n] system id
    const uint8_t *flags = nullptr;      // [n] kFlag*
    const float *bond_r0 = nullptr;      // [n] r0 of bond (i, i+1), < 0 when i is the last bead of its chain
    const double *bond_r0d = nullptr;    // [n] the same in FP64
    const int32_t *nat_row = nullptr;    // [n+1] CSR rows, both directions, ascending
    const int32_t *nat_col = nullptr;    // [nnz]
    const float *nat_r0sq = nullptr;     // [nnz] r0^2 rounded to FP32
    const uint2 *nat_ent = nullptr;      // [nnz] (nat_col, nat_r0sq as float bits): one load per entry
    const double *nat_r0 = nullptr;      // [nnz] FP64 r0
    const int32_t *sys_lo = nullptr;     // [n_sys+1] first bead of each system
    const int32_t *sys_ree_last = nullptr;  // [n_sys] last bead of the system's first chain
    const int32_t *sys_nat_pairs = nullptr; // [n_sys] native contacts (i < j) per system
    const int32_t *xb_row = nullptr;     // [n+1] cross-link CSR (both directions, ascending); NULL: none
    const int32_t *xb_col = nullptr;     // [n_xb]
    const float *xb_r0 = nullptr;        // [n_xb] native length, FP32
    const double *xb_r0d = nullptr;      // [n_xb] the same in FP64
};

// Cantilevers (per system) and the indenter, FP64.
struct DevExternal {
    const int32_t *pull_of_sys = nullptr;  // [n_sys] pull index or -1
    const int32_t *pull_anchor = nullptr;  // [n_pull]
    const int32_t *pull_bead = nullptr;    // [n_pull]
    const double *pull_ks = nullptr;       // [n_pull]
    const double *pull_v = nullptr;        // [n_pull]
    const double *pull_dir = nullptr;      // [3 n_pull]
    const double *pull_n0 = nullptr;       // [n_pull] start step
    const double *pull_tip0 = nullptr;     // [R * n_pull * 3] tip at the start, per replica
    int32_t n_pull = 0;
    int32_t has_indenter = 0;
    double ind_c0[3] = {0, 0, 0};
    double ind_dir[3] = {0, 0, 0};
    double ind_radius = 0, ind_v = 0, ind_n0 = 0;
};

// Everything the per-step kernels read.
struct StepArgs {
    DevTopo topo;
    DevExternal ext;
    ForceParams fp;
    float cut2_f = 0;
    double cut2_d = 0;
    double k_fene = 0, R0 = 0, eps_h = 0, eps_l = 0, sigma = 0;   // FP64 copies for observables
    uint64_t seed = 0;
    int32_t R = 0;
    const int64_t *d_step = nullptr;   // device step counter (step of the first kernel of a sequence)
    int32_t *rep_status = nullptr;     // [R]
    int32_t *halt = nullptr;           // [1] nonzero: every kernel copies state through
    uint4 *taus = nullptr;             // [R*n] Hybrid Taus state per bead; null: Philox noise
    float4 *vel = nullptr;             // [R*n] underdamped (BAOAB) velocity per bead; null: overdamped
    float h_m = 0, half_h = 0, c1 = 0, c2 = 0;   // BAOAB: h/m, h/2, exp(-zeta h/m), sqrt(kT (1 - c1^2)/m)
};

// Streamed-schedule Verlet list (row starts are arbitrary; rows are sorted).
struct DevPairList {
    int32_t *start = nullptr;          // [R*n]
    int32_t *len = nullptr;            // [R*n]
    int32_t *col = nullptr;            // [cap] replica-local partner index
    int32_t *cursor = nullptr;         // [n_seg] next free column of each segment
    const int64_t *seg_base = nullptr; // [n_seg] first column of each segment
    const int64_t *seg_end = nullptr;  // [n_seg] one past the last column of each segment
    int64_t cap = 0;
};

// Host-known extent of a range of segments [g_lo, g_hi).
struct SegRange {
    int32_t g_lo = 0, g_hi = 0;   // segments
    int32_t b_lo = 0, b_hi = 0;   // global beads
    int32_t c_lo = 0, c_hi = 0;   // cells
    int32_t max_seg = 0;          // beads of the largest segment (0: unknown)
    int32_t k_lo = 0, k_hi = 0;   // CTAs of the all-pairs list build (DevCells::brute_cta_lo)
};

// Cell-list scratch of the streamed rebuild.
struct DevCells {
    int32_t n_seg = 0;
    const int32_t *seg_bead_lo = nullptr;   // [n_seg+1] global bead offsets (replica-major)
    const int32_t *seg_cell_base = nullptr; // [n_seg+1] cell offsets
    float4 *seg_lo = nullptr;               // [n_seg] grid origin (w = inverse cell edge)
    int4 *seg_dims = nullptr;               // [n_seg] dims (w = cells used)
    int32_t *cell_of = nullptr;             // [R*n] global cell index of each bead
    int32_t *cell_cnt = nullptr;            // [n_cells] zero between rebuilds
    int32_t *cell_start = nullptr;          // [n_cells+1]
    float4 *sorted = nullptr;               // [R*n] positions grouped by cell, bead index (int bits) in w
    int32_t *seg_box = nullptr;             // [n_seg*8] bounding-box keys of large segments (reset after use)
    const int32_t *brute_cta_lo = nullptr;  // [n_seg+1] first CTA of each segment in the all-pairs build
    int32_t *brute_done = nullptr;          // [n_seg] CTAs done in the current all-pairs build (0 between)
    int32_t *brute_used = nullptr;          // [n_seg] list entries of each segment after its last build
    int32_t *scan_tmp = nullptr;            // scan block sums
    int64_t n_cells = 0;
};

// Observable scratch.
struct DevObs {
    int32_t n_chunks = 0;
    const int32_t *chunk_seg = nullptr;     // [n_chunks]
    const int32_t *chunk_lo = nullptr;      // [n_chunks] global bead range
    const int32_t *chunk_hi = nullptr;
    const int32_t *seg_chunk_lo = nullptr;  // [n_seg+1]
    int32_t max_seg_chunks = 0;             // most chunks of one segment
    double *partial = nullptr;              // [n_chunks * 8]
    sop_record *ring = nullptr;             // [cap]
    int64_t cap = 0;
    int64_t *events = nullptr;              // [1] cadence events recorded
    int32_t obs_every = 0;
    int32_t q_every = 0;                    // records at steps not a multiple of this carry NaN in q (0: none)
};

// Set the text returned by sop_last_error(NULL) (sop_api.cu).
void set_global_error(const std::string &msg);

// ---- launchers (k_stream.cu) ----
// Elements one block of the scan covers, and candidates one Verlet row of the streamed
// builder may hold (more is an overflow of that row).
constexpr int kScanTileElems = 2048;
constexpr int kRowCandidates = 256;

// Scan: out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total.
void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s, int64_t *launches);
int64_t scan_tmp_elems(int64_t n);

void launch_setup_bonds(const double *native_xyz, const int32_t *chain, float *bond_r0, double *bond_r0d,
                        int32_t n, cudaStream_t s);
void launch_native_count(const double *native_xyz, const int32_t *chain, const int32_t *sys,
                         const int32_t *sys_lo, int32_t n, double cut, int32_t *count, cudaStream_t s);
void launch_native_fill(const double *native_xyz, const int32_t *chain, const int32_t *sys,
                        const int32_t *sys_lo, int32_t n, double cut, const int32_t *row, int32_t *col,
                        double *r0, float *r0sq, cudaStream_t s);

// Streamed rebuild of the Verlet list for global beads [b_lo, b_hi) = segments [g_lo, g_hi).
// pos: the positions to build from; snap (may be null) receives a copy of them.
// Beads per chunk of the FP64 observable sums of the streamed forms (one CTA each).
constexpr int kObsChunkBeads = 32;
// Segments up to this many beads build their Verlet rows without a cell list: each bead
// tests the blocks of 64 consecutive beads whose bounding box lies within the cutoff;
// kBruteSliceBeads beads per CTA.
constexpr int kBruteMaxBeads = 8192;
constexpr int kBruteSliceBeads = 16;
// Put every segment's bounding-box accumulator in its empty state (once, after allocation).
void launch_seg_box_init(int32_t *seg_box, int32_t n_seg, cudaStream_t s);
void launch_rebuild(const StepArgs &a, const DevCells &c, const DevPairList &pl, const float4 *pos, float4 *snap,
                    const SegRange &rg, cudaStream_t s, int64_t *launches);

// One fused force + noise + update step for global beads [b_lo, b_hi), step = *d_step + k_off.
void launch_step(const StepArgs &a, const DevPairList &pl, const float4 *pos_in, float4 *pos_out, float4 *comp,
                 int32_t b_lo, int32_t b_hi, int32_t k_off, int lanes, cudaStream_t s, int64_t *launches);

// k_steps fused steps of the beads [b_lo, b_hi) in one cooperative launch (grid barriers
// between steps; layers alternate from pos_a, so after an odd count the result is in pos_b).
// bar: two zero-initialised words of device memory owned by the caller.
cudaError_t launch_step_coop(const StepArgs &a, const DevPairList &pl, float4 *pos_a, float4 *pos_b, float4 *comp,
                             int32_t b_lo, int32_t b_hi, int32_t k_off, int32_t k_steps, int lanes, unsigned *bar,
                             cudaStream_t s, int64_t *launches);

// Forces only (no update) at pos for global beads [b_lo, b_hi) with `lanes` (4, 8, 16)
// lanes per bead; writes F (xyz, w unused).
void launch_forces(const StepArgs &a, const DevPairList &pl, const float4 *pos, float4 *force, int32_t b_lo,
                   int32_t b_hi, int64_t step, cudaStream_t s, int64_t *launches, int lanes = 8);

// Observables (FP64) of all segments at pos; step = *d_step + k_off. If gate > 0 the record
// is written only when the step is a multiple of gate. Writes into the ring.
void launch_observables(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t n_seg,
                        int32_t k_off, int32_t gate, cudaStream_t s, int64_t *launches);

// Observables of segment g alone (chunks [ch_lo, ch_hi)) at step *d_step + k_off, written as
// cadence event *events + event_off.
void launch_observables_seg(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t g,
                            int32_t n_seg, int32_t ch_lo, int32_t ch_hi, int32_t k_off, int64_t event_off,
                            cudaStream_t s, int64_t *launches);

// FP64 energy of the segments [g_lo, g_hi) at pos into *out (device), via the observable partials.
// Chunks [ch_lo, ch_hi) must be exactly the chunks of segments [g_lo, g_hi).
void launch_energy(const StepArgs &a, const DevPairList &pl, const DevObs &o, const float4 *pos, int32_t g_lo,
                   int32_t g_hi, int32_t ch_lo, int32_t ch_hi, double *out, cudaStream_t s, int64_t *launches);

// Advance the device step counter by k; add one cadence event when gate > 0 and the new step
// is a multiple of gate, else add n_events.
void launch_tick(int64_t *d_step, int64_t k, int64_t *events, int32_t gate, int64_t n_events, cudaStream_t s,
                 int64_t *launches);

// ---- pair-based form (k_pairs.cu), Algorithms 4 and 5 ----
// Pair lists and force tables. Each pair (i < j) is evaluated once; +df goes to the slot of
// entry (i -> j), -df to the slot of the reverse entry (j -> i). Slots are laid out like the
// rows, so a bead's gathering reads its own slots in row order.
struct DevPairTables {
    const int32_t *nat_half = nullptr;    // [n_nat_half] native CSR entries q with col[q] > row(q)
    const int32_t *nat_owner = nullptr;   // [nnz] row (replica-local bead) of entry q
    const int32_t *nat_mirror = nullptr;  // [nnz] reverse entry of q
    int32_t n_nat_half = 0;
    int64_t nnz = 0;
    int4 *vpair = nullptr;                // [vcap] Verlet half pairs (entry, reverse entry or -1, gb, gj)
    int32_t *vcount = nullptr;            // [beads of the range] upper entries per row
    int32_t *voff = nullptr;              // [beads + 1] exclusive offsets; voff[beads] = total
    int32_t *scan_tmp = nullptr;          // scan block sums
    int64_t vcap = 0;
    float4 *fb = nullptr;                 // [2 R n] bond slots: 2 gb left bond, 2 gb + 1 right bond; w = 1 if broken
    float4 *fn = nullptr;                 // [R nnz] native slots, replica r at r * nnz
    float4 *fv = nullptr;                 // [pl cap] Verlet slots, aligned with the list's columns
};

// Half list of the Verlet list for the beads of range rg (whole replicas): count, scan, fill.
void launch_pair_index(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const SegRange &rg,
                       cudaStream_t s, int64_t *launches);

// One step in the pair-based form: the pair kernel (Algorithm 4) over bonds, natives and the
// Verlet half list, then the gathering (Algorithm 5) fused with noise and the update.
void launch_pairs_step(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const float4 *pos_in,
                       float4 *pos_out, float4 *comp, const SegRange &rg, int32_t k_off, int lanes, cudaStream_t s,
                       int64_t *launches);

// Forces only in the pair-based form (pair kernel + gathering), as launch_forces.
void launch_pairs_forces(const StepArgs &a, const DevPairList &pl, const DevPairTables &t, const float4 *pos,
                         float4 *force, const SegRange &rg, int64_t step, cudaStream_t s, int64_t *launches);

// ---- batched schedule (k_batched.cu) ----
struct BatchedArgs {
    StepArgs sa;
    // work items (replica, system), heaviest first
    int32_t n_items = 0;
    const int32_t *item_rep = nullptr;
    const int32_t *item_sys = nullptr;
    // native lists in ELL form per system, column-major within a system:
    // entry k of local bead b of system s is at nat_ell_off[s] + k * n_s + b
    const int32_t *nat_ell_off = nullptr;  // [n_sys]
    const int32_t *nat_ell_cnt = nullptr;  // [n] count per bead
    const uint16_t *nat_ell_col = nullptr; // system-local partner
    const float *nat_ell_r0sq = nullptr;
    // the same table in native-slot order: slot t of system s holds local bead
    // nat_slot_bead[sys_lo[s] + t] (beads by native count, descending: the warps of the native
    // phase get beads of equal count), entry k at nat_ell_off[s] + k * n_s + t
    const uint16_t *nat_slot_bead = nullptr;  // [n]
    const uint16_t *nat_slot_cnt = nullptr;   // [n]
    const uint2 *nat_slot_ent = nullptr;     // (partner, r0^2 as float bits) per entry
    // pair form: each native pair belongs to the row of one of its beads (balanced
    // orientation); ELL tables per system like the ones above, entry k of bead b at
    // off[s] + k * n_s + b. own: the partners of b's own pairs (ascending) and their r0^2;
    // rev: the partners whose row holds the pair with b (ascending) and the index of b
    // among that partner's own natives
    const int32_t *nat_own_off = nullptr;  // [n_sys]
    const int32_t *nat_own_cnt = nullptr;  // [n]
    const uint16_t *nat_own_col = nullptr;
    const float *nat_own_r0sq = nullptr;
    const int32_t *nat_rev_off = nullptr;  // [n_sys]
    const int32_t *nat_rev_cnt = nullptr;  // [n]
    const uint16_t *nat_rev_col = nullptr;
    const uint16_t *nat_rev_k = nullptr;
    int32_t pair_pool = 0;      // pair form: bytes of shared memory for rows, reverse lists and coefficients
    // static exclusions of the rebuild scan for systems of at most 256 beads: bit t of
    // excl[excl_off[s] + blk * n_s + b] marks candidate 32 blk + t of bead b as the bead itself,
    // a bonded neighbour or a native partner; excl_off[s] < 0 for larger systems
    const int32_t *excl_off = nullptr;   // [n_sys]
    const uint32_t *excl = nullptr;
    float4 *pos = nullptr;      // [R*n] current positions (read at start, written at end)
    float4 *comp = nullptr;     // [R*n]
    float4 *snap = nullptr;     // [R*n] positions at the last rebuild
    int32_t *pl_dump_start = nullptr;  // optional: dump the list of the first rebuild (forces mode)
    int32_t *pl_dump_len = nullptr;
    int32_t *pl_dump_col = nullptr;
    int32_t pl_dump_stride = 0;
    float4 *force_out = nullptr;       // forces mode: F at the start positions
    const int64_t *d_step = nullptr;    // step at launch start (device, read-only here)
    const int64_t *d_events = nullptr;  // records taken before this launch (device)
    int32_t n_steps = 0;
    int32_t K = 10;             // rebuild_every
    int32_t cap = 64;           // Verlet capacity per bead
    int32_t max_n = 0;          // largest system in the launch
    uint16_t *row_global = nullptr;  // rows in global memory: [n_items][row_width][max_n]
    int32_t row_width = 0;      // natives + Verlet capacity per row
    DevObs obs;
    int32_t obs_every = 0;
    int32_t n_seg = 0;
};

struct BatchedConfig {
    int threads = 128;
    int beads_per_thread = 1;
    int min_blocks = 4;        // register cap 65536 / (max threads of the instance * min_blocks)
    bool rows_global = false;  // neighbour rows in global memory instead of shared memory
    int row_width = 0;
    size_t smem = 0;
    int cluster = 0;           // > 0: the cluster form, one system over `cluster` CTAs of 2^m_shift beads each
    int m_shift = 0;
    bool pair_form = false;    // each pair evaluated once (k_bpair) instead of the particle-based gather
    int lanes = 1;             // cluster form: lanes per bead (1, 2 or 4)
};

// A configuration for systems of at most max_n beads whose merged rows hold up to
// row_width entries (natives + Verlet capacity); false when no compiled instance fits.
bool batched_config(int max_n, int row_width, int threads, bool rows_global, int min_blocks, BatchedConfig *cfg);
// The cluster form: each system is split over ceil(max_n / 2^m_shift) CTAs (at most 16)
// of `threads` threads that own 2^m_shift consecutive beads each, served by groups of
// `lanes` lanes per bead (1, 2 or 4); false when it does not fit.
bool cluster_config(int max_n, int row_width, int threads, int m_shift, int lanes, BatchedConfig *cfg);
cudaError_t launch_cluster(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s);
// The pair form (Newton's third law inside the CTA) for systems of at most max_n <= 256
// beads with `pool` bytes (a multiple of 16) of shared memory for the rows, reverse lists and
// coefficients of one item; false when it does not fit.
bool pair_config(int max_n, int pool, int threads, int min_blocks, BatchedConfig *cfg);
// Pool bytes for so own entries and sr reverse entries (group padding included) in a system
// of n beads.
size_t pair_pool_bytes(int so, int sr, int n);
constexpr int kPairMaxBeads = 256;
// CTAs of the configuration the device holds at once (cluster form: clusters x size); 0 when
// the occupancy query fails.
int batched_resident_ctas(const BatchedConfig &cfg);
// Clusters of the configuration that fit the device at once (0: it cannot launch).
int cluster_capacity(const BatchedConfig &cfg);
// Run n_steps (or forces only when a.force_out != null and n_steps == 0).
cudaError_t launch_bpair(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s);
int bpair_resident_ctas(const BatchedConfig &cfg);
cudaError_t launch_batched(const BatchedArgs &a, const BatchedConfig &cfg, cudaStream_t s, int64_t *launches);

}  // namespace sop
