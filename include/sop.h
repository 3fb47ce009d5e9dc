/*
 * sop.h - C ABI of the GB300 (sm_103a) SOP-model overdamped Langevin library.
 *
 * The library advances Calpha-level Self-Organized-Polymer models of proteins
 * with the first-order (Ermak-McCammon) Langevin update, as described in
 * Zhmurov, Dima, Kholodov, Barsegov, "Langevin dynamics simulations of
 * biomolecules on graphics processors" (arXiv 1003.1148):
 *   - forces of Eq. 1: FENE bonds (i, i+1), the native-contact 12-6 attraction
 *     eps_h [(r0/r)^12 - 2 (r0/r)^6] and the non-native repulsion
 *     eps_l (sigma/r)^6 over a Verlet pair list (Sec. IV.A, Sec. III.A);
 *   - Gaussian random forces (Sec. III.C), drawn from counter-based
 *     Philox4x32-10 and transformed by Box-Muller;
 *   - the update r += F h/zeta + g sqrt(2 kT h/zeta) (Algorithm 7);
 *   - the Verlet list rebuilt every K steps (Algorithm 3), here from a cell
 *     list built by counting sort;
 *   - constant-velocity cantilever pulling (Sec. IV.B) and a repulsive
 *     spherical indenter (force-indentation runs named in the Conclusion).
 *
 * Conventions for every entry point:
 *   - Units: Angstrom, kcal/mol, ps, K. Bead indices are 0-based and count
 *     beads of one replica (0 .. n_beads-1).
 *   - Host arrays are owned by the caller and only read or written during the
 *     call. The context owns all device memory it allocates.
 *   - Positions cross the boundary as FP64 xyz triples ([3*n] doubles, bead
 *     major); inside they are FP32 with a compensated (Kahan) update, so a
 *     value read back is the FP32 state converted exactly to FP64.
 *   - Work is queued on params.cuda_stream (NULL = the legacy default stream).
 *     Calls that return data to the host synchronise that stream.
 *   - No C++ exception crosses the ABI. Every call returns a sop_status; the
 *     text of the last error of a context is sop_last_error(ctx).
 *   - A context is used by one host thread at a time.
 *   - Replica r of a context is an independent copy of the whole topology;
 *     its random forces use the Philox key seed + r and the counter
 *     (step, bead, 0).
 */
#ifndef SOP_H
#define SOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Not in the paper: the version of this interface (also stamped into checkpoints). */
#define SOP_ABI_VERSION 3

/* Not in the paper: the status every call returns. The failure conditions follow
 * Eq. 1 (the FENE term is undefined at |r - r0| >= R0) and Sec. III.A (the Verlet
 * list's capacity). */
typedef enum {
    SOP_OK = 0,
    SOP_ERR_INVALID_ARG = 1,       /* a pointer, size or parameter was rejected */
    SOP_ERR_CUDA = 2,              /* a CUDA runtime call failed (see sop_last_error) */
    SOP_ERR_OOM = 3,               /* device allocation failed */
    SOP_ERR_FENE_BREAK = 4,        /* a bond reached |r - r0| >= R0; that replica is frozen */
    SOP_ERR_NONFINITE = 5,         /* a position became NaN/Inf; that replica is frozen */
    SOP_ERR_PAIRLIST_OVERFLOW = 6, /* the Verlet list outgrew its capacity; the run stopped */
    SOP_ERR_ABORTED = 7,           /* sop_abort() stopped the run */
    SOP_ERR_TIMEOUT = 8,           /* a bounded device-side wait gave up */
    SOP_ERR_INDENTER_OVERLAP = 9,  /* a bead entered the indenter sphere; that replica is frozen */
    SOP_ERR_UNSUPPORTED = 10,      /* the request is valid but this build cannot serve it */
    SOP_ERR_CAPACITY = 11          /* a caller-provided output buffer is too small */
} sop_status;

/* How the steps are executed (the schedule): Sec. III's kernels (particle-based,
 * Sec. III.A; pair-based, Sec. III.B; the fused integration kernel, Sec. III.D) in
 * forms of this library's own (the persistent batched kernel, graph replay). */
typedef enum {
    SOP_SCHED_AUTO = 0,      /* choose per workload (autotuned) */
    SOP_SCHED_BATCHED = 1,   /* persistent fused kernel, one CTA per (replica, system), state in shared memory */
    SOP_SCHED_STREAMED = 2,  /* per-step kernels over global memory, cell-list rebuilds, CUDA-graph replay */
    SOP_SCHED_PLAIN = 3,     /* the plain form: per-step launches, one system after another, no graph */
    SOP_SCHED_PAIRS = 4,     /* the streamed schedule with pair-based forces (Sec. III.B, Algorithms 4 and 5):
                                one thread per interacting pair writes +df and -df into per-entry force
                                slots; the per-bead gathering is fused into the update */
    SOP_SCHED_BATCHED_PAIRS = 5  /* the batched schedule with each pair evaluated once (Sec. III.B, Algorithms
                                4 and 5, inside one CTA): a pair belongs to the row of one of its beads,
                                whose thread adds the force to it and leaves the coefficient for the other
                                bead to add after a barrier; systems of up to 256 beads (larger systems
                                of the context take the particle-based gather). SOP_SCHED_BATCHED keeps the
                                gather everywhere; SOP_SCHED_AUTO times both forms per size bucket, so its
                                summation order (and so its trajectory bits) may follow the timing */
} sop_schedule;

/* Source of the Gaussian random force (Sec. III.C). */
typedef enum {
    SOP_RNG_PHILOX = 0,       /* counter-based Philox4x32-10: key seed + replica, counter (step, bead); no state */
    SOP_RNG_HYBRID_TAUS = 1   /* Hybrid Taus (Algorithm 6): three Tausworthe generators and an LCG per bead,
                                 16 bytes of state each, four outputs per bead and step; a bead's generator
                                 advances only in steps in which the bead moves */
} sop_rng;

/* Equations of motion (Eq. 2 and Algorithm 7; the underdamped form is the extension the
 * Conclusion names). */
typedef enum {
    SOP_INTEGRATOR_OVERDAMPED = 0,   /* Algorithm 7: r += F h/zeta + g sqrt(2 kT h/zeta) */
    SOP_INTEGRATOR_BAOAB = 1         /* underdamped Langevin dynamics (the limit the Conclusion names), by the
                                        BAOAB splitting of Leimkuhler and Matthews (2013): bead mass `mass`,
                                        friction zeta; per step, with F = F(r_n) and w the stored velocity:
                                        v' = w + (h/m) F; v'' = c1 v' + c2 g; r += (h/2)(v' + v''); w = v'',
                                        c1 = exp(-zeta h/m), c2 = sqrt(kT (1 - c1^2)/m). The stored velocity
                                        is the one after the O sub-step (0 at the start). */
} sop_integrator;

/* Not in the paper: the opaque handle that owns a simulation's device memory. */
typedef struct sop_ctx sop_ctx;

/* Topology of one replica (the SOP model's chains of C-alpha beads, Sec. IV.A; bonds
 * join consecutive beads of a chain, Eq. 1's first term). Chains are contiguous bead
 * ranges; systems are contiguous chain ranges. Beads interact (native contacts,
 * repulsion) only with beads of the same system. */
typedef struct {
    int32_t n_beads;                 /* beads per replica, >= 1 */
    int32_t n_chains;                /* >= 1 */
    const int32_t *chain_offsets;    /* [n_chains+1], 0 = off[0] < off[1] < ... = n_beads */
    int32_t n_systems;               /* 0: every chain is its own system */
    const int32_t *system_offsets;   /* [n_systems+1] in chains, or NULL when n_systems == 0 */
    const uint8_t *fixed_mask;       /* [n_beads], 1 = bead never moves; NULL = none fixed */
    int32_t n_extra_bonds;           /* cross-links: covalent bonds beyond (i, i+1) of a chain (Table I
                                        counts such bonds among the covalent ones), e.g. disulfide
                                        bridges or links between chains; 0 = none */
    const int32_t *extra_bonds;      /* [2*n_extra_bonds] bead pairs (i, j): one system, i != j, not
                                        consecutive beads of one chain, no pair twice. Each is a FENE
                                        term of Eq. 1 with its native length; the pair is neither a
                                        native contact nor a Verlet-list pair. The streamed schedules
                                        take them; the batched ones answer SOP_ERR_UNSUPPORTED (AUTO
                                        then runs streamed). NULL when n_extra_bonds == 0 */
} sop_topology;

/* Parameters (Eq. 1, Algorithm 7, the Verlet list and the run). */
typedef struct {
    double k_fene;          /* FENE spring constant k, kcal/(mol A^2) */
    double R0;              /* FENE tolerance R0, A (paper: 2) */
    double eps_h;           /* native contact depth, kcal/mol */
    double native_cut;      /* native contact cutoff R_C, A (paper: 8) */
    double eps_l;           /* repulsion strength, kcal/mol (paper: 1) */
    double sigma;           /* repulsion range, A (paper: 3.8) */
    double T;               /* temperature, K */
    double zeta;            /* friction, (kcal/mol) ps / A^2 */
    double dt;              /* time step h, ps */
    double pair_cut;        /* Verlet-list cutoff, A */
    int32_t rebuild_every;  /* K: the list is rebuilt at steps 0, K, 2K, ... */
    int32_t n_replicas;     /* >= 1 */
    uint64_t seed;          /* Philox key of replica r is seed + r */
    int32_t obs_every;      /* observable cadence in steps (0 = none) */
    int32_t obs_capacity;   /* ring-buffer capacity in records (0 = 4096) */
    int32_t pairs_per_bead; /* Verlet-list capacity per bead (0 = automatic) */
    int32_t schedule;       /* a sop_schedule */
    void *cuda_stream;      /* cudaStream_t to queue work on (NULL = default stream) */
    int32_t rng;            /* a sop_rng (0 = Philox) */
    int32_t integrator;     /* a sop_integrator (0 = overdamped) */
    double mass;            /* bead mass, (kcal/mol) ps^2 / A^2 (> 0 for SOP_INTEGRATOR_BAOAB) */
    int32_t obs_every_q;    /* cadence of Q in steps: 0 = every record; else a multiple of obs_every, and
                               records at other steps carry NaN in q. Sec. IV.B reads the force-extension
                               curve f(R) along the pull; Q is a slower structural readout, so the two get
                               their own cadences (the values are the caller's; the paper gives none) */
} sop_params;

/* Cantilever on one system (Sec. IV.B): `anchor` is held fixed; a spring of
 * constant k_s acts on `pulled`, whose tip starts at the pulled bead's
 * position when sop_pull is called and moves at v A/step along the unit
 * vector from anchor to pulled at that moment. */
typedef struct {
    int32_t system;
    int32_t anchor;
    int32_t pulled;
    double k_s;             /* kcal/(mol A^2) */
    double v;               /* A per step */
} sop_pull_params;

/* One observable record (all FP64): Eq. 1's energy and the readouts of Sec. IV.B
 * (force f and extension R of the force-extension curve, Fig. 3), plus Q and the
 * end-to-end distance. */
typedef struct {
    double step;            /* step at which the record was taken */
    double replica;
    double system;
    double energy;          /* Eq. 1 energy of the system (FENE + native + listed repulsion) */
    double f_ext;           /* pull: k_s (tip - r_pulled) . dir; indenter: force on the system's beads along its motion */
    double extension;       /* pull: |r_pulled - r_anchor|; indenter: distance travelled */
    double q;               /* fraction of native contacts with r < r0 + 2 A */
    double r_ee;            /* end-to-end distance of the system's first chain */
} sop_record;

/* Not in the paper: counters of the work queued so far. */
typedef struct {
    int64_t steps;                /* steps completed (the global step counter) */
    int64_t kernel_launches;      /* kernels launched by this context (graph nodes counted) */
    int64_t graph_launches;       /* CUDA-graph launches */
    int64_t rebuilds;             /* Verlet-list rebuilds */
    int32_t schedule;             /* the sop_schedule in use */
    int32_t block_threads;        /* CTA size of the step kernel */
    int32_t pairs_per_bead;       /* Verlet-list capacity per bead */
    int32_t beads_per_thread;     /* batched schedule: beads owned by one thread */
    int32_t min_blocks;           /* batched schedule: register cap 65536 / (256 * min_blocks); 0 = rows in global memory */
    int32_t buckets;              /* batched schedule: size buckets (one kernel launch each per chunk) */
    int64_t pairlist_entries;     /* entries in the last Verlet list of replica 0 */
    int64_t native_entries;       /* native contacts (i < j) */
    double tune_ms;               /* batched schedule: trial time of the chosen configuration */
    int32_t cluster_buckets;      /* batched schedule: buckets run in the cluster form (one system over a
                                     thread-block cluster) */
    int32_t cluster_size;         /* CTAs per cluster in the bucket with the most systems (0: not clustered) */
    int32_t pair_buckets;         /* batched schedule: buckets run in the pair form (each pair evaluated once) */
} sop_stats;

/* Create a context: validates the arguments, builds the bonds (r0 from the
 * native coordinates) and the native contact map (pairs |i-j| > 2 in a chain,
 * or in different chains of one system, with FP64 native distance below
 * native_cut; Eq. 1, Sec. IV.A) on the GPU, uploads the native coordinates as
 * the starting positions of every replica and builds the first Verlet list.
 * native_xyz: [3*n_beads] FP64, host. On success *out owns the device state;
 * on failure *out is NULL. */
sop_status sop_create(const sop_topology *topo, const double *native_xyz, const sop_params *params,
                      sop_ctx **out);

/* Advance every replica by n_steps >= 0 steps (Algorithm 7 with the forces of
 * Eq. 1, the Verlet list rebuilt at multiples of rebuild_every). Returns after
 * the work is queued and the status word has been read (one stream sync).
 * A replica whose bond breaks, whose position becomes non-finite or whose bead
 * enters the indenter is frozen and reported; the others continue. */
sop_status sop_step(sop_ctx *ctx, int64_t n_steps);

/* Forces (FP32 arithmetic) at the current positions of `replica`, with a
 * Verlet list built from those positions, and the Eq. 1 energy (FP64
 * accumulation). out_f: [3*n_beads] FP64 host (may be NULL); out_energy: one
 * double (may be NULL). Does not change the simulation state. */
sop_status sop_forces(sop_ctx *ctx, int32_t replica, double *out_f, double *out_energy);

/* Rebuild the Verlet list of every replica from the current positions now (Sec. III.A,
 * Algorithm 3: pairs within pair_cut, not bonded, not native). */
sop_status sop_pairlist_rebuild(sop_ctx *ctx);

/* Start (or replace) cantilever pulling on the listed systems (all replicas), the
 * protocol of Sec. IV.B (one end fixed, the other pulled by a spring whose end moves at
 * constant speed). Anchors become fixed. n = 0 removes all springs. */
sop_status sop_pull(sop_ctx *ctx, int32_t n, const sop_pull_params *pulls);

/* Start (or replace) a repulsive spherical indenter acting on every bead of
 * every replica (the force-indentation application of the Conclusion; the wall
 * repels with Eq. 1's (sigma/r)^6 form measured from the sphere's surface): V = eps_l (sigma / (|r - c| - radius))^6, centre c starting
 * at `center` and moving v A/step along unit `direction`. radius <= 0 removes it. */
sop_status sop_indenter(sop_ctx *ctx, const double center[3], const double direction[3], double radius,
                        double v);

/* Not in the paper (state access): positions of one replica ([3*n_beads] FP64 host),
 * or of all replicas when replica == -1 ([3*n_beads*n_replicas], replica major). */
sop_status sop_get_positions(sop_ctx *ctx, int32_t replica, double *out_xyz);
/* Not in the paper (state access): set positions (converted to FP32, compensation
 * reset; Algorithm 7's compensated sum). replica == -1 sets
 * all replicas from a [3*n_beads*n_replicas] array. The Verlet list is rebuilt from
 * the new positions at once (they replace the snapshot of the last rebuild), so a
 * list built from other positions is never used with them; the step counter, and with
 * it the cantilever tips and the indenter, is unchanged. */
sop_status sop_set_positions(sop_ctx *ctx, int32_t replica, const double *xyz);

/* Not in the paper (state access): stored velocities of the underdamped integrator (A/ps, the velocity after the O
 * sub-step of the last step), FP64 host [3*n_beads] (replica >= 0) or
 * [3*n_beads*n_replicas] (replica == -1). SOP_ERR_UNSUPPORTED for the overdamped
 * integrator. Part of the checkpoint. */
sop_status sop_get_velocities(sop_ctx *ctx, int32_t replica, double *out_v);
sop_status sop_set_velocities(sop_ctx *ctx, int32_t replica, const double *v);

/* The Verlet list of Sec. III.A (Algorithm 3) of `replica`, as canonical CSR over its
 * beads: row i holds every partner j (both directions, ascending). row_ptr: [n_beads+1]; col: [cap].
 * *nnz receives the entry count; SOP_ERR_CAPACITY when cap < nnz. */
sop_status sop_get_pairlist(sop_ctx *ctx, int32_t replica, int32_t *row_ptr, int32_t *col, int64_t cap,
                            int64_t *nnz);

/* The native contacts of Eq. 1's second term (Sec. IV.A: pairs closer than native_cut
 * in the native structure) as canonical CSR (both directions, ascending) with the FP64
 * native distance r0 of each entry. */
sop_status sop_get_native_map(sop_ctx *ctx, int32_t *row_ptr, int32_t *col, double *r0, int64_t cap,
                              int64_t *nnz);

/* The readouts of Sec. IV.B (see sop_record). Copy out and clear the records taken
 * since the last call, in
 * order of step, then replica, then system. When more records were taken than
 * the ring holds, the oldest are lost and *n_lost says how many. */
sop_status sop_get_observables(sop_ctx *ctx, sop_record *out, int64_t cap, int64_t *n_records, int64_t *n_lost);

/* Not in the paper: checkpoint and resume. Saves the step counter, positions, compensation terms, pulling and
 * indenter set-up, status, the Hybrid Taus state and the velocities (when used).
 * Resuming from it continues bit-exactly.
 * With buf == NULL, *size receives the byte count needed. */
sop_status sop_get_state(sop_ctx *ctx, void *buf, int64_t cap, int64_t *size);
sop_status sop_set_state(sop_ctx *ctx, const void *buf, int64_t size);

/* State of the Hybrid Taus generator of Sec. III.C (Algorithm 6), every bead of every
 * replica (SOP_RNG_HYBRID_TAUS only):
 * n_words = 4 * n_replicas * n_beads uint32 host words, replica-major, bead i of
 * replica r at 4 (r n_beads + i), words (y1, y2, y3, y4). sop_create seeds them from
 * params.seed with SplitMix64 (Steele, Lea, Flood, OOPSLA'14): for replica r and bead i
 * the SplitMix64 state starts at ((seed + r) << 32) + i and two outputs give
 * y1 y2 (first, low word first) and y3 y4 (second); y1 < 2, y2 < 8, y3 < 16 are raised
 * by 2, 8, 16 (a Tausworthe component needs a nonzero top k bits).
 * sop_set_rng_state rejects y1 < 2, y2 < 8 or y3 < 16 (SOP_ERR_INVALID_ARG);
 * SOP_ERR_UNSUPPORTED when the context draws from Philox, SOP_ERR_CAPACITY when
 * n_words is too small. The state is part of the checkpoint. */
sop_status sop_get_rng_state(sop_ctx *ctx, uint32_t *state, int64_t n_words);
sop_status sop_set_rng_state(sop_ctx *ctx, const uint32_t *state, int64_t n_words);

/* Accuracy of the first-order integrator (Sec. IV.C): n_runs independent Brownian
 * particles in the harmonic potential K X^2 / 2 (minimum at 0) driven by the ramp force
 * r_f t, started at X0 and advanced n_steps steps of
 *     X += (r_f t_n / xi - X / tau) h  [+ (X / (2 tau^2) - r_f t_n / (2 tau xi)) h^2]
 *          [+ r_f h^2 / (2 xi)] + sqrt(2 kT h / xi) g_n,     t_n = n h, tau = xi / K,
 * the first bracket for order >= 2 (Eq. 5 as printed), the second for order 3 (the
 * complete second-order Taylor step; Eq. 5 as printed lacks it and is first-order
 * accurate). FP32 arithmetic with a compensated (Kahan) position, one thread per run.
 * Noise: Philox4x32-10, key = seed, counter = (n/4 lo, n/4 hi, run, 1); step n takes
 * normal n mod 4 of its block (Box-Muller on (x0, x1) and (x2, x3), cosine then sine).
 * Units are the caller's (any consistent set). */
typedef struct {
    double K;          /* spring constant, > 0 */
    double xi;         /* friction, > 0 */
    double kT;         /* thermal energy, >= 0 (0: no noise) */
    double h;          /* time step, > 0 */
    double r_f;        /* loading rate of the ramp force */
    double X0;         /* position at t = 0 */
    int64_t n_runs;    /* 1 .. 2^31 - 1 */
    int64_t n_steps;   /* >= 1 */
    int32_t order;     /* 1, 2 or 3 */
    int32_t n_out;     /* checkpoints, 1 .. n_steps: after steps n_steps (k + 1) / n_out, k < n_out */
    uint64_t seed;
} sop_ramp_params;

/* Runs the experiment on the device behind cuda_stream (NULL = default stream) and
 * blocks until it ends. mean[k], var[k] (host, [n_out], FP64): mean and population
 * variance over runs of X at checkpoint k; x_final (host, [n_runs] or NULL): every
 * run's final X. X is read as the FP32 value minus its compensation, in FP64.
 * Allocates and frees its own device memory (8 bytes per run plus reduction scratch).
 * SOP_ERR_INVALID_ARG on a parameter out of range; SOP_ERR_CUDA / SOP_ERR_OOM on
 * device failure (text in sop_last_error(NULL)). */
sop_status sop_brownian_ramp(const sop_ramp_params *params, double *mean, double *var, double *x_final,
                             void *cuda_stream);

/* The noise of the step (Sec. III.C) on its own, for checking it against other
 * implementations; both calls use the device functions that every step kernel uses.
 *
 * sop_box_muller: for each k < n, the four words x[4k .. 4k + 3] (host, uint32) give three
 * standard normals out[3k .. 3k + 2] (host, FP64 widened from the FP32 results):
 * radius sqrt(-2 ln u) with u = (x0 + 1) 2^-32 in (0, 1], angle 2 pi x1 2^-32 (cosine,
 * then sine); the third normal is sqrt(-2 ln((x2 + 1) 2^-32)) cos(2 pi x3 2^-32).
 *
 * sop_bead_noise: the three normals out[3k .. 3k + 2] that the step kernels draw for bead
 * bead_lo + k at step `step` of the replica keyed by `key` (= sop_params.seed + replica):
 * Philox4x32-10 with key (key lo, key hi) and counter (step lo, step hi, bead, 0), then
 * the map above. Requires bead_lo + n <= 2^32.
 *
 * Both: 0 <= n <= 2^26; they allocate and free their own device memory on cuda_stream
 * (NULL = default stream) and synchronise it. SOP_ERR_INVALID_ARG on n or a pointer out
 * of range, SOP_ERR_CUDA / SOP_ERR_OOM on device failure (text in sop_last_error(NULL)). */
sop_status sop_box_muller(const uint32_t *x, int64_t n, double *out, void *cuda_stream);
sop_status sop_bead_noise(uint64_t key, int64_t step, uint32_t bead_lo, int64_t n, double *out, void *cuda_stream);

/* FP32 FMA throughput of the current device, the denominator of the FP32 roofline of
 * the batched kernels (the paper has no counterpart; a measurement utility). A kernel
 * of independent fmaf chains (four CTAs of 256 threads per SM, eight chains per thread)
 * runs on the default stream, its launches growing until one lasts about `seconds`
 * (0 < seconds <= 10); *tflops receives the best rate of the launches (2 FLOP per
 * FMA), *elapsed_ms (may be NULL) the duration of the last launch and *sm_count (may
 * be NULL) the SMs of the device. Allocates and frees a small output buffer.
 * SOP_ERR_INVALID_ARG on an argument out of range, SOP_ERR_CUDA on device failure
 * (text in sop_last_error(NULL)). */
sop_status sop_fp32_peak(double seconds, double *tflops, double *elapsed_ms, int32_t *sm_count);

/* Not in the paper: per-replica status ([n_replicas] int32 host), a sop_status value each
 * (a replica whose FENE bond breaks, Eq. 1, is frozen and reported here). */
sop_status sop_replica_status(sop_ctx *ctx, int32_t *out);

/* Not in the paper: ask a running sop_step to stop at the next check (thread-safe, async). */
void sop_abort(sop_ctx *ctx);

/* Not in the paper: counters and the schedule in use. */
sop_status sop_get_stats(sop_ctx *ctx, sop_stats *out);

/* Not in the paper: text of the last error of ctx (or of the last failed sop_create when ctx is NULL). */
const char *sop_last_error(const sop_ctx *ctx);

/* Not in the paper: free all device and host memory of ctx. NULL is allowed. */
void sop_destroy(sop_ctx *ctx);

/* Not in the paper: largest system sop_pairlist_build_noalloc accepts. */
#define SOP_NOALLOC_MAX_BEADS 65536

/*
 * Verlet list of one system, built without allocating any device memory.
 * The paper has no counterpart: this is an interface for callers that cannot
 * call cudaMalloc -- hosts whose device memory all belongs to their own pool
 * allocator, or services that must not allocate after start-up. It runs the
 * same cell-list rebuild as the streamed schedule on caller-provided device
 * buffers; its scratch (2.5 MiB for at most SOP_NOALLOC_MAX_BEADS beads) is a
 * fixed array inside this library that every GPU which loads the library holds
 * until the process exits.
 *
 * Inputs (device pointers, read only): pos4 [4*n] floats, bead-major (x, y, z,
 * unused), 16-byte aligned; chain [n] chain id of each bead (beads i, i+1 of
 * one chain are bonded); nat_row [n+1], nat_col: the native contact map as CSR
 * with both directions, each row ascending (as sop_get_native_map returns it;
 * a row that is not ascending may leave native partners in the list). Outputs (device
 * pointers): row_start [n], row_len [n] and col [cap]: row i is
 * col[row_start[i] .. row_start[i] + row_len[i]), ascending partner indices;
 * rows are packed in no particular order. *nnz (host) receives the number of
 * entries. The pair set equals that of sop_get_pairlist.
 *
 * Errors: SOP_ERR_INVALID_ARG when n is outside [1, SOP_NOALLOC_MAX_BEADS], a
 * pointer is NULL or misaligned, or pair_cut <= 0; SOP_ERR_PAIRLIST_OVERFLOW
 * when cap is too small or a row meets more than 256 candidates within
 * pair_cut (whatever cap is); SOP_ERR_NONFINITE when a position is NaN or
 * infinite, or when no grid of at most 2 n + 8 cells of edge >= pair_cut covers
 * the system (every row is then empty); SOP_ERR_CUDA for a CUDA failure. The
 * text is sop_last_error(NULL). The call reads its counters back and
 * synchronises cuda_stream (NULL = the legacy default stream) before it
 * returns.
 *
 * The first call on a device looks up the scratch array's device address for
 * that device (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture begins. Every call
 * shares the one scratch array and overwrites it, so calls whose GPU work
 * overlaps (two host threads, or two streams) race and must be serialised by
 * the caller.
 */
sop_status sop_pairlist_build_noalloc(const float *pos4, int32_t n, const int32_t *chain, const int32_t *nat_row,
                                      const int32_t *nat_col, double pair_cut, int32_t *row_start, int32_t *row_len,
                                      int32_t *col, int64_t cap, int64_t *nnz, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SOP_H */
