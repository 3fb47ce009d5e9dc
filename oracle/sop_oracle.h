/*
 * FP64 CPU oracle for the SOP-model overdamped Langevin step.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct
 * restatement of what the simulation computes, used to check the CUDA path.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it. It shares no code, header or constant with the CUDA library.
 *
 * Units: A, kcal/mol, ps, K. Bead indices are 0-based.
 */
#ifndef SOP_ORACLE_H
#define SOP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cantilever on one system (Sec. IV.B: N-terminus fixed, C-terminus pulled). */
typedef struct {
    int32_t system;        /* system the spring acts on */
    int32_t anchor;        /* bead held fixed */
    int32_t pulled;        /* bead the spring acts on */
    double k_s;            /* spring constant, kcal/mol/A^2 */
    double v;              /* tip speed, A/step */
    double dir[3];         /* unit pulling direction */
    double tip0[3];        /* tip position at step n0 */
    int64_t n0;            /* step at which pulling started */
} orc_pull;

/* Repulsive spherical indenter (force-indentation runs, Conclusion). */
typedef struct {
    double c0[3];          /* centre at step n0 */
    double dir[3];         /* unit direction of motion */
    double radius;         /* A */
    double v;              /* A/step */
    int64_t n0;
} orc_indenter;

typedef struct {
    /* topology of one replica */
    int32_t n;                       /* beads */
    const int32_t *chain;            /* [n] chain id; chains are contiguous ranges */
    const int32_t *sys;              /* [n] system id; different systems never interact */
    const uint8_t *fixed;            /* [n] 1 = never moved; may be NULL */
    int32_t n_bonds;                 /* FENE bonds: (i, i+1) within chains, then any cross-links */
    const int32_t *bond_i, *bond_j;
    const double *bond_r0;
    int64_t n_nat;                   /* native contacts, i < j */
    const int32_t *nat_i, *nat_j;
    const double *nat_r0;
    /* Eq. 1 parameters */
    double k_fene, R0, eps_h, eps_l, sigma;
    /* Langevin parameters */
    double T, zeta, dt;
    /* Verlet list */
    double pair_cut;
    int32_t rebuild_every;
    int32_t use_cells;               /* 0: brute-force list (the definition), 1: cell list */
    int32_t noise_offset;            /* added to the bead index in the noise counter (a chain
                                        checked out of a larger topology keeps its draws) */
    /* external forces */
    int32_t n_pull;
    const orc_pull *pulls;
    const orc_indenter *indenter;    /* may be NULL */
    /* noise source: NULL = Philox4x32-10 keyed by the replica seed; else the Hybrid
     * Taus state of every bead ([n][4] words y1..y4), advanced in place */
    uint32_t *taus;
    /* integrator: 0 = overdamped first-order update (Algorithm 7); 1 = underdamped
     * Langevin dynamics by the BAOAB splitting (Leimkuhler and Matthews, 2013) with
     * bead mass `mass` and friction coefficient zeta; `vel` ([n][3]) holds each bead's
     * velocity after the O step of the previous step (0 at the start), advanced in place */
    int32_t integrator;
    double mass;
    double *vel;
} orc_model;

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,
    ORC_ERR_CAPACITY = 2,
    ORC_ERR_FENE_BREAK = 3,
    ORC_ERR_INDENTER_OVERLAP = 4,
    ORC_ERR_NONFINITE = 5
};

/* Boltzmann constant in kcal/(mol K): the molar gas constant
 * 8.314462618 J/(mol K) divided by 4184 J/kcal. */
double orc_kB(void);

/* Bonds (i, i+1) of every chain, r0 = native distance. Returns the count. */
int32_t orc_bonds(int32_t n, const double *xyz, const int32_t *chain, int32_t *out_i, int32_t *out_j,
                  double *out_r0);

/* Native contacts: pairs i < j of one system with |i-j| > 2 inside a chain (or
 * in different chains) and native distance below `cut`. Returns the count, or
 * -1 when cap is too small. */
int64_t orc_native_pairs(int32_t n, const double *xyz, const int32_t *chain, const int32_t *sys, double cut,
                         int32_t *out_i, int32_t *out_j, double *out_r0, int64_t cap);

/* The same set from a uniform cell grid (faster; must equal orc_native_pairs). */
int64_t orc_native_pairs_cells(int32_t n, const double *xyz, const int32_t *chain, const int32_t *sys, double cut,
                               int32_t *out_i, int32_t *out_j, double *out_r0, int64_t cap);

/* Verlet list of the non-native repulsion: pairs i < j of one system that are
 * not bonded, not native and closer than m->pair_cut. Brute force over all
 * pairs (the definition). Sorted by (i, j). Returns count or -1 (cap). */
int64_t orc_pairlist_brute(const orc_model *m, const double *xyz, int32_t *out_i, int32_t *out_j, int64_t cap);

/* The same set from a uniform cell grid (faster; must equal the brute force). */
int64_t orc_pairlist_cells(const orc_model *m, const double *xyz, int32_t *out_i, int32_t *out_j, int64_t cap);

/* Forces F = -grad V of Eq. 1 over bonds, natives and the given list, plus the
 * external forces at step `step`. F and A are [3n]; A (may be NULL) receives,
 * per component, the sum over terms of the term evaluated with every
 * subtraction replaced by an addition of magnitudes (a bound on rounding
 * error scale). E_parts (may be NULL) receives [FENE, native, repulsion,
 * indenter wall]. Returns ORC_OK or an error. */
int orc_forces(const orc_model *m, const double *xyz, int64_t n_pl, const int32_t *pl_i, const int32_t *pl_j,
               int64_t step, double *F, double *A, double *E_parts);

/* Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Three standard normals from one Philox block by Box-Muller. */
void orc_box_muller(const uint32_t x[4], double g[3]);

/* Hybrid Taus (Algorithm 6): one output of the generator with state s = (y1, y2,
 * y3, y4): the three Tausworthe components and the LCG each take one step and the
 * output is y1 ^ y2 ^ y3 ^ y4 (as an integer; times 2^-32 it is the uniform). */
uint32_t orc_taus_next(uint32_t s[4]);

/* Three standard normals from four successive Hybrid Taus outputs (Box-Muller as
 * for a Philox block), advancing s by four outputs. */
void orc_taus_noise(uint32_t s[4], double g[3]);

/* Gaussian vector of bead `bead` at step `step` for the replica keyed by seed. */
void orc_noise(uint64_t seed, int64_t step, int32_t bead, double g[3]);

/* One first-order (Ermak-McCammon) update of all non-fixed beads given forces F:
 * r += F h/zeta + g sqrt(2 kT h / zeta), g from orc_noise(seed, step, i), or from
 * the bead's Hybrid Taus state when m->taus is set (only moved beads draw). */
void orc_ermak_update(const orc_model *m, double *xyz, const double *F, uint64_t seed, int64_t step);

/* Accuracy of the integrator (Sec. IV.C): a Brownian particle in the harmonic
 * potential K X^2 / 2 driven by the ramp force r_f t, started at X0 (the reading:
 * the minimum is at 0 and X0 is the start, as Eqs. 3-5 have it). tau = xi / K. */
typedef struct {
    double K, xi, kT, h, r_f, X0;
    int32_t order;                   /* 1: Eq. 4; 2: Eq. 5 as printed; 3: Eq. 5 with the r_f h^2 / (2 xi)
                                        term of the second-order Taylor step, which the printed
                                        equation lacks (without it the scheme is first order) */
} orc_ramp;

/* Eq. 3: X0 e^(-t/tau) + (r_f tau / xi)(t - tau (1 - e^(-t/tau))). */
double orc_ramp_theory(const orc_ramp *p, double t);

/* The mean after n steps: Eq. 4 (or Eq. 5) iterated from X0 with t_n = n h. */
double orc_ramp_mean(const orc_ramp *p, int64_t n);

/* Four standard normals from one Philox block (Box-Muller on (x0, x1) and (x2, x3),
 * cosine then sine of each pair). */
void orc_box_muller4(const uint32_t x[4], double g[4]);

/* One stochastic run (`run` = its index): X += drift_n + sqrt(2 kT h / xi) g_n, with
 * g_n normal n % 4 of the Philox block of key seed, counter (n/4 lo, n/4 hi, run, 1).
 * Returns X after n_steps. */
double orc_ramp_run(const orc_ramp *p, uint64_t seed, int64_t run, int64_t n_steps);

/* One underdamped step (m->integrator == 1) of all non-fixed beads from x_n with
 * forces F = F(x_n) and stored velocities w = m->vel: the B, A, O, A sub-steps of
 * BAOAB with the closing B of the previous step merged into this step's opening B:
 *   v' = w + (h / m) F        (the previous step's closing half kick and this one's opening)
 *   x  = x + (h / 2) v'
 *   v'' = c1 v' + c2 g,  c1 = exp(-zeta h / m), c2 = sqrt(kT (1 - c1^2) / m)
 *   x  = x + (h / 2) v'',  w = v''
 * so the first step from w = 0 starts from the velocity (h / 2m) F(x_0). */
void orc_baoab_update(const orc_model *m, double *xyz, const double *F, uint64_t seed, int64_t step);

/* Observables of every system at positions xyz and step `step`. Per system 8
 * doubles: step, system, energy (Eq. 1 over the list), external force, extension,
 * fraction of native contacts Q (r < r0 + 2 A), end-to-end distance of the
 * system's first chain (its first bead to that chain's last bead), 0.
 * External force and extension: a system on a cantilever (Sec. IV.B) gives
 * k_s (X_tip(n) - r_pulled) . d with X_tip(n) = tip0 + v (n - n0) d, and
 * |r_pulled - r_anchor|; any other system, when an indenter is set, gives the sum
 * over its beads of the wall force projected on the indenter's direction of
 * motion, and the distance v (n - n0) the indenter has travelled; else 0, 0. */
int orc_observables(const orc_model *m, const double *xyz, int64_t n_pl, const int32_t *pl_i,
                    const int32_t *pl_j, int64_t step, int32_t n_systems, double *out);

/* Run n_steps steps of one replica from step0 (a multiple of rebuild_every):
 * at each step n, rebuild the list when n % rebuild_every == 0, compute forces,
 * update. After the update to step n+1, when obs_every > 0 and (n+1) % obs_every
 * == 0, append one record per system to obs (capacity obs_cap records).
 * Returns ORC_OK or an error; *n_obs receives the records written;
 * *fail_step the step of the first error. */
int orc_run(const orc_model *m, double *xyz, int64_t step0, int64_t n_steps, uint64_t seed, int32_t n_systems,
            int32_t obs_every, double *obs, int64_t obs_cap, int64_t *n_obs, int64_t *fail_step);

#ifdef __cplusplus
}
#endif
#endif
