/*
 * FP64 CPU oracle for the SOP-model overdamped Langevin step.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct restatement of
 * what the simulation computes, written from the paper (Zhmurov, Dima,
 * Kholodov, Barsegov, "Langevin dynamics simulations of biomolecules on
 * graphics processors"). Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it. It shares no code, header, table or
 * constant with the CUDA library. Built with -O2 -ffp-contract=off and without
 * fast-math, so every expression is evaluated as written.
 *
 * What each function follows:
 *   orc_bonds, orc_native_pairs   Eq. 1 and Sec. IV.A (FENE bonds i,i+1 with
 *                                 native r0; native contacts |i-j|>2 within R_C)
 *   orc_pairlist_*                Sec. III.A "Verlet lists" and Algorithm 3
 *                                 (pairs closer than the cutoff)
 *   orc_forces                    Algorithm 1 (serial loop over pairs, +df to
 *                                 i and -df to j) applied to the three pair
 *                                 terms of Eq. 1; pulling as in Sec. IV.B
 *   orc_philox4x32_10, orc_noise  counter-based Philox4x32-10 as published by
 *                                 Salmon et al. (SC'11); the paper's own
 *                                 generator is Hybrid Taus (Algorithm 6)
 *   orc_taus_next, orc_taus_noise Algorithm 6 (Hybrid Taus: three Tausworthe
 *                                 generators and an LCG), Sec. III.C
 *   orc_box_muller                Sec. III.C (Box-Muller transformation)
 *   orc_ermak_update              Algorithm 7 (the first-order Ermak-McCammon
 *                                 update, Eq. 2)
 *   orc_run                       the step sequence of Fig. 2 / Sec. III.D
 *   orc_observables               the readouts of Sec. IV.B and Fig. 3: energy of
 *                                 Eq. 1, the cantilever force along the pulling
 *                                 direction and the extension, the end-to-end
 *                                 distance, and the fraction of native contacts
 *   orc_baoab_update              the underdamped limit named in the Conclusion, as the
 *                                 BAOAB splitting of Leimkuhler and Matthews (2013)
 *   orc_ramp_*                    Sec. IV.C: the harmonic Brownian particle under a
 *                                 ramp force, Eqs. 3, 4 and 5
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes): the integrator follows Algorithm 7 (r += f h/xi + g
 * sqrt(2kTh/xi)), not the garbled Eq. 2; the i,i+2 repulsion of Eq. 1 is folded
 * into the non-native list (same sigma and epsilon); the list is rebuilt at
 * steps 0, K, 2K, ... before that step's forces; a listed pair interacts with
 * no further distance test; F_i = -grad_i V; a FENE bond stretched to
 * |r - r0| >= R0 is a failure; the indenter is V = eps_l (sigma / (|r-c| -
 * R_ind))^6; a native contact counts as formed when r < r0 + 2 A; a
 * cross-link (a covalent bond joining beads other than i, i+1 of a chain, which
 * Table I counts among the covalent bonds) is one more FENE term of Eq. 1 with
 * its native length, and its two beads are neither a native contact nor a
 * Verlet-list pair (the model's bond list holds it; the lists exclude every
 * bonded partner).
 */
#include "sop_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_kB(void) { return 8.314462618 / 4184.0; }

/* |a - b|^2 evaluated as ((dx*dx + dy*dy) + dz*dz). */
static double dist2(const double *a, const double *b) {
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    double dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* ------------------------------------------------------------------------ */
/* Topology: bonds and the native map (Eq. 1, Sec. IV.A)                     */
/* ------------------------------------------------------------------------ */
int32_t orc_bonds(int32_t n, const double *xyz, const int32_t *chain, int32_t *out_i, int32_t *out_j,
                  double *out_r0) {
    int32_t nb = 0;
    for (int32_t i = 0; i + 1 < n; ++i) {
        if (chain[i] != chain[i + 1]) continue;
        out_i[nb] = i;
        out_j[nb] = i + 1;
        out_r0[nb] = sqrt(dist2(xyz + 3 * i, xyz + 3 * (i + 1)));
        ++nb;
    }
    return nb;
}

/* May i and j (i < j) form a native contact? Same system, and more than two
 * residues apart when in the same chain (Delta_ij is defined for |i-j| > 2). */
static int native_candidate(const int32_t *chain, const int32_t *sys, int32_t i, int32_t j) {
    if (sys[i] != sys[j]) return 0;
    if (chain[i] == chain[j] && j - i <= 2) return 0;
    return 1;
}

int64_t orc_native_pairs(int32_t n, const double *xyz, const int32_t *chain, const int32_t *sys, double cut,
                         int32_t *out_i, int32_t *out_j, double *out_r0, int64_t cap) {
    int64_t cnt = 0;
    double cut2 = cut * cut;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) {
            if (!native_candidate(chain, sys, i, j)) continue;
            double d2 = dist2(xyz + 3 * i, xyz + 3 * j);
            if (d2 < cut2) {
                if (cnt >= cap) return -1;
                out_i[cnt] = i;
                out_j[cnt] = j;
                out_r0[cnt] = sqrt(d2);
                ++cnt;
            }
        }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Verlet list of the repulsive term (Sec. III.A, Algorithm 3)               */
/* ------------------------------------------------------------------------ */
/* Per-bead native partners, so that "is (i, j) native" is a table lookup. */
typedef struct {
    int64_t *row;   /* [n+1] */
    int32_t *col;   /* [2*n_nat] */
} adjacency;

static int adjacency_build(int32_t n, int64_t m, const int32_t *a, const int32_t *b, adjacency *adj) {
    adj->row = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    adj->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    if (!adj->row || !adj->col) return -1;
    for (int64_t p = 0; p < m; ++p) { adj->row[a[p] + 1]++; adj->row[b[p] + 1]++; }
    for (int32_t i = 0; i < n; ++i) adj->row[i + 1] += adj->row[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!fill) return -1;
    memcpy(fill, adj->row, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t p = 0; p < m; ++p) { adj->col[fill[a[p]]++] = b[p]; adj->col[fill[b[p]]++] = a[p]; }
    free(fill);
    return 0;
}

static void adjacency_free(adjacency *adj) { free(adj->row); free(adj->col); }

/* Bonded: (i, i+1) inside one chain. Cross-links (bonds of the model's list that join
 * other pairs) are excluded through the bond adjacency instead. */
static int bonded(const orc_model *m, int32_t i, int32_t j) {
    int32_t lo = i < j ? i : j, hi = i < j ? j : i;
    return hi == lo + 1 && m->chain[lo] == m->chain[hi];
}

/* Mark (val = 1) or unmark (val = 0) the partners of bead i in adj. */
static void mark(const adjacency *adj, int32_t i, unsigned char *flag, unsigned char val) {
    for (int64_t p = adj->row[i]; p < adj->row[i + 1]; ++p) flag[adj->col[p]] = val;
}

int64_t orc_pairlist_brute(const orc_model *m, const double *xyz, int32_t *out_i, int32_t *out_j, int64_t cap) {
    int32_t n = m->n;
    adjacency adj, badj;
    if (adjacency_build(n, m->n_nat, m->nat_i, m->nat_j, &adj) != 0) return -1;
    if (adjacency_build(n, m->n_bonds, m->bond_i, m->bond_j, &badj) != 0) return -1;
    unsigned char *is_nat = (unsigned char *)calloc((size_t)n, 1);
    double cut2 = m->pair_cut * m->pair_cut;
    int64_t cnt = 0;
    for (int32_t i = 0; i < n && cnt >= 0; ++i) {
        mark(&adj, i, is_nat, 1);
        mark(&badj, i, is_nat, 1);   /* every covalent partner, cross-links included */
        for (int32_t j = i + 1; j < n; ++j) {
            if (m->sys[i] != m->sys[j] || bonded(m, i, j) || is_nat[j]) continue;
            if (dist2(xyz + 3 * i, xyz + 3 * j) < cut2) {
                if (cnt >= cap) { cnt = -1; break; }
                out_i[cnt] = i;
                out_j[cnt] = j;
                ++cnt;
            }
        }
        mark(&adj, i, is_nat, 0);
        mark(&badj, i, is_nat, 0);
    }
    free(is_nat);
    adjacency_free(&adj);
    adjacency_free(&badj);
    return cnt;
}

/* A uniform grid of cubic cells of edge >= cut over each system's bounding
 * box; beads sorted by cell. Used to enumerate candidate pairs quickly. */
typedef struct {
    int32_t n_sys;
    double *lo;          /* [3*n_sys] */
    int64_t *dims;       /* [3*n_sys] */
    int64_t *base;       /* [n_sys+1] first cell of each system */
    int64_t *start;      /* [n_cells+1] */
    int32_t *beads;      /* [n] */
    int64_t *cell_of;    /* [n] */
    double edge;
} cellgrid;

static int cellgrid_build(int32_t n, const double *xyz, const int32_t *sys, double cut, cellgrid *g) {
    int32_t ns = 0;
    for (int32_t i = 0; i < n; ++i) if (sys[i] + 1 > ns) ns = sys[i] + 1;
    g->n_sys = ns;
    g->edge = cut;
    g->lo = (double *)malloc(sizeof(double) * 3 * (size_t)ns);
    double *hi = (double *)malloc(sizeof(double) * 3 * (size_t)ns);
    g->dims = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)ns);
    g->base = (int64_t *)calloc((size_t)ns + 1, sizeof(int64_t));
    g->cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    g->beads = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!g->lo || !hi || !g->dims || !g->base || !g->cell_of || !g->beads) return -1;
    for (int32_t s = 0; s < ns; ++s)
        for (int k = 0; k < 3; ++k) { g->lo[3 * s + k] = INFINITY; hi[3 * s + k] = -INFINITY; }
    for (int32_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double x = xyz[3 * i + k];
            if (x < g->lo[3 * sys[i] + k]) g->lo[3 * sys[i] + k] = x;
            if (x > hi[3 * sys[i] + k]) hi[3 * sys[i] + k] = x;
        }
    for (int32_t s = 0; s < ns; ++s) {
        int64_t cells = 1;
        for (int k = 0; k < 3; ++k) {
            int64_t d = isfinite(g->lo[3 * s + k]) ? (int64_t)floor((hi[3 * s + k] - g->lo[3 * s + k]) / cut) + 1 : 1;
            g->dims[3 * s + k] = d;
            cells *= d;
        }
        g->base[s + 1] = g->base[s] + cells;
    }
    free(hi);
    int64_t nc = g->base[ns];
    g->start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!g->start) return -1;
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = sys[i];
        int64_t c[3];
        for (int k = 0; k < 3; ++k) {
            c[k] = (int64_t)floor((xyz[3 * i + k] - g->lo[3 * s + k]) / cut);
            if (c[k] >= g->dims[3 * s + k]) c[k] = g->dims[3 * s + k] - 1;
        }
        g->cell_of[i] = g->base[s] + (c[2] * g->dims[3 * s + 1] + c[1]) * g->dims[3 * s] + c[0];
        g->start[g->cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) g->start[c + 1] += g->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nc + 1));
    if (!fill) return -1;
    memcpy(fill, g->start, sizeof(int64_t) * ((size_t)nc + 1));
    for (int32_t i = 0; i < n; ++i) g->beads[fill[g->cell_of[i]]++] = i;
    free(fill);
    return 0;
}

static void cellgrid_free(cellgrid *g) {
    free(g->lo); free(g->dims); free(g->base); free(g->start); free(g->beads); free(g->cell_of);
}

/* All beads j > i in the 27 cells around bead i (same system). Returns count. */
static int64_t cellgrid_candidates(const cellgrid *g, const int32_t *sys, int32_t i, int32_t *buf) {
    int32_t s = sys[i];
    int64_t local = g->cell_of[i] - g->base[s];
    int64_t dx_ = g->dims[3 * s], dy_ = g->dims[3 * s + 1], dz_ = g->dims[3 * s + 2];
    int64_t cx = local % dx_, cy = (local / dx_) % dy_, cz = local / (dx_ * dy_);
    int64_t cnt = 0;
    for (int64_t z = cz - 1; z <= cz + 1; ++z) {
        if (z < 0 || z >= dz_) continue;
        for (int64_t y = cy - 1; y <= cy + 1; ++y) {
            if (y < 0 || y >= dy_) continue;
            for (int64_t x = cx - 1; x <= cx + 1; ++x) {
                if (x < 0 || x >= dx_) continue;
                int64_t c = g->base[s] + (z * dy_ + y) * dx_ + x;
                for (int64_t p = g->start[c]; p < g->start[c + 1]; ++p)
                    if (g->beads[p] > i) buf[cnt++] = g->beads[p];
            }
        }
    }
    return cnt;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_pairlist_cells(const orc_model *m, const double *xyz, int32_t *out_i, int32_t *out_j, int64_t cap) {
    int32_t n = m->n;
    cellgrid g;
    if (cellgrid_build(n, xyz, m->sys, m->pair_cut, &g) != 0) return -1;
    adjacency adj, badj;
    if (adjacency_build(n, m->n_nat, m->nat_i, m->nat_j, &adj) != 0) return -1;
    if (adjacency_build(n, m->n_bonds, m->bond_i, m->bond_j, &badj) != 0) return -1;
    unsigned char *is_nat = (unsigned char *)calloc((size_t)n + 1, 1);
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    double cut2 = m->pair_cut * m->pair_cut;
    int64_t cnt = 0;
    for (int32_t i = 0; i < n && cnt >= 0; ++i) {
        int64_t nb = cellgrid_candidates(&g, m->sys, i, buf);
        qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        mark(&adj, i, is_nat, 1);
        mark(&badj, i, is_nat, 1);
        for (int64_t q = 0; q < nb; ++q) {
            int32_t j = buf[q];
            if (bonded(m, i, j) || is_nat[j]) continue;
            if (dist2(xyz + 3 * i, xyz + 3 * j) < cut2) {
                if (cnt >= cap) { cnt = -1; break; }
                out_i[cnt] = i;
                out_j[cnt] = j;
                ++cnt;
            }
        }
        mark(&adj, i, is_nat, 0);
        mark(&badj, i, is_nat, 0);
    }
    free(buf);
    free(is_nat);
    adjacency_free(&adj);
    adjacency_free(&badj);
    cellgrid_free(&g);
    return cnt;
}

/* Native map from a cell grid (same set as orc_native_pairs, faster). */
int64_t orc_native_pairs_cells(int32_t n, const double *xyz, const int32_t *chain, const int32_t *sys, double cut,
                               int32_t *out_i, int32_t *out_j, double *out_r0, int64_t cap) {
    cellgrid g;
    if (cellgrid_build(n, xyz, sys, cut, &g) != 0) return -1;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    double cut2 = cut * cut;
    int64_t cnt = 0;
    for (int32_t i = 0; i < n && cnt >= 0; ++i) {
        int64_t nb = cellgrid_candidates(&g, sys, i, buf);
        qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < nb; ++q) {
            int32_t j = buf[q];
            if (!native_candidate(chain, sys, i, j)) continue;
            double d2 = dist2(xyz + 3 * i, xyz + 3 * j);
            if (d2 < cut2) {
                if (cnt >= cap) { cnt = -1; break; }
                out_i[cnt] = i;
                out_j[cnt] = j;
                out_r0[cnt] = sqrt(d2);
                ++cnt;
            }
        }
    }
    free(buf);
    cellgrid_free(&g);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Forces: Algorithm 1 over the three pair terms of Eq. 1                     */
/* ------------------------------------------------------------------------ */
/* Scatter a pair increment: f[i] += df, f[j] -= df (Algorithm 1). The scale
 * a >= 0 goes to both beads' rounding-scale accumulator. */
static void scatter(double *F, double *A, int32_t i, int32_t j, const double d[3], double coef, double acoef) {
    for (int k = 0; k < 3; ++k) {
        double df = coef * d[k];
        F[3 * i + k] += df;
        F[3 * j + k] -= df;
        if (A) {
            double a = acoef * fabs(d[k]);
            A[3 * i + k] += a;
            A[3 * j + k] += a;
        }
    }
}

int orc_forces(const orc_model *m, const double *xyz, int64_t n_pl, const int32_t *pl_i, const int32_t *pl_j,
               int64_t step, double *F, double *A, double *E_parts) {
    int32_t n = m->n;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (A) memset(A, 0, sizeof(double) * 3 * (size_t)n);
    double e_fene = 0.0, e_nat = 0.0, e_rep = 0.0, e_wall = 0.0;
    const double R02 = m->R0 * m->R0;

    /* FENE: V = -(k/2) R0^2 log(1 - (r - r0)^2 / R0^2).
     * -dV/dr = -k (r - r0) / (1 - (r - r0)^2 / R0^2); F_i = (-dV/dr) d / r. */
    for (int32_t b = 0; b < m->n_bonds; ++b) {
        int32_t i = m->bond_i[b], j = m->bond_j[b];
        double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1], xyz[3 * i + 2] - xyz[3 * j + 2]};
        double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        double dr = r - m->bond_r0[b];
        double arg = 1.0 - dr * dr / R02;
        if (!(arg > 0.0)) return ORC_ERR_FENE_BREAK;
        e_fene += -0.5 * m->k_fene * R02 * log(arg);
        double coef = -m->k_fene * dr / arg / r;
        double acoef = m->k_fene * (r + m->bond_r0[b]) / arg / r;
        scatter(F, A, i, j, d, coef, acoef);
    }

    /* Native attraction: V = eps_h [(r0/r)^12 - 2 (r0/r)^6].
     * F_i = (12 eps_h / r^2) [s^6 - s^3] d with s = (r0/r)^2. */
    for (int64_t p = 0; p < m->n_nat; ++p) {
        int32_t i = m->nat_i[p], j = m->nat_j[p];
        double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1], xyz[3 * i + 2] - xyz[3 * j + 2]};
        double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        double s = m->nat_r0[p] * m->nat_r0[p] / r2;
        double s3 = s * s * s;
        double s6 = s3 * s3;
        e_nat += m->eps_h * (s6 - 2.0 * s3);
        double coef = 12.0 * m->eps_h / r2 * (s6 - s3);
        double acoef = 12.0 * m->eps_h / r2 * (s6 + s3);
        scatter(F, A, i, j, d, coef, acoef);
    }

    /* Non-native repulsion over the Verlet list: V = eps_l (sigma/r)^6.
     * F_i = (6 eps_l / r^2) (sigma^2/r^2)^3 d. */
    for (int64_t p = 0; p < n_pl; ++p) {
        int32_t i = pl_i[p], j = pl_j[p];
        double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1], xyz[3 * i + 2] - xyz[3 * j + 2]};
        double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        double q = m->sigma * m->sigma / r2;
        double q3 = q * q * q;
        e_rep += m->eps_l * q3;
        double coef = 6.0 * m->eps_l / r2 * q3;
        scatter(F, A, i, j, d, coef, coef);
    }

    /* Cantilever (Sec. IV.B): tip at tip0 + v (step - n0) dir, spring k_s on the pulled bead. */
    for (int32_t p = 0; p < m->n_pull; ++p) {
        const orc_pull *pl = &m->pulls[p];
        double t = pl->v * (double)(step - pl->n0);
        for (int k = 0; k < 3; ++k) {
            double tip = pl->tip0[k] + t * pl->dir[k];
            double x = xyz[3 * pl->pulled + k];
            F[3 * pl->pulled + k] += pl->k_s * (tip - x);
            if (A) A[3 * pl->pulled + k] += pl->k_s * (fabs(tip) + fabs(x));
        }
    }

    /* Indenter: V = eps_l (sigma / rho)^6 with rho = |r - c| - R_ind, on every bead. */
    if (m->indenter) {
        const orc_indenter *in = m->indenter;
        double t = in->v * (double)(step - in->n0);
        double c[3] = {in->c0[0] + t * in->dir[0], in->c0[1] + t * in->dir[1], in->c0[2] + t * in->dir[2]};
        for (int32_t i = 0; i < n; ++i) {
            double e[3] = {xyz[3 * i] - c[0], xyz[3 * i + 1] - c[1], xyz[3 * i + 2] - c[2]};
            double r = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
            double rho = r - in->radius;
            if (!(rho > 0.0)) return ORC_ERR_INDENTER_OVERLAP;
            double q = m->sigma / rho;
            double q2 = q * q;
            double q6 = q2 * q2 * q2;
            e_wall += m->eps_l * q6;
            double coef = 6.0 * m->eps_l * q6 / rho / r;
            double acoef = 6.0 * m->eps_l * q6 / rho * (r + in->radius) / rho / r;
            for (int k = 0; k < 3; ++k) {
                F[3 * i + k] += coef * e[k];
                if (A) A[3 * i + k] += acoef * fabs(e[k]);
            }
        }
    }
    if (E_parts) { E_parts[0] = e_fene; E_parts[1] = e_nat; E_parts[2] = e_rep; E_parts[3] = e_wall; }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Random force: Philox4x32-10 + Box-Muller (Sec. III.C)                     */
/* ------------------------------------------------------------------------ */
/* Philox4x32: each of the 10 rounds multiplies words 0 and 2 by fixed odd
 * constants, swaps the halves of the products across lanes and mixes in the
 * key; the key is advanced by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u1 = (x0 + 1) 2^-32 in (0, 1], u2 = x1 2^-32 in [0, 1);
 * g0 = sqrt(-2 ln u1) cos(2 pi u2), g1 = sqrt(-2 ln u1) sin(2 pi u2);
 * g2 from (x2, x3) like g0. The fourth normal is not used. */
void orc_box_muller(const uint32_t x[4], double g[3]) {
    const double two_m32 = 1.0 / 4294967296.0;
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = ((double)x[0] + 1.0) * two_m32;
    double u2 = (double)x[1] * two_m32;
    double u3 = ((double)x[2] + 1.0) * two_m32;
    double u4 = (double)x[3] * two_m32;
    double ra = sqrt(-2.0 * log(u1));
    double rb = sqrt(-2.0 * log(u3));
    g[0] = ra * cos(two_pi * u2);
    g[1] = ra * sin(two_pi * u2);
    g[2] = rb * cos(two_pi * u4);
}

/* One step of a Tausworthe component (L'Ecuyer's shift form of a trinomial
 * recurrence of degree k): b = ((y << q) ^ y) >> (k - s); y = ((y & mask) << s) ^ b,
 * mask keeping the top k bits. The three components of Algorithm 6, read as
 * (q, k - s, s, mask): (13, 19, 12, 4294967294), (2, 25, 4, 4294967288),
 * (3, 11, 17, 4294967280); the listing's subscripts are garbled, and these are
 * the values of L'Ecuyer's taus88, degrees k = 31, 29, 28 (periods 2^31-1,
 * 2^29-1, 2^28-1; the text gives 2^30-1 for the second). */
static uint32_t taus_component(uint32_t y, int q, int k_minus_s, int s, uint32_t mask) {
    uint32_t b = ((y << q) ^ y) >> k_minus_s;
    return ((y & mask) << s) ^ b;
}

uint32_t orc_taus_next(uint32_t s[4]) {
    s[0] = taus_component(s[0], 13, 19, 12, 4294967294u);
    s[1] = taus_component(s[1], 2, 25, 4, 4294967288u);
    s[2] = taus_component(s[2], 3, 11, 17, 4294967280u);
    s[3] = 1664525u * s[3] + 1013904223u;   /* LCG modulo 2^32 */
    return s[0] ^ s[1] ^ s[2] ^ s[3];
}

void orc_taus_noise(uint32_t s[4], double g[3]) {
    uint32_t x[4];
    for (int k = 0; k < 4; ++k) x[k] = orc_taus_next(s);
    orc_box_muller(x, g);
}

/* Key = the replica's 64-bit seed; counter = (step lo, step hi, bead, 0). */
void orc_noise(uint64_t seed, int64_t step, int32_t bead, double g[3]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t s = (uint64_t)step;
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)bead, 0u};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    orc_box_muller(x, g);
}

/* ------------------------------------------------------------------------ */
/* Integration: Algorithm 7                                                  */
/* ------------------------------------------------------------------------ */
static int is_held(const orc_model *m, int32_t i) {
    if (m->fixed && m->fixed[i]) return 1;
    for (int32_t p = 0; p < m->n_pull; ++p)
        if (m->pulls[p].anchor == i) return 1;
    return 0;
}

void orc_ermak_update(const orc_model *m, double *xyz, const double *F, uint64_t seed, int64_t step) {
    double kT = orc_kB() * m->T;
    double mob = m->dt / m->zeta;
    double amp = sqrt(2.0 * kT * m->dt / m->zeta);
    for (int32_t i = 0; i < m->n; ++i) {
        if (is_held(m, i)) continue;
        double g[3];
        if (m->taus) orc_taus_noise(m->taus + 4 * (size_t)i, g);
        else orc_noise(seed, step, i + m->noise_offset, g);
        for (int k = 0; k < 3; ++k) xyz[3 * i + k] = xyz[3 * i + k] + F[3 * i + k] * mob + g[k] * amp;
    }
}

void orc_baoab_update(const orc_model *m, double *xyz, const double *F, uint64_t seed, int64_t step) {
    double kT = orc_kB() * m->T;
    double h = m->dt;
    double c1 = exp(-m->zeta * h / m->mass);
    double c2 = sqrt(kT * (1.0 - c1 * c1) / m->mass);
    for (int32_t i = 0; i < m->n; ++i) {
        if (is_held(m, i)) continue;
        double g[3];
        if (m->taus) orc_taus_noise(m->taus + 4 * (size_t)i, g);
        else orc_noise(seed, step, i + m->noise_offset, g);
        for (int k = 0; k < 3; ++k) {
            double v1 = m->vel[3 * i + k] + h / m->mass * F[3 * i + k];
            double x = xyz[3 * i + k] + 0.5 * h * v1;
            double v2 = c1 * v1 + c2 * g[k];
            xyz[3 * i + k] = x + 0.5 * h * v2;
            m->vel[3 * i + k] = v2;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Integrator accuracy: Sec. IV.C, Eqs. 3-5                                  */
/* ------------------------------------------------------------------------ */
double orc_ramp_theory(const orc_ramp *p, double t) {
    double tau = p->xi / p->K;
    double e = exp(-t / tau);
    return p->X0 * e + p->r_f * tau / p->xi * (t - tau * (1.0 - e));
}

/* drift of one step at X and t_n: Eq. 4's increment, plus Eq. 5's h^2 term (order 2),
 * plus the h^2 term of the ramp's own time derivative (order 3: the full Taylor step
 * X'' h^2 / 2 with X'' = r_f / xi - X' / tau) */
static double ramp_drift(const orc_ramp *p, double X, double t) {
    double tau = p->xi / p->K;
    double d = (p->r_f * t / p->xi - X / tau) * p->h;
    if (p->order >= 2) d += (X / (2.0 * tau * tau) - p->r_f * t / (2.0 * tau * p->xi)) * p->h * p->h;
    if (p->order == 3) d += p->r_f / (2.0 * p->xi) * p->h * p->h;
    return d;
}

double orc_ramp_mean(const orc_ramp *p, int64_t n) {
    double X = p->X0;
    for (int64_t k = 0; k < n; ++k) X = X + ramp_drift(p, X, (double)k * p->h);
    return X;
}

void orc_box_muller4(const uint32_t x[4], double g[4]) {
    const double two_m32 = 1.0 / 4294967296.0;
    const double two_pi = 6.283185307179586476925286766559;
    double ra = sqrt(-2.0 * log(((double)x[0] + 1.0) * two_m32));
    double rb = sqrt(-2.0 * log(((double)x[2] + 1.0) * two_m32));
    g[0] = ra * cos(two_pi * (double)x[1] * two_m32);
    g[1] = ra * sin(two_pi * (double)x[1] * two_m32);
    g[2] = rb * cos(two_pi * (double)x[3] * two_m32);
    g[3] = rb * sin(two_pi * (double)x[3] * two_m32);
}

double orc_ramp_run(const orc_ramp *p, uint64_t seed, int64_t run, int64_t n_steps) {
    double amp = sqrt(2.0 * p->kT * p->h / p->xi);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double X = p->X0, g[4] = {0, 0, 0, 0};
    for (int64_t n = 0; n < n_steps; ++n) {
        if (n % 4 == 0) {
            uint64_t b = (uint64_t)(n / 4);
            uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), (uint32_t)run, 1u};
            uint32_t x[4];
            orc_philox4x32_10(ctr, key, x);
            orc_box_muller4(x, g);
        }
        X = X + ramp_drift(p, X, (double)n * p->h) + amp * g[n % 4];
    }
    return X;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */
int orc_observables(const orc_model *m, const double *xyz, int64_t n_pl, const int32_t *pl_i,
                    const int32_t *pl_j, int64_t step, int32_t n_systems, double *out) {
    int32_t n = m->n;
    double *E = (double *)calloc((size_t)n_systems, sizeof(double));
    double *fx = (double *)calloc((size_t)n_systems, sizeof(double));
    double *ex = (double *)calloc((size_t)n_systems, sizeof(double));
    double *fw = (double *)calloc((size_t)n_systems, sizeof(double));
    int *pulled = (int *)calloc((size_t)n_systems, sizeof(int));
    int64_t *qf = (int64_t *)calloc((size_t)n_systems, sizeof(int64_t));
    int64_t *qn = (int64_t *)calloc((size_t)n_systems, sizeof(int64_t));
    if (!E || !fx || !ex || !fw || !pulled || !qf || !qn) return ORC_ERR_ARG;
    const double R02 = m->R0 * m->R0;
    int rc = ORC_OK;
    for (int32_t b = 0; b < m->n_bonds; ++b) {
        int32_t i = m->bond_i[b], j = m->bond_j[b];
        double r = sqrt(dist2(xyz + 3 * i, xyz + 3 * j));
        double dr = r - m->bond_r0[b];
        double arg = 1.0 - dr * dr / R02;
        if (!(arg > 0.0)) { rc = ORC_ERR_FENE_BREAK; continue; }
        E[m->sys[i]] += -0.5 * m->k_fene * R02 * log(arg);
    }
    for (int64_t p = 0; p < m->n_nat; ++p) {
        int32_t i = m->nat_i[p], j = m->nat_j[p];
        double r2 = dist2(xyz + 3 * i, xyz + 3 * j);
        double s = m->nat_r0[p] * m->nat_r0[p] / r2;
        double s3 = s * s * s;
        E[m->sys[i]] += m->eps_h * (s3 * s3 - 2.0 * s3);
        qn[m->sys[i]] += 1;
        if (sqrt(r2) < m->nat_r0[p] + 2.0) qf[m->sys[i]] += 1;
    }
    for (int64_t p = 0; p < n_pl; ++p) {
        int32_t i = pl_i[p], j = pl_j[p];
        double q = m->sigma * m->sigma / dist2(xyz + 3 * i, xyz + 3 * j);
        E[m->sys[i]] += m->eps_l * q * q * q;
    }
    for (int32_t p = 0; p < m->n_pull; ++p) {
        const orc_pull *pl = &m->pulls[p];
        double t = pl->v * (double)(step - pl->n0);
        double f = 0.0;
        for (int k = 0; k < 3; ++k)
            f += pl->k_s * (pl->tip0[k] + t * pl->dir[k] - xyz[3 * pl->pulled + k]) * pl->dir[k];
        fx[pl->system] = f;
        ex[pl->system] = sqrt(dist2(xyz + 3 * pl->pulled, xyz + 3 * pl->anchor));
        pulled[pl->system] = 1;
    }
    if (m->indenter) {
        const orc_indenter *in = m->indenter;
        double t = in->v * (double)(step - in->n0);
        double c[3] = {in->c0[0] + t * in->dir[0], in->c0[1] + t * in->dir[1], in->c0[2] + t * in->dir[2]};
        for (int32_t i = 0; i < n; ++i) {
            double e[3] = {xyz[3 * i] - c[0], xyz[3 * i + 1] - c[1], xyz[3 * i + 2] - c[2]};
            double r = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
            double rho = r - in->radius;
            if (!(rho > 0.0)) { rc = ORC_ERR_INDENTER_OVERLAP; continue; }
            double q = m->sigma / rho;
            double q2 = q * q;
            double q6 = q2 * q2 * q2;
            double coef = 6.0 * m->eps_l * q6 / rho / r;
            fw[m->sys[i]] += coef * ((e[0] * in->dir[0] + e[1] * in->dir[1]) + e[2] * in->dir[2]);
        }
        /* a system on a cantilever reports its spring; every other one the indenter's
           push along its motion and the distance the indenter has travelled */
        for (int32_t s = 0; s < n_systems; ++s)
            if (!pulled[s]) { fx[s] = fw[s]; ex[s] = t; }
    }
    /* first chain of each system: from the system's first bead to the last bead of that chain */
    int32_t *first = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_systems);
    int32_t *last = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_systems);
    if (!first || !last) return ORC_ERR_ARG;
    for (int32_t s = 0; s < n_systems; ++s) first[s] = last[s] = -1;
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = m->sys[i];
        if (first[s] < 0) first[s] = i;
        if (m->chain[i] == m->chain[first[s]]) last[s] = i;
    }
    for (int32_t s = 0; s < n_systems; ++s) {
        double *o = out + 8 * (size_t)s;
        o[0] = (double)step;
        o[1] = (double)s;
        o[2] = E[s];
        o[3] = fx[s];
        o[4] = ex[s];
        o[5] = qn[s] > 0 ? (double)qf[s] / (double)qn[s] : 0.0;
        o[6] = first[s] >= 0 ? sqrt(dist2(xyz + 3 * first[s], xyz + 3 * last[s])) : 0.0;
        o[7] = 0.0;
    }
    free(first); free(last);
    free(E); free(fx); free(ex); free(fw); free(pulled); free(qf); free(qn);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The step sequence                                                         */
/* ------------------------------------------------------------------------ */
static int64_t build_list(const orc_model *m, const double *xyz, int32_t *pi, int32_t *pj, int64_t cap) {
    return m->use_cells ? orc_pairlist_cells(m, xyz, pi, pj, cap) : orc_pairlist_brute(m, xyz, pi, pj, cap);
}

int orc_run(const orc_model *m, double *xyz, int64_t step0, int64_t n_steps, uint64_t seed, int32_t n_systems,
            int32_t obs_every, double *obs, int64_t obs_cap, int64_t *n_obs, int64_t *fail_step) {
    int32_t n = m->n;
    int32_t K = m->rebuild_every;
    if (n <= 0 || K <= 0 || step0 % K != 0) return ORC_ERR_ARG;
    if (n_obs) *n_obs = 0;
    if (fail_step) *fail_step = -1;
    /* capacity: a bead has fewer than 512 partners within any sane cutoff */
    int64_t cap = (int64_t)n * 512;
    int32_t *pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *pj = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!pi || !pj || !F) { free(pi); free(pj); free(F); return ORC_ERR_ARG; }
    int rc = ORC_OK;
    int64_t n_pl = 0, list_step = -1, written = 0, step;
    for (step = step0; step < step0 + n_steps; ++step) {
        if (step % K == 0 && list_step != step) {
            n_pl = build_list(m, xyz, pi, pj, cap);
            if (n_pl < 0) { rc = ORC_ERR_CAPACITY; break; }
            list_step = step;
        }
        rc = orc_forces(m, xyz, n_pl, pi, pj, step, F, NULL, NULL);
        if (rc != ORC_OK) break;
        if (m->integrator == 1) orc_baoab_update(m, xyz, F, seed, step);
        else orc_ermak_update(m, xyz, F, seed, step);
        for (int64_t k = 0; k < 3 * (int64_t)n; ++k)
            if (!isfinite(xyz[k])) { rc = ORC_ERR_NONFINITE; break; }
        if (rc != ORC_OK) break;
        int64_t s = step + 1;
        if (obs_every > 0 && s % obs_every == 0 && obs) {
            if (s % K == 0 && list_step != s) {
                n_pl = build_list(m, xyz, pi, pj, cap);
                if (n_pl < 0) { rc = ORC_ERR_CAPACITY; break; }
                list_step = s;
            }
            if (written + n_systems > obs_cap) { rc = ORC_ERR_CAPACITY; break; }
            rc = orc_observables(m, xyz, n_pl, pi, pj, s, n_systems, obs + 8 * (size_t)written);
            if (rc != ORC_OK) break;
            written += n_systems;
        }
    }
    if (rc != ORC_OK && fail_step) *fail_step = step;
    if (n_obs) *n_obs = written;
    free(pi); free(pj); free(F);
    return rc;
}
