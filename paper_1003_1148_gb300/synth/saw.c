/*
 * Seeded synthetic inputs for the SOP-model workloads: compact self-avoiding
 * random walks that stand in for the Calpha traces of the paper's PDB systems
 * (Table I), which are not available here.
 *
 * A walk places beads one after another. Consecutive beads are exactly `bond`
 * apart (3.8 A, the Calpha-Calpha virtual bond). Each new bead goes in a
 * uniformly random direction from its predecessor and is rejected when it lies
 * outside the confinement region or closer than `min_dist` to any bead already
 * placed other than that predecessor. After `TRIES` rejections in a row the
 * walk backs up, removing 1, 2, 4, ... 64 of the most recent beads.
 *
 * The confinement region sets the density: a sphere, a cylinder (fiber-like
 * chains) or one angular cell of a spherical shell (one copy of an assembly;
 * copies are grown one after another in a shared grid so that they also avoid
 * each other).
 *
 * Random numbers: xoshiro256** seeded through SplitMix64, both as published by
 * Blackman and Vigna ("Scrambled linear pseudorandom number generators", ACM
 * TOMS 2021). Nothing in this file computes any part of the simulation method;
 * it only makes coordinates.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TRIES 64
#define MAX_BACK_LOG2 6

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xoshiro_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_uniform(rng_t *r) { return (double)(xoshiro_next(r) >> 11) * 0x1.0p-53; }

static void rng_unit_vector(rng_t *r, double v[3]) {
    double z = 2.0 * rng_uniform(r) - 1.0;
    double phi = 2.0 * M_PI * rng_uniform(r);
    double s = sqrt(fmax(0.0, 1.0 - z * z));
    v[0] = s * cos(phi);
    v[1] = s * sin(phi);
    v[2] = z;
}

/* ---------------- confinement regions ---------------- */
enum { REGION_SPHERE = 0, REGION_CYLINDER = 1, REGION_SHELL_CELL = 2 };

typedef struct {
    int kind;
    double a, b;          /* sphere: a = radius; cylinder: a = radius, b = half length (z axis);
                             shell cell: a = inner radius, b = outer radius */
    const double *dirs;   /* shell cell: unit vectors of all cells */
    int n_dirs, cell;     /* shell cell: number of cells, this copy's cell */
} region_t;

static int region_inside(const region_t *g, const double p[3]) {
    double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    switch (g->kind) {
    case REGION_SPHERE:
        return r2 <= g->a * g->a;
    case REGION_CYLINDER:
        return (p[0] * p[0] + p[1] * p[1] <= g->a * g->a) && fabs(p[2]) <= g->b;
    case REGION_SHELL_CELL: {
        if (r2 < g->a * g->a || r2 > g->b * g->b) return 0;
        int best = 0;
        double bd = -2.0;
        for (int k = 0; k < g->n_dirs; ++k) {
            double d = p[0] * g->dirs[3 * k] + p[1] * g->dirs[3 * k + 1] + p[2] * g->dirs[3 * k + 2];
            if (d > bd) { bd = d; best = k; }
        }
        return best == g->cell;
    }
    }
    return 0;
}

/* ---------------- hashed uniform grid for the clash test ---------------- */
typedef struct {
    int32_t *head, *next;
    uint32_t mask;
    double cell;
} grid_t;

static int grid_init(grid_t *gr, int32_t n_total, double cell) {
    uint32_t t = 1024;
    while (t < 4u * (uint32_t)n_total) t <<= 1;
    gr->head = (int32_t *)malloc(sizeof(int32_t) * t);
    gr->next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_total);
    if (!gr->head || !gr->next) return -1;
    for (uint32_t i = 0; i < t; ++i) gr->head[i] = -1;
    gr->mask = t - 1;
    gr->cell = cell;
    return 0;
}

static void grid_free(grid_t *gr) { free(gr->head); free(gr->next); }

static uint32_t grid_hash(int64_t cx, int64_t cy, int64_t cz, uint32_t mask) {
    uint32_t h = (uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u;
    return h & mask;
}

static void grid_cell_of(const grid_t *gr, const double p[3], int64_t c[3]) {
    for (int k = 0; k < 3; ++k) c[k] = (int64_t)floor(p[k] / gr->cell);
}

static void grid_insert(grid_t *gr, const double *xyz, int32_t i) {
    int64_t c[3];
    grid_cell_of(gr, xyz + 3 * (size_t)i, c);
    uint32_t h = grid_hash(c[0], c[1], c[2], gr->mask);
    gr->next[i] = gr->head[h];
    gr->head[h] = i;
}

/* Beads leave the grid in the reverse order of insertion, so bead i is the
 * head of its bucket when it is removed. */
static void grid_remove_last(grid_t *gr, const double *xyz, int32_t i) {
    int64_t c[3];
    grid_cell_of(gr, xyz + 3 * (size_t)i, c);
    uint32_t h = grid_hash(c[0], c[1], c[2], gr->mask);
    gr->head[h] = gr->next[i];
}

/* 1 when p is closer than min_dist to a placed bead other than `skip`. */
static int grid_clash(const grid_t *gr, const double *xyz, const double p[3], int32_t skip, double min_dist) {
    int64_t c[3];
    grid_cell_of(gr, p, c);
    double md2 = min_dist * min_dist;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                uint32_t h = grid_hash(c[0] + dx, c[1] + dy, c[2] + dz, gr->mask);
                for (int32_t j = gr->head[h]; j >= 0; j = gr->next[j]) {
                    if (j == skip) continue;
                    const double *q = xyz + 3 * (size_t)j;
                    double ex = p[0] - q[0], ey = p[1] - q[1], ez = p[2] - q[2];
                    if (ex * ex + ey * ey + ez * ez < md2) return 1;
                }
            }
    return 0;
}

/* Grow one chain of n beads into xyz[3*base ...], inside region g, avoiding every
 * bead already in the grid. Returns 0 on success, -1 when the budget runs out
 * (the chain's beads are then removed from the grid again). */
static int grow_chain(rng_t *rng, grid_t *gr, double *xyz, int32_t base, int32_t n, const region_t *g,
                      const double start[3], double bond, double min_dist, int64_t budget) {
    double v[3], p[3];
    /* first bead: the start point, or a random point near it */
    int placed = 0;
    for (int t = 0; t < 100000 && !placed; ++t) {
        double s = (t == 0) ? 0.0 : 0.5 * bond * (1.0 + t / 64);
        rng_unit_vector(rng, v);
        for (int k = 0; k < 3; ++k) p[k] = start[k] + s * v[k];
        if (region_inside(g, p) && !grid_clash(gr, xyz, p, -1, min_dist)) placed = 1;
    }
    if (!placed) return -1;
    memcpy(xyz + 3 * (size_t)base, p, sizeof(p));
    grid_insert(gr, xyz, base);

    int32_t i = 1;
    int fails = 0;
    int64_t spent = 0;
    while (i < n) {
        const double *prev = xyz + 3 * (size_t)(base + i - 1);
        int ok = 0;
        for (int t = 0; t < TRIES; ++t) {
            rng_unit_vector(rng, v);
            for (int k = 0; k < 3; ++k) p[k] = prev[k] + bond * v[k];
            if (region_inside(g, p) && !grid_clash(gr, xyz, p, base + i - 1, min_dist)) { ok = 1; break; }
        }
        if (ok) {
            memcpy(xyz + 3 * (size_t)(base + i), p, sizeof(p));
            grid_insert(gr, xyz, base + i);
            ++i;
            fails = 0;
            continue;
        }
        if (++spent > budget) {
            for (int32_t k = i - 1; k >= 0; --k) grid_remove_last(gr, xyz, base + k);
            return -1;
        }
        ++fails;
        int lg = fails - 1 < MAX_BACK_LOG2 ? fails - 1 : MAX_BACK_LOG2;
        int32_t back = (int32_t)1 << lg;
        if (back > i - 1) back = i - 1;
        for (int32_t k = 0; k < back; ++k) grid_remove_last(gr, xyz, base + i - 1 - k);
        i -= back;
        if (i < 1) i = 1;
    }
    return 0;
}

/*
 * One chain of n beads. kind 0: sphere of radius a centred at the origin, the
 * walk starts at the centre. kind 1: cylinder of radius a and half length b
 * along z, the walk starts near the z = -b end. On failure the walk restarts
 * with the next random numbers; after 8 failed restarts the region grows by 2%.
 * Returns the number of restarts used, or -1.
 */
int synth_walk(int32_t n, uint64_t seed, int32_t kind, double a, double b, double bond, double min_dist,
               double *xyz) {
    if (n <= 0 || !xyz || (kind != REGION_SPHERE && kind != REGION_CYLINDER)) return -1;
    rng_t rng;
    rng_seed(&rng, seed);
    grid_t gr;
    if (grid_init(&gr, n, min_dist) != 0) return -1;
    region_t g = {kind, a, b, NULL, 0, 0};
    int restarts = 0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        double start[3] = {0.0, 0.0, kind == REGION_CYLINDER ? -g.b + bond : 0.0};
        if (grow_chain(&rng, &gr, xyz, 0, n, &g, start, bond, min_dist, 200LL * n + 10000) == 0) {
            grid_free(&gr);
            return restarts;
        }
        ++restarts;
        if (restarts % 8 == 0) { g.a *= 1.02; g.b *= 1.02; }
    }
    grid_free(&gr);
    return -1;
}

/*
 * An assembly of n_copies chains of n_per beads, each grown inside its own
 * angular cell (nearest of n_copies Fibonacci-sphere directions) of the shell
 * r_in <= |r| <= r_out, starting at the cell's direction times the mid radius.
 * All copies share one clash grid. Returns total restarts, or -1.
 */
int synth_shell(int32_t n_copies, int32_t n_per, uint64_t seed, double r_in, double r_out, double bond,
                double min_dist, double *xyz) {
    if (n_copies <= 0 || n_per <= 0 || !xyz) return -1;
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)n_copies);
    if (!dirs) return -1;
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int k = 0; k < n_copies; ++k) {
        double z = 1.0 - (2.0 * k + 1.0) / n_copies;
        double r = sqrt(fmax(0.0, 1.0 - z * z));
        dirs[3 * k] = r * cos(golden * k);
        dirs[3 * k + 1] = r * sin(golden * k);
        dirs[3 * k + 2] = z;
    }
    rng_t rng;
    rng_seed(&rng, seed);
    grid_t gr;
    if (grid_init(&gr, n_copies * n_per, min_dist) != 0) { free(dirs); return -1; }
    int restarts = 0;
    double rm = 0.5 * (r_in + r_out);
    for (int k = 0; k < n_copies; ++k) {
        region_t g = {REGION_SHELL_CELL, r_in, r_out, dirs, n_copies, k};
        double start[3] = {dirs[3 * k] * rm, dirs[3 * k + 1] * rm, dirs[3 * k + 2] * rm};
        int ok = 0;
        for (int attempt = 0; attempt < 64 && !ok; ++attempt) {
            if (grow_chain(&rng, &gr, xyz, k * n_per, n_per, &g, start, bond, min_dist, 200LL * n_per + 10000) == 0)
                ok = 1;
            else
                ++restarts;
        }
        if (!ok) { grid_free(&gr); free(dirs); return -1; }
    }
    grid_free(&gr);
    free(dirs);
    return restarts;
}

/* ---------------- many independent sphere-confined chains, in parallel ---------------- */
typedef struct {
    int32_t n_chains;
    const int32_t *sizes;
    const uint64_t *seeds;
    const int64_t *offsets;
    double v, bond, min_dist;
    double *xyz;
    int32_t next;              /* next chain to take */
    int32_t failed;
    pthread_mutex_t mu;
} many_job_t;

static void *many_worker(void *arg) {
    many_job_t *job = (many_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        int32_t c = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (c >= job->n_chains) break;
        int32_t n = job->sizes[c];
        double radius = cbrt(3.0 * n * job->v / (4.0 * M_PI));
        int rc = synth_walk(n, job->seeds[c], REGION_SPHERE, radius, 0.0, job->bond, job->min_dist,
                            job->xyz + 3 * job->offsets[c]);
        if (rc < 0) {
            pthread_mutex_lock(&job->mu);
            job->failed = 1;
            pthread_mutex_unlock(&job->mu);
        }
    }
    return NULL;
}

/*
 * n_chains independent chains, chain c of sizes[c] beads grown with seed seeds[c]
 * in the sphere of volume sizes[c]*v, written at xyz[3*offsets[c] ...]. The
 * result does not depend on n_threads. Returns 0, or -1 if any chain failed.
 */
int synth_walk_many(int32_t n_chains, const int32_t *sizes, const uint64_t *seeds, const int64_t *offsets,
                    double v, double bond, double min_dist, int32_t n_threads, double *xyz) {
    if (n_chains <= 0 || !sizes || !seeds || !offsets || !xyz) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    many_job_t job = {n_chains, sizes, seeds, offsets, v, bond, min_dist, xyz, 0, 0};
    pthread_mutex_init(&job.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < n_threads; ++t)
        if (pthread_create(&th[t], NULL, many_worker, &job) == 0) ++started;
    if (started == 0) many_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&job.mu);
    return job.failed ? -1 : 0;
}
