/*
 * CPU FP64 oracle for the single-GPU short-range MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Plain, slow and
 * written to be checked against the paper by eye; see oracle.h for the
 * section each function follows.  Build with -ffp-contract=off.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Periodic box, minimum image (Sec. 4.1: "the usual minimum image convention
 * for periodic boundaries").                                                */

static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* Separation x_i - x_j under minimum image, and r^2 = (dx dx + dy dy) + dz dz. */
static double separation(const double *pi, const double *pj, const double *L,
                         double *d) {
    for (int k = 0; k < 3; k++) d[k] = min_image(pi[k] - pj[k], L[k]);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* Compensated (Neumaier) accumulation keeps each per-particle sum accurate to
 * a few ulps of the result, independent of summation order. */
typedef struct { double s, c; } acc_t;

static void acc_add(acc_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double acc_get(const acc_t *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Cell list (Sec. 4.3.3 mentions the cell list; Sec. 5.1 looks up the cell
 * neighbours of particle i).                                                */

int32_t orc_cells_per_dim(double L, double r_list) {
    /* cells at least r_list (1 + 1e-12) wide, so that rounding in x / h
     * cannot put two particles closer than r_list two cells apart even when
     * L is an exact multiple of r_list */
    double m = floor(L / (r_list * (1.0 + 1e-12)));
    if (m > 512.0) m = 512.0;
    if (m < 3.0) return 0;
    return (int32_t)m;
}

static int32_t cell_of(double x, int32_t nc, double L) {
    double inv_h = (double)nc / L;
    int32_t c = (int32_t)floor(x * inv_h);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

void orc_cell_coords(int64_t n, const double *pos, const double *L,
                     const int32_t *nc, int32_t *cell) {
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) cell[3 * i + k] = cell_of(pos[4 * i + k], nc[k], L[k]);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* Neighbour rows (Sec. 5.1, Fig. "nlist"): row i holds every j != i within
 * the list radius; the order inside a row is not part of the result, so the
 * oracle stores it ascending.                                               */

int32_t orc_neighbors_brute(int64_t n, const double *pos, const double *L,
                            double r_list, int32_t *counts, int32_t *rows,
                            int32_t max_nb) {
    double rl2 = r_list * r_list;
    int32_t longest = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : longest)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            if (separation(pos + 4 * i, pos + 4 * j, L, d) < rl2) {
                if (c < max_nb) rows[i * max_nb + c] = (int32_t)j;
                c++;
            }
        }
        counts[i] = c;
        if (c > longest) longest = c;
    }
    return longest;
}

int32_t orc_neighbors_cells(int64_t n, const double *pos, const double *L,
                            double r_list, int32_t *counts, int32_t *rows,
                            int32_t max_nb) {
    int32_t nc[3];
    for (int k = 0; k < 3; k++) {
        nc[k] = orc_cells_per_dim(L[k], r_list);
        /* fewer than 3 cells per edge: the 27-cell stencil would repeat
         * cells, so use the all-pairs definition instead */
        if (nc[k] == 0) return orc_neighbors_brute(n, pos, L, r_list, counts, rows, max_nb);
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell = malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *fill = calloc((size_t)ncell, sizeof(int64_t));
    int32_t *members = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    orc_cell_coords(n, pos, L, nc, cell);
    /* counting sort of the particles into cells, ascending index per cell */
    for (int64_t i = 0; i < n; i++) {
        int64_t id = cell[3 * i] + (int64_t)nc[0] * (cell[3 * i + 1] + (int64_t)nc[1] * cell[3 * i + 2]);
        start[id + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; i++) {
        int64_t id = cell[3 * i] + (int64_t)nc[0] * (cell[3 * i + 1] + (int64_t)nc[1] * cell[3 * i + 2]);
        members[start[id] + fill[id]++] = (int32_t)i;
    }
    double rl2 = r_list * r_list;
    int32_t longest = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : longest)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = 0;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int64_t cx = (cell[3 * i] + dx + nc[0]) % nc[0];
                    int64_t cy = (cell[3 * i + 1] + dy + nc[1]) % nc[1];
                    int64_t cz = (cell[3 * i + 2] + dz + nc[2]) % nc[2];
                    int64_t id = cx + nc[0] * (cy + nc[1] * cz);
                    for (int64_t m = start[id]; m < start[id + 1]; m++) {
                        int32_t j = members[m];
                        if (j == i) continue;
                        double d[3];
                        if (separation(pos + 4 * i, pos + 4 * (int64_t)j, L, d) < rl2) {
                            if (c < max_nb) rows[i * max_nb + c] = j;
                            c++;
                        }
                    }
                }
        counts[i] = c;
        if (c > longest) longest = c;
        qsort(rows + i * max_nb, (size_t)(c < max_nb ? c : max_nb), sizeof(int32_t), cmp_i32);
    }
    free(cell);
    free(start);
    free(fill);
    free(members);
    return longest;
}

/* ------------------------------------------------------------------------ */
/* LJ 12-6 (Sec. 3 lists LJ; the benchmarks of Sec. 6 and 8.3 use it with
 * eps = sigma = 1).  V(r) = 4 eps ((s/r)^12 - (s/r)^6);
 * F_i = -dV/dr (x_i - x_j)/r = 24 eps (2 (s/r)^12 - (s/r)^6) / r^2 (x_i - x_j). */

double orc_lj_pair(double r2, double eps, double sigma, double *v) {
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *v = 4.0 * eps * (s12 - s6);
    return 24.0 * eps * (2.0 * s12 - s6) / r2;
}

typedef struct {
    acc_t f[3], pe, w[6], absf;
} pacc_t;

static void pacc_clear(pacc_t *a) { memset(a, 0, sizeof(*a)); }

/* Add the pair force fr * d (d = x_i - x_j) and pair energy v to particle i;
 * energy and virial are split half / half between the two particles. */
static void pacc_pair(pacc_t *a, const double *d, double fr, double v) {
    double f[3] = {fr * d[0], fr * d[1], fr * d[2]};
    for (int k = 0; k < 3; k++) acc_add(&a->f[k], f[k]);
    acc_add(&a->pe, 0.5 * v);
    acc_add(&a->w[0], 0.5 * d[0] * f[0]);
    acc_add(&a->w[1], 0.5 * d[0] * f[1]);
    acc_add(&a->w[2], 0.5 * d[0] * f[2]);
    acc_add(&a->w[3], 0.5 * d[1] * f[1]);
    acc_add(&a->w[4], 0.5 * d[1] * f[2]);
    acc_add(&a->w[5], 0.5 * d[2] * f[2]);
    acc_add(&a->absf, sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]));
}

static void pacc_store(const pacc_t *a, int64_t i, double *force, double *virial,
                       double *absf) {
    for (int k = 0; k < 3; k++) force[4 * i + k] = acc_get(&a->f[k]);
    force[4 * i + 3] = acc_get(&a->pe);
    if (virial)
        for (int k = 0; k < 6; k++) virial[6 * i + k] = acc_get(&a->w[k]);
    if (absf) absf[i] = acc_get(&a->absf);
}

static void lj_one(pacc_t *a, const double *d, double r2, int32_t ti, int32_t tj,
                   int32_t ntypes, const double *coeff, double r_cut,
                   int32_t shift_energy) {
    const double *c = coeff + 2 * (ti * ntypes + tj);
    double v;
    double fr = orc_lj_pair(r2, c[0], c[1], &v);
    if (shift_energy) {
        double vc;
        orc_lj_pair(r_cut * r_cut, c[0], c[1], &vc);
        v -= vc;
    }
    pacc_pair(a, d, fr, v);
}

int32_t orc_pair_ncoeff(int32_t kind) { return kind == 3 ? 3 : 2; }

/* Gaussian: V = eps e^(-r^2 / 2 sigma^2), -dV/dr = (r / sigma^2) V. */
static double gauss_pair(double r2, double eps, double sigma, double *v) {
    *v = eps * exp(-r2 / (2.0 * sigma * sigma));
    return *v / (sigma * sigma);
}

/* Morse: with x = e^(-alpha (r - r0)), V = D0 (x^2 - 2 x) and
 * -dV/dr = 2 D0 alpha (x^2 - x). */
static double morse_pair(double r2, double d0, double alpha, double r0, double *v) {
    double r = sqrt(r2);
    double x = exp(-alpha * (r - r0));
    *v = d0 * (x * x - 2.0 * x);
    return 2.0 * d0 * alpha * (x * x - x) / r;
}

/* Yukawa: V = eps e^(-kappa r) / r, -dV/dr = V (1 + kappa r) / r. */
static double yukawa_pair(double r2, double eps, double kappa, double *v) {
    double r = sqrt(r2);
    *v = eps * exp(-kappa * r) / r;
    return *v * (1.0 + kappa * r) / r2;
}

double orc_pair_eval(int32_t kind, double r2, const double *c, double *v) {
    switch (kind) {
        case 0: return orc_lj_pair(r2, c[0], c[1], v);
        case 2: return gauss_pair(r2, c[0], c[1], v);
        case 3: return morse_pair(r2, c[0], c[1], c[2], v);
        case 4: return yukawa_pair(r2, c[0], c[1], v);
        default: *v = 0.0; return 0.0;
    }
}

static void pair_one(pacc_t *a, int32_t kind, const double *d, double r2, int32_t ti,
                     int32_t tj, int32_t ntypes, const double *coeff, double r_cut,
                     int32_t shift_energy) {
    const double *c = coeff + (size_t)orc_pair_ncoeff(kind) * (size_t)(ti * ntypes + tj);
    double v;
    double fr = orc_pair_eval(kind, r2, c, &v);
    if (shift_energy) {
        double vc;
        orc_pair_eval(kind, r_cut * r_cut, c, &vc);
        v -= vc;
    }
    pacc_pair(a, d, fr, v);
}

void orc_pair_forces_brute(int32_t kind, int64_t n, const double *pos, const int32_t *type,
                           const double *L, double r_cut, int32_t ntypes,
                           const double *coeff, int32_t shift_energy,
                           double *force, double *virial, double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                pair_one(&a, kind, d, r2, type[i], type[j], ntypes, coeff, r_cut, shift_energy);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

void orc_pair_forces_nlist(int32_t kind, int64_t n, const double *pos, const int32_t *type,
                           const double *L, double r_cut, int32_t ntypes,
                           const double *coeff, int32_t shift_energy,
                           const int32_t *counts, const int32_t *rows,
                           int32_t max_nb, double *force, double *virial,
                           double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int32_t k = 0; k < counts[i] && k < max_nb; k++) {
            int64_t j = rows[i * max_nb + k];
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                pair_one(&a, kind, d, r2, type[i], type[j], ntypes, coeff, r_cut, shift_energy);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

double orc_table_eval(double r2, const double *tab, int32_t n_points, double r_min,
                      double r_cut, double *v) {
    double r = sqrt(r2);
    double dr = (r_cut - r_min) / (double)(n_points - 1);
    double x = (r - r_min) / dr;
    int32_t k = 0;
    double t = 0.0;
    if (x > 0.0) {
        k = (int32_t)floor(x);
        if (k > n_points - 2) k = n_points - 2;
        t = x - (double)k;
    }
    const double *a = tab + 2 * k, *b = tab + 2 * (k + 1);
    *v = a[0] + t * (b[0] - a[0]);
    return (a[1] + t * (b[1] - a[1])) / r;
}

void orc_table_forces_brute(int64_t n, const double *pos, const int32_t *type,
                            const double *L, double r_cut, int32_t ntypes,
                            const double *table, int32_t n_points, double r_min,
                            double *force, double *virial, double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2) {
                const double *tab = table + (size_t)2 * n_points * (size_t)(type[i] * ntypes + type[j]);
                double v;
                double fr = orc_table_eval(r2, tab, n_points, r_min, r_cut, &v);
                pacc_pair(&a, d, fr, v);
            }
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

void orc_lj_forces_brute(int64_t n, const double *pos, const int32_t *type,
                         const double *L, double r_cut, int32_t ntypes,
                         const double *coeff, int32_t shift_energy,
                         double *force, double *virial, double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                lj_one(&a, d, r2, type[i], type[j], ntypes, coeff, r_cut, shift_energy);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

void orc_lj_forces_nlist(int64_t n, const double *pos, const int32_t *type,
                         const double *L, double r_cut, int32_t ntypes,
                         const double *coeff, int32_t shift_energy,
                         const int32_t *counts, const int32_t *rows,
                         int32_t max_nb, double *force, double *virial,
                         double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int32_t k = 0; k < counts[i] && k < max_nb; k++) {
            int64_t j = rows[i * max_nb + k];
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                lj_one(&a, d, r2, type[i], type[j], ntypes, coeff, r_cut, shift_energy);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as easy as
 * 1, 2, 3"): ten rounds of two 32x32->64 multiplies on the even counter words,
 * outputs permuted and XORed with the odd words and the round key; the key is
 * advanced by the Weyl constants between rounds.                            */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    for (int k = 0; k < 4; k++) out[k] = c[k];
}

double orc_dpd_theta(int32_t tag_i, int32_t tag_j, uint64_t step, uint64_t seed) {
    uint32_t a = (uint32_t)tag_i, b = (uint32_t)tag_j;
    uint32_t ctr[4] = {a < b ? a : b, a < b ? b : a, (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double u = ((double)w[0] + 0.5) * 0x1p-32;
    return sqrt(3.0) * (2.0 * u - 1.0);
}

/* DPD pair (Sec. 9 benchmarks A = 25, gamma = 4.5, rho = 3; the random force
 * uses a per-pair generator seeded with global particle IDs).  Groot-Warren
 * form with w = 1 - r / r_cut:
 *   F_i = [A w - gamma w^2 (e . v_ij) + sigma w theta / sqrt(dt)] e,
 *   e = (x_i - x_j) / r, v_ij = v_i - v_j, sigma = sqrt(2 gamma kT),
 *   V = A r_cut w^2 / 2.                                                     */
static void dpd_one(pacc_t *a, const double *d, double r2, const double *vi,
                    const double *vj, int32_t ti, int32_t tj, int32_t tag_i,
                    int32_t tag_j, int32_t ntypes, const double *coeff,
                    double r_cut, double kT, double dt, uint64_t step,
                    uint64_t seed) {
    const double *c = coeff + 2 * (ti * ntypes + tj);
    double A = c[0], gamma = c[1];
    double r = sqrt(r2);
    double w = 1.0 - r / r_cut;
    double e[3] = {d[0] / r, d[1] / r, d[2] / r};
    double ev = e[0] * (vi[0] - vj[0]) + e[1] * (vi[1] - vj[1]) + e[2] * (vi[2] - vj[2]);
    double sigma = sqrt(2.0 * gamma * kT);
    double theta = orc_dpd_theta(tag_i, tag_j, step, seed);
    double fmag = A * w - gamma * w * w * ev + sigma * w * theta / sqrt(dt);
    double v = 0.5 * A * r_cut * w * w;
    /* express as fr * d with fr = fmag / r */
    pacc_pair(a, d, fmag / r, v);
}

void orc_dpd_forces_brute(int64_t n, const double *pos, const double *vel,
                          const int32_t *type, const int32_t *tag,
                          const double *L, double r_cut, int32_t ntypes,
                          const double *coeff, double kT, double dt,
                          uint64_t step, uint64_t seed, double *force,
                          double *virial, double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                dpd_one(&a, d, r2, vel + 4 * i, vel + 4 * j, type[i], type[j], tag[i],
                        tag[j], ntypes, coeff, r_cut, kT, dt, step, seed);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

void orc_dpd_forces_nlist(int64_t n, const double *pos, const double *vel,
                          const int32_t *type, const int32_t *tag,
                          const double *L, double r_cut, int32_t ntypes,
                          const double *coeff, double kT, double dt,
                          uint64_t step, uint64_t seed, const int32_t *counts,
                          const int32_t *rows, int32_t max_nb, double *force,
                          double *virial, double *absf) {
    double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        pacc_t a;
        pacc_clear(&a);
        for (int32_t k = 0; k < counts[i] && k < max_nb; k++) {
            int64_t j = rows[i * max_nb + k];
            double d[3];
            double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
            if (r2 < rc2)
                dpd_one(&a, d, r2, vel + 4 * i, vel + 4 * j, type[i], type[j], tag[i],
                        tag[j], ntypes, coeff, r_cut, kT, dt, step, seed);
        }
        pacc_store(&a, i, force, virial, absf);
    }
}

/* ------------------------------------------------------------------------ */
/* Harmonic bond (Sec. 3 lists harmonic bonds; Sec. 4.3.4 defines a bond as an
 * unordered pair of particle IDs): V = K/2 (r - r0)^2,
 * F_i = -K (r - r0) (x_i - x_j) / r, and F_j = -F_i.                        */

/* FENE bond (Sec. 3 lists FENE bonds; the finitely extensible nonlinear
 * elastic spring of Kremer and Grest, without the repulsive core):
 * V = -K R0^2 / 2 ln(1 - (r / R0)^2), -dV/dr = -K r / (1 - (r / R0)^2).
 * Returns the number of bonds at r >= R0 (undefined; skipped). */
int64_t orc_fene_bond_forces(int64_t n_bonds, const int32_t *bonds, const double *pos,
                             const double *L, double K, double R0, double *force,
                             double *virial, double *absf) {
    int64_t broken = 0;
    for (int64_t b = 0; b < n_bonds; b++) {
        int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
        double q = r2 / (R0 * R0);
        if (!(q < 1.0)) {
            broken++;
            continue;
        }
        double fr = -K / (1.0 - q);
        double v = -0.5 * K * R0 * R0 * log(1.0 - q);
        double f[3] = {fr * d[0], fr * d[1], fr * d[2]};
        for (int k = 0; k < 3; k++) {
            force[4 * i + k] += f[k];
            force[4 * j + k] -= f[k];
        }
        force[4 * i + 3] += 0.5 * v;
        force[4 * j + 3] += 0.5 * v;
        if (virial) {
            double w[6] = {d[0] * f[0], d[0] * f[1], d[0] * f[2],
                           d[1] * f[1], d[1] * f[2], d[2] * f[2]};
            for (int k = 0; k < 6; k++) {
                virial[6 * i + k] += 0.5 * w[k];
                virial[6 * j + k] += 0.5 * w[k];
            }
        }
        if (absf) {
            double m = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
            absf[i] += m;
            absf[j] += m;
        }
    }
    return broken;
}

/* Harmonic angle (Sec. 3 lists harmonic angle potentials): for a triplet
 * (a, b, c) with vertex b, u = x_a - x_b and w = x_c - x_b (minimum image),
 * theta = acos(u.w / (|u| |w|)) and V = K/2 (theta - theta0)^2.  With
 * c = cos(theta) and s = sin(theta):
 *   F_a = K (theta - theta0) / s (w / (|u| |w|) - c u / |u|^2),
 *   F_c = K (theta - theta0) / s (u / (|u| |w|) - c w / |w|^2),
 *   F_b = -(F_a + F_c).
 * Each particle of the triplet gets a third of V and of the angle's virial
 * u (x) F_a + w (x) F_c.  s is floored at 1e-12 (a straight or folded
 * triplet). */
void orc_angle_forces(int64_t n_angles, const int32_t *tri, const double *pos,
                      const double *L, double K, double theta0, double *force,
                      double *virial, double *absf) {
    for (int64_t t = 0; t < n_angles; t++) {
        int64_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        double u[3], w[3];
        double uu = separation(pos + 4 * a, pos + 4 * b, L, u);
        double ww = separation(pos + 4 * c, pos + 4 * b, L, w);
        double ru = sqrt(uu), rw = sqrt(ww);
        double cs = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / (ru * rw);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double th = acos(cs);
        double sn = sqrt(1.0 - cs * cs);
        if (sn < 1e-12) sn = 1e-12;
        double g = K * (th - theta0) / sn;
        double fa[3], fc[3], fb[3];
        for (int k = 0; k < 3; k++) {
            fa[k] = g * (w[k] / (ru * rw) - cs * u[k] / uu);
            fc[k] = g * (u[k] / (ru * rw) - cs * w[k] / ww);
            fb[k] = -(fa[k] + fc[k]);
        }
        double v = 0.5 * K * (th - theta0) * (th - theta0);
        double vir[6] = {u[0] * fa[0] + w[0] * fc[0], u[0] * fa[1] + w[0] * fc[1],
                         u[0] * fa[2] + w[0] * fc[2], u[1] * fa[1] + w[1] * fc[1],
                         u[1] * fa[2] + w[1] * fc[2], u[2] * fa[2] + w[2] * fc[2]};
        int64_t who[3] = {a, b, c};
        double *fs[3] = {fa, fb, fc};
        for (int m = 0; m < 3; m++) {
            for (int k = 0; k < 3; k++) force[4 * who[m] + k] += fs[m][k];
            force[4 * who[m] + 3] += v / 3.0;
            if (virial)
                for (int k = 0; k < 6; k++) virial[6 * who[m] + k] += vir[k] / 3.0;
            if (absf)
                absf[who[m]] += sqrt(fs[m][0] * fs[m][0] + fs[m][1] * fs[m][1] + fs[m][2] * fs[m][2]);
        }
    }
}

void orc_bond_forces(int64_t n_bonds, const int32_t *bonds, const double *pos,
                     const double *L, double K, double r0, double *force,
                     double *virial, double *absf) {
    for (int64_t b = 0; b < n_bonds; b++) {
        int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        double r2 = separation(pos + 4 * i, pos + 4 * j, L, d);
        double r = sqrt(r2);
        double fr = (r0 == 0.0) ? -K : (r > 0.0 ? -K * (r - r0) / r : 0.0);
        double v = 0.5 * K * (r - r0) * (r - r0);
        for (int k = 0; k < 3; k++) {
            force[4 * i + k] += fr * d[k];
            force[4 * j + k] -= fr * d[k];
        }
        force[4 * i + 3] += 0.5 * v;
        force[4 * j + 3] += 0.5 * v;
        double f[3] = {fr * d[0], fr * d[1], fr * d[2]};
        if (virial) {
            double w[6] = {d[0] * f[0], d[0] * f[1], d[0] * f[2],
                           d[1] * f[1], d[1] * f[2], d[2] * f[2]};
            for (int k = 0; k < 6; k++) {
                virial[6 * i + k] += 0.5 * w[k];
                virial[6 * j + k] += 0.5 * w[k];
            }
        }
        if (absf) {
            double m = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
            absf[i] += m;
            absf[j] += m;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet (Sec. 3: NVE integration with the velocity-Verlet update;
 * DPD uses the same update with the DPD pair force).                        */

void orc_vv_first(int64_t n, double *pos, double *vel, int32_t *image,
                  const double *force, double dt, double mass, const double *L) {
    double h = 0.5 * dt / mass;
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++) {
            double v = vel[4 * i + k] + h * force[4 * i + k];
            double x = pos[4 * i + k] + dt * v;
            int32_t img = image[4 * i + k];
            while (x >= L[k]) { x -= L[k]; img++; }
            while (x < 0.0) { x += L[k]; img--; }
            if (x >= L[k]) { x -= L[k]; img++; }
            vel[4 * i + k] = v;
            pos[4 * i + k] = x;
            image[4 * i + k] = img;
        }
    }
}

void orc_vv_second(int64_t n, double *vel, const double *force, double dt,
                   double mass) {
    double h = 0.5 * dt / mass;
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) vel[4 * i + k] += h * force[4 * i + k];
}

/* ------------------------------------------------------------------------ */
/* Thermostats (Sec. 3: NVT with the Martyna-Tobias-Klein update equations,
 * Langevin dynamics; Sec. 6.1 runs NVT with a Nose-Hoover thermostat that
 * needs one kinetic-energy sum per step).                                  */

void orc_langevin_noise(int32_t tag, uint64_t step, uint64_t seed, double *theta) {
    uint32_t ctr[4] = {(uint32_t)tag, 0xFFFFFFFFu, (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int k = 0; k < 3; k++) {
        double u = ((double)w[k] + 0.5) * 0x1p-32;
        theta[k] = sqrt(3.0) * (2.0 * u - 1.0);
    }
}

void orc_baoab_first(int64_t n, double *pos, double *vel, int32_t *image,
                     const double *force, const int32_t *tag, double dt,
                     double mass, double gamma, double kT, uint64_t step,
                     uint64_t seed, const double *L) {
    double h = 0.5 * dt / mass;
    double c = exp(-gamma * dt);
    double sigma = sqrt((1.0 - c * c) * kT / mass);
    for (int64_t i = 0; i < n; i++) {
        double theta[3];
        orc_langevin_noise(tag[i], step, seed, theta);
        for (int k = 0; k < 3; k++) {
            double v = vel[4 * i + k] + h * force[4 * i + k];   /* B */
            double x = pos[4 * i + k] + 0.5 * dt * v;           /* A */
            v = c * v + sigma * theta[k];                       /* O */
            x = x + 0.5 * dt * v;                               /* A */
            int32_t img = image[4 * i + k];
            while (x >= L[k]) { x -= L[k]; img++; }
            while (x < 0.0) { x += L[k]; img--; }
            if (x >= L[k]) { x -= L[k]; img++; }
            vel[4 * i + k] = v;
            pos[4 * i + k] = x;
            image[4 * i + k] = img;
        }
    }
}

double orc_nh_half(int64_t n, double *vel, double mass, double kT, double tau,
                   double dt, double *state) {
    acc_t ke = {0, 0};
    for (int64_t i = 0; i < n; i++) {
        const double *v = vel + 4 * i;
        acc_add(&ke, 0.5 * mass * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
    double g = 3.0 * (double)n - 3.0;
    double KE = acc_get(&ke);
    state[0] += 0.25 * dt * ((2.0 * KE / g) / kT - 1.0) / (tau * tau);
    double s = exp(-0.5 * dt * state[0]);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) vel[4 * i + k] *= s;
    state[1] += 0.5 * dt * state[0];
    KE *= s * s;
    state[0] += 0.25 * dt * ((2.0 * KE / g) / kT - 1.0) / (tau * tau);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Thermodynamic reductions (Sec. 4.3.3: kinetic energy, virial etc. grouped
 * into one global synchronization per step).                               */

void orc_thermo(int64_t n, const double *vel, const double *force,
                const double *virial, double mass, const double *L, double *out) {
    acc_t ke = {0, 0}, pe = {0, 0}, w = {0, 0}, p[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = 0; i < n; i++) {
        const double *v = vel + 4 * i;
        acc_add(&ke, 0.5 * mass * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
        acc_add(&pe, force[4 * i + 3]);
        if (virial) acc_add(&w, virial[6 * i] + virial[6 * i + 3] + virial[6 * i + 5]);
        for (int k = 0; k < 3; k++) acc_add(&p[k], mass * v[k]);
    }
    double volume = L[0] * L[1] * L[2];
    out[0] = acc_get(&ke);
    out[1] = acc_get(&pe);
    out[2] = acc_get(&w);
    out[3] = (2.0 * out[0] + out[2]) / (3.0 * volume);
    out[4] = n > 1 ? 2.0 * out[0] / (3.0 * (double)n - 3.0) : 0.0;
    for (int k = 0; k < 3; k++) out[5 + k] = acc_get(&p[k]);
}

/* ------------------------------------------------------------------------ */
/* Hilbert curve (Skilling 2004).  The transpose form of the index is built by
 * undoing the curve's reflections and exchanges from the top bit down, then
 * Gray-coding; the index reads its bits MSB first, axis 0 first.            */

uint64_t orc_hilbert3(uint32_t x, uint32_t y, uint32_t z, int32_t bits) {
    uint32_t X[3] = {x, y, z};
    uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        uint32_t low = q - 1;
        for (int i = 0; i < 3; i++) {
            if (X[i] & q) {
                X[0] ^= low;
            } else {
                uint32_t t = (X[0] ^ X[i]) & low;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[2] & q) flip ^= q - 1;
    for (int i = 0; i < 3; i++) X[i] ^= flip;
    uint64_t h = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int i = 0; i < 3; i++) h = (h << 1) | ((X[i] >> b) & 1u);
    return h;
}

typedef struct { uint64_t key; int64_t idx; } keyidx_t;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Space-filling-curve order (Sec. 4.3.1 reorders all particle arrays
 * together, at list rebuilds; the curve, a 3-D Hilbert curve, is the
 * benchmark configuration's choice, not the paper's): the key of a particle is the
 * Hilbert index of the brick of 2 x 2 x 2 cells holding its cell, on a grid
 * of ceil(nc / 2) bricks per edge; particles with equal keys keep their index
 * order.  Nothing finer is fixed by the method: the order of the cells of a
 * brick and of the particles of a cell is left to the implementation. */
void orc_sfc_order(int64_t n, const double *pos, const double *L, double r_list,
                   int32_t *order) {
    int32_t nc[3];
    int32_t nmax = 1;
    for (int k = 0; k < 3; k++) {
        nc[k] = orc_cells_per_dim(L[k], r_list);
        if (nc[k] == 0) nc[k] = 1;
        if (nc[k] > nmax) nmax = nc[k];
    }
    int32_t bmax = (nmax + 1) / 2;
    int32_t bits = 1; /* bits >= 1 even for a single brick per edge */
    while ((1 << bits) < bmax) bits++;
    keyidx_t *ki = malloc(sizeof(keyidx_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        uint32_t c[3];
        for (int k = 0; k < 3; k++) c[k] = (uint32_t)cell_of(pos[4 * i + k], nc[k], L[k]);
        ki[i].key = orc_hilbert3(c[0] >> 1, c[1] >> 1, c[2] >> 1, bits);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t i = 0; i < n; i++) order[i] = (int32_t)ki[i].idx;
    free(ki);
}

/* ------------------------------------------------------------------------ */
/* MD loop (Sec. 4.2: the list is rebuilt when particles move more than half of
 * the buffer length; forces are then exact for every pair within r_cut).    */

static void compute_forces(int64_t n, const double *pos, const double *vel,
                           const int32_t *type, const int32_t *tag,
                           const orc_params *p, uint64_t step,
                           const int32_t *counts, const int32_t *rows,
                           double *force, double *virial) {
    if (p->pair != 1)
        orc_pair_forces_nlist(p->pair, n, pos, type, p->L, p->r_cut, p->ntypes, p->coeff,
                              p->shift_energy, counts, rows, p->max_nb, force, virial, NULL);
    else
        orc_dpd_forces_nlist(n, pos, vel, type, tag, p->L, p->r_cut, p->ntypes, p->coeff,
                             p->kT, p->dt, step, p->seed, counts, rows, p->max_nb, force,
                             virial, NULL);
    if (p->n_bonds > 0)
    {
        if (p->bond_style == 1)
            orc_fene_bond_forces(p->n_bonds, p->bonds, pos, p->L, p->K, p->r0, force, virial, NULL);
        else
            orc_bond_forces(p->n_bonds, p->bonds, pos, p->L, p->K, p->r0, force, virial, NULL);
    }
    if (p->n_angles > 0)
        orc_angle_forces(p->n_angles, p->angles, pos, p->L, p->angle_K, p->angle_theta0, force,
                         virial, NULL);
}

int64_t orc_run(int64_t n, double *pos, double *vel, int32_t *image,
                const int32_t *type, const int32_t *tag, double *force,
                const orc_params *p, int64_t n_steps, double *thermo_out) {
    double r_list = p->r_cut + p->r_skin;
    int32_t max_nb = p->max_nb;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *counts = malloc(sizeof(int32_t) * nn);
    int32_t *rows = malloc(sizeof(int32_t) * nn * (size_t)max_nb);
    double *ref = malloc(sizeof(double) * 4 * nn);
    double *virial = malloc(sizeof(double) * 6 * nn);
    int64_t builds = 0, n_out = 0;
    double half2 = 0.25 * p->r_skin * p->r_skin;

#define ORC_BUILD()                                                            \
    do {                                                                       \
        if (orc_neighbors_cells(n, pos, p->L, r_list, counts, rows, max_nb) > max_nb) { \
            builds = -1;                                                       \
            goto done;                                                         \
        }                                                                      \
        memcpy(ref, pos, sizeof(double) * 4 * nn);                            \
        builds++;                                                              \
    } while (0)

    double nh_local[2] = {0.0, 0.0};
    double *nh = p->nh_state ? p->nh_state : nh_local;
    ORC_BUILD();
    compute_forces(n, pos, vel, type, tag, p, p->step0, counts, rows, force, virial);
    for (int64_t s = 1; s <= n_steps; s++) {
        uint64_t t = (uint64_t)(p->step0 + s);
        if (p->integrator == 2) orc_nh_half(n, vel, p->mass, p->t_kT, p->t_tau, p->dt, nh);
        if (p->integrator == 1)
            orc_baoab_first(n, pos, vel, image, force, tag, p->dt, p->mass, p->t_gamma,
                            p->t_kT, t, p->t_seed, p->L);
        else
            orc_vv_first(n, pos, vel, image, force, p->dt, p->mass, p->L);
        int rebuild = 0;
        for (int64_t i = 0; i < n && !rebuild; i++) {
            double d[3];
            if (separation(pos + 4 * i, ref + 4 * i, p->L, d) > half2) rebuild = 1;
        }
        if (rebuild) ORC_BUILD();
        compute_forces(n, pos, vel, type, tag, p, t, counts, rows, force, virial);
        orc_vv_second(n, vel, force, p->dt, p->mass);
        if (p->integrator == 2) orc_nh_half(n, vel, p->mass, p->t_kT, p->t_tau, p->dt, nh);
        if (p->thermo_period > 0 && t % (uint64_t)p->thermo_period == 0 && thermo_out) {
            orc_thermo(n, vel, force, virial, p->mass, p->L, thermo_out + 8 * n_out);
            n_out++;
        }
    }
done:
#undef ORC_BUILD
    free(counts);
    free(rows);
    free(ref);
    free(virial);
    return builds;
}
