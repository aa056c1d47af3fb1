/*
 * CPU FP64 oracle for the single-GPU short-range MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Every function is a plain, slow, obviously correct statement of what the
 * method computes (Glaser et al., "Strong scaling of general-purpose molecular
 * dynamics simulations on GPUs"):
 *   - periodic box with the minimum-image convention (Sec. 4.1),
 *   - Verlet neighbour list of radius r_cut + r_buff, rebuilt when a particle
 *     moved more than half the buffer length (Sec. 4.2),
 *   - cell-list binning (Sec. 4.3.3) and the per-particle neighbour rows of
 *     the cooperative-thread-array algorithm (Sec. 5.1, Fig. "nlist"),
 *   - LJ 12-6 and DPD pair forces, DPD random numbers seeded with global
 *     particle IDs (Sec. 3, Sec. 9),
 *   - harmonic bonds between an unordered pair of particle IDs (Sec. 4.3.4),
 *   - velocity-Verlet NVE / DPD integration (Sec. 3),
 *   - grouped thermodynamic reductions (Sec. 4.3.3).
 *
 * Layouts: positions / velocities / forces are double[N][4]; force w holds the
 * per-particle potential energy.  Image counters are int32[N][4].  Virials are
 * double[N][6] (xx, xy, xz, yy, yz, zz).  Pair coefficients are per ordered
 * type pair: coeff[2 * (ti * ntypes + tj) + {0,1}] = (eps, sigma) for LJ and
 * (A, gamma) for DPD.
 *
 * Floating-point contract: compiled with -ffp-contract=off, so every product
 * and sum is rounded separately, in source order.
 */
#ifndef MD_ORACLE_H
#define MD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of cells per box edge for a cell list of minimum width r_list:
 * floor(L / (r_list (1 + 1e-12))), capped at 512 (the margin keeps cells
 * strictly wider than r_list when L is an exact multiple of it).  Returns 0
 * when fewer than 3 fit. */
int32_t orc_cells_per_dim(double L, double r_list);

/* Integer cell coordinates of every particle, cell[i][d] in [0, nc[d]). */
void orc_cell_coords(int64_t n, const double *pos, const double *L,
                     const int32_t *nc, int32_t *cell);

/* Full neighbour rows by brute force: j != i with r^2 < r_list^2 (strict).
 * rows[i * max_nb + k] in ascending j.  Returns the largest row length
 * (rows longer than max_nb are truncated but counted). */
int32_t orc_neighbors_brute(int64_t n, const double *pos, const double *L,
                            double r_list, int32_t *counts, int32_t *rows,
                            int32_t max_nb);

/* The same neighbour rows through a cell list (O(N)); boxes with fewer than
 * 3 cells per edge use the all-pairs loop. */
int32_t orc_neighbors_cells(int64_t n, const double *pos, const double *L,
                            double r_list, int32_t *counts, int32_t *rows,
                            int32_t max_nb);

/* LJ 12-6 pair: returns force magnitude divided by r, writes V(r). */
double orc_lj_pair(double r2, double eps, double sigma, double *v);

/* LJ forces over all pairs within r_cut.  force[i] = (F_i, PE_i); PE_i is half
 * the sum of the pair energies (shifted by V(r_cut) when shift_energy != 0).
 * virial and absf (sum over j of |f_ij|) may be NULL. */
void orc_lj_forces_brute(int64_t n, const double *pos, const int32_t *type,
                         const double *L, double r_cut, int32_t ntypes,
                         const double *coeff, int32_t shift_energy,
                         double *force, double *virial, double *absf);

/* LJ forces from full neighbour rows (as written by orc_neighbors_*). */
void orc_lj_forces_nlist(int64_t n, const double *pos, const int32_t *type,
                         const double *L, double r_cut, int32_t ntypes,
                         const double *coeff, int32_t shift_energy,
                         const int32_t *counts, const int32_t *rows,
                         int32_t max_nb, double *force, double *virial,
                         double *absf);

/* Pair kinds: 0 = LJ (eps, sigma), 1 = DPD (A, gamma), and the other
 * pair potentials of Sec. 3's list in their textbook forms:
 *   2 = Gaussian (eps, sigma):   V = eps exp(-r^2 / (2 sigma^2))
 *   3 = Morse (D0, alpha, r0):   V = D0 [exp(-2 alpha (r - r0)) - 2 exp(-alpha (r - r0))]
 *   4 = Yukawa (eps, kappa):     V = eps exp(-kappa r) / r
 * Coefficients per ordered type pair, orc_pair_ncoeff(kind) doubles each. */
int32_t orc_pair_ncoeff(int32_t kind);

/* Potential of kind 0, 2, 3 or 4 at r^2 with coefficients c: returns
 * -dV/dr / r (the factor of d = x_i - x_j in f_ij), writes V(r). */
double orc_pair_eval(int32_t kind, double r2, const double *c, double *v);

/* As orc_lj_forces_brute / orc_lj_forces_nlist for any kind 0, 2, 3, 4. */
void orc_pair_forces_brute(int32_t kind, int64_t n, const double *pos, const int32_t *type,
                           const double *L, double r_cut, int32_t ntypes,
                           const double *coeff, int32_t shift_energy,
                           double *force, double *virial, double *absf);
void orc_pair_forces_nlist(int32_t kind, int64_t n, const double *pos, const int32_t *type,
                           const double *L, double r_cut, int32_t ntypes,
                           const double *coeff, int32_t shift_energy,
                           const int32_t *counts, const int32_t *rows,
                           int32_t max_nb, double *force, double *virial,
                           double *absf);

/* Tabulated pair potential (Sec. 3 lists tabulated potentials): per ordered
 * type pair, n_points samples (V_j, F_j) at r_j = r_min + j dr,
 * dr = (r_cut - r_min) / (n_points - 1), F = -dV/dr; between samples V and
 * F are interpolated linearly in r; below r_min they take their values at
 * r_min.  table: [ntypes][ntypes][n_points][2].  Force factor F(r) / r. */
double orc_table_eval(double r2, const double *tab, int32_t n_points, double r_min,
                      double r_cut, double *v);
void orc_table_forces_brute(int64_t n, const double *pos, const int32_t *type,
                            const double *L, double r_cut, int32_t ntypes,
                            const double *table, int32_t n_points, double r_min,
                            double *force, double *virial, double *absf);

/* Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* DPD pair noise theta_ij = sqrt(3) (2u - 1), u = (w0 + 1/2) 2^-32, where w0
 * is word 0 of Philox-4x32-10 with counter (min tag, max tag, step lo,
 * step hi) and key (seed lo, seed hi).  Symmetric in (tag_i, tag_j). */
double orc_dpd_theta(int32_t tag_i, int32_t tag_j, uint64_t step, uint64_t seed);

/* DPD (Groot-Warren) forces over all pairs within r_cut. */
void orc_dpd_forces_brute(int64_t n, const double *pos, const double *vel,
                          const int32_t *type, const int32_t *tag,
                          const double *L, double r_cut, int32_t ntypes,
                          const double *coeff, double kT, double dt,
                          uint64_t step, uint64_t seed, double *force,
                          double *virial, double *absf);

/* DPD forces from full neighbour rows. */
void orc_dpd_forces_nlist(int64_t n, const double *pos, const double *vel,
                          const int32_t *type, const int32_t *tag,
                          const double *L, double r_cut, int32_t ntypes,
                          const double *coeff, double kT, double dt,
                          uint64_t step, uint64_t seed, const int32_t *counts,
                          const int32_t *rows, int32_t max_nb, double *force,
                          double *virial, double *absf);

/* Harmonic bonds V = K/2 (r - r0)^2 between particle indices bonds[2b],
 * bonds[2b+1].  ADDS to force (and PE in force w, half per end), virial, absf
 * (any of virial / absf may be NULL). */
/* FENE bonds: V = -K R0^2 / 2 ln(1 - (r/R0)^2); returns the number of
 * bonds at r >= R0 (skipped). */
int64_t orc_fene_bond_forces(int64_t n_bonds, const int32_t *bonds, const double *pos,
                             const double *L, double K, double R0, double *force,
                             double *virial, double *absf);

/* Harmonic angles V = K/2 (theta - theta0)^2 over triplets (a, b, c) with
 * vertex b; each particle gets a third of V and of the angle's virial. */
void orc_angle_forces(int64_t n_angles, const int32_t *tri, const double *pos,
                      const double *L, double K, double theta0, double *force,
                      double *virial, double *absf);

void orc_bond_forces(int64_t n_bonds, const int32_t *bonds, const double *pos,
                     const double *L, double K, double r0, double *force,
                     double *virial, double *absf);

/* Velocity Verlet, first half: v += dt/2 F/m; x += dt v; wrap into [0, L)
 * and count the crossings in image. */
void orc_vv_first(int64_t n, double *pos, double *vel, int32_t *image,
                  const double *force, double dt, double mass, const double *L);

/* Velocity Verlet, second half: v += dt/2 F/m. */
void orc_vv_second(int64_t n, double *vel, const double *force, double dt,
                   double mass);

/* out = {KE, PE, W, P, T, px, py, pz}: kinetic and potential energy, virial
 * trace W, pressure (2 KE + W) / (3 V), temperature 2 KE / (3N - 3), momentum.
 * virial may be NULL (then W = P's virial part = 0). */
void orc_thermo(int64_t n, const double *vel, const double *force,
                const double *virial, double mass, const double *L, double *out);

/* 3-D Hilbert index of a cell of a 2^bits grid (Skilling, AIP Conf. Proc. 707,
 * 2004: axes-to-transpose, then bit interleave). */
uint64_t orc_hilbert3(uint32_t x, uint32_t y, uint32_t z, int32_t bits);

/* Space-filling-curve order (Sec. 4.3.1: all particle arrays reordered
 * together at list rebuilds; the Hilbert curve is the benchmark
 * configuration's choice): particles ordered by the Hilbert index of the brick of 2 x 2 x 2
 * cells (cell list of minimum width r_list) holding their cell, ties by
 * index.  The order inside a brick is not part of the method. */
void orc_sfc_order(int64_t n, const double *pos, const double *L, double r_list,
                   int32_t *order);

/* Langevin noise of one particle and step: theta_k = sqrt(3) (2 u_k - 1),
 * u_k = (w_k + 1/2) 2^-32 (k = 0, 1, 2), words 0..2 of Philox-4x32-10 with
 * counter (tag, 0xFFFFFFFF, step lo, step hi) and key (seed lo, seed hi).
 * Unit variance, mean zero. */
void orc_langevin_noise(int32_t tag, uint64_t step, uint64_t seed, double *theta);

/* Langevin dynamics, BAOAB splitting (Leimkuhler & Matthews 2013), first
 * part of a step: v += dt/2 F/m; x += dt/2 v; v = c v + sqrt((1 - c^2) kT/m)
 * theta (c = exp(-gamma dt)); x += dt/2 v; wrap into [0, L) counting images.
 * The step's last part is orc_vv_second (v += dt/2 F/m). */
void orc_baoab_first(int64_t n, double *pos, double *vel, int32_t *image,
                     const double *force, const int32_t *tag, double dt,
                     double mass, double gamma, double kT, uint64_t step,
                     uint64_t seed, const double *L);

/* Half a step of one Nose-Hoover thermostat of period tau (the Trotter
 * factor exp(iL_T dt/2) of Martyna, Tuckerman, Tobias & Klein 1996 with one
 * thermostat): with g = 3N - 3 degrees of freedom, G = (2 KE / g) / kT - 1,
 *   xi += dt/4 G / tau^2;  s = exp(-xi dt/2);  v *= s;  eta += xi dt/2;
 *   xi += dt/4 G' / tau^2 (G' with the scaled KE).
 * state = {xi, eta}.  Returns the scale s applied to the velocities. */
double orc_nh_half(int64_t n, double *vel, double mass, double kT, double tau,
                   double dt, double *state);

typedef struct {
    double L[3];
    double r_cut, r_skin, dt, mass, kT;
    uint64_t seed;
    int32_t pair;          /* pair kind (orc_pair_ncoeff) */
    int32_t ntypes;
    const double *coeff;
    int32_t shift_energy;
    int32_t thermo_period; /* 0 = never */
    double K, r0;          /* harmonic bonds */
    int64_t n_bonds;
    const int32_t *bonds;  /* index pairs */
    int64_t step0;         /* time step of the initial state */
    int32_t max_nb;
    int32_t integrator;    /* 0 = NVE velocity Verlet, 1 = Langevin (BAOAB),
                              2 = Nose-Hoover (one thermostat, MTK splitting) */
    double t_kT;           /* thermostat temperature */
    double t_gamma;        /* Langevin friction */
    double t_tau;          /* Nose-Hoover period */
    uint64_t t_seed;       /* Langevin noise key */
    double *nh_state;      /* Nose-Hoover {xi, eta}, updated in place (or NULL) */
    int32_t bond_style;    /* 0 = harmonic (K, r0), 1 = FENE (K, R0 = r0) */
    int64_t n_angles;      /* harmonic angles (index triplets, vertex in the middle) */
    const int32_t *angles;
    double angle_K, angle_theta0;
} orc_params;

/* Whole MD loop: forces at step0, then n_steps steps of the chosen
 * integrator (velocity Verlet, BAOAB Langevin, or velocity Verlet between
 * two Nose-Hoover half steps) with a Verlet list rebuilt when any particle
 * moved more than r_skin/2 since the last build.  thermo_out receives 8 doubles (orc_thermo) at every step t
 * with t % thermo_period == 0, t > step0.  force holds the final forces.
 * Returns the number of neighbour-list builds, or -1 on row overflow. */
int64_t orc_run(int64_t n, double *pos, double *vel, int32_t *image,
                const int32_t *type, const int32_t *tag, double *force,
                const orc_params *p, int64_t n_steps, double *thermo_out);

#ifdef __cplusplus
}
#endif
#endif
