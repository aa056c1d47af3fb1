/*
 * md.h -- C ABI of the GB300 short-range molecular-dynamics hot path.
 *
 * The library implements, on one GPU, the per-timestep path of the method of
 * Glaser et al., "Strong scaling of general-purpose molecular dynamics
 * simulations on GPUs" (HOOMD-blue 1.0): cell-list binning, a Verlet
 * neighbour list with a buffer (skin) rebuilt when a particle moved more than
 * half the buffer length, LJ and DPD pair forces, harmonic bonds and
 * velocity-Verlet integration in a periodic box, for one system or for a
 * batch of independent replicas in one launch per kernel.
 *
 * Conventions shared by every entry point
 *   - Plain C: pointers, sizes and status codes; no C++ or framework types.
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are host memory read during the call only.
 *   - Calls taking a stream only enqueue work on it and return without
 *     synchronising, unless stated otherwise.  Argument errors are reported
 *     immediately by the return code.  Errors found on the device (neighbour
 *     row overflow, a non-finite position, an over-full cell, a force
 *     evaluation on a list that does not match the current binning, a timed-
 *     out internal wait) are recorded in a device error word that
 *     md_poll_error() reads.
 *   - The library never allocates device memory: the caller passes one
 *     workspace buffer sized by md_workspace_size().  The system handle itself
 *     lives in host memory owned by the library (md_destroy_system frees it).
 *   - Indices are int32: at most 134,217,728 (2^27) particles per system.
 *     Neighbour-list entries are 16-bit slots of a brick's shared-memory
 *     stage, not particle indices (md_get_nlist decodes them).
 *   - Units are LJ / DPD reduced units, k_B = 1.
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_ABI_VERSION 8

typedef struct md_system md_system;
typedef struct CUstream_st *md_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID_ARG = 1,          /* bad pointer, size or parameter */
    MD_ERR_CUDA = 2,                 /* a CUDA runtime call failed */
    MD_ERR_WORKSPACE_TOO_SMALL = 3,  /* ws_bytes < md_workspace_size() */
    MD_ERR_NLIST_OVERFLOW = 4,       /* a neighbour row exceeded max_nb; detail = needed */
    MD_ERR_CELL_GRID = 5,            /* fewer than 3 cells per box edge */
    MD_ERR_NONFINITE = 6,            /* non-finite position after integration, or a finite
                                        one the periodic wrap cannot bring into the box */
    MD_ERR_CELL_OVERFLOW = 7,        /* a cell held more particles than can be ordered */
    MD_ERR_STATE = 8,                /* call not valid in the current state */
    MD_ERR_TIMEOUT = 9,              /* a kernel's wait for its own shared-memory copies gave
                                        up after about a second (an internal error); the
                                        kernel returned early */
    MD_ERR_BOND = 10                 /* a FENE bond reached its maximum extension R0;
                                        detail = the particle index */
} md_status;

/* Bond styles (Sec. 3 lists harmonic and FENE bonds). */
typedef enum { MD_BOND_HARMONIC = 0, MD_BOND_FENE = 1 } md_bond_style;

typedef enum { MD_FP64 = 0, MD_MIXED = 1 } md_precision;
/* Pair potentials (Sec. 3 lists LJ, DPD, Gaussian, Morse and Yukawa among
 * the supported pairs; textbook forms, force truncated at r_cut):
 *   MD_PAIR_LJ      (eps, sigma):       V = 4 eps [(sigma/r)^12 - (sigma/r)^6]
 *   MD_PAIR_DPD     (A, gamma):         Groot-Warren, see md_params.kT / seed
 *   MD_PAIR_GAUSS   (eps, sigma):       V = eps exp(-r^2 / (2 sigma^2))
 *   MD_PAIR_MORSE   (D0, alpha, r0):    V = D0 [e^(-2 alpha (r - r0)) - 2 e^(-alpha (r - r0))]
 *   MD_PAIR_YUKAWA  (eps, kappa):       V = eps e^(-kappa r) / r
 *   MD_PAIR_TABLE   (no coefficients):  V and F = -dV/dr sampled per type pair
 *                                       (md_set_pair_table), linear in r between
 *                                       samples; zero until a table is set */
typedef enum {
    MD_PAIR_LJ = 0,
    MD_PAIR_DPD = 1,
    MD_PAIR_GAUSS = 2,
    MD_PAIR_MORSE = 3,
    MD_PAIR_YUKAWA = 4,
    MD_PAIR_TABLE = 5
} md_pair_kind;
typedef enum { MD_KERNEL_NLIST = 0, MD_KERNEL_PAIR = 1 } md_kernel;
typedef enum { MD_NVE = 0, MD_LANGEVIN = 1, MD_NOSE_HOOVER = 2 } md_integrator;

/* Caller-owned particle state, all DEVICE arrays of N = n_total entries,
 * concatenated over replicas (replica r owns [replica_offset[r],
 * replica_offset[r+1])).  md_sort_particles permutes all five in place. */
typedef struct {
    double *pos;    /* [N][4] x, y, z in [0, L) of the particle's replica; w kept */
    double *vel;    /* [N][4] vx, vy, vz; w kept */
    int32_t *image; /* [N][4] periodic image counters; w kept */
    int32_t *tag;   /* [N] global particle IDs: a permutation of 0..N-1 */
    int32_t *type;  /* [N] particle type in [0, n_types) */
} md_particles;

/* Run parameters.  Paper references: list radius r_cut + r_buff and the
 * half-buffer rebuild rule (Sec. 4.2); w threads per particle and the block
 * size, set per kernel by md_autotune (Sec. 5.1-5.2). */
typedef struct {
    int64_t n_total;               /* N, summed over replicas */
    int32_t n_replicas;            /* R >= 1 */
    const int64_t *replica_offset; /* host [R+1], offset[0] = 0, offset[R] = N */
    const double *box;             /* host [R][3] orthorhombic edge lengths */
    double r_cut;                  /* pair cut-off */
    double r_skin;                 /* buffer length r_buff (> 0) */
    double dt;                     /* time step */
    double mass;                   /* particle mass (all particles) */
    double kT;                     /* DPD temperature */
    uint64_t seed;                 /* DPD noise key */
    int32_t pair;                  /* md_pair_kind */
    int32_t n_types;               /* >= 1, <= 32 */
    const double *pair_coeff;      /* host [n_types][n_types][k], k = 3 for
                                      Morse, 0 for the table (may be NULL),
                                      else 2 (coefficients of md_pair_kind, in
                                      its order); finite */
    int32_t precision;             /* md_precision */
    int32_t shift_energy;          /* LJ, Gaussian, Morse, Yukawa: report
                                      V(r) - V(r_cut) as energy */
    int32_t max_nb;                /* neighbour row capacity (rounded up to 32) */
    int32_t sort_period;           /* sort at the first rebuild >= this many
                                      steps after the last sort; 0 = never */
    int32_t thermo_period;         /* md_run: thermo row every this many steps;
                                      0 = none */
    int32_t graph_steps;           /* md_run: steps per captured CUDA graph
                                      (multiple of thermo_period); 0 = eager */
    int32_t max_bonds;             /* bonds per particle capacity; 0 = no bonds */
    int32_t max_angles;            /* angles per particle capacity (as an end or the
                                      vertex); 0 = no angles */
    int32_t table_points;          /* MD_PAIR_TABLE: samples per type pair, 2..65536 */
} md_params;

/* Thermodynamic row per replica, 8 doubles (Sec. 4.3.3 groups these global
 * reductions into one synchronisation per step):
 * {KE, PE, W, P, T, px, py, pz} = kinetic energy, potential energy, virial
 * trace, pressure (2 KE + W) / (3 V), temperature 2 KE / (3 N - 3), momentum.
 * PE and W are those of the last force evaluation made with want_virial = 1. */
#define MD_THERMO_FIELDS 8

int32_t md_abi_version(void);
const char *md_status_string(md_status s);

/* Bytes of device workspace a system with these parameters needs.
 * Errors: MD_ERR_INVALID_ARG, MD_ERR_CELL_GRID. */
md_status md_workspace_size(const md_params *p, size_t *bytes);

/* Creates a system over caller-owned particle arrays and workspace (both must
 * stay valid until md_destroy_system).  Sec. 4.1: the single-GPU code path
 * keeps all simulation data on the device and transfers nothing significant
 * between host and device while it runs; the host only plans and launches.
 * Builds the per-replica cell grids and space-filling-curve cell order on the
 * host, uploads them, and binds `parts`.
 * Enqueues initialisation on `stream`; does not build the neighbour list.
 * Errors: MD_ERR_INVALID_ARG, MD_ERR_CELL_GRID, MD_ERR_WORKSPACE_TOO_SMALL,
 * MD_ERR_CUDA. */
md_status md_create_system(const md_params *p, const md_particles *parts,
                           void *workspace, size_t ws_bytes, md_stream stream,
                           md_system **out);

/* Frees the host handle and any captured graph; the caller frees its memory.
 * Not in the paper (resource handling of this interface).  Errors:
 * MD_ERR_INVALID_ARG for a NULL handle. */
md_status md_destroy_system(md_system *s);

/* Harmonic bonds V = K/2 (r - r0)^2 between unordered pairs of particle IDs
 * (tags) (Sec. 4.3.4: a bond is an unordered pair of particle IDs with a
 * type).  bond_tags: HOST [n_bonds][2].  Stores, per particle ID, the IDs of
 * its partners; fails with MD_ERR_INVALID_ARG if any particle has more than
 * max_bonds partners.  Synchronises `stream`. */
md_status md_set_bonds(md_system *s, const int32_t *bond_tags, int64_t n_bonds,
                       double K, double r0, md_stream stream);

/* Tabulated pair potential (Sec. 3 lists tabulated potentials), for a
 * system created with pair = MD_PAIR_TABLE: table HOST double
 * [n_types][n_types][table_points][2] = (V_j, F_j) at r_j = r_min + j dr,
 * dr = (r_cut - r_min) / (table_points - 1), F = -dV/dr.  Between samples V and
 * F are linear in r; below r_min they keep their values at r_min; the force
 * on i is F(r) (x_i - x_j) / r for r < r_cut.  Energies are used as given
 * (shift_energy does not apply).  Uploads the table (FP32 in mixed systems,
 * FP64 otherwise) and synchronises `stream`.  Errors: MD_ERR_INVALID_ARG
 * (another pair kind, 0 <= r_min < r_cut violated, non-finite samples),
 * MD_ERR_CUDA. */
md_status md_set_pair_table(md_system *s, const double *table, double r_min,
                            md_stream stream);

/* Harmonic angles V = K/2 (theta - theta0)^2 (Sec. 3 lists harmonic angle
 * potentials; Sec. 4.3.4 treats angles like bonds, as groups of particle
 * IDs).  angle_tags: HOST [n_angles][3] particle IDs (a, b, c), b the
 * vertex, theta the angle between x_a - x_b and x_c - x_b (minimum image);
 * K >= 0, 0 <= theta0 <= pi.  Stores, per particle ID, the angles it takes
 * part in; each particle then sums its own force from them (no atomics),
 * and gets a third of each angle's energy and virial.  The forces are added
 * with the bonds' (md_compute_bonds, md_step, md_run).  Errors:
 * MD_ERR_INVALID_ARG (bad IDs, repeated IDs in a triplet, a particle in more
 * than max_angles angles, K or theta0 out of range).  Synchronises
 * `stream`. */
md_status md_set_angles(md_system *s, const int32_t *angle_tags, int64_t n_angles,
                        double K, double theta0, md_stream stream);

/* Bond style of md_set_bonds' bonds (Sec. 3 lists harmonic and FENE bonds):
 *   MD_BOND_HARMONIC  V = K/2 (r - r0)^2 (the default)
 *   MD_BOND_FENE      V = -K R0^2 / 2 ln(1 - (r / R0)^2), R0 = the r0 given to
 *                     md_set_bonds (> 0); finitely extensible, no repulsive
 *                     core (add it through the pair potential).  A bond at
 *                     r >= R0 contributes nothing and raises MD_ERR_BOND in the
 *                     device error word.
 * Errors: MD_ERR_INVALID_ARG (unknown style; FENE with r0 <= 0). */
md_status md_set_bond_style(md_system *s, int32_t style);

/* Space-filling-curve sort (Sec. 4.3.1: the particle arrays, positions,
 * velocities and the rest, are reordered together, infrequently, at list
 * rebuilds; the choice of a Hilbert curve over bricks of 2 x 2 x 2 cells is
 * this library's): reorders every caller particle array into the cell list's
 * order, i.e. bricks along the Hilbert curve, then the binning's order inside
 * each brick (cells x first, then y, then z; in a cell by x offset from the
 * cell centre, then index).  Errors: MD_ERR_INVALID_ARG, MD_ERR_STATE (no
 * binning yet), MD_ERR_CUDA.
 * force = 0: only replicas that rebuild now and whose last sort is
 * >= sort_period steps old.  Requires md_build_cells to have binned the
 * current positions (it sorts by that binning). */
md_status md_sort_particles(md_system *s, int32_t force, md_stream stream);

/* Cell-list binning (Sec. 4.3.3, Sec. 5.1): counts per cell, exclusive scan,
 * scatter, then the members of each cell ordered by their FP32 x offset from
 * the cell centre, ties by particle index.  force = 0: only
 * replicas whose rebuild flag was raised by md_integrate(half = 1).  The
 * neighbour list refers to the binning it was built from: after a forced
 * binning, md_compute_pair returns MD_ERR_STATE until md_build_nlist ran. */
md_status md_build_cells(md_system *s, int32_t force, md_stream stream);

/* Neighbour list (Sec. 5.1, Fig. "nlist"): w threads per particle stride over
 * the 27 cells around it and compact every j != i with
 * |x_i - x_j|^2 < (r_cut + r_skin)^2 (minimum image, FP64 decision) into
 * row i.  Records the build positions for the half-buffer test.
 * force = 0: only replicas whose rebuild flag is raised.  The build reads the
 * binning's member order; if particles moved through this API since the last
 * md_build_cells (md_integrate, md_step, md_run), it bins them again first.
 * After writing positions into the particle arrays directly, call
 * md_build_cells before this.
 * Row overflow: MD_ERR_NLIST_OVERFLOW in the device error word. */
md_status md_build_nlist(md_system *s, int32_t force, md_stream stream);

/* Pair forces from the neighbour list (Sec. 5.1: w threads per particle,
 * intra-warp reduction).  LJ 12-6 or DPD (Groot-Warren, noise from
 * Philox-4x32-10 keyed on (min tag, max tag, step, seed)), FP64 or mixed
 * precision.  want_virial = 1 also writes per-particle energy and virial.
 * Overwrites the force array. */
md_status md_compute_pair(md_system *s, int32_t want_virial, md_stream stream);

/* Adds harmonic-bond forces (md_set_bonds) to the force array: each particle
 * sums V = K/2 (r - r0)^2 over its own bonds (Sec. 3 lists harmonic bonds;
 * Sec. 4.3.4: a bond is an unordered pair of particle IDs, so the partner is
 * found through the tag table after any sort).  Per-particle energy gets half
 * of each bond's V and the virial half of r f when want_virial = 1.  No-op
 * without bonds.  Errors: MD_ERR_INVALID_ARG, MD_ERR_CUDA. */
md_status md_compute_bonds(md_system *s, int32_t want_virial, md_stream stream);

/* Velocity Verlet (Sec. 3).  half = 1: v += dt/2 F/m, x += dt v, wrap into the
 * box, advance the device step counter, and raise the replica's rebuild flag
 * if a particle moved more than r_skin/2 since the last list build
 * (Sec. 4.2).  half = 2: v += dt/2 F/m. */
md_status md_integrate(md_system *s, int32_t half, md_stream stream);

/* One full step: integrate(1), conditional sort / cells / nlist, pair, bonds,
 * integrate(2). want_virial as in md_compute_pair. */
md_status md_step(md_system *s, int32_t want_virial, md_stream stream);

/* Thermo reduction (FP64, fixed summation tree: bitwise reproducible):
 * writes R rows of MD_THERMO_FIELDS doubles to DEVICE memory dev_out. */
md_status md_reduce_thermo(md_system *s, double *dev_out, md_stream stream);

/* Runs n_steps full steps; segments of graph_steps steps replay one captured
 * CUDA graph (captured on first use, re-captured after md_autotune or
 * md_set_tuning).  Inside a graph each step's second half-kick is folded into
 * the next step's first (velocities hold v(t + 1/2) in between); thermo steps
 * and the last step of every graph end with the plain second half-kick, so
 * the velocities are full-step ones wherever thermo reads them and when the
 * call returns.  If thermo_out (DEVICE, [n_steps / thermo_period][R][8]) is
 * not NULL, a thermo row is written after every step t with
 * t % thermo_period == 0, in order.  While the device error word holds a
 * non-finite position or an over-full cell, list builds are skipped (the
 * steps' results are invalid; md_poll_error reports the error). */
md_status md_run(md_system *s, int64_t n_steps, double *thermo_out, md_stream stream);

/* Integrator (Sec. 3 lists NVE, NVT with the Martyna-Tobias-Klein update
 * equations, and Langevin dynamics; Sec. 6.1 runs NVT with a Nose-Hoover
 * thermostat that sums the kinetic energy once per step).  Default MD_NVE.
 *   MD_NVE          velocity Verlet; kT, param, seed unused.
 *   MD_LANGEVIN     BAOAB splitting with friction gamma = param >= 0:
 *                   v += dt/2 F/m; x += dt/2 v; v = c v + sqrt((1 - c^2) kT/m)
 *                   theta; x += dt/2 v; [forces]; v += dt/2 F/m, c =
 *                   exp(-gamma dt); theta = sqrt(3) (2u - 1) per component,
 *                   u from words 0..2 of Philox-4x32-10 with counter (tag,
 *                   0xFFFFFFFF, step lo, step hi) and key (seed lo, seed hi),
 *                   step = the time step being computed.
 *   MD_NOSE_HOOVER  one Nose-Hoover thermostat per replica, period tau =
 *                   param > 0, in the Trotter splitting exp(iL_T dt/2)
 *                   exp(iL_v dt/2) exp(iL_x dt) exp(iL_v dt/2) exp(iL_T dt/2);
 *                   each thermostat half step, with g = 3N - 3 and G =
 *                   (2 KE / g) / kT - 1: xi += dt/4 G / tau^2; v *= exp(-xi
 *                   dt/2); eta += xi dt/2; xi += dt/4 G' / tau^2 (G' after the
 *                   scaling).  The kinetic energy is summed once per step, in
 *                   the second half-kick; the resulting velocity scales are
 *                   applied by the next first half (md_integrate(1)), and by
 *                   md_step / md_run before they return.  Conserved:
 *                   KE + PE + g kT tau^2 xi^2 / 2 + g kT eta.
 * Resets the thermostat state (xi = eta = 0); the next step computes its
 * first half step from the velocities at that time (call this again after
 * writing velocities directly).  Not valid with DPD pair forces (their
 * noise and friction are the thermostat).  Errors: MD_ERR_INVALID_ARG. */
md_status md_set_integrator(md_system *s, int32_t kind, double kT, double param,
                            uint64_t seed);

/* Half neighbour list with Newton's third law, FP64 forms only (not in the
 * paper, whose Sec. 5.1 kernels use full lists): with enable = 1 each
 * pair within r_list is listed once, in the row of the particle with the
 * smaller cell-list position, and the pair kernel evaluates it once, adding
 * f_ij to that particle and -f_ij (and half the pair energy and virial) to
 * the partner with FP64 atomic adds.  Halves the FP64 pair arithmetic, the
 * bound of the FP64 form.  The order of the atomic adds varies from run to
 * run, so FP64 forces are reproducible only to rounding (within the 1e-12
 * rule), not bit for bit; md_get_nlist then returns the half rows.  The
 * list is rebuilt at the next step.  Errors: MD_ERR_INVALID_ARG (enable not
 * 0 or 1, or a mixed-precision system). */
md_status md_set_newton(md_system *s, int32_t enable);

/* Nose-Hoover state between steps (after the last completed step's end half
 * step), HOST [R][2] = (xi, eta) per replica.  Synchronises. */
md_status md_get_thermostat(md_system *s, double *host_out);

/* Autotuner (Sec. 5.2): for the pair and neighbour-list kernels, times every
 * (block size b = 32 k <= 512, threads per particle w = 2^m <= 32) pair with
 * the median of n_samples launches (paper: 5), and keeps the fastest.  Both
 * kernels are persistent: a block keeps one brick's data in shared memory
 * while the next brick's is copied in.  The list build's w is
 * at most the pair kernel's (the pair kernel's w fixes the list layout, and a
 * build pass must cover whole row groups of it).  block_stride (>= 1) thins
 * the block sizes to every block_stride-th multiple of 32.  Synchronises
 * `stream`; rebuilds the neighbour list. */
md_status md_autotune(md_system *s, int32_t n_samples, int32_t block_stride,
                      md_stream stream);

/* Sets / reads the launch parameters of one kernel (md_kernel): b threads per
 * block (a multiple of 32, at most the kernel's limit) and w threads per
 * particle.  Changing the pair kernel's w changes the list layout and forces
 * a rebuild; a list-build w above the pair kernel's runs at the pair
 * kernel's. */
md_status md_set_tuning(md_system *s, int32_t kernel, int32_t block, int32_t w);
md_status md_get_tuning(md_system *s, int32_t kernel, int32_t *block, int32_t *w);

/* Device step counter (time step of the current positions). */
md_status md_set_step(md_system *s, int64_t step, md_stream stream);
md_status md_get_step(md_system *s, int64_t *step); /* synchronises */

/* Synchronises the system's work and reads the device error word.  Not in
 * the paper (error reporting of this interface).  Returns MD_OK or the first
 * recorded error, in this order of precedence: MD_ERR_NLIST_OVERFLOW
 * (*detail = the max_nb needed), MD_ERR_NONFINITE (*detail = the index of a
 * particle with a non-finite position, or a finite one more than 1e9 box
 * lengths outside the box), MD_ERR_BOND (*detail = the index of a particle
 * with a FENE bond at or beyond R0), MD_ERR_CELL_OVERFLOW, MD_ERR_STATE (a
 * force evaluation found its replica's list stale and computed nothing),
 * MD_ERR_TIMEOUT.  The word is not cleared.  detail may be NULL. */
md_status md_poll_error(md_system *s, int64_t *detail);

/* --- inspection (tests, diagnostics) ------------------------------------ */

/* Forces as DEVICE double [N][4] (F, per-particle energy); virial (may be
 * NULL) as DEVICE double [N][6] (xx, xy, xz, yy, yz, zz). */
md_status md_get_forces(md_system *s, double *dev_force, double *dev_virial,
                        md_stream stream);

/* Neighbour rows as DEVICE int32 counts [N] and rows [N][max_nb] (plain
 * particle indices; entries past counts[i] are -1). */
md_status md_get_nlist(md_system *s, int32_t *dev_counts, int32_t *dev_rows,
                       md_stream stream);

/* Cell list as DEVICE arrays: cell_start / cell_count [total cells] (cells
 * in Hilbert order per replica, replicas concatenated), cell_idx [N]. */
md_status md_get_cells(md_system *s, int32_t *dev_start, int32_t *dev_count,
                       int32_t *dev_idx, md_stream stream);

/* Sizes: total cells, max_nb in use, number of list builds so far (syncs). */
md_status md_get_info(md_system *s, int64_t *n_cells, int32_t *max_nb,
                      int64_t *n_builds);

/* The device Philox-4x32-10 used for the DPD noise, exposed for bitwise
 * checks: in DEVICE [n][6] (ctr0..3, key0..1), out DEVICE [n][4]. */
md_status md_philox4x32_10(const uint32_t *dev_in, uint32_t *dev_out, int64_t n,
                           md_stream stream);

/* --- allocation-free entry point ----------------------------------------- */

/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory at all (a plugin whose host program owns every
 * device allocation, a real-time loop that cannot afford cudaMalloc's implicit
 * synchronisation): it computes FP64 LJ 12-6 forces of ONE periodic system
 * without a workspace, binning the particles into cells of width at least
 * r_cut (1 + 1e-12) and summing every pair within r_cut over the 27
 * surrounding cells (minimum image).
 *   dev_pos    DEVICE double [n][4] (x, y, z; w ignored), 16-B aligned; any
 *              finite coordinates (each is wrapped into [0, box) for binning)
 *   box        HOST double [3] edge lengths
 *   dev_force  DEVICE double [n][4] output: F, per-particle energy (half of each
 *              pair's unshifted V)
 * Scratch: a 4 MiB array in the library's device memory (1,048,576 int32),
 * reserved on every device the library is used on, until the process exits.
 * A call needs 3 n + 2 n_cells of them, n_cells = product over the edges of
 * min(floor(box / (r_cut (1 + 1e-12))), 1024); larger systems get MD_ERR_WORKSPACE_TOO_SMALL
 * before any launch.  Boxes under 3 cells per edge: MD_ERR_CELL_GRID.
 * The first call on a device looks up the array's device address (with that
 * device current): make that first call before any stream capture.  Calls use
 * no cudaMalloc / cudaFree.  All calls share the one array, so calls that may
 * overlap on the GPU (different streams, or different host threads) race:
 * serialise them.  Enqueues on `stream` and returns without synchronising. */
md_status md_lj_forces_noalloc(const double *dev_pos, int64_t n, const double *box,
                               double r_cut, double epsilon, double sigma,
                               double *dev_force, md_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* MD_GB300_H */
