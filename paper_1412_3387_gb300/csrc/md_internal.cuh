// Internal definitions shared by the CUDA translation units of libmdgb.
// Not part of the public ABI (include/md.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/md.h"

namespace mdgb {

constexpr int kMaxTypes = 32;
constexpr int kChunkCells = 2048;     // cells per scan chunk (256 threads x 8)
constexpr int kThermoChunk = 4096;    // particles per thermo partial sum
constexpr int kNhFields = 6;          // Nose-Hoover state doubles per replica
constexpr int kMaxCellSort = 256;     // largest cell the in-cell sort handles
constexpr int kCellBits = 9;          // packed cell coordinate bits (nc <= 512)
// Largest system: 2^27 particles (about 80 GB of state and list at the
// benchmark's density); int32 indices and cell-list positions everywhere.
constexpr int64_t kMaxParticles = (int64_t)1 << 27;

// Device error word bits.
enum : uint32_t {
  kErrNlistOverflow = 1u << 0,
  kErrNonfinite = 1u << 1,
  kErrCellOverflow = 1u << 2,
  kErrBadInput = 1u << 3,
  kErrTimeout = 1u << 4,
  kErrStaleList = 1u << 5,  // pair forces asked for before the list of a new binning
  kErrBond = 1u << 6,       // a FENE bond at or beyond its maximum extension
};

// Per-replica constants (device-resident copy + host mirror).
struct Rep {
  int64_t p0, p1;     // particle range [p0, p1)
  int64_t cell0;      // first cell slot (chunk aligned) in the cell arrays
  int64_t chunk0;     // first scan chunk
  int64_t tchunk0;    // first thermo chunk
  int64_t brick0;     // first brick (brick.cuh)
  int64_t nbrick;     // bricks
  int32_t nc[3];      // cells per edge
  int32_t ncell;      // nc0 nc1 nc2
  int32_t nchunk;     // scan chunks
  int32_t ntchunk;    // thermo chunks
  double L[3];
  double inv_L[3];
  double h[3];        // L / nc
  double half_h[3];   // h / 2
  double inv_h[3];    // nc / L
  // Stage frame (brick.cuh): FP32 offsets and stage coordinates are exact
  // multiples of the grid gq (a power of two), frame cells are hq apart (h
  // rounded to a multiple of 2 gq) and a periodic image shifts by wq (L - nc hq
  // rounded to gq).  Every stage coordinate and every separation is then an
  // exactly computed FP32 number: x_i - x_j seen from i's brick is exactly
  // minus x_j - x_i seen from j's, so pair forces are exactly antisymmetric.
  float hq[3];
  float gq[3];
  float wq[3];
  float cq[3];        // 1.5 2^23 gq: the frame centres in ctab are shifted down by it
  float weps;         // slack of the list build's x-windows (covers h - hq drift)
  float Lf[3];        // float(L)
  int64_t ctab0;      // first entry of the replica's cell-centre table (x, then y, then z)
  float band;         // FP32 r^2 uncertainty band around r_list^2 and r_cut^2
  double volume;
};

struct BrickDesc;  // brick.cuh

// Global device state (one per system, in the workspace).
struct DevState {
  int64_t step;          // time step of the current positions
  int64_t run_base;      // md_run: step before the first step of the run
  double *thermo_out;    // md_run: device output rows (or null)
  int64_t thermo_period;
  uint32_t error;        // OR of kErr* bits
  int32_t need_max_nb;   // largest row seen when overflowing
  int64_t error_detail;  // particle index of the first non-finite position
  uint32_t blocks_done;  // integrate(1) last-block ticket
  int32_t rebuild_any;   // some replica's rebuild flag is raised for the current step
  int64_t n_builds;      // replica list builds so far
  int64_t thermo_rows;   // md_run: capacity of thermo_out in rows
  uint32_t nh_done;      // Nose-Hoover reduction last-block ticket
};

// Pair coefficients, prepared on the host.
struct LJCoeffD { double lj1, lj2, lj3, lj4, vshift, pad0, pad1, pad2; };  // 64 B
struct LJCoeffF { float lj1, lj2, lj3, lj4, vshift, pad0, pad1, pad2; };
struct DPDCoeffD { double A, gamma, sigma_rdt, pad; };  // sigma / sqrt(dt)
struct DPDCoeffF { float A, gamma, sigma_rdt, pad; };
// Gaussian (c0 = 1 / (2 sigma^2), c1 = eps / sigma^2, c2 = eps), Morse
// (c0 = alpha, c1 = r0, c2 = 2 D0 alpha, c3 = D0), Yukawa (c0 = kappa,
// c1 = eps); vshift = V(r_cut) when energies are shifted.  Table: c0 = r_min,
// c1 = 1 / dr, c2 = the last segment's index, c3 = the type pair's first
// segment (integer bits); each segment is (V_j, F_j, V_j+1 - V_j, F_j+1 - F_j).
struct PotCoeffD { double c0, c1, c2, c3, vshift, pad0, pad1, pad2; };  // 64 B
struct PotCoeffF { float c0, c1, c2, c3, vshift, pad0, pad1, pad2; };

// Everything a kernel needs, passed by value (< 4 KB).
struct KArgs {
  int64_t n;           // particles
  int64_t n_pad;       // padded particle count (list pitch)
  int32_t R;
  int32_t ntypes;
  const int64_t *rep_off;  // [R+1]
  const Rep *rep;          // [R]
  const int32_t *chunk_rep;   // [n chunks] replica of each scan chunk
  const int32_t *tchunk_rep;  // [n thermo chunks]
  // caller state
  double4 *pos;
  double4 *vel;
  int4 *image;
  int32_t *tag;
  int32_t *type;
  // internal
  float4 *pos4f;       // [cell-list position] frame-relative FP32 position, packed frame cell + type
  float4 *oref;        // [particle] frame-relative position at the last build
  float4 *vel4f;       // [cell-list position] FP32 velocity, tag bits in w (DPD)
  int32_t *cellpos;    // [particle] cell-list position
  int32_t *cell_rank;  // [cells] linear cell -> rank in brick order (per replica)
  const double *ctab;  // frame centres (c + 1/2) hq - cq per replica and axis (FP64)
  const int32_t *brick_stage;  // [bricks][64] cell slot of each stage cell (brick.cuh)
  const int4 *brick_info;      // [bricks] first cell slot, cell mask, replica
  const int32_t *brick_rep;    // [bricks] replica
  BrickDesc *brick_desc;       // [bricks] stage layouts of the current binning
  int32_t *cell_count; // [cells]
  int32_t *cell_start; // [cells] first particle (global index)
  int32_t *chunk_sum;  // [chunks]
  int32_t *cell_idx;   // [N]
  int32_t *pcell;      // [N] cell slot of each particle (binning)
  int32_t *pslot;      // [N] rank inside its cell (binning)
  uint16_t *nl;        // [n_pad * max_nb] 1 + stage slot, row groups (brick.cuh)
  int32_t *nl_tiles;   // [n_pad] tiles of the row group starting at this cell-list position
  int32_t *n_nb;       // [n_pad] row lengths, indexed by cell position
  int32_t stage_cap;   // staged particles per brick buffer
  void *force;         // double4[N] (FP64) or float4[N] (mixed)
  void *virial;        // double[N][6] or float[N][6]
  double *tpart;       // [thermo chunks][8]
  DevState *ds;
  int32_t *rebuild;    // [R][2]
  int32_t *sort_now;   // [R]
  int64_t *last_sort;  // [R]
  int32_t *rtag;       // [N] tag -> index
  int32_t *ident;      // [R] 1 while the replica's particles are in cell order
  int32_t *list_ok;    // [R] 1 while the replica's list matches its binning
  int32_t *btab;       // [N][max_bonds] partner tags (-1 = none)
  int32_t *atab;       // [N][max_angles][3] angle triplets by tag (-1 = none)
  // sort scratch
  double4 *s_pos, *s_vel;
  int4 *s_img;
  int32_t *s_tag, *s_type;
  float4 *s_oref;
  const void *coeff;   // LJCoeff* / DPDCoeff* / PotCoeff* [ntypes^2], precision-matched
  const void *table;   // float4* / double4* segments of tabulated pairs
  // the single type pair's FP32 coefficients, as kernel parameters: the
  // mixed pair loops take them as constant operands instead of re-loading
  // them from memory
  LJCoeffF lj1f;
  DPDCoeffF dpd1f;
  PotCoeffF pot1f;
  // parameters
  int32_t max_nb;        // a multiple of 32
  int32_t w_store_log2;  // neighbour-list tile width (pair kernel's w)
  int32_t sort_period;
  int32_t max_bonds;
  int32_t mixed;
  int32_t pair;
  // half list (md_set_newton): each pair's row entry only in the row of the
  // particle with the smaller cell-list position; the FP64 pair kernel adds
  // -f_ij to the partner with atomics
  int32_t half;
  double r_cut, rc2, rl2;
  float rc2f, rl2f;
  double dt, mass, kT;
  double half_dt_m;    // dt / (2 m), computed once on the host
  double bond_K, bond_r0;
  int32_t bond_style;  // md_bond_style
  int32_t max_angles;
  double angle_K, angle_th0;
  // thermostat (md_set_integrator)
  int32_t integ;         // md_integrator
  double t_kT, t_c, t_sig, t_tau;  // kT; Langevin exp(-gamma dt), sqrt((1 - c^2) kT / m); NH tau
  uint64_t t_seed;
  double *nh;            // [R][kNhFields] Nose-Hoover: xi, eta (for the next step), start-of-step
                         // scale, pending end-of-step scale, xi, eta between steps (reported)
  double *nh_part;       // [thermo chunks] kinetic-energy partial sums
  float disp2_f;       // (r_skin / 2)^2, slightly reduced
  uint64_t seed;
  int64_t n_chunks, n_tchunks, n_cells, n_bricks;
};

// ---- device helpers -------------------------------------------------------

__device__ __forceinline__ int replica_of(const KArgs &a, int64_t i) {
  if (a.R == 1) return 0;
  int lo = 0, hi = a.R - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(a.rep_off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz, int type) {
  return (uint32_t)cx | ((uint32_t)cy << kCellBits) | ((uint32_t)cz << (2 * kCellBits)) |
         ((uint32_t)type << (3 * kCellBits));
}
__device__ __forceinline__ int cell_x(uint32_t w) { return (int)(w & 511u); }
__device__ __forceinline__ int cell_y(uint32_t w) { return (int)((w >> kCellBits) & 511u); }
__device__ __forceinline__ int cell_z(uint32_t w) { return (int)((w >> (2 * kCellBits)) & 511u); }
__device__ __forceinline__ int cell_type(uint32_t w) { return (int)(w >> (3 * kCellBits)); }

// Cell coordinate exactly as floor(x * (nc / L)) clamped to [0, nc).
__device__ __forceinline__ int cell_coord(double x, double inv_h, int nc) {
  int c = (int)floor(__dmul_rn(x, inv_h));
  c = c >= nc ? nc - 1 : c;
  return c < 0 ? 0 : c;
}

// FP32 offset of x from the centre (c + 1/2) hq of its frame cell c,
// rounded once to the replica's grid gq (a power of two).  ctr_q is that
// centre minus cq = 1.5 2^23 gq (exact in FP64): x - ctr_q lies in
// [2^23 gq, 2^24 gq) while |offset| < 2^22 gq, and there the FP32 numbers are
// exactly the multiples of gq, so the conversion rounds the offset to the
// grid and subtracting cq is exact.  FP64 instructions are scarce on GB300
// (a few per clock per SM), so the centre comes from a table and the periodic
// fold (needed only once the particle has crossed the box since its frame
// was set) is decided on the FP32 value: offsets stay below h + skin << L/2.
// The periodic image of the offset (a particle that crossed the box since its
// frame cell was chosen).  Out of line: the FP64 work stays off the common
// path instead of being issued there under a predicate.
static __device__ __noinline__ float frame_offset_image(double d, double L, float cq, float o) {
  return (float)(d + (o > 0.f ? -L : L)) - cq;
}

__device__ __forceinline__ float frame_offset(double x, double ctr_q, float cq, float Lf, double L) {
  const double d = x - ctr_q;
  const float o = (float)d - cq;
  if (fabsf(o) > 0.5f * Lf) return frame_offset_image(d, L, cq, o);
  return o;
}

// Frame centre of cell c along axis ax of replica rp, minus cq.
__device__ __forceinline__ double cell_centre(const KArgs &a, const Rep &rp, int ax, int c) {
  const int off = ax == 0 ? 0 : ax == 1 ? rp.nc[0] : rp.nc[0] + rp.nc[1];
  return __ldg(a.ctab + rp.ctab0 + off + c);
}

// Exact FP64 minimum-image r^2 with a fixed operation order and no FMA:
// dx = (x_i - x_j) - L rint((x_i - x_j) / L); r2 = (dx dx + dy dy) + dz dz.
__device__ __forceinline__ double exact_r2(const double4 &pi, const double4 &pj, const Rep &rp,
                                           double *d) {
  double dx = __dsub_rn(pi.x, pj.x);
  double dy = __dsub_rn(pi.y, pj.y);
  double dz = __dsub_rn(pi.z, pj.z);
  dx = __dsub_rn(dx, __dmul_rn(rp.L[0], rint(__dmul_rn(dx, rp.inv_L[0]))));
  dy = __dsub_rn(dy, __dmul_rn(rp.L[1], rint(__dmul_rn(dy, rp.inv_L[1]))));
  dz = __dsub_rn(dz, __dmul_rn(rp.L[2], rint(__dmul_rn(dz, rp.inv_L[2]))));
  d[0] = dx; d[1] = dy; d[2] = dz;
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ double4 ld_d4(const double4 *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ void set_error(DevState *ds, uint32_t bit) { atomicOr(&ds->error, bit); }

// ---- Philox-4x32-10 (Salmon et al., SC'11) --------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

__device__ __forceinline__ uint32_t dpd_word(int32_t ti, int32_t tj, uint64_t step, uint64_t seed) {
  uint32_t a = (uint32_t)ti, b = (uint32_t)tj;
  U4 c{a < b ? a : b, a < b ? b : a, (uint32_t)step, (uint32_t)(step >> 32)};
  return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32)).x;
}

// ---- launch wrappers (defined in the k_*.cu files) ------------------------
struct Launch { int block; int w; };

// fold_kick: also apply the previous step's second half-kick (it was left out)
cudaError_t launch_integrate1(const KArgs &a, cudaStream_t st, bool fold_kick = false);
cudaError_t launch_integrate2(const KArgs &a, cudaStream_t st);
// Nose-Hoover: sum the kinetic energy and take the thermostat's half step
// (begin = 1: at the start of a sequence of steps, without a kick); flush:
// apply the pending end-of-step scale to the velocities.
cudaError_t launch_nh_begin(const KArgs &a, cudaStream_t st);
cudaError_t launch_nh_flush(const KArgs &a, cudaStream_t st);
cudaError_t launch_nh_reset(const KArgs &a, cudaStream_t st);
cudaError_t launch_bin(const KArgs &a, int force, cudaStream_t st);
cudaError_t launch_sort(const KArgs &a, int force, cudaStream_t st);
cudaError_t launch_nlist(const KArgs &a, Launch l, int force, cudaStream_t st);
cudaError_t launch_pair(const KArgs &a, Launch l, int want_virial, cudaStream_t st);
void pair_init_attributes();
void nlist_init_attributes();
cudaError_t launch_bonds(const KArgs &a, int want_virial, cudaStream_t st);
cudaError_t launch_thermo(const KArgs &a, double *out, int from_run, cudaStream_t st);
cudaError_t launch_set_step(const KArgs &a, int64_t step, cudaStream_t st);
cudaError_t launch_run_begin(const KArgs &a, double *out, int64_t period, int64_t rows,
                             cudaStream_t st);
cudaError_t launch_clear_state(const KArgs &a, cudaStream_t st);
cudaError_t launch_force_rebuild_flags(const KArgs &a, cudaStream_t st);
cudaError_t launch_export_forces(const KArgs &a, double *f, double *v, cudaStream_t st);
cudaError_t launch_export_nlist(const KArgs &a, int32_t *counts, int32_t *rows, cudaStream_t st);
cudaError_t launch_export_cells(const KArgs &a, int32_t *start, int32_t *count, int32_t *idx,
                                cudaStream_t st);
cudaError_t launch_philox(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t st);
cudaError_t launch_init_frames(const KArgs &a, cudaStream_t st);
int max_block_nlist(const KArgs &a, int w);
int max_block_pair(const KArgs &a, int w, int want_virial);
// Blocks of a persistent launch: resident blocks per SM x SMs, at most `work`.
int persistent_grid(const void *kernel, int threads, size_t smem, int64_t work);

}  // namespace mdgb
