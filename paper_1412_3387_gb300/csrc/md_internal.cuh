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
constexpr int kIdxBits = 27;          // neighbour entry: index bits, code in the top 5
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;
constexpr int kMaxCellSort = 256;     // largest cell the in-cell sort handles
constexpr int kCellBits = 9;          // packed cell coordinate bits (nc <= 512)
constexpr int64_t kMaxParticles = (int64_t)1 << kIdxBits;

// Device error word bits.
enum : uint32_t {
  kErrNlistOverflow = 1u << 0,
  kErrNonfinite = 1u << 1,
  kErrCellOverflow = 1u << 2,
  kErrBadInput = 1u << 3,
};

// Per-replica constants (device-resident copy + host mirror).
struct Rep {
  int64_t p0, p1;     // particle range [p0, p1)
  int64_t cell0;      // first cell slot (chunk aligned) in the cell arrays
  int64_t chunk0;     // first scan chunk
  int64_t tchunk0;    // first thermo chunk
  int32_t nc[3];      // cells per edge
  int32_t ncell;      // nc0 nc1 nc2
  int32_t nchunk;     // scan chunks
  int32_t ntchunk;    // thermo chunks
  double L[3];
  double inv_L[3];
  double h[3];        // L / nc
  double half_h[3];   // h / 2
  double inv_h[3];    // nc / L
  float hf[3];        // float(h): shift of a neighbouring cell's frame
  float band;         // FP32 r^2 uncertainty band (see DESIGN: exact decisions)
  double volume;
};

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
  uint32_t pad0;
  int64_t n_builds;      // replica list builds so far
  int64_t thermo_rows;   // md_run: capacity of thermo_out in rows
};

// Pair coefficients, prepared on the host.
struct LJCoeffD { double lj1, lj2, lj3, lj4, vshift, pad0, pad1, pad2; };  // 64 B
struct LJCoeffF { float lj1, lj2, lj3, lj4, vshift, pad0, pad1, pad2; };
struct DPDCoeffD { double A, gamma, sigma_rdt, pad; };  // sigma / sqrt(dt)
struct DPDCoeffF { float A, gamma, sigma_rdt, pad; };

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
  float4 *pos4f;       // frame-relative FP32 position, packed frame cell + type
  float4 *oref;        // frame-relative position at the last build
  float4 *vel4f;       // FP32 velocity, tag bits in w (DPD mixed)
  int32_t *cell_rank;  // [cells] linear cell -> Hilbert rank (per replica)
  const uint32_t *stencil;  // [cells][27] neighbour cells by ascending rank | code << 27
  int32_t *cell_count; // [cells]
  int32_t *cell_start; // [cells] first particle (global index)
  int32_t *chunk_sum;  // [chunks]
  int32_t *cell_idx;   // [N]
  int32_t *pcell;      // [N] cell slot of each particle (binning)
  int32_t *pslot;      // [N] rank inside its cell (binning)
  uint16_t *nl;        // [max_nb * n_pad] stage slots, rows indexed by cell position
  int32_t *n_nb;       // [n_pad] row lengths, indexed by cell position
  int32_t stage_cap;   // stage slots per warp (pair / list kernels)
  void *force;         // double4[N] (FP64) or float4[N] (mixed)
  void *virial;        // double[N][6] or float[N][6]
  double *tpart;       // [thermo chunks][8]
  DevState *ds;
  int32_t *rebuild;    // [R][2]
  int32_t *sort_now;   // [R]
  int64_t *last_sort;  // [R]
  int32_t *rtag;       // [N] tag -> index
  int32_t *ident;      // [R] 1 while the replica's particles are in cell order
  int32_t *btab;       // [N][max_bonds] partner tags (-1 = none)
  // sort scratch
  double4 *s_pos, *s_vel;
  int4 *s_img;
  int32_t *s_tag, *s_type;
  float4 *s_pos4f, *s_oref, *s_vel4f;
  const void *coeff;   // LJCoeff* / DPDCoeff* [ntypes^2], precision-matched
  // parameters
  int32_t max_nb;
  int32_t w_store_log2;  // neighbour-list tile width (pair kernel's w)
  int32_t sort_period;
  int32_t max_bonds;
  int32_t mixed;
  int32_t pair;
  double r_cut, rc2, rl2;
  float rc2f, rl2f;
  double dt, mass, kT;
  double half_dt_m;    // dt / (2 m), computed once on the host
  double bond_K, bond_r0;
  float disp2_f;       // (r_skin / 2)^2, slightly reduced
  uint64_t seed;
  int64_t n_chunks, n_tchunks, n_cells;
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

// FP32 offset of x from the centre (c + 1/2) h of frame cell c, folded into
// (-L/2, L/2].  FP64 instructions are scarce on GB300, so the centre is one
// FP64 multiply-add and the periodic fold (needed only once the particle has
// crossed the box since its frame was set) is decided on the FP32 value: the
// offsets stay below h + skin << L/2, far from the fold's threshold.
__device__ __forceinline__ float frame_offset_fast(double x, int c, double h, double half_h,
                                                   double L) {
  double d = x - fma((double)c, h, half_h);
  const float df = (float)d;
  if (fabsf(df) > 0.5f * (float)L) d += df > 0.f ? -L : L;
  return (float)d;
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

// ---- cell stage ------------------------------------------------------------
// The stage of home cell g is the concatenation, in ascending Hilbert rank,
// of the members of the 27 cells around g (g included).  Slot s holds the
// member's FP32 frame offset plus the offset d h of its cell relative to g
// (d in {-1,0,1}^3), so that x_i - x_j = o_i - stage[s] for a home particle
// i.  Rows of the neighbour list hold stage slots (16 bits: a stage has at
// most 27 x kMaxCellSort slots).  A block stages at most `stage_cap` slots at
// a time; denser neighbourhoods are processed in windows of that size (rows
// are in ascending slot order, so each window is a contiguous part of a row).
struct StageInfo {
  int off[28];          // first slot of each stencil cell; off[27] = total
  int start[27];        // cell_start of each stencil cell
  float sx[27], sy[27], sz[27];  // image shift d h of each stencil cell
  int self;             // first slot of the home cell's own members
  int pad[3];
};

// Filled by the first warp of the block (lanes 0..26: one stencil cell each);
// the caller synchronises the block before use.
__device__ __forceinline__ void stage_info(const KArgs &a, const Rep &rp, int64_t g, StageInfo &si) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  int cnt = 0, code = -1;
  if (lane < 27) {
    const uint32_t e = __ldg(a.stencil + g * 27 + lane);
    const int64_t cell = rp.cell0 + (int64_t)(e & kIdxMask);
    code = (int)(e >> kIdxBits);
    cnt = __ldg(a.cell_count + cell);
    si.start[lane] = __ldg(a.cell_start + cell);
    si.sx[lane] = (float)(code % 3 - 1) * rp.hf[0];
    si.sy[lane] = (float)((code / 3) % 3 - 1) * rp.hf[1];
    si.sz[lane] = (float)(code / 9 - 1) * rp.hf[2];
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < 27) si.off[lane] = incl - cnt;
  if (lane == 26) si.off[27] = incl;
  if (code == 13) si.self = incl - cnt;
}

// Stencil cell holding stage slot `slot` (largest s with off[s] <= slot).
__device__ __forceinline__ int stage_cell(const StageInfo &si, int slot) {
  int s = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1)
    if (s + step < 27 && si.off[s + step] <= slot) s += step;
  return s;
}

// Fills window slots [w0, w0 + m) of the stage with all threads of the block:
// positions (pre-shifted), and particle indices / FP32 velocities when idx /
// vel are given.  Each thread takes slots tid, tid + blockDim, ...; kUnroll of
// them are looked up and loaded independently before any is stored, so a
// stage costs about one memory latency.  When the replica's particles are in
// cell order (`ident`: after each space-filling-curve sort, until the next
// binning) cell members are index ranges and the cell_idx lookup is skipped.
// The caller synchronises the block before and after.
__device__ __forceinline__ void stage_fill(const KArgs &a, const StageInfo &si, int w0, int m,
                                           bool ident, float4 *pos, int32_t *idx, float4 *vel) {
  constexpr int kUnroll = 4;
  const int nt = blockDim.x;
  for (int b = 0; b < m; b += nt * kUnroll) {
    int32_t j[kUnroll];
    int sc[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const int k = b + u * nt + threadIdx.x;
      j[u] = -1;
      sc[u] = 0;
      if (k < m) {
        const int slot = w0 + k;
        const int s = stage_cell(si, slot);
        sc[u] = s;
        const int at = si.start[s] + (slot - si.off[s]);
        j[u] = ident ? at : __ldg(a.cell_idx + at);
      }
    }
    float4 o[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
      o[u] = j[u] >= 0 ? __ldg(a.pos4f + j[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      if (j[u] < 0) continue;
      const int k = b + u * nt + threadIdx.x;
      const int s = sc[u];
      pos[k] = make_float4(o[u].x + si.sx[s], o[u].y + si.sy[s], o[u].z + si.sz[s], o[u].w);
      if (idx) idx[k] = j[u];
      if (vel) vel[k] = __ldg(a.vel4f + j[u]);
    }
  }
}

// Shared memory of one block: StageInfo, then stage_cap slots of positions,
// indices and (DPD) velocities.
__host__ __device__ __forceinline__ size_t stage_bytes(int cap, bool with_vel) {
  return sizeof(StageInfo) + (size_t)cap * (sizeof(float4) + sizeof(int32_t)) +
         (with_vel ? (size_t)cap * sizeof(float4) : 0);
}

// Neighbour-list address of entry k of row p for tile width 2^lw.
__device__ __forceinline__ size_t nl_addr(int64_t i, int k, int lw, int64_t n_pad) {
  return ((((size_t)(k >> lw)) * (size_t)n_pad + (size_t)i) << lw) | (size_t)(k & ((1 << lw) - 1));
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

cudaError_t launch_integrate1(const KArgs &a, cudaStream_t st);
cudaError_t launch_integrate2(const KArgs &a, cudaStream_t st);
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
int max_block_nlist(int w, int cap);
int max_block_pair(const KArgs &a, int w, int want_virial);

}  // namespace mdgb
