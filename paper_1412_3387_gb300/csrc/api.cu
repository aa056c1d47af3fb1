// C ABI of libmdgb (include/md.h): system set-up, workspace layout, the step
// sequence, CUDA-graph capture of multi-step runs and the autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "md_internal.cuh"
#include "brick.cuh"

using namespace mdgb;


struct md_system {
  md_params p{};
  std::vector<int64_t> off;
  std::vector<double> box;
  std::vector<double> coeff;
  md_particles parts{};
  KArgs a{};
  std::vector<Rep> reps;
  Launch tune[2]{{128, 2}, {128, 2}};  // nlist, pair (computing threads, w)
  bool built = false;   // list built and forces computed (ready to step)
  bool binned = false;  // cells binned at least once
  bool listed = false;  // list built in the current layout
  // The binning is current (no particle moved since): for every replica, or
  // for the replicas that rebuild.  The list build needs it (it searches
  // x-windows in the cells' member order).
  bool bin_all = false, bin_cond = false;
  int64_t step = 0;
  int64_t n_bonds = 0;
  int64_t n_angles = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool gvalid = false;
  // Nose-Hoover: the start-of-step thermostat scale has been computed for the
  // current velocities
  bool nh_primed = false;
};

namespace {

#define MD_CUDA(x)                                  \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return MD_ERR_CUDA;      \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kMaxTuneBlock = 512;  // largest computing-thread count the tuner tries

int ilog2(int w) { int l = 0; while ((1 << l) < w) l++; return l; }

// 3-D Hilbert index of cell (x, y, z) on a 2^bits grid (Skilling, AIP Conf.
// Proc. 707, 2004).  The coordinates are turned into the curve's "transposed"
// index by walking the bit levels from the top, reflecting or exchanging the
// lower bits at each level; a Gray decode across the axes and the bit
// interleave then give the index.  Written independently of the oracle's copy.
uint64_t hilbert_key(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint32_t c[3] = {x, y, z};
  for (int lvl = bits - 1; lvl >= 1; --lvl) {
    const uint32_t bit = 1u << lvl, below = bit - 1u;
    for (int ax = 0; ax < 3; ++ax) {
      if (c[ax] & bit) {
        c[0] ^= below;  // reflect axis 0's lower bits
      } else {
        const uint32_t swap = (c[0] ^ c[ax]) & below;  // exchange lower bits
        c[0] ^= swap;
        c[ax] ^= swap;
      }
    }
  }
  for (int ax = 1; ax < 3; ++ax) c[ax] ^= c[ax - 1];
  uint32_t mask = 0;
  for (int lvl = bits - 1; lvl >= 1; --lvl)
    if (c[2] & (1u << lvl)) mask ^= (1u << lvl) - 1u;
  for (int ax = 0; ax < 3; ++ax) c[ax] ^= mask;
  uint64_t key = 0;
  for (int lvl = bits - 1; lvl >= 0; --lvl)
    for (int ax = 0; ax < 3; ++ax) key = (key << 1) | ((c[ax] >> lvl) & 1u);
  return key;
}

struct Plan {
  std::vector<Rep> reps;
  int64_t n = 0, n_pad = 0, n_cells = 0, n_chunks = 0, n_tchunks = 0;
  int32_t max_nb = 0;
  int32_t stage_cap = 0;
  int64_t n_bricks = 0, n_ctab = 0;
  // byte offsets into the workspace
  size_t o_rep, o_off, o_chunk_rep, o_tchunk_rep, o_cell_rank, o_ctab, o_brick_stage, o_brick_info,
      o_brick_rep, o_brick_desc, o_cell_count, o_cell_start,
      o_chunk_sum, o_cell_idx, o_cellpos, o_pcell, o_pslot, o_n_nb, o_rtag, o_pos4f, o_oref, o_vel4f,
      o_nl, o_nl_tiles, o_force, o_virial, o_tpart, o_ds, o_rebuild, o_sort_now, o_last_sort, o_ident,
      o_list_ok, o_coeff, o_table, o_btab, o_atab, o_s_pos, o_s_vel, o_s_img, o_s_tag, o_s_type, o_s_oref, o_nh,
      o_nh_part;
  size_t total = 0;
};

// Coefficients per ordered type pair of each pair kind (md.h).
int pair_ncoeff(int32_t pair) {
  return pair == MD_PAIR_MORSE ? 3 : pair == MD_PAIR_TABLE ? 0 : 2;
}

// The float whose bits are those of the integer i (host side).
float int_bits_as_float(int i) {
  float f;
  std::memcpy(&f, &i, sizeof(f));
  return f;
}

md_status validate(const md_params *p) {
  if (!p) return MD_ERR_INVALID_ARG;
  if (p->n_total < 0 || p->n_total > kMaxParticles) return MD_ERR_INVALID_ARG;
  if (p->n_replicas < 1 || !p->replica_offset || !p->box) return MD_ERR_INVALID_ARG;
  if (p->replica_offset[0] != 0 || p->replica_offset[p->n_replicas] != p->n_total)
    return MD_ERR_INVALID_ARG;
  for (int r = 0; r < p->n_replicas; r++)
    if (p->replica_offset[r + 1] < p->replica_offset[r]) return MD_ERR_INVALID_ARG;
  if (!(p->r_cut > 0) || !(p->r_skin > 0) || !(p->dt > 0) || !(p->mass > 0))
    return MD_ERR_INVALID_ARG;
  if (!std::isfinite(p->r_cut) || !std::isfinite(p->r_skin) || !std::isfinite(p->dt))
    return MD_ERR_INVALID_ARG;
  if (p->pair < MD_PAIR_LJ || p->pair > MD_PAIR_TABLE) return MD_ERR_INVALID_ARG;
  if (p->pair == MD_PAIR_TABLE && (p->table_points < 2 || p->table_points > 65536))
    return MD_ERR_INVALID_ARG;
  if (p->precision != MD_FP64 && p->precision != MD_MIXED) return MD_ERR_INVALID_ARG;
  if (p->n_types < 1 || p->n_types > kMaxTypes) return MD_ERR_INVALID_ARG;
  if (pair_ncoeff(p->pair) > 0 && !p->pair_coeff) return MD_ERR_INVALID_ARG;
  if (p->pair == MD_PAIR_DPD && !(p->kT >= 0)) return MD_ERR_INVALID_ARG;
  for (int k = 0; k < pair_ncoeff(p->pair) * p->n_types * p->n_types; k++)
    if (!std::isfinite(p->pair_coeff[k])) return MD_ERR_INVALID_ARG;
  if (p->max_nb < 1 || p->max_nb > (1 << 20)) return MD_ERR_INVALID_ARG;
  if (p->sort_period < 0 || p->thermo_period < 0 || p->graph_steps < 0 || p->max_bonds < 0 ||
      p->max_angles < 0 || p->max_angles > 64)
    return MD_ERR_INVALID_ARG;
  if (p->graph_steps > 0 && p->thermo_period > 0 && p->graph_steps % p->thermo_period != 0)
    return MD_ERR_INVALID_ARG;
  for (int k = 0; k < 3 * p->n_replicas; k++)
    if (!(p->box[k] > 0) || !std::isfinite(p->box[k])) return MD_ERR_INVALID_ARG;
  return MD_OK;
}

md_status make_plan(const md_params *p, Plan &pl) {
  md_status st = validate(p);
  if (st != MD_OK) return st;
  const int R = p->n_replicas;
  const double rl = p->r_cut + p->r_skin;
  pl.n = p->n_total;
  pl.n_pad = std::max<int64_t>(128, (p->n_total + 127) / 128 * 128);
  pl.max_nb = (p->max_nb + 31) / 32 * 32;
  pl.reps.resize(R);
  int64_t cell0 = 0, chunk0 = 0, tchunk0 = 0;
  for (int r = 0; r < R; r++) {
    Rep &rp = pl.reps[r];
    std::memset(&rp, 0, sizeof(rp));
    rp.p0 = p->replica_offset[r];
    rp.p1 = p->replica_offset[r + 1];
    double hmax = 0;
    for (int d = 0; d < 3; d++) {
      const double L = p->box[3 * r + d];
      // cells at least r_list (1 + 1e-12) wide: with cells exactly r_list wide
      // (a box an exact multiple of r_list), the rounding of x / h could put
      // two particles closer than r_list two cells apart
      double m = std::floor(L / (rl * (1.0 + 1e-12)));
      if (m > 512.0) m = 512.0;
      if (m < 3.0) return MD_ERR_CELL_GRID;
      rp.nc[d] = (int32_t)m;
      rp.L[d] = L;
      rp.inv_L[d] = 1.0 / L;
      rp.h[d] = L / (double)rp.nc[d];
      rp.half_h[d] = 0.5 * rp.h[d];
      rp.inv_h[d] = (double)rp.nc[d] / L;
      rp.Lf[d] = (float)L;
      hmax = std::max(hmax, rp.h[d]);
    }
    // Stage frame (brick.cuh), per axis: the smallest power-of-two grid gq for
    // which every frame offset, |o| <= h/2 + skin/2 + drift, stays below
    // 2^22 gq (frame_offset's rounding trick) and every stage coordinate,
    // |o| + 1.5 hq + |wq|, below 2^24 gq (exact FP32 sums and differences).
    // hq = h rounded to a multiple of 2 gq; the frame centres (c + 1/2) hq
    // drift from the cell centres by at most nc |hq - h|.
    double gmax = 0.0, drift_max = 0.0;
    for (int d = 0; d < 3; d++) {
      const double h = rp.h[d], L = rp.L[d];
      const int nc = rp.nc[d];
      double g = std::ldexp(1.0, -40), hq = h, wq = 0.0, drift = 0.0;
      for (;;) {
        hq = 2.0 * g * std::nearbyint(h / (2.0 * g));
        wq = g * std::nearbyint((L - nc * hq) / g);
        drift = nc * std::fabs(hq - h) + g;
        const double omax = 0.5 * h + 0.5 * p->r_skin + drift;
        if (omax < std::ldexp(g, 22) && omax + 1.5 * hq + std::fabs(wq) < std::ldexp(g, 24)) break;
        g *= 2.0;
      }
      rp.gq[d] = (float)g;
      rp.hq[d] = (float)hq;
      rp.wq[d] = (float)wq;
      rp.cq[d] = (float)(1.5 * std::ldexp(g, 23));
      gmax = std::max(gmax, g);
      drift_max = std::max(drift_max, drift);
    }
    rp.weps = (float)(1e-4 * hmax + 2.0 * drift_max + 4.0 * gmax);
    // FP32 r^2 uncertainty: each separation component is exact up to the grid
    // rounding of two offsets and of wq (<= 1.5 gq), and r^2 = dx^2 + dy^2 +
    // dz^2 is rounded three times, so near r_list
    //   |dr^2| <= 2 r_list sqrt(3) 1.5 gq + 3 2^-24 r_list^2.
    // The band is the larger of 64 2^-24 (h + skin)^2 and four times that.
    {
      const double rl = p->r_cut + p->r_skin;
      const double err = 2.0 * rl * std::sqrt(3.0) * 1.5 * gmax + 3.0 * std::ldexp(rl * rl, -24);
      rp.band = (float)std::max(64.0 * std::ldexp(1.0, -24) * (hmax + p->r_skin) * (hmax + p->r_skin),
                                4.0 * err);
    }
    rp.volume = rp.L[0] * rp.L[1] * rp.L[2];
    rp.ncell = rp.nc[0] * rp.nc[1] * rp.nc[2];
    rp.nchunk = (rp.ncell + kChunkCells - 1) / kChunkCells;
    const int64_t np = rp.p1 - rp.p0;
    rp.ntchunk = (int32_t)((np + kThermoChunk - 1) / kThermoChunk);
    rp.cell0 = cell0;
    rp.chunk0 = chunk0;
    rp.tchunk0 = tchunk0;
    rp.brick0 = pl.n_bricks;
    rp.ctab0 = pl.n_ctab;
    pl.n_ctab += rp.nc[0] + rp.nc[1] + rp.nc[2];
    rp.nbrick = ((rp.nc[0] + 1) / 2) * ((rp.nc[1] + 1) / 2) * ((rp.nc[2] + 1) / 2);
    pl.n_bricks += rp.nbrick;
    cell0 += (int64_t)rp.nchunk * kChunkCells;
    chunk0 += rp.nchunk;
    tchunk0 += rp.ntchunk;
  }
  // Brick stage buffers (brick.cuh): room for the mean population m of the 64
  // stage cells of the densest replica plus six Poisson standard deviations
  // (a liquid fluctuates less); a brick beyond that is served from global
  // memory instead.  Two buffers (positions, and velocities for
  // mixed-precision DPD) must fit well inside shared memory.
  double dens = 0.0;
  for (const Rep &rp : pl.reps)
    if (rp.ncell > 0) dens = std::max(dens, (double)(rp.p1 - rp.p0) / rp.ncell);
  const bool vel = p->pair == MD_PAIR_DPD && p->precision == MD_MIXED;
  const double m = 64.0 * dens;
  int cap = (int)std::ceil((m + 6.0 * std::sqrt(m) + 64.0) / 32.0) * 32;
  cap = std::min(cap, 64 * kMaxCellSort);
  while (BrickSmem::bytes(cap, vel, 0) > 160u * 1024u) cap /= 2;
  pl.stage_cap = std::max(cap, 32);
  pl.n_cells = cell0;
  if (pl.n_cells > (int64_t)INT32_MAX) return MD_ERR_CELL_GRID;
  pl.n_chunks = chunk0;
  pl.n_tchunks = tchunk0;
  const bool mixed = p->precision == MD_MIXED;
  const bool dpd = p->pair == MD_PAIR_DPD;
  const int64_t N = pl.n, NP = pl.n_pad;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + std::max<size_t>(bytes, 1)); return at; };
  pl.o_rep = take(sizeof(Rep) * R);
  pl.o_off = take(sizeof(int64_t) * (R + 1));
  pl.o_chunk_rep = take(sizeof(int32_t) * pl.n_chunks);
  pl.o_tchunk_rep = take(sizeof(int32_t) * pl.n_tchunks);
  pl.o_cell_rank = take(sizeof(int32_t) * pl.n_cells);
  pl.o_ctab = take(sizeof(double) * (size_t)pl.n_ctab);
  pl.o_brick_stage = take(sizeof(int32_t) * kStageCells * (size_t)pl.n_bricks);
  pl.o_brick_info = take(sizeof(int4) * (size_t)pl.n_bricks);
  pl.o_brick_rep = take(sizeof(int32_t) * (size_t)pl.n_bricks);
  pl.o_brick_desc = take(sizeof(BrickDesc) * (size_t)pl.n_bricks);
  pl.o_cell_count = take(sizeof(int32_t) * pl.n_cells);
  pl.o_cell_start = take(sizeof(int32_t) * pl.n_cells);
  pl.o_chunk_sum = take(sizeof(int32_t) * pl.n_chunks);
  pl.o_cell_idx = take(sizeof(int32_t) * N);
  pl.o_cellpos = take(sizeof(int32_t) * N);
  pl.o_pcell = take(sizeof(int32_t) * N);
  pl.o_pslot = take(sizeof(int32_t) * N);
  pl.o_n_nb = take(sizeof(int32_t) * NP);
  pl.o_rtag = take(sizeof(int32_t) * N);
  pl.o_pos4f = take(sizeof(float4) * NP);
  pl.o_oref = take(sizeof(float4) * NP);
  pl.o_vel4f = dpd ? take(sizeof(float4) * NP) : 0;
  pl.o_nl = take(sizeof(uint16_t) * (size_t)pl.max_nb * NP);
  pl.o_nl_tiles = take(sizeof(int32_t) * NP);
  pl.o_force = take((mixed ? sizeof(float4) : sizeof(double4)) * NP);
  pl.o_virial = take((mixed ? sizeof(float) : sizeof(double)) * 6 * NP);
  pl.o_tpart = take(sizeof(double) * 8 * pl.n_tchunks);
  pl.o_ds = take(sizeof(DevState));
  pl.o_rebuild = take(sizeof(int32_t) * 2 * R);
  pl.o_sort_now = take(sizeof(int32_t) * R);
  pl.o_last_sort = take(sizeof(int64_t) * R);
  pl.o_ident = take(sizeof(int32_t) * R);
  pl.o_list_ok = take(sizeof(int32_t) * R);
  pl.o_coeff = take(64 * (size_t)p->n_types * p->n_types);
  pl.o_table = take(p->pair == MD_PAIR_TABLE
                        ? (p->precision == MD_MIXED ? 16 : 32) * (size_t)p->n_types * p->n_types *
                              (size_t)p->table_points
                        : 0);
  pl.o_btab = take(sizeof(int32_t) * (size_t)std::max(p->max_bonds, 0) * N);
  pl.o_atab = take(sizeof(int32_t) * 3 * (size_t)std::max(p->max_angles, 0) * N);
  pl.o_s_pos = take(sizeof(double4) * N);
  pl.o_s_vel = take(sizeof(double4) * N);
  pl.o_s_img = take(sizeof(int4) * N);
  pl.o_s_tag = take(sizeof(int32_t) * N);
  pl.o_s_type = take(sizeof(int32_t) * N);
  pl.o_s_oref = take(sizeof(float4) * N);
  pl.o_nh = take(sizeof(double) * kNhFields * R);
  pl.o_nh_part = take(sizeof(double) * (size_t)pl.n_tchunks);
  pl.total = o;
  return MD_OK;
}

template <class T>
T *at(void *base, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(base) + off); }

// One step.  fold_in: the previous step left its second half-kick out, this
// step's first half applies both.  close: apply this step's second half-kick
// (else it is left to the next step; velocities then hold v(t + 1/2)).
md_status enqueue_step(md_system *s, int want_virial, cudaStream_t st, bool fold_in = false,
                       bool close = true) {
  const KArgs &a = s->a;
  if (a.integ == MD_NOSE_HOOVER) {
    // the thermostat needs every step's second half-kick (its kinetic-energy
    // sum lives there): no folding
    fold_in = false;
    close = true;
  }
  MD_CUDA(launch_integrate1(a, st, fold_in));
  MD_CUDA(launch_bin(a, 0, st));
  if (s->p.sort_period > 0) MD_CUDA(launch_sort(a, 0, st));
  MD_CUDA(launch_nlist(a, s->tune[MD_KERNEL_NLIST], 0, st));
  MD_CUDA(launch_pair(a, s->tune[MD_KERNEL_PAIR], want_virial, st));
  if (s->n_bonds > 0 || s->n_angles > 0) MD_CUDA(launch_bonds(a, want_virial, st));
  if (close) MD_CUDA(launch_integrate2(a, st));
  return MD_OK;
}

md_status prepare(md_system *s, cudaStream_t st) {
  if (s->built) return MD_OK;
  MD_CUDA(launch_bin(s->a, 1, st));
  s->binned = s->bin_all = s->bin_cond = true;
  MD_CUDA(launch_nlist(s->a, s->tune[MD_KERNEL_NLIST], 1, st));
  s->listed = true;
  MD_CUDA(launch_pair(s->a, s->tune[MD_KERNEL_PAIR], 0, st));
  if (s->n_bonds > 0 || s->n_angles > 0) MD_CUDA(launch_bonds(s->a, 0, st));
  s->built = true;
  return MD_OK;
}

void set_pair_w(md_system *s, Launch l) {
  s->tune[MD_KERNEL_PAIR] = l;
  s->a.w_store_log2 = ilog2(l.w);
  s->gvalid = false;
}

// Nose-Hoover: the first step of a sequence needs the thermostat's
// start-of-step half step from the current velocities.
cudaError_t nh_prime(md_system *s, cudaStream_t st) {
  if (s->a.integ != MD_NOSE_HOOVER || s->nh_primed) return cudaSuccess;
  s->nh_primed = true;
  return launch_nh_begin(s->a, st);
}

bool valid_launch(int block, int w) {
  return block >= 32 && block <= 1024 && block % 32 == 0 &&
         (w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32);
}

}  // namespace

namespace mdgb {

int persistent_grid(const void *kernel, int threads, size_t smem, int64_t work) {
  static int dev = -1, nsm = 0;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return 0;
  if (d != dev) {
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) return 0;
    dev = d;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess)
    return 0;
  if (per <= 0) return 0;
  const int64_t g = std::min<int64_t>((int64_t)per * nsm, std::max<int64_t>(work, 1));
  return (int)g;
}

}  // namespace mdgb

extern "C" {

int32_t md_abi_version(void) { return MD_ABI_VERSION; }

const char *md_status_string(md_status s) {
  switch (s) {
    case MD_OK: return "ok";
    case MD_ERR_INVALID_ARG: return "invalid argument";
    case MD_ERR_CUDA: return "CUDA runtime error";
    case MD_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case MD_ERR_NLIST_OVERFLOW: return "neighbour row overflow (raise max_nb)";
    case MD_ERR_CELL_GRID: return "box smaller than 3 cells of r_cut + r_skin per edge";
    case MD_ERR_NONFINITE: return "non-finite particle position";
    case MD_ERR_CELL_OVERFLOW: return "cell occupancy above the in-cell sort limit";
    case MD_ERR_STATE: return "call not valid in the current state";
    case MD_ERR_TIMEOUT: return "a kernel's internal wait timed out (internal error)";
    case MD_ERR_BOND: return "a FENE bond reached its maximum extension";
  }
  return "unknown status";
}

md_status md_workspace_size(const md_params *p, size_t *bytes) {
  if (!bytes) return MD_ERR_INVALID_ARG;
  Plan pl;
  md_status st = make_plan(p, pl);
  if (st != MD_OK) return st;
  *bytes = pl.total;
  return MD_OK;
}

md_status md_create_system(const md_params *p, const md_particles *parts, void *workspace,
                           size_t ws_bytes, md_stream stream_, md_system **out) {
  if (!out || !parts) return MD_ERR_INVALID_ARG;
  *out = nullptr;
  Plan pl;
  md_status st = make_plan(p, pl);
  if (st != MD_OK) return st;
  if (!workspace || ws_bytes < pl.total) return MD_ERR_WORKSPACE_TOO_SMALL;
  if (((uintptr_t)workspace & 255) != 0) return MD_ERR_INVALID_ARG;
  if (p->n_total > 0 && (!parts->pos || !parts->vel || !parts->image || !parts->tag || !parts->type))
    return MD_ERR_INVALID_ARG;
  if (((uintptr_t)parts->pos & 15) || ((uintptr_t)parts->vel & 15) || ((uintptr_t)parts->image & 15))
    return MD_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);

  static bool attributes_set = false;  // opt the kernels into large shared memory once
  if (!attributes_set) {
    nlist_init_attributes();
    pair_init_attributes();
    attributes_set = true;
  }
  md_system *s = new (std::nothrow) md_system();
  if (!s) return MD_ERR_INVALID_ARG;
  s->p = *p;
  const int R = p->n_replicas;
  s->off.assign(p->replica_offset, p->replica_offset + R + 1);
  s->box.assign(p->box, p->box + 3 * R);
  if (pair_ncoeff(p->pair) > 0)
    s->coeff.assign(p->pair_coeff, p->pair_coeff + pair_ncoeff(p->pair) * p->n_types * p->n_types);
  s->p.replica_offset = s->off.data();
  s->p.box = s->box.data();
  s->p.pair_coeff = s->coeff.data();
  s->p.max_nb = pl.max_nb;
  s->parts = *parts;
  s->reps = pl.reps;

  KArgs &a = s->a;
  std::memset(&a, 0, sizeof(a));
  void *ws = workspace;
  const bool mixed = p->precision == MD_MIXED, dpd = p->pair == MD_PAIR_DPD;
  a.n = pl.n;
  a.n_pad = pl.n_pad;
  a.R = R;
  a.ntypes = p->n_types;
  a.rep_off = at<int64_t>(ws, pl.o_off);
  a.rep = at<Rep>(ws, pl.o_rep);
  a.chunk_rep = at<int32_t>(ws, pl.o_chunk_rep);
  a.tchunk_rep = at<int32_t>(ws, pl.o_tchunk_rep);
  a.pos = reinterpret_cast<double4 *>(parts->pos);
  a.vel = reinterpret_cast<double4 *>(parts->vel);
  a.image = reinterpret_cast<int4 *>(parts->image);
  a.tag = parts->tag;
  a.type = parts->type;
  a.pos4f = at<float4>(ws, pl.o_pos4f);
  a.oref = at<float4>(ws, pl.o_oref);
  a.vel4f = dpd ? at<float4>(ws, pl.o_vel4f) : nullptr;
  a.cell_rank = at<int32_t>(ws, pl.o_cell_rank);
  a.ctab = at<double>(ws, pl.o_ctab);
  a.brick_stage = at<int32_t>(ws, pl.o_brick_stage);
  a.brick_info = at<int4>(ws, pl.o_brick_info);
  a.brick_rep = at<int32_t>(ws, pl.o_brick_rep);
  a.brick_desc = at<BrickDesc>(ws, pl.o_brick_desc);
  a.cell_count = at<int32_t>(ws, pl.o_cell_count);
  a.cell_start = at<int32_t>(ws, pl.o_cell_start);
  a.chunk_sum = at<int32_t>(ws, pl.o_chunk_sum);
  a.cell_idx = at<int32_t>(ws, pl.o_cell_idx);
  a.cellpos = at<int32_t>(ws, pl.o_cellpos);
  a.pcell = at<int32_t>(ws, pl.o_pcell);
  a.pslot = at<int32_t>(ws, pl.o_pslot);
  a.nl = at<uint16_t>(ws, pl.o_nl);
  a.nl_tiles = at<int32_t>(ws, pl.o_nl_tiles);
  a.stage_cap = pl.stage_cap;
  a.n_nb = at<int32_t>(ws, pl.o_n_nb);
  a.force = at<void>(ws, pl.o_force);
  a.virial = at<void>(ws, pl.o_virial);
  a.tpart = at<double>(ws, pl.o_tpart);
  a.ds = at<DevState>(ws, pl.o_ds);
  a.rebuild = at<int32_t>(ws, pl.o_rebuild);
  a.sort_now = at<int32_t>(ws, pl.o_sort_now);
  a.last_sort = at<int64_t>(ws, pl.o_last_sort);
  a.ident = at<int32_t>(ws, pl.o_ident);
  a.list_ok = at<int32_t>(ws, pl.o_list_ok);
  a.rtag = at<int32_t>(ws, pl.o_rtag);
  a.btab = p->max_bonds > 0 ? at<int32_t>(ws, pl.o_btab) : nullptr;
  a.atab = p->max_angles > 0 ? at<int32_t>(ws, pl.o_atab) : nullptr;
  a.max_angles = p->max_angles;
  a.s_pos = at<double4>(ws, pl.o_s_pos);
  a.s_vel = at<double4>(ws, pl.o_s_vel);
  a.s_img = at<int4>(ws, pl.o_s_img);
  a.s_tag = at<int32_t>(ws, pl.o_s_tag);
  a.s_type = at<int32_t>(ws, pl.o_s_type);
  a.s_oref = at<float4>(ws, pl.o_s_oref);
  a.coeff = at<void>(ws, pl.o_coeff);
  a.table = at<void>(ws, pl.o_table);
  a.nh = at<double>(ws, pl.o_nh);
  a.nh_part = at<double>(ws, pl.o_nh_part);
  a.integ = MD_NVE;
  a.t_kT = 1.0;
  a.t_c = 1.0;
  a.t_tau = 1.0;
  a.max_nb = pl.max_nb;
  a.sort_period = p->sort_period;
  a.max_bonds = p->max_bonds;
  a.mixed = mixed;
  a.pair = p->pair;
  const double rl = p->r_cut + p->r_skin;
  a.r_cut = p->r_cut;
  a.rc2 = p->r_cut * p->r_cut;
  a.rl2 = rl * rl;
  a.rc2f = (float)a.rc2;
  a.rl2f = (float)a.rl2;
  a.dt = p->dt;
  a.mass = p->mass;
  a.kT = p->kT;
  a.half_dt_m = 0.5 * p->dt / p->mass;
  a.seed = p->seed;
  a.disp2_f = (float)(0.25 * p->r_skin * p->r_skin * (1.0 - 1e-4));
  a.n_chunks = pl.n_chunks;
  a.n_tchunks = pl.n_tchunks;
  a.n_cells = pl.n_cells;
  a.n_bricks = pl.n_bricks;

  // host tables: cell ranks (bricks of 2 x 2 x 2 cells along a Hilbert curve,
  // the cells of a brick x first, then y, then z) and per brick its 64 stage
  // cells and its own cells
  std::vector<int32_t> chunk_rep(pl.n_chunks), tchunk_rep(pl.n_tchunks);
  std::vector<int32_t> rank(pl.n_cells, 0);
  std::vector<int32_t> bstage((size_t)pl.n_bricks * kStageCells, 0);
  std::vector<int4> binfo((size_t)pl.n_bricks);
  std::vector<int32_t> brep((size_t)pl.n_bricks, 0);
  std::vector<double> ctab((size_t)pl.n_ctab, 0.0);
  for (int r = 0; r < R; r++) {
    const Rep &rp = pl.reps[r];
    for (int c = 0; c < rp.nchunk; c++) chunk_rep[rp.chunk0 + c] = r;
    for (int c = 0; c < rp.ntchunk; c++) tchunk_rep[rp.tchunk0 + c] = r;
    for (int d = 0, off = 0; d < 3; off += rp.nc[d], d++)
      for (int c = 0; c < rp.nc[d]; c++)  // exact: (c + 1/2) hq and cq are multiples of gq
        ctab[rp.ctab0 + off + c] = ((double)c + 0.5) * (double)rp.hq[d] - (double)rp.cq[d];
    const int nb[3] = {(rp.nc[0] + 1) / 2, (rp.nc[1] + 1) / 2, (rp.nc[2] + 1) / 2};
    const int nmax = std::max(nb[0], std::max(nb[1], nb[2]));
    int bits = 1;
    while ((1 << bits) < nmax) bits++;
    std::vector<std::pair<uint64_t, int32_t>> keys((size_t)rp.nbrick);
    for (int z = 0; z < nb[2]; z++)
      for (int y = 0; y < nb[1]; y++)
        for (int x = 0; x < nb[0]; x++) {
          const int32_t lin = x + nb[0] * (y + nb[1] * z);
          keys[lin] = {hilbert_key(x, y, z, bits), lin};
        }
    std::sort(keys.begin(), keys.end());
    auto cell_lin = [&](int x, int y, int z) {
      x = ((x % rp.nc[0]) + rp.nc[0]) % rp.nc[0];
      y = ((y % rp.nc[1]) + rp.nc[1]) % rp.nc[1];
      z = ((z % rp.nc[2]) + rp.nc[2]) % rp.nc[2];
      return x + rp.nc[0] * (y + rp.nc[1] * z);
    };
    int32_t k = 0;
    for (int64_t bi = 0; bi < rp.nbrick; bi++) {
      const int32_t lin = keys[bi].second;
      const int bx = lin % nb[0], by = (lin / nb[0]) % nb[1], bz = lin / (nb[0] * nb[1]);
      const int64_t B = rp.brick0 + bi;
      int mask = 0;
      const int32_t first = k;
      for (int q = 0; q < 8; q++) {
        const int x = 2 * bx + (q & 1), y = 2 * by + ((q >> 1) & 1), z = 2 * bz + (q >> 2);
        if (x >= rp.nc[0] || y >= rp.nc[1] || z >= rp.nc[2]) continue;
        rank[rp.cell0 + cell_lin(x, y, z)] = k++;
        mask |= 1 << q;
      }
      binfo[B] = make_int4((int)(rp.cell0 + first), mask, r, bx | (by << 10) | (bz << 20));
      brep[B] = r;
    }
    for (int64_t bi = 0; bi < rp.nbrick; bi++) {
      const int32_t lin = keys[bi].second;
      const int bx = lin % nb[0], by = (lin / nb[0]) % nb[1], bz = lin / (nb[0] * nb[1]);
      const int64_t B = rp.brick0 + bi;
      for (int s = 0; s < kStageCells; s++) {
        const int x = 2 * bx - 1 + (s & 3), y = 2 * by - 1 + ((s >> 2) & 3), z = 2 * bz - 1 + (s >> 4);
        bstage[(size_t)B * kStageCells + s] = (int32_t)(rp.cell0 + rank[rp.cell0 + cell_lin(x, y, z)]);
      }
    }
  }
  std::vector<unsigned char> coeff(64 * (size_t)p->n_types * p->n_types, 0);
  for (int ti = 0; ti < p->n_types; ti++)
    for (int tj = 0; tj < p->n_types; tj++) {
      const int c = ti * p->n_types + tj;
      const int nk = pair_ncoeff(p->pair);
      if (nk == 0) continue;  // the table's coefficients come with md_set_pair_table
      const double c0 = p->pair_coeff[nk * c], c1 = p->pair_coeff[nk * c + 1];
      if (p->pair == MD_PAIR_GAUSS || p->pair == MD_PAIR_MORSE || p->pair == MD_PAIR_YUKAWA) {
        // Gaussian (eps, sigma), Morse (D0, alpha, r0), Yukawa (eps, kappa)
        double k0 = 0, k1 = 0, k2 = 0, k3 = 0, vc = 0;
        const double rc = p->r_cut;
        if (p->pair == MD_PAIR_GAUSS) {
          k0 = 1.0 / (2.0 * c1 * c1), k1 = c0 / (c1 * c1), k2 = c0;
          vc = c0 * std::exp(-rc * rc * k0);
        } else if (p->pair == MD_PAIR_MORSE) {
          const double r0 = p->pair_coeff[nk * c + 2];
          k0 = c1, k1 = r0, k2 = 2.0 * c0 * c1, k3 = c0;
          const double x = std::exp(-c1 * (rc - r0));
          vc = c0 * x * (x - 2.0);
        } else {
          k0 = c1, k1 = c0;
          vc = c0 * std::exp(-c1 * rc) / rc;
        }
        if (!p->shift_energy) vc = 0.0;
        if (mixed) {
          PotCoeffF f{(float)k0, (float)k1, (float)k2, (float)k3, (float)vc, 0, 0, 0};
          std::memcpy(coeff.data() + sizeof(PotCoeffF) * c, &f, sizeof(f));
          if (c == 0) a.pot1f = f;
        } else {
          PotCoeffD d{k0, k1, k2, k3, vc, 0, 0, 0};
          std::memcpy(coeff.data() + sizeof(PotCoeffD) * c, &d, sizeof(d));
        }
      } else if (p->pair == MD_PAIR_LJ) {
        const double eps = c0, sig = c1;
        const double s6 = std::pow(sig, 6), s12 = s6 * s6;
        const double sr6 = s6 / std::pow(p->r_cut, 6);
        const double vc = p->shift_energy ? 4.0 * eps * (sr6 * sr6 - sr6) : 0.0;
        if (mixed) {
          LJCoeffF f{(float)(48 * eps * s12), (float)(24 * eps * s6), (float)(4 * eps * s12),
                     (float)(4 * eps * s6), (float)vc, 0, 0, 0};
          std::memcpy(coeff.data() + sizeof(LJCoeffF) * c, &f, sizeof(f));
          if (c == 0) a.lj1f = f;
        } else {
          LJCoeffD d{48 * eps * s12, 24 * eps * s6, 4 * eps * s12, 4 * eps * s6, vc, 0, 0, 0};
          std::memcpy(coeff.data() + sizeof(LJCoeffD) * c, &d, sizeof(d));
        }
      } else {
        const double A = c0, gamma = c1;
        const double srdt = std::sqrt(2.0 * gamma * p->kT) / std::sqrt(p->dt);
        if (mixed) {
          DPDCoeffF f{(float)A, (float)gamma, (float)srdt, 0};
          std::memcpy(coeff.data() + sizeof(DPDCoeffF) * c, &f, sizeof(f));
          if (c == 0) a.dpd1f = f;
        } else {
          DPDCoeffD d{A, gamma, srdt, 0};
          std::memcpy(coeff.data() + sizeof(DPDCoeffD) * c, &d, sizeof(d));
        }
      }
    }

  auto fail = [&](md_status e) { delete s; return e; };
  if (cudaMemcpyAsync(at<void>(ws, pl.o_rep), pl.reps.data(), sizeof(Rep) * R, cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_off), s->off.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_chunk_rep), chunk_rep.data(), sizeof(int32_t) * pl.n_chunks, cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_tchunk_rep), tchunk_rep.data(), sizeof(int32_t) * pl.n_tchunks, cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_cell_rank), rank.data(), sizeof(int32_t) * pl.n_cells, cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_ctab), ctab.data(), sizeof(double) * ctab.size(), cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_brick_stage), bstage.data(), sizeof(int32_t) * bstage.size(), cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_brick_info), binfo.data(), sizeof(int4) * binfo.size(), cudaMemcpyHostToDevice, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_brick_rep), brep.data(), sizeof(int32_t) * brep.size(), cudaMemcpyHostToDevice, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_brick_desc), 0, sizeof(BrickDesc) * (size_t)pl.n_bricks, stream) ||
      cudaMemcpyAsync(at<void>(ws, pl.o_coeff), coeff.data(), coeff.size(), cudaMemcpyHostToDevice, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_table), 0,
                      p->pair == MD_PAIR_TABLE
                          ? (mixed ? 16 : 32) * (size_t)p->n_types * p->n_types * (size_t)p->table_points
                          : 0,
                      stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_cell_count), 0, sizeof(int32_t) * pl.n_cells, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_cell_start), 0, sizeof(int32_t) * pl.n_cells, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_n_nb), 0, sizeof(int32_t) * pl.n_pad, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_nl), 0, sizeof(uint16_t) * (size_t)pl.max_nb * pl.n_pad, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_nl_tiles), 0, sizeof(int32_t) * pl.n_pad, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_rtag), 0, sizeof(int32_t) * pl.n, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_pcell), 0, sizeof(int32_t) * pl.n, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_pslot), 0, sizeof(int32_t) * pl.n, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_force), 0, (mixed ? 16 : 32) * pl.n_pad, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_virial), 0, (mixed ? 4 : 8) * 6 * pl.n_pad, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_ds), 0, sizeof(DevState), stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_rebuild), 0, sizeof(int32_t) * 2 * R, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_sort_now), 0, sizeof(int32_t) * R, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_last_sort), 0, sizeof(int64_t) * R, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_ident), 0, sizeof(int32_t) * R, stream) ||
      cudaMemsetAsync(at<void>(ws, pl.o_list_ok), 0, sizeof(int32_t) * R, stream))
    return fail(MD_ERR_CUDA);
  if (p->max_bonds > 0 &&
      cudaMemsetAsync(at<void>(ws, pl.o_btab), 0xff, sizeof(int32_t) * (size_t)p->max_bonds * pl.n, stream))
    return fail(MD_ERR_CUDA);
  if (p->max_angles > 0 &&
      cudaMemsetAsync(at<void>(ws, pl.o_atab), 0xff, sizeof(int32_t) * 3 * (size_t)p->max_angles * pl.n,
                      stream))
    return fail(MD_ERR_CUDA);
  if (launch_init_frames(a, stream) != cudaSuccess) return fail(MD_ERR_CUDA);
  if (launch_nh_reset(a, stream) != cudaSuccess) return fail(MD_ERR_CUDA);
  if (cudaStreamSynchronize(stream) != cudaSuccess) return fail(MD_ERR_CUDA);
  uint32_t err = 0;
  if (cudaMemcpy(&err, &a.ds->error, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MD_ERR_CUDA);
  if (err & kErrBadInput) return fail(MD_ERR_INVALID_ARG);
  if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(MD_ERR_CUDA);
  set_pair_w(s, s->tune[MD_KERNEL_PAIR]);
  *out = s;
  return MD_OK;
}

md_status md_destroy_system(md_system *s) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->cap) cudaStreamDestroy(s->cap);
  delete s;
  return MD_OK;
}

md_status md_set_bonds(md_system *s, const int32_t *bond_tags, int64_t n_bonds, double K,
                       double r0, md_stream stream_) {
  if (!s || n_bonds < 0 || (n_bonds > 0 && !bond_tags)) return MD_ERR_INVALID_ARG;
  if (n_bonds > 0 && s->p.max_bonds == 0) return MD_ERR_INVALID_ARG;
  if (!(K >= 0) || !(r0 >= 0)) return MD_ERR_INVALID_ARG;
  if (s->a.bond_style == MD_BOND_FENE && !(r0 > 0)) return MD_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const int64_t N = s->a.n;
  const int mb = s->p.max_bonds;
  if (mb > 0) {
    std::vector<int32_t> tab((size_t)N * mb, -1);
    std::vector<int32_t> cnt(N, 0);
    for (int64_t b = 0; b < n_bonds; b++) {
      const int32_t x = bond_tags[2 * b], y = bond_tags[2 * b + 1];
      if (x < 0 || y < 0 || x >= N || y >= N || x == y) return MD_ERR_INVALID_ARG;
      if (cnt[x] >= mb || cnt[y] >= mb) return MD_ERR_INVALID_ARG;
      tab[(size_t)x * mb + cnt[x]++] = y;
      tab[(size_t)y * mb + cnt[y]++] = x;
    }
    MD_CUDA(cudaMemcpyAsync(s->a.btab, tab.data(), sizeof(int32_t) * tab.size(),
                            cudaMemcpyHostToDevice, stream));
    MD_CUDA(cudaStreamSynchronize(stream));
  }
  s->n_bonds = n_bonds;
  s->a.bond_K = K;
  s->a.bond_r0 = r0;
  s->gvalid = false;
  s->built = false;  // forces must include the bonds before the next step
  return MD_OK;
}

md_status md_set_pair_table(md_system *s, const double *table, double r_min, md_stream stream_) {
  if (!s || !table || s->p.pair != MD_PAIR_TABLE) return MD_ERR_INVALID_ARG;
  const double rc = s->p.r_cut;
  if (!(r_min >= 0) || !(r_min < rc)) return MD_ERR_INVALID_ARG;
  const int nt = s->p.n_types, np = s->p.table_points;
  const size_t npairs = (size_t)nt * nt;
  for (size_t k = 0; k < npairs * np * 2; k++)
    if (!std::isfinite(table[k])) return MD_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const bool mixed = s->p.precision == MD_MIXED;
  const double inv_dr = (double)(np - 1) / (rc - r_min);
  // segments (V_j, F_j, V_j+1 - V_j, F_j+1 - F_j), j = 0 .. np - 2, per
  // ordered type pair at np * pair; the last slot of a pair is unused
  std::vector<double> seg(npairs * np * 4, 0.0);
  std::vector<unsigned char> coeff(64 * npairs, 0);
  for (size_t c = 0; c < npairs; c++) {
    const double *t = table + c * np * 2;
    for (int j = 0; j + 1 < np; j++) {
      double *g = seg.data() + (c * np + j) * 4;
      g[0] = t[2 * j], g[1] = t[2 * j + 1];
      g[2] = t[2 * j + 2] - t[2 * j], g[3] = t[2 * j + 3] - t[2 * j + 1];
    }
    const int first = (int)(c * np);
    if (mixed) {
      PotCoeffF f{(float)r_min, (float)inv_dr, (float)(np - 2), int_bits_as_float(first), 0, 0, 0, 0};
      std::memcpy(coeff.data() + sizeof(PotCoeffF) * c, &f, sizeof(f));
      if (c == 0) s->a.pot1f = f;
    } else {
      PotCoeffD d{r_min, inv_dr, (double)(np - 2), (double)first, 0, 0, 0, 0};
      std::memcpy(coeff.data() + sizeof(PotCoeffD) * c, &d, sizeof(d));
    }
  }
  if (mixed) {
    std::vector<float> f(seg.size());
    for (size_t k = 0; k < seg.size(); k++) f[k] = (float)seg[k];
    MD_CUDA(cudaMemcpyAsync(const_cast<void *>(s->a.table), f.data(), sizeof(float) * f.size(),
                            cudaMemcpyHostToDevice, stream));
    MD_CUDA(cudaMemcpyAsync(const_cast<void *>(s->a.coeff), coeff.data(), sizeof(PotCoeffF) * npairs,
                            cudaMemcpyHostToDevice, stream));
  } else {
    MD_CUDA(cudaMemcpyAsync(const_cast<void *>(s->a.table), seg.data(), sizeof(double) * seg.size(),
                            cudaMemcpyHostToDevice, stream));
    MD_CUDA(cudaMemcpyAsync(const_cast<void *>(s->a.coeff), coeff.data(), sizeof(PotCoeffD) * npairs,
                            cudaMemcpyHostToDevice, stream));
  }
  MD_CUDA(cudaStreamSynchronize(stream));
  s->gvalid = false;
  s->built = false;  // forces of the new table before the next step
  return MD_OK;
}

md_status md_set_angles(md_system *s, const int32_t *angle_tags, int64_t n_angles, double K,
                        double theta0, md_stream stream_) {
  if (!s || n_angles < 0 || (n_angles > 0 && !angle_tags)) return MD_ERR_INVALID_ARG;
  if (n_angles > 0 && s->p.max_angles == 0) return MD_ERR_INVALID_ARG;
  if (!(K >= 0) || !std::isfinite(K) || !(theta0 >= 0) || !(theta0 <= 3.14159265358979324))
    return MD_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const int64_t N = s->a.n;
  const int ma = s->p.max_angles;
  if (ma > 0) {
    std::vector<int32_t> tab((size_t)N * ma * 3, -1);
    std::vector<int32_t> cnt(N, 0);
    for (int64_t t = 0; t < n_angles; t++) {
      const int32_t *q = angle_tags + 3 * t;
      for (int k = 0; k < 3; k++)
        if (q[k] < 0 || q[k] >= N) return MD_ERR_INVALID_ARG;
      if (q[0] == q[1] || q[1] == q[2] || q[0] == q[2]) return MD_ERR_INVALID_ARG;
      for (int k = 0; k < 3; k++) {
        const int32_t x = q[k];
        if (cnt[x] >= ma) return MD_ERR_INVALID_ARG;
        int32_t *e = tab.data() + ((size_t)x * ma + cnt[x]++) * 3;
        e[0] = q[0], e[1] = q[1], e[2] = q[2];
      }
    }
    MD_CUDA(cudaMemcpyAsync(s->a.atab, tab.data(), sizeof(int32_t) * tab.size(),
                            cudaMemcpyHostToDevice, stream));
    MD_CUDA(cudaStreamSynchronize(stream));
  }
  s->n_angles = n_angles;
  s->a.angle_K = K;
  s->a.angle_th0 = theta0;
  s->gvalid = false;
  s->built = false;  // forces must include the angles before the next step
  return MD_OK;
}

md_status md_set_bond_style(md_system *s, int32_t style) {
  if (!s || (style != MD_BOND_HARMONIC && style != MD_BOND_FENE)) return MD_ERR_INVALID_ARG;
  if (style == MD_BOND_FENE && !(s->a.bond_r0 > 0)) return MD_ERR_INVALID_ARG;
  s->a.bond_style = style;
  s->gvalid = false;
  s->built = false;  // forces must include the bonds of the new style
  return MD_OK;
}

md_status md_sort_particles(md_system *s, int32_t force, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (!s->binned) return MD_ERR_STATE;
  MD_CUDA(launch_sort(s->a, force ? 1 : 0, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_build_cells(md_system *s, int32_t force, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_bin(s->a, force ? 1 : 0, reinterpret_cast<cudaStream_t>(stream)));
  s->bin_cond = true;
  if (force) {
    s->binned = s->bin_all = true;
    s->listed = false;  // rows refer to the cell stages of the previous binning
    s->built = false;
  }
  return MD_OK;
}

md_status md_build_nlist(md_system *s, int32_t force, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (!s->binned) return MD_ERR_STATE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (force ? !s->bin_all : !s->bin_cond) {
    // particles moved since the last binning: bin them again first
    MD_CUDA(launch_bin(s->a, force ? 1 : 0, st));
    s->bin_cond = true;
    if (force) s->bin_all = true;
  }
  MD_CUDA(launch_nlist(s->a, s->tune[MD_KERNEL_NLIST], force ? 1 : 0, st));
  if (force) s->listed = true;
  return MD_OK;
}

md_status md_compute_pair(md_system *s, int32_t want_virial, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (!s->listed) return MD_ERR_STATE;  // no list in the current layout yet
  MD_CUDA(launch_pair(s->a, s->tune[MD_KERNEL_PAIR], want_virial ? 1 : 0,
                      reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_compute_bonds(md_system *s, int32_t want_virial, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (s->n_bonds == 0 && s->n_angles == 0) return MD_OK;
  MD_CUDA(launch_bonds(s->a, want_virial ? 1 : 0, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_integrate(md_system *s, int32_t half, md_stream stream) {
  if (!s || (half != 1 && half != 2)) return MD_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (half == 1) {
    MD_CUDA(nh_prime(s, st));
    MD_CUDA(launch_integrate1(s->a, st));
    s->bin_all = s->bin_cond = false;
    s->step++;
  } else {
    MD_CUDA(launch_integrate2(s->a, st));
    if (s->a.integ == MD_NOSE_HOOVER) s->nh_primed = true;
  }
  return MD_OK;
}

md_status md_step(md_system *s, int32_t want_virial, md_stream stream) {
  if (!s) return MD_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  md_status e = prepare(s, st);
  if (e != MD_OK) return e;
  MD_CUDA(nh_prime(s, st));
  e = enqueue_step(s, want_virial ? 1 : 0, st);
  s->bin_all = s->bin_cond = false;
  if (e == MD_OK) s->step++;
  if (e == MD_OK && s->a.integ == MD_NOSE_HOOVER) MD_CUDA(launch_nh_flush(s->a, st));
  return e;
}

md_status md_reduce_thermo(md_system *s, double *dev_out, md_stream stream) {
  if (!s || !dev_out) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_thermo(s->a, dev_out, 0, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_run(md_system *s, int64_t n_steps, double *thermo_out, md_stream stream) {
  if (!s || n_steps < 0) return MD_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  md_status e = prepare(s, st);
  if (e != MD_OK) return e;
  const int64_t period = s->p.thermo_period;
  const int gsteps = s->p.graph_steps;
  const int64_t rows = period > 0 ? (s->step + n_steps) / period - s->step / period : 0;
  MD_CUDA(launch_run_begin(s->a, thermo_out, period, rows, st));
  if (n_steps > 0) s->bin_all = s->bin_cond = false;
  if (n_steps > 0) MD_CUDA(nh_prime(s, st));
  int64_t left = n_steps;
  while (left > 0) {
    if (gsteps > 0 && left >= gsteps && (period == 0 || s->step % period == 0)) {
      if (!s->gvalid) {
        if (s->gexec) { cudaGraphExecDestroy(s->gexec); s->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        MD_CUDA(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        md_status ce = MD_OK;
        // inside the graph a step's second half-kick is folded into the next
        // step's first half, except on thermo steps (they need full-step
        // velocities) and the last step (the graph ends in a full step)
        for (int l = 0; l < gsteps && ce == MD_OK; l++) {
          const int th = period > 0 && (l + 1) % period == 0;
          const bool prev_open = l > 0 && !(period > 0 && l % period == 0);
          const bool close = th || l == gsteps - 1;
          ce = enqueue_step(s, th, s->cap, prev_open, close);
          if (ce == MD_OK && th && launch_thermo(s->a, nullptr, 1, s->cap) != cudaSuccess) ce = MD_ERR_CUDA;
        }
        cudaError_t ee = cudaStreamEndCapture(s->cap, &g);
        if (ce != MD_OK) { if (g) cudaGraphDestroy(g); return ce; }
        if (ee != cudaSuccess) return MD_ERR_CUDA;
        cudaError_t ie = cudaGraphInstantiate(&s->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { s->gexec = nullptr; return MD_ERR_CUDA; }
        s->gvalid = true;
      }
      MD_CUDA(cudaGraphLaunch(s->gexec, st));
      s->step += gsteps;
      left -= gsteps;
    } else {
      const int th = period > 0 && (s->step + 1) % period == 0;
      e = enqueue_step(s, th, st);
      if (e != MD_OK) return e;
      if (th) MD_CUDA(launch_thermo(s->a, nullptr, 1, st));
      s->step++;
      left--;
    }
  }
  // Nose-Hoover: leave full-step velocities (the end-of-step scale applied)
  if (n_steps > 0 && s->a.integ == MD_NOSE_HOOVER) MD_CUDA(launch_nh_flush(s->a, st));
  return MD_OK;
}

md_status md_set_newton(md_system *s, int32_t enable) {
  if (!s || (enable != 0 && enable != 1)) return MD_ERR_INVALID_ARG;
  if (enable && s->p.precision != MD_FP64) return MD_ERR_INVALID_ARG;
  if (s->a.half != enable) {
    s->a.half = enable;
    s->built = s->listed = false;  // rows must be rebuilt in the new form
    s->gvalid = false;
  }
  return MD_OK;
}

md_status md_set_integrator(md_system *s, int32_t kind, double kT, double param, uint64_t seed) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (kind != MD_NVE && kind != MD_LANGEVIN && kind != MD_NOSE_HOOVER) return MD_ERR_INVALID_ARG;
  if (kind != MD_NVE) {
    if (s->p.pair == MD_PAIR_DPD) return MD_ERR_INVALID_ARG;
    if (!(kT > 0) || !std::isfinite(kT) || !std::isfinite(param)) return MD_ERR_INVALID_ARG;
    if (kind == MD_LANGEVIN && !(param >= 0)) return MD_ERR_INVALID_ARG;
    if (kind == MD_NOSE_HOOVER && !(param > 0)) return MD_ERR_INVALID_ARG;
  }
  KArgs &a = s->a;
  a.integ = kind;
  a.t_kT = kind == MD_NVE ? 1.0 : kT;
  a.t_seed = seed;
  a.t_tau = kind == MD_NOSE_HOOVER ? param : 1.0;
  a.t_c = kind == MD_LANGEVIN ? std::exp(-param * a.dt) : 1.0;
  a.t_sig = kind == MD_LANGEVIN ? std::sqrt((1.0 - a.t_c * a.t_c) * kT / a.mass) : 0.0;
  std::vector<double> nh(kNhFields * (size_t)a.R, 0.0);
  for (int r = 0; r < a.R; r++) nh[kNhFields * r + 2] = nh[kNhFields * r + 3] = 1.0;
  MD_CUDA(cudaDeviceSynchronize());
  MD_CUDA(cudaMemcpy(a.nh, nh.data(), sizeof(double) * nh.size(), cudaMemcpyHostToDevice));
  s->nh_primed = false;
  s->gvalid = false;
  return MD_OK;
}

md_status md_get_thermostat(md_system *s, double *host_out) {
  if (!s || !host_out) return MD_ERR_INVALID_ARG;
  std::vector<double> nh(kNhFields * (size_t)s->a.R);
  MD_CUDA(cudaDeviceSynchronize());
  MD_CUDA(cudaMemcpy(nh.data(), s->a.nh, sizeof(double) * nh.size(), cudaMemcpyDeviceToHost));
  for (int r = 0; r < s->a.R; r++) {  // the state between steps
    host_out[2 * r] = nh[kNhFields * r + 4];
    host_out[2 * r + 1] = nh[kNhFields * r + 5];
  }
  return MD_OK;
}

md_status md_set_tuning(md_system *s, int32_t kernel, int32_t block, int32_t w) {
  if (!s || (kernel != MD_KERNEL_NLIST && kernel != MD_KERNEL_PAIR) || !valid_launch(block, w))
    return MD_ERR_INVALID_ARG;
  const int mb = kernel == MD_KERNEL_NLIST
                     ? max_block_nlist(s->a, w)
                     : std::min(max_block_pair(s->a, w, 0), max_block_pair(s->a, w, 1));
  if (block > mb) return MD_ERR_INVALID_ARG;
  if (kernel == MD_KERNEL_NLIST) {
    s->tune[MD_KERNEL_NLIST] = Launch{block, w};
    s->gvalid = false;
  } else {
    const bool relayout = w != s->tune[MD_KERNEL_PAIR].w;
    set_pair_w(s, Launch{block, w});
    if (relayout) s->built = s->listed = false;  // rows must be rewritten in the new layout
  }
  return MD_OK;
}

md_status md_get_tuning(md_system *s, int32_t kernel, int32_t *block, int32_t *w) {
  if (!s || !block || !w || (kernel != MD_KERNEL_NLIST && kernel != MD_KERNEL_PAIR))
    return MD_ERR_INVALID_ARG;
  *block = s->tune[kernel].block;
  *w = s->tune[kernel].w;
  return MD_OK;
}

md_status md_autotune(md_system *s, int32_t n_samples, int32_t block_stride, md_stream stream) {
  if (!s || n_samples < 1 || block_stride < 1) return MD_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  md_status e = prepare(s, st);
  if (e != MD_OK) return e;
  if (!s->bin_all) {  // the timed builds need a current binning
    MD_CUDA(launch_bin(s->a, 1, st));
    s->bin_all = s->bin_cond = true;
  }
  cudaEvent_t e0, e1;
  MD_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MD_ERR_CUDA; }
  auto median_time = [&](auto &&launch) -> float {
    std::vector<float> t;
    for (int k = 0; k < n_samples; k++) {
      cudaEventRecord(e0, st);
      if (launch() != cudaSuccess) return -1.f;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
  };
  static const int ws[6] = {1, 2, 4, 8, 16, 32};
  md_status result = MD_OK;
  // pair kernel: (block, w); each w needs its own list layout
  Launch best_pair = s->tune[MD_KERNEL_PAIR];
  float best_t = 1e30f;
  for (int w : ws) {
    set_pair_w(s, Launch{std::max(32, w), w});
    if (launch_nlist(s->a, s->tune[MD_KERNEL_NLIST], 1, st) != cudaSuccess) { result = MD_ERR_CUDA; break; }
    const int mb = std::min(max_block_pair(s->a, w, 0), max_block_pair(s->a, w, 1));
    for (int b = 32 * block_stride; b <= std::min(kMaxTuneBlock, mb); b += 32 * block_stride) {
      set_pair_w(s, Launch{b, w});
      const float t = median_time([&] { return launch_pair(s->a, Launch{b, w}, 0, st); });
      if (t < 0) { cudaGetLastError(); continue; }
      if (t < best_t) { best_t = t; best_pair = Launch{b, w}; }
    }
  }
  set_pair_w(s, best_pair);
  // neighbour-list kernel: (block, w) over the chosen layout
  Launch best_nl = s->tune[MD_KERNEL_NLIST];
  best_t = 1e30f;
  for (int w : ws) {
    if (result != MD_OK) break;
    if (w > best_pair.w) break;  // the build's w is capped by the pair kernel's
    const int mb = max_block_nlist(s->a, w);
    for (int b = 32 * block_stride; b <= std::min(kMaxTuneBlock, mb); b += 32 * block_stride) {
      const float t = median_time([&] { return launch_nlist(s->a, Launch{b, w}, 1, st); });
      if (t < 0) { cudaGetLastError(); continue; }
      if (t < best_t) { best_t = t; best_nl = Launch{b, w}; }
    }
  }
  s->tune[MD_KERNEL_NLIST] = best_nl;
  if (result == MD_OK && launch_nlist(s->a, best_nl, 1, st) != cudaSuccess) result = MD_ERR_CUDA;
  if (result == MD_OK && launch_pair(s->a, best_pair, 0, st) != cudaSuccess) result = MD_ERR_CUDA;
  if (result == MD_OK && (s->n_bonds > 0 || s->n_angles > 0) && launch_bonds(s->a, 0, st) != cudaSuccess) result = MD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) result = MD_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->gvalid = false;
  return result;
}

md_status md_set_step(md_system *s, int64_t step, md_stream stream) {
  if (!s || step < 0) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_set_step(s->a, step, reinterpret_cast<cudaStream_t>(stream)));
  s->step = step;
  return MD_OK;
}

md_status md_get_step(md_system *s, int64_t *step) {
  if (!s || !step) return MD_ERR_INVALID_ARG;
  MD_CUDA(cudaDeviceSynchronize());
  MD_CUDA(cudaMemcpy(step, &s->a.ds->step, sizeof(int64_t), cudaMemcpyDeviceToHost));
  return MD_OK;
}

md_status md_poll_error(md_system *s, int64_t *detail) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (detail) *detail = 0;
  MD_CUDA(cudaDeviceSynchronize());
  DevState ds;
  MD_CUDA(cudaMemcpy(&ds, s->a.ds, sizeof(ds), cudaMemcpyDeviceToHost));
  if (ds.error & kErrNlistOverflow) {
    if (detail) *detail = ds.need_max_nb;
    return MD_ERR_NLIST_OVERFLOW;
  }
  if (ds.error & kErrNonfinite) {
    if (detail) *detail = ds.error_detail;
    return MD_ERR_NONFINITE;
  }
  if (ds.error & kErrBond) {
    if (detail) *detail = ds.error_detail;
    return MD_ERR_BOND;
  }
  if (ds.error & kErrCellOverflow) return MD_ERR_CELL_OVERFLOW;
  if (ds.error & kErrStaleList) return MD_ERR_STATE;
  if (ds.error & kErrTimeout) {
    if (detail) *detail = ds.error_detail;
    return MD_ERR_TIMEOUT;
  }
  return MD_OK;
}

md_status md_get_forces(md_system *s, double *dev_force, double *dev_virial, md_stream stream) {
  if (!s || !dev_force) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_export_forces(s->a, dev_force, dev_virial, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_get_nlist(md_system *s, int32_t *dev_counts, int32_t *dev_rows, md_stream stream) {
  if (!s || !dev_counts || !dev_rows) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_export_nlist(s->a, dev_counts, dev_rows, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_get_cells(md_system *s, int32_t *dev_start, int32_t *dev_count, int32_t *dev_idx,
                       md_stream stream) {
  if (!s || !dev_start || !dev_count || !dev_idx) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_export_cells(s->a, dev_start, dev_count, dev_idx, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_get_info(md_system *s, int64_t *n_cells, int32_t *max_nb, int64_t *n_builds) {
  if (!s) return MD_ERR_INVALID_ARG;
  if (n_cells) *n_cells = s->a.n_cells;
  if (max_nb) *max_nb = s->a.max_nb;
  if (n_builds) {
    MD_CUDA(cudaDeviceSynchronize());
    MD_CUDA(cudaMemcpy(n_builds, &s->a.ds->n_builds, sizeof(int64_t), cudaMemcpyDeviceToHost));
  }
  return MD_OK;
}

md_status md_philox4x32_10(const uint32_t *dev_in, uint32_t *dev_out, int64_t n, md_stream stream) {
  if (n < 0 || (n > 0 && (!dev_in || !dev_out))) return MD_ERR_INVALID_ARG;
  MD_CUDA(launch_philox(dev_in, dev_out, n, reinterpret_cast<cudaStream_t>(stream)));
  return MD_OK;
}

}  // extern "C"
