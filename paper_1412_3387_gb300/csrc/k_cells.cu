// Cell-list binning and the space-filling-curve particle sort.
//
// Binning (Sec. 4.3.3 uses a cell list built with atomics; Sec. 5.1 looks up
// the cell neighbours of each particle): count per cell with atomics ->
// exclusive scan -> scatter -> order each cell's members by their FP32 x
// offset from the cell centre, ties by particle index, which makes the result
// independent of the atomics' order (Sec. 4.3.3 notes the atomics make plain
// cell lists non-deterministic).  Cells are numbered brick by brick along a
// 3-D Hilbert curve over bricks of 2 x 2 x 2 cells per replica, so the cell
// list's particle order IS the space-filling-curve order used by the sort.
#include "brick.cuh"

namespace mdgb {

namespace {

__device__ __forceinline__ bool rebuilding(const KArgs &a, int r, int force) {
  return force || a.rebuild[2 * r + (int)(a.ds->step & 1)] != 0;
}

// Quiet step (no replica rebuilds): every thread leaves at once.
__device__ __forceinline__ bool quiet(const KArgs &a, int force) {
  return !force && !a.ds->rebuild_any;
}

__global__ void k_bin_zero(KArgs a, int force) {
  if (quiet(a, force)) return;
  int64_t ch = blockIdx.x;
  int r = a.chunk_rep[ch];
  if (!rebuilding(a, r, force)) return;
  int32_t *cnt = a.cell_count + ch * kChunkCells;
  for (int k = threadIdx.x; k < kChunkCells; k += blockDim.x) cnt[k] = 0;
}

__device__ __forceinline__ void k_bin_count_one(const KArgs &a, int64_t i, int force) {
  int r = replica_of(a, i);
  if (!rebuilding(a, r, force)) return;
  const Rep &rp = a.rep[r];
  double4 x = ld_d4(a.pos + i);
  int cx = cell_coord(x.x, rp.inv_h[0], rp.nc[0]);
  int cy = cell_coord(x.y, rp.inv_h[1], rp.nc[1]);
  int cz = cell_coord(x.z, rp.inv_h[2], rp.nc[2]);
  int64_t lin = cx + (int64_t)rp.nc[0] * (cy + (int64_t)rp.nc[1] * cz);
  int64_t g = rp.cell0 + a.cell_rank[rp.cell0 + lin];
  a.pcell[i] = (int32_t)g;
  a.pslot[i] = atomicAdd(a.cell_count + g, 1);
}

__global__ void k_bin_count(KArgs a, int force) {
  if (quiet(a, force)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x)
    k_bin_count_one(a, i, force);
}

// Block-wide exclusive scan of 8 values per thread (256 threads).
__device__ __forceinline__ int block_excl_scan8(int v[8], int *total) {
  __shared__ int warp_tot[32];
  int s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) { int t = v[k]; v[k] = s; s += t; }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int t = lane < nw ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == nw - 1) warp_tot[31] = ti;   // block total (nw <= 31 here)
  }
  __syncthreads();
  int base = warp_tot[wid] + (incl - s);
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] += base;
  int tot = warp_tot[31];
  __syncthreads();
  *total = tot;
  return base;
}

__global__ void __launch_bounds__(256) k_scan_chunk_sum(KArgs a, int force) {
  if (quiet(a, force)) return;
  int64_t ch = blockIdx.x;
  int r = a.chunk_rep[ch];
  if (!rebuilding(a, r, force)) return;
  const int32_t *cnt = a.cell_count + ch * kChunkCells + threadIdx.x * 8;
  int v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = cnt[k];
  int tot;
  block_excl_scan8(v, &tot);
  if (threadIdx.x == 0) a.chunk_sum[ch] = tot;
}

// One warp per replica: exclusive scan of its chunk sums, in place.
__global__ void k_scan_chunks(KArgs a, int force) {
  if (quiet(a, force)) return;
  int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (r >= a.R) return;
  if (!rebuilding(a, r, force)) return;
  const Rep &rp = a.rep[r];
  int carry = 0;
  for (int base = 0; base < rp.nchunk; base += 32) {
    int k = base + lane;
    int v = k < rp.nchunk ? a.chunk_sum[rp.chunk0 + k] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (k < rp.nchunk) a.chunk_sum[rp.chunk0 + k] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) atomicAdd((unsigned long long *)&a.ds->n_builds, 1ull);
}

__global__ void __launch_bounds__(256) k_scan_cells(KArgs a, int force) {
  if (quiet(a, force)) return;
  int64_t ch = blockIdx.x;
  int r = a.chunk_rep[ch];
  if (!rebuilding(a, r, force)) return;
  const Rep &rp = a.rep[r];
  int64_t c0 = ch * kChunkCells + threadIdx.x * 8;
  int v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = a.cell_count[c0 + k];
  int tot;
  block_excl_scan8(v, &tot);
  int off = (int)rp.p0 + a.chunk_sum[ch];
#pragma unroll
  for (int k = 0; k < 8; k++) a.cell_start[c0 + k] = off + v[k];
}

__device__ __forceinline__ void k_bin_scatter_one(const KArgs &a, int64_t i, int force) {
  int r = replica_of(a, i);
  if (!rebuilding(a, r, force)) return;
  const Rep &rp = a.rep[r];
  a.cell_idx[a.cell_start[a.pcell[i]] + a.pslot[i]] = (int32_t)i;
  if (i == rp.p0) {
    a.ident[r] = 0;    // the new binning is not in particle order
    a.list_ok[r] = 0;  // and the rows refer to the old one
  }
  double4 x = ld_d4(a.pos + i);
  int cx = cell_coord(x.x, rp.inv_h[0], rp.nc[0]);
  int cy = cell_coord(x.y, rp.inv_h[1], rp.nc[1]);
  int cz = cell_coord(x.z, rp.inv_h[2], rp.nc[2]);
  float4 o;
  o.x = frame_offset(x.x, cell_centre(a, rp, 0, cx), rp.cq[0], rp.Lf[0], rp.L[0]);
  o.y = frame_offset(x.y, cell_centre(a, rp, 1, cy), rp.cq[1], rp.Lf[1], rp.L[1]);
  o.z = frame_offset(x.z, cell_centre(a, rp, 2, cz), rp.cq[2], rp.Lf[2], rp.L[2]);
  o.w = __uint_as_float(pack_cell(cx, cy, cz, a.type[i]));
  a.oref[i] = o;
}

__global__ void k_bin_scatter(KArgs a, int force) {
  if (quiet(a, force)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x)
    k_bin_scatter_one(a, i, force);
}

// Particle v goes to cell-list position p: the index maps both ways, and the
// FP32 copies the staged kernels read (kept in cell-list order) are set.
__device__ __forceinline__ void place(const KArgs &a, int p, int32_t v) {
  a.cell_idx[p] = v;
  a.cellpos[v] = p;
  a.pos4f[p] = a.oref[v];
  if (a.vel4f) {
    const double4 u = ld_d4(a.vel + v);
    a.vel4f[p] = make_float4((float)u.x, (float)u.y, (float)u.z, __int_as_float(a.tag[v]));
  }
}

// One warp per cell: order the cell's members by their FP32 x offset from the
// cell centre, ties by particle index.  At a build every member lies inside
// its cell, so each run of x-adjacent cells is then sorted by x (the list
// build searches windows in such runs).
__device__ __forceinline__ void cell_sort_one(const KArgs &a, int64_t cell, int force,
                                              int32_t *buf, float *bx) {
  const int lane = threadIdx.x & 31;
  const int r = a.chunk_rep[cell / kChunkCells];
  if (!rebuilding(a, r, force)) return;
  const int cnt = a.cell_count[cell];
  if (cnt == 0) return;
  const int start = a.cell_start[cell];
  const int32_t *idx = a.cell_idx + start;
  if (cnt > kMaxCellSort) {
    // flagged; the members keep their binning order
    if (lane == 0) set_error(a.ds, kErrCellOverflow);
    for (int k = lane; k < cnt; k += 32) place(a, start + k, idx[k]);
    return;
  }
  for (int k = lane; k < cnt; k += 32) {
    const int32_t v = idx[k];
    buf[k] = v;
    // a non-finite offset (flagged elsewhere) ranks as +inf: the order stays
    // strict, so every member gets its own place
    const float x = a.oref[v].x;
    bx[k] = x == x ? x : INFINITY;
  }
  __syncwarp();
  for (int k = lane; k < cnt; k += 32) {
    const int32_t v = buf[k];
    const float x = bx[k];
    int rank = 0;
    for (int m = 0; m < cnt; m++) {
      const float xm = bx[m];
      rank += (xm < x || (xm == x && buf[m] < v)) ? 1 : 0;
    }
    place(a, start + rank, v);
  }
  __syncwarp();
}

__global__ void k_cell_sort(KArgs a, int force) {
  if (quiet(a, force)) return;
  __shared__ int32_t buf[8][kMaxCellSort];
  __shared__ float bx[8][kMaxCellSort];
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; cell < a.n_cells;
       cell += warps)
    cell_sort_one(a, cell, force, buf[threadIdx.x >> 5], bx[threadIdx.x >> 5]);
}

// One warp per brick: the stage layout of its 64 stage cells (first slot and
// cell-list start of each) and the cell-list range of its own cells.
__global__ void k_brick_desc(KArgs a, int force) {
  if (quiet(a, force)) return;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= a.n_bricks) return;
  const int4 info = a.brick_info[b];
  if (!rebuilding(a, info.z, force)) return;
  BrickDesc &d = a.brick_desc[b];
  const int32_t c0 = a.brick_stage[b * kStageCells + lane];
  const int32_t c1 = a.brick_stage[b * kStageCells + 32 + lane];
  const int n0 = a.cell_count[c0], n1 = a.cell_count[c1];
  const int st0 = a.cell_start[c0], st1 = a.cell_start[c1];
  d.start[lane] = st0;
  d.start[32 + lane] = st1;
  int i0 = n0, i1 = n1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y0 = __shfl_up_sync(0xffffffffu, i0, o), y1 = __shfl_up_sync(0xffffffffu, i1, o);
    if (lane >= o) {
      i0 += y0;
      i1 += y1;
    }
  }
  const int t0 = __shfl_sync(0xffffffffu, i0, 31);
  d.off[lane] = i0 - n0;
  d.off[32 + lane] = t0 + i1 - n1;
  if (lane == 31) d.off[64] = t0 + i1;
  // the brick's own cells are the consecutive cell slots info.x, info.x + 1, ...
  const int nh = __popc(info.y);
  const int hc = lane < nh ? a.cell_count[info.x + lane] : 0;
  int hi = hc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, hi, o);
    if (lane >= o) hi += y;
  }
  if (lane < 9) d.hoff[lane] = hi - hc;
  if (lane == 31) d.nhome = hi;
  // per own cell: its stage cell and the slot offset of its members
  const int hs = home_stage_cell(info.y, lane < 8 ? lane : 0);
  const int src = hs & 31;
  const int off_lo = __shfl_sync(0xffffffffu, i0 - n0, src);
  const int off_hi = __shfl_sync(0xffffffffu, t0 + i1 - n1, src);
  const int st_lo = __shfl_sync(0xffffffffu, st0, src), st_hi = __shfl_sync(0xffffffffu, st1, src);
  if (lane < 8) {
    d.hcell[lane] = hs;
    d.hbase[lane] = hs < 32 ? off_lo - st_lo : off_hi - st_hi;
  }
  if (lane == 0) {
    d.r = info.z;
    d.hstart = a.cell_start[info.x];
    d.hmask = info.y;
    d.bc = info.w;
  }
}

// ---- space-filling-curve sort --------------------------------------------

__global__ void k_sort_flags(KArgs a, int value) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  a.sort_now[r] = value;
  if (value) a.last_sort[r] = a.ds->step;
}

__device__ __forceinline__ void k_sort_gather_one(const KArgs &a, int64_t k) {
  int r = replica_of(a, k);
  if (!a.sort_now[r]) return;
  int32_t old = a.cell_idx[k];
  a.s_pos[k] = a.pos[old];
  a.s_vel[k] = a.vel[old];
  a.s_img[k] = a.image[old];
  a.s_tag[k] = a.tag[old];
  a.s_type[k] = a.type[old];
  a.s_oref[k] = a.oref[old];
}

__global__ void k_sort_gather(KArgs a, int force) {
  if (quiet(a, force)) return;  // sorts happen only at rebuilds
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x)
    k_sort_gather_one(a, k);
}

__device__ __forceinline__ void k_sort_scatter_one(const KArgs &a, int64_t k) {
  int r = replica_of(a, k);
  if (!a.sort_now[r]) return;
  a.pos[k] = a.s_pos[k];
  a.vel[k] = a.s_vel[k];
  a.image[k] = a.s_img[k];
  int32_t t = a.s_tag[k];
  a.tag[k] = t;
  a.type[k] = a.s_type[k];
  a.oref[k] = a.s_oref[k];
  a.rtag[t] = (int32_t)k;
  // the particle order is now the cell-list order; the FP32 copies, kept in
  // cell-list order, stay where they are
  a.cell_idx[k] = (int32_t)k;
  a.cellpos[k] = (int32_t)k;
  if (k == a.rep[r].p0) a.ident[r] = 1;
}

__global__ void k_sort_scatter(KArgs a, int force) {
  if (quiet(a, force)) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x)
    k_sort_scatter_one(a, k);
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Grid of the grid-stride kernels: enough blocks to fill the GPU, never more
// than the work needs.
inline unsigned stride_blocks(int64_t n, int b) {
  const unsigned need = blocks_for(n, b);
  return need < 152u * 8u ? need : 152u * 8u;
}

}  // namespace

cudaError_t launch_bin(const KArgs &a, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_bin_zero<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_bin_count<<<stride_blocks(a.n, 256), 256, 0, st>>>(a, force);
  k_scan_chunk_sum<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_scan_chunks<<<blocks_for((int64_t)a.R * 32, 256), 256, 0, st>>>(a, force);
  k_scan_cells<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_bin_scatter<<<stride_blocks(a.n, 256), 256, 0, st>>>(a, force);
  k_cell_sort<<<stride_blocks(a.n_cells * 32, 256), 256, 0, st>>>(a, force);
  if (a.n_bricks > 0) k_brick_desc<<<blocks_for(a.n_bricks * 32, 256), 256, 0, st>>>(a, force);
  return cudaGetLastError();
}

cudaError_t launch_sort(const KArgs &a, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (force) k_sort_flags<<<blocks_for(a.R, 128), 128, 0, st>>>(a, 1);
  k_sort_gather<<<stride_blocks(a.n, 256), 256, 0, st>>>(a, force);
  k_sort_scatter<<<stride_blocks(a.n, 256), 256, 0, st>>>(a, force);
  if (force) k_sort_flags<<<blocks_for(a.R, 128), 128, 0, st>>>(a, 0);
  return cudaGetLastError();
}

}  // namespace mdgb
