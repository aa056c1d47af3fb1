// Cell-list binning and the space-filling-curve particle sort.
//
// Binning (Sec. 4.3.3 uses a cell list built with atomics; Sec. 5.1 looks up
// the cell neighbours of each particle): count per cell with atomics ->
// exclusive scan -> scatter -> order each cell's members by index, which makes
// the result independent of the atomics' order (Sec. 4.3.3 notes the atomics
// make plain cell lists non-deterministic).  Cells are numbered along a 3-D
// Hilbert curve per replica, so the cell list's particle order IS the
// space-filling-curve order used by the sort.
#include "md_internal.cuh"

namespace mdgb {

namespace {

__device__ __forceinline__ bool rebuilding(const KArgs &a, int r, int force) {
  return force || a.rebuild[2 * r + (int)(a.ds->step & 1)] != 0;
}

__global__ void k_bin_zero(KArgs a, int force) {
  int64_t ch = blockIdx.x;
  int r = a.chunk_rep[ch];
  if (!rebuilding(a, r, force)) return;
  int32_t *cnt = a.cell_count + ch * kChunkCells;
  for (int k = threadIdx.x; k < kChunkCells; k += blockDim.x) cnt[k] = 0;
}

__global__ void k_bin_count(KArgs a, int force) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
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

__global__ void k_bin_scatter(KArgs a, int force) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int r = replica_of(a, i);
  if (!rebuilding(a, r, force)) return;
  const Rep &rp = a.rep[r];
  a.cell_idx[a.cell_start[a.pcell[i]] + a.pslot[i]] = (int32_t)i;
  if (i == rp.p0) a.ident[r] = 0;  // the new binning is not in particle order
  double4 x = ld_d4(a.pos + i);
  int cx = cell_coord(x.x, rp.inv_h[0], rp.nc[0]);
  int cy = cell_coord(x.y, rp.inv_h[1], rp.nc[1]);
  int cz = cell_coord(x.z, rp.inv_h[2], rp.nc[2]);
  float4 o;
  o.x = frame_offset_fast(x.x, cx, rp.h[0], rp.half_h[0], rp.L[0]);
  o.y = frame_offset_fast(x.y, cy, rp.h[1], rp.half_h[1], rp.L[1]);
  o.z = frame_offset_fast(x.z, cz, rp.h[2], rp.half_h[2], rp.L[2]);
  o.w = __uint_as_float(pack_cell(cx, cy, cz, a.type[i]));
  a.pos4f[i] = o;
  a.oref[i] = o;
}

// One warp per cell: order the cell's members by particle index.
__global__ void k_cell_sort(KArgs a, int force) {
  __shared__ int32_t buf[8][kMaxCellSort];
  int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (cell >= a.n_cells) return;
  int r = a.chunk_rep[cell / kChunkCells];
  if (!rebuilding(a, r, force)) return;
  int cnt = a.cell_count[cell];
  if (cnt <= 1) return;
  if (cnt > kMaxCellSort) {
    if (lane == 0) set_error(a.ds, kErrCellOverflow);
    return;
  }
  int32_t *idx = a.cell_idx + a.cell_start[cell];
  for (int k = lane; k < cnt; k += 32) buf[wid][k] = idx[k];
  __syncwarp();
  for (int k = lane; k < cnt; k += 32) {
    int32_t v = buf[wid][k];
    int rank = 0;
    for (int m = 0; m < cnt; m++) rank += buf[wid][m] < v;
    idx[rank] = v;
  }
}

// ---- space-filling-curve sort --------------------------------------------

__global__ void k_sort_flags(KArgs a, int value) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  a.sort_now[r] = value;
  if (value) a.last_sort[r] = a.ds->step;
}

__global__ void k_sort_gather(KArgs a) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  int r = replica_of(a, k);
  if (!a.sort_now[r]) return;
  int32_t old = a.cell_idx[k];
  a.s_pos[k] = a.pos[old];
  a.s_vel[k] = a.vel[old];
  a.s_img[k] = a.image[old];
  a.s_tag[k] = a.tag[old];
  a.s_type[k] = a.type[old];
  a.s_pos4f[k] = a.pos4f[old];
  a.s_oref[k] = a.oref[old];
  if (a.vel4f) a.s_vel4f[k] = a.vel4f[old];
}

__global__ void k_sort_scatter(KArgs a) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  int r = replica_of(a, k);
  if (!a.sort_now[r]) return;
  a.pos[k] = a.s_pos[k];
  a.vel[k] = a.s_vel[k];
  a.image[k] = a.s_img[k];
  int32_t t = a.s_tag[k];
  a.tag[k] = t;
  a.type[k] = a.s_type[k];
  a.pos4f[k] = a.s_pos4f[k];
  a.oref[k] = a.s_oref[k];
  if (a.vel4f) a.vel4f[k] = a.s_vel4f[k];
  a.rtag[t] = (int32_t)k;
  a.cell_idx[k] = (int32_t)k;  // the cell list order is now the particle order
  if (k == a.rep[r].p0) a.ident[r] = 1;
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_bin(const KArgs &a, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_bin_zero<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_bin_count<<<blocks_for(a.n, 256), 256, 0, st>>>(a, force);
  k_scan_chunk_sum<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_scan_chunks<<<blocks_for((int64_t)a.R * 32, 256), 256, 0, st>>>(a, force);
  k_scan_cells<<<(unsigned)a.n_chunks, 256, 0, st>>>(a, force);
  k_bin_scatter<<<blocks_for(a.n, 256), 256, 0, st>>>(a, force);
  k_cell_sort<<<blocks_for(a.n_cells * 32, 256), 256, 0, st>>>(a, force);
  return cudaGetLastError();
}

cudaError_t launch_sort(const KArgs &a, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (force) k_sort_flags<<<blocks_for(a.R, 128), 128, 0, st>>>(a, 1);
  k_sort_gather<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  k_sort_scatter<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  if (force) k_sort_flags<<<blocks_for(a.R, 128), 128, 0, st>>>(a, 0);
  return cudaGetLastError();
}

}  // namespace mdgb
