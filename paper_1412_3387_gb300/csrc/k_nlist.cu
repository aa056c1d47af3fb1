// Neighbour-list build (Sec. 5.1, Fig. "nlist").
//
// Each particle i is served by a segment of W lanes of one warp (W = 2^m <= 32;
// a warp holds 32/W segments).  The segment walks the 27 cells around i's
// cell; inside each cell the W lanes take candidates with a stride of W, test
// r^2 < r_list^2, and the hits are compacted into row i with a warp ballot and
// a population count over the segment's bits (the intra-warp prefix sum of the
// paper's algorithm).  The running row length n_tot advances by the
// segment's hit count after every stride.
//
// Distance test.  Candidates are first screened in FP32 from frame-relative
// offsets (see md_internal.cuh: frame_offset); only candidates whose FP32 r^2
// lies within a proven error band of r_list^2 are re-tested with the FP64
// minimum-image distance in the fixed operation order.  The set of neighbours
// is therefore exactly the FP64 set, at FP32 cost.
//
// Storage: entry = j | (stencil code << 27); the code (0..26) names the
// neighbouring cell, i.e. the periodic image shift the pair kernel applies.
// Entry k of row i sits at ((k / ws) * n_pad + i) * ws + k % ws, ws = the
// pair kernel's W, so the pair kernel's W lanes read consecutive words.
#include "md_internal.cuh"

namespace mdgb {

namespace {

__device__ __forceinline__ bool rebuilding(const KArgs &a, int r, int force) {
  return force || a.rebuild[2 * r + (int)(a.ds->step & 1)] != 0;
}

template <int W>
__global__ void k_nlist(KArgs a, int force) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int sl = lane & (W - 1);
  const unsigned segmask = (W == 32) ? FULL : (((1u << W) - 1u) << (lane & ~(W - 1)));
  const unsigned lt_mask = (1u << lane) - 1u;
  const int per_block = blockDim.x / W;
  const int64_t i = (int64_t)blockIdx.x * per_block + threadIdx.x / W;
  const bool valid = i < a.n;
  const int r = valid ? replica_of(a, i) : 0;
  const bool active = valid && rebuilding(a, r, force);
  if (!__any_sync(FULL, active)) return;

  const Rep &rp = a.rep[r];
  float4 oi = active ? a.pos4f[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const uint32_t wi = __float_as_uint(oi.w);
  const int cx = cell_x(wi), cy = cell_y(wi), cz = cell_z(wi);
  const float lo = a.rl2f - rp.band, hi = a.rl2f + rp.band;
  const int lw = a.w_store_log2;
  int n = 0;

  for (int s = 0; s < 27; s++) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    int start = 0, cnt = 0;
    float shx = 0.f, shy = 0.f, shz = 0.f;
    if (active) {
      int nx = cx + dx, ny = cy + dy, nz = cz + dz;
      nx += nx < 0 ? rp.nc[0] : 0;  nx -= nx >= rp.nc[0] ? rp.nc[0] : 0;
      ny += ny < 0 ? rp.nc[1] : 0;  ny -= ny >= rp.nc[1] ? rp.nc[1] : 0;
      nz += nz < 0 ? rp.nc[2] : 0;  nz -= nz >= rp.nc[2] ? rp.nc[2] : 0;
      int64_t lin = nx + (int64_t)rp.nc[0] * (ny + (int64_t)rp.nc[1] * nz);
      int64_t g = rp.cell0 + __ldg(a.cell_rank + rp.cell0 + lin);
      start = __ldg(a.cell_start + g);
      cnt = __ldg(a.cell_count + g);
      shx = (float)dx * rp.hf[0];
      shy = (float)dy * rp.hf[1];
      shz = (float)dz * rp.hf[2];
    }
    const int iters = __reduce_max_sync(FULL, (unsigned)((cnt + W - 1) / W));
    for (int t = 0; t < iters; t++) {
      const int k = t * W + sl;
      bool in = false;
      int32_t j = 0;
      if (k < cnt) {
        j = __ldg(a.cell_idx + start + k);
        if ((int64_t)j != i) {
          float4 oj = __ldg(a.pos4f + j);
          float ddx = (oi.x - oj.x) - shx;
          float ddy = (oi.y - oj.y) - shy;
          float ddz = (oi.z - oj.z) - shz;
          float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, ddx * ddx));
          if (r2 < lo) {
            in = true;
          } else if (r2 < hi) {
            double d[3];
            in = exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + j), rp, d) < a.rl2;
          }
        }
      }
      const unsigned b = __ballot_sync(FULL, in) & segmask;
      if (in) {
        const int p = n + __popc(b & lt_mask);
        if (p < a.max_nb) a.nl[nl_addr(i, p, lw, a.n_pad)] = (uint32_t)j | ((uint32_t)s << kIdxBits);
      }
      n += __popc(b);
    }
  }
  if (active && sl == 0) {
    a.n_nb[i] = n;
    if (n > a.max_nb) {
      atomicMax(&a.ds->need_max_nb, n);
      set_error(a.ds, kErrNlistOverflow);
    }
  }
}

template <int W>
cudaError_t launch_w(const KArgs &a, int block, int force, cudaStream_t st) {
  int per_block = block / W;
  unsigned grid = (unsigned)((a.n + per_block - 1) / per_block);
  k_nlist<W><<<grid, block, 0, st>>>(a, force);
  return cudaGetLastError();
}

template <int W>
int max_block_w() {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_nlist<W>) != cudaSuccess) return 0;
  return at.maxThreadsPerBlock;
}

}  // namespace

cudaError_t launch_nlist(const KArgs &a, Launch l, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  switch (l.w) {
    case 1: return launch_w<1>(a, l.block, force, st);
    case 2: return launch_w<2>(a, l.block, force, st);
    case 4: return launch_w<4>(a, l.block, force, st);
    case 8: return launch_w<8>(a, l.block, force, st);
    case 16: return launch_w<16>(a, l.block, force, st);
    case 32: return launch_w<32>(a, l.block, force, st);
    default: return cudaErrorInvalidValue;
  }
}

int max_block_nlist(int w) {
  switch (w) {
    case 1: return max_block_w<1>();
    case 2: return max_block_w<2>();
    case 4: return max_block_w<4>();
    case 8: return max_block_w<8>();
    case 16: return max_block_w<16>();
    case 32: return max_block_w<32>();
    default: return 0;
  }
}

}  // namespace mdgb
