// Neighbour-list build (Sec. 5.1, Fig. "nlist").
//
// One warp serves one home cell.  Its lanes form 32/W segments of W lanes
// (W = 2^m <= 32, the paper's threads per particle); each segment owns one
// home particle i of the cell at a time.  The warp walks the 27 cells around
// the home cell, stages each cell's members (index + FP32 position) in shared
// memory 32 at a time, and each segment's W lanes test the staged candidates
// with a stride of W; hits are compacted into row i with a warp ballot and a
// population count over the segment's bits (the intra-warp prefix sum of the
// paper's algorithm), and the row length advances by the segment's hit count.
// Because every lane of the warp shares the home cell, all loops are uniform
// across the warp.
//
// The 27 surrounding cells are visited in ascending Hilbert rank (a per-cell
// table built at creation) and members inside a cell are in ascending index
// order, so every row lists its neighbours in ascending particle index.
//
// Distance test.  Candidates are screened in FP32 from frame-relative offsets;
// only those whose FP32 r^2 lies within a proven error band of r_list^2 are
// re-tested with the FP64 minimum-image distance in the oracle's operation
// order.  The neighbour sets are therefore exactly the FP64 sets.
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
  constexpr int SEGS = 32 / W;
  __shared__ int32_t s_idx[32][32];
  __shared__ float4 s_pos[32][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int sl = lane & (W - 1), seg = lane / W;
  const unsigned segmask = (W == 32) ? FULL : (((1u << W) - 1u) << (seg * W));
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;  // home cell
  if (g >= a.n_cells) return;
  const int r = a.chunk_rep[g / kChunkCells];
  if (!rebuilding(a, r, force)) return;
  const int cnt = a.cell_count[g];
  if (cnt == 0) return;
  const Rep &rp = a.rep[r];
  const int start = a.cell_start[g];
  const float lo = a.rl2f - rp.band, hi = a.rl2f + rp.band;
  const int lw = a.w_store_log2;
  const uint32_t *stencil = a.stencil + g * 27;
  int32_t *cidx = s_idx[wid];
  float4 *cpos = s_pos[wid];

  for (int q0 = 0; q0 < cnt; q0 += SEGS) {
    const int q = q0 + seg;
    const bool active = q < cnt;
    const int32_t i = active ? a.cell_idx[start + q] : -1;
    const float4 oi = active ? a.pos4f[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int n = 0;
    // W == 1 write pointer into row i: entries advance by one word inside a
    // tile of ws words and jump to the next tile row after ws entries
    const int ws = 1 << lw;
    const size_t tile_jump = ((size_t)a.n_pad << lw) - (size_t)(ws - 1);
    uint32_t *wp = a.nl + nl_addr(active ? i : 0, 0, lw, a.n_pad);
    for (int s = 0; s < 27; s++) {
      const uint32_t e = __ldg(stencil + s);
      const int64_t g2 = rp.cell0 + (int64_t)(e & kIdxMask);
      const int code = (int)(e >> kIdxBits);
      // x_i - x_j = (o_i - shift) - o_j with shift = d * h, d in {-1,0,1}^3
      const float px = oi.x - (float)(code % 3 - 1) * rp.hf[0];
      const float py = oi.y - (float)((code / 3) % 3 - 1) * rp.hf[1];
      const float pz = oi.z - (float)(code / 9 - 1) * rp.hf[2];
      const int st2 = __ldg(a.cell_start + g2), cnt2 = __ldg(a.cell_count + g2);
      for (int c0 = 0; c0 < cnt2; c0 += 32) {
        const int m = min(32, cnt2 - c0);
        __syncwarp();
        if (lane < m) {
          const int32_t j = __ldg(a.cell_idx + st2 + c0 + lane);
          cidx[lane] = j;
          cpos[lane] = __ldg(a.pos4f + j);
        }
        __syncwarp();
        if constexpr (W == 1) {
          // one lane per home particle: each lane appends to its own row
          for (int c = 0; c < m; c++) {
            const int32_t j = cidx[c];
            const float4 oj = cpos[c];
            const float dx = px - oj.x, dy = py - oj.y, dz = pz - oj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool in = active && j != i && r2 < lo;
            const bool band = active && j != i && r2 >= lo && r2 < hi;
            if (__any_sync(FULL, band) && band) {
              double d[3];
              in = exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + j), rp, d) < a.rl2;
            }
            if (in) {
              if (n < a.max_nb) *wp = (uint32_t)j | ((uint32_t)code << kIdxBits);
              n++;
              wp += ((n & (ws - 1)) == 0) ? tile_jump : 1;
            }
          }
        } else {
          for (int t = 0; t < m; t += W) {
            const int c = t + sl;
            bool in = false;
            int32_t j = 0;
            if (active && c < m) {
              j = cidx[c];
              const float4 oj = cpos[c];
              const float dx = px - oj.x, dy = py - oj.y, dz = pz - oj.z;
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              if (j != i) {
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
              if (p < a.max_nb)
                a.nl[nl_addr(i, p, lw, a.n_pad)] = (uint32_t)j | ((uint32_t)code << kIdxBits);
            }
            n += __popc(b);
          }
        }
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
}

template <int W>
cudaError_t launch_w(const KArgs &a, int block, int force, cudaStream_t st) {
  const int cells_per_block = block / 32;
  unsigned grid = (unsigned)((a.n_cells + cells_per_block - 1) / cells_per_block);
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
