// Neighbour-list build (Sec. 5.1, Fig. "nlist").
//
// One thread block serves one home cell.  Its threads form segments of W
// lanes (W = 2^m <= 32, the paper's threads per particle; the block size is
// the paper's other tuning parameter); each segment owns one home particle at
// a time.  The block stages the members of the 27 cells around the home cell
// (see md_internal.cuh, "cell stage") in shared memory, and each segment's W
// lanes test the staged candidates with a stride of W.
// A chunk of 32 candidates yields one hit mask per home particle (the
// segment's lanes OR their partial masks together); the hits are then
// written in ascending order, the rank of each hit inside the chunk giving
// its position in the row (the paper's intra-warp prefix sum), and the row
// length advances by the chunk's hit count.  All loops are uniform across the
// block because every thread shares the home cell.
//
// The 27 cells are staged in ascending Hilbert rank and members in ascending
// index, so row entries (stage slots) ascend, and so do the particles they
// name.
//
// Distance test.  Candidates are screened in FP32 from the frame-relative
// offsets; a candidate whose FP32 r^2 lies within a proven error band of
// r_list^2 is re-tested with the FP64 minimum-image distance in the oracle's
// operation order.  The neighbour sets are therefore exactly the FP64 sets.
//
// Storage: 16-bit stage slots.  Row p (the cell-list position of the home
// particle) keeps entry k at ((k / ws) * n_pad + p) * ws + k % ws, ws = the
// pair kernel's W, so that kernel's W lanes read consecutive entries and a
// warp reads the rows of one cell side by side.
#include "md_internal.cuh"

namespace mdgb {

namespace {

__device__ __forceinline__ bool rebuilding(const KArgs &a, int r, int force) {
  return force || a.rebuild[2 * r + (int)(a.ds->step & 1)] != 0;
}

// w = 1: one thread per home particle, the leanest form.  The stage is padded
// to a multiple of 32 slots with far-away dummies, so every chunk of 32
// candidates is a straight-line sequence (broadcast shared-memory load,
// distance, compare, predicated append to the row kept in shared memory).
// The rare candidate in the FP64 tie-break band makes the warp redo that
// chunk in order with the exact test.  Rows are written out at the end,
// coalesced, in the pair kernel's tile layout.
constexpr int kRowsPerPass = 32;

__global__ void k_nlist_w1(KArgs a, int force) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int cap = a.stage_cap;  // a multiple of 32
  StageInfo &si = *reinterpret_cast<StageInfo *>(smem);
  float4 *spos = reinterpret_cast<float4 *>(smem + sizeof(StageInfo));
  int32_t *sidx = reinterpret_cast<int32_t *>(spos + cap);
  uint16_t *rows = reinterpret_cast<uint16_t *>(sidx + cap);  // [kRowsPerPass][max_nb]

  const int64_t g = blockIdx.x;
  const int r = a.chunk_rep[g / kChunkCells];
  if (!rebuilding(a, r, force)) return;
  const int cnt = a.cell_count[g];
  if (cnt == 0) return;
  const Rep &rp = a.rep[r];
  const int start = a.cell_start[g];
  stage_info(a, rp, g, si);
  __syncthreads();
  const bool ident = a.ident[r] != 0;
  const int total = si.off[27], self0 = si.self;
  const float lo = a.rl2f - rp.band, hi = a.rl2f + rp.band;
  const int lw = a.w_store_log2;
  const int max_nb = a.max_nb;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int q0 = 0; q0 < cnt; q0 += kRowsPerPass) {
    const int nq = min(kRowsPerPass, cnt - q0);
    int n = 0;  // this thread's row length (threads >= nq hold no particle)
    const int q = q0 + tid;
    const bool active = tid < nq;
    const int32_t i = a.cell_idx[start + (active ? q : 0)];
    // Threads without a particle, and the padding slots of the stage, hold NaN
    // positions: every comparison with NaN is false, so they never hit (a
    // finite "far away" value would, against an equal far-away padding slot).
    const float qnan = __int_as_float(0x7fc00000);
    float4 oi = __ldg(a.pos4f + i);
    if (!active) oi = make_float4(qnan, qnan, qnan, 0.f);
    uint16_t *myrow = rows + (size_t)(active ? tid : 0) * max_nb;
    const int me = self0 + q;
    for (int w0 = 0; w0 < total; w0 += cap) {
      const int mw = min(cap, total - w0);
      const int mpad = (mw + 31) & ~31;
      __syncthreads();
      stage_fill(a, si, w0, mw, ident, spos, sidx, nullptr);
      for (int k = mw + tid; k < mpad; k += nt) spos[k] = make_float4(qnan, qnan, qnan, 0.f);
      __syncthreads();
      for (int b = 0; b < mpad; b += 32) {
        const int n0 = n;
        bool band = false;
#pragma unroll
        for (int c = 0; c < 32; c++) {
          const float4 oj = spos[b + c];
          const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const bool hit = (r2 < lo) & (w0 + b + c != me);
          band |= (r2 >= lo) & (r2 < hi);
          if (hit) {
            if (n < max_nb) myrow[n] = (uint16_t)(w0 + b + c);
            n++;
          }
        }
        if (__any_sync(0xffffffffu, band)) {
          // redo the chunk in order, deciding band candidates in FP64
          n = n0;
          for (int c = 0; c < 32 && b + c < mw; c++) {
            const float4 oj = spos[b + c];
            const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool hit = active && (r2 < lo) && (w0 + b + c != me);
            if (active && r2 >= lo && r2 < hi && w0 + b + c != me) {
              double d[3];
              hit = exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + sidx[b + c]), rp, d) < a.rl2;
            }
            if (hit) {
              if (n < max_nb) myrow[n] = (uint16_t)(w0 + b + c);
              n++;
            }
          }
        }
      }
    }
    if (active) {
      a.n_nb[start + q] = n;
      if (n > max_nb) {
        atomicMax(&a.ds->need_max_nb, n);
        set_error(a.ds, kErrNlistOverflow);
      }
    }
    // coalesced copy of the pass's rows into the tile layout
    __shared__ int s_len[kRowsPerPass];
    __shared__ int s_kmax;
    if (tid == 0) s_kmax = 0;
    __syncthreads();
    if (active) {
      s_len[tid] = min(n, max_nb);
      atomicMax(&s_kmax, min(n, max_nb));
    }
    __syncthreads();
    const int ws = 1 << lw, kmax = s_kmax;
    const int tiles = (kmax + ws - 1) >> lw;
    const int per_tile = nq << lw;  // words of one tile row of this pass
    for (int e = tid; e < tiles * per_tile; e += nt) {
      const int tile = e / per_tile, rem = e - tile * per_tile;
      const int qq = rem >> lw, k = (tile << lw) + (rem & (ws - 1));
      if (k < s_len[qq])
        a.nl[nl_addr(start + q0 + qq, k, lw, a.n_pad)] = rows[(size_t)qq * max_nb + k];
    }
  }
}

template <int W>
__global__ void k_nlist(KArgs a, int force) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int sl = lane & (W - 1), seg = threadIdx.x / W;
  const int segs = blockDim.x / W;
  const int cap = a.stage_cap;
  StageInfo &si = *reinterpret_cast<StageInfo *>(smem);
  float4 *spos = reinterpret_cast<float4 *>(smem + sizeof(StageInfo));
  int32_t *sidx = reinterpret_cast<int32_t *>(spos + cap);

  const int64_t g = blockIdx.x;  // home cell
  const int r = a.chunk_rep[g / kChunkCells];
  if (!rebuilding(a, r, force)) return;
  const int cnt = a.cell_count[g];
  if (cnt == 0) return;
  const Rep &rp = a.rep[r];
  const int start = a.cell_start[g];
  stage_info(a, rp, g, si);
  __syncthreads();
  const bool ident = a.ident[r] != 0;
  const int total = si.off[27], self0 = si.self;
  const float lo = a.rl2f - rp.band, hi = a.rl2f + rp.band;
  const int lw = a.w_store_log2;
  const bool single = total <= cap;
  if (single) {
    stage_fill(a, si, 0, total, ident, spos, sidx, nullptr);
    __syncthreads();
  }

  for (int q0 = 0; q0 < cnt; q0 += segs) {
    const int q = q0 + seg;
    const bool active = q < cnt;
    const int p = start + (active ? q : 0);
    const int32_t i = a.cell_idx[p];
    // inactive segments hold NaN positions: no comparison with them is true
    const float qnan = __int_as_float(0x7fc00000);
    float4 oi = __ldg(a.pos4f + i);
    if (!active) oi = make_float4(qnan, qnan, qnan, 0.f);
    const int me = self0 + q;  // own stage slot (excluded)
    int n = 0;
    for (int w0 = 0; w0 < total; w0 += cap) {
      const int mw = min(cap, total - w0);
      if (!single) {
        __syncthreads();
        stage_fill(a, si, w0, mw, ident, spos, sidx, nullptr);
        __syncthreads();
      }
      for (int b = 0; b < mw; b += 32) {
        const int mm = min(32, mw - b);
        uint32_t in = 0, maybe = 0;
        for (int c = sl; c < mm; c += W) {
          const float4 oj = spos[b + c];
          const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          in |= (uint32_t)(r2 < lo) << c;
          maybe |= (uint32_t)(r2 < hi) << c;
        }
#pragma unroll
        for (int o = W / 2; o >= 1; o >>= 1) {
          in |= __shfl_xor_sync(FULL, in, o);
          maybe |= __shfl_xor_sync(FULL, maybe, o);
        }
        const int self_bit = me - (w0 + b);
        if (self_bit >= 0 && self_bit < 32) {
          in &= ~(1u << self_bit);
          maybe &= ~(1u << self_bit);
        }
        uint32_t band = maybe & ~in;
        if (__any_sync(FULL, band != 0)) {
          // rare: decide in FP64 with the oracle's operation order
          while (band) {
            const int c = __ffs(band) - 1;
            band &= band - 1;
            double d[3];
            if (exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + sidx[b + c]), rp, d) < a.rl2)
              in |= 1u << c;
          }
        }
        // write the hits in ascending order; hit number h goes to lane h % W
        uint32_t m2 = in;
        int h = 0;
        while (m2) {
          const int c = __ffs(m2) - 1;
          m2 &= m2 - 1;
          if ((h & (W - 1)) == sl) {
            const int k = n + h;
            if (k < a.max_nb) a.nl[nl_addr(p, k, lw, a.n_pad)] = (uint16_t)(w0 + b + c);
          }
          h++;
        }
        n += h;
      }
    }
    if (active && sl == 0) {
      a.n_nb[p] = n;
      if (n > a.max_nb) {
        atomicMax(&a.ds->need_max_nb, n);
        set_error(a.ds, kErrNlistOverflow);
      }
    }
  }
}

template <int W>
cudaError_t launch_w(const KArgs &a, int block, int force, cudaStream_t st) {
  if (W == 1) {
    // one thread per home particle: one warp, rows staged in shared memory
    const size_t smem = stage_bytes(a.stage_cap, false) +
                        (size_t)kRowsPerPass * a.max_nb * sizeof(uint16_t);
    k_nlist_w1<<<(unsigned)a.n_cells, 32, smem, st>>>(a, force);
  } else {
    const size_t smem = stage_bytes(a.stage_cap, false);
    k_nlist<W><<<(unsigned)a.n_cells, block, smem, st>>>(a, force);
  }
  return cudaGetLastError();
}

template <int W>
int max_block_w(int cap) {
  (void)cap;  // one stage per block, independent of the block size
  if (W == 1) return 1024;  // the w = 1 form runs one warp per cell whatever the block
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_nlist<W>) != cudaSuccess) return 0;
  return at.maxThreadsPerBlock;
}

template <int W>
void allow_smem() {
  cudaFuncSetAttribute(k_nlist<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

void nlist_init_attributes() {
  cudaFuncSetAttribute(k_nlist_w1, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  allow_smem<1>(); allow_smem<2>(); allow_smem<4>();
  allow_smem<8>(); allow_smem<16>(); allow_smem<32>();
}

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

int max_block_nlist(int w, int cap) {
  switch (w) {
    case 1: return max_block_w<1>(cap);
    case 2: return max_block_w<2>(cap);
    case 4: return max_block_w<4>(cap);
    case 8: return max_block_w<8>(cap);
    case 16: return max_block_w<16>(cap);
    case 32: return max_block_w<32>(cap);
    default: return 0;
  }
}

}  // namespace mdgb
