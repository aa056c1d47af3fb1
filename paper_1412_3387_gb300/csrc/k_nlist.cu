// Neighbour-list build (Sec. 5.1, Fig. "nlist").
//
// Persistent kernel over brick stages (brick.cuh): while a block's warps work
// on one brick, the next brick's stage is copied into shared memory.  A warp
// takes passes of P = 32 / W particles of the brick (W = 2^m <= 32 lanes per
// particle, the paper's threads per particle; the block size is the paper's
// other tuning parameter).  A particle's candidates are the members of the
// 27 cells around its cell: a 3 x 3 x 3 sub-block of the stage, i.e. nine
// contiguous runs of slots.  The W lanes of a particle split every run into W
// contiguous parts; each lane appends its hits to a row in its own
// shared-memory scratch, so the candidate loop is a straight line (stage load,
// distance, compare, branch-free append).  The W partial rows of a particle,
// concatenated in lane order, form its row (a fixed, deterministic order), and
// are written out, coalesced, in the pair kernel's group-tile layout
// (brick.cuh) with the sentinel padding.
//
// Distance test.  Candidates are screened in FP32; a candidate whose FP32 r^2
// lies within a proven error band of r_list^2 is re-tested with the FP64
// minimum-image distance in the oracle's operation order.  The neighbour sets
// are therefore exactly the FP64 sets.
#include <algorithm>

#include "brick.cuh"

namespace mdgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Scratch of one warp: 32 partial rows of max_nb + 1 entries, stored entry
// by entry across the lanes (entry k of lane l at k * 32 + l, so the lanes'
// appends fall in different banks), then the lanes' row lengths and their
// offsets inside the particle's row.
__host__ __device__ inline size_t warp_scratch_bytes(int max_nb) {
  return ((size_t)32 * (max_nb + 1) * 2 + 64 * 4 + 15) / 16 * 16;
}

template <int WB, bool DIRECT>
__device__ __forceinline__ void build_pass(const KArgs &a, const BrickDesc &d, const float4 *spos,
                                           uint16_t *scr, int *meta, int j) {
  constexpr int PB = 32 / WB;
  constexpr int U = 8;
  const int lane = threadIdx.x & 31;
  const int qq = lane / WB, sl = lane & (WB - 1);
  const int q = j * PB + qq;
  const bool active = q < d.nhome;
  const int qe = active ? qq : 0;
  const Rep &rp = a.rep[d.r];
  const bool ident = a.ident[d.r] != 0;
  const HomeSlot hs = home_slot(d, j * PB + qe);
  const int p = hs.p;
  const StageSrc<DIRECT> src{a, d, rp, smem_u32(spos), 0u};
  const float4 oi = src.pos((uint32_t)(hs.slot + 1));
  const float lo2 = a.rl2f - rp.band, hi2 = a.rl2f + rp.band;
  const int max_nb = a.max_nb;
  uint16_t *row = scr + lane;  // entry k at row[k * 32]
  const uint32_t row_s = smem_u32(row);
  // the nine runs of the particle's 3 x 3 x 3 stencil: stage cells
  // (hx .. hx + 2, hy + dy, hz + dz) for the home cell (hx + 1, hy + 1, hz + 1)
  const int c0 = (hs.s & 3) - 1 + 4 * (((hs.s >> 2) & 3) - 1) + 16 * ((hs.s >> 4) - 1);
  int n = 0;
  for (int rr = 0; rr < 9; rr++) {
    const int s = c0 + 4 * (rr % 3) + 16 * (rr / 3);
    const int rlo = d.off[s], len = d.off[s + 3] - rlo;
    // this lane's part of the run; all lanes take part in every run, and the
    // loop runs to the warp's longest part so that the warp-wide vote below
    // sees every lane
    const int part = (len + WB - 1) / WB;
    const int beg = rlo + sl * part;
    const int mylen = min(max(len - sl * part, 0), part);
    const int wlen = (int)__reduce_max_sync(FULL, (unsigned)mylen);
    for (int x0 = 0; x0 < wlen; x0 += U) {
      const int n0 = n;
      bool band = false;
      // all loads of the group first: the appends below store to shared
      // memory, which the compiler would otherwise not let later loads pass
      float4 oju[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int slot = beg + x0 + u;
        const bool valid = active && x0 + u < mylen && slot != hs.slot;
        oju[u] = src.pos(valid ? (uint32_t)(slot + 1) : 0u);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const float4 oj = oju[u];
        const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        band |= (r2 >= lo2) & (r2 < hi2);
        // branch-free append: the store is kept only if the count moves on
        // (the scratch row has room for max_nb + 1 entries)
        sts16(row_s + (uint32_t)min(n, max_nb) * 64u, (uint16_t)(beg + x0 + u + 1));
        n += r2 < lo2 ? 1 : 0;
      }
      if (__any_sync(FULL, band)) {
        // rare: redo the group in order, deciding band candidates in FP64 with
        // the oracle's operation order
        n = n0;
        const int32_t i = ident ? p : __ldg(a.cell_idx + p);
        for (int u = 0; u < U; u++) {
          const int slot = beg + x0 + u;
          const bool valid = active && x0 + u < mylen && slot != hs.slot;
          if (!valid) continue;
          const float4 oj = src.pos((uint32_t)(slot + 1));
          const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          bool hit = r2 < lo2;
          if (r2 >= lo2 && r2 < hi2) {
            double dd[3];
            hit = exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + src.index((uint32_t)(slot + 1), ident)),
                           rp, dd) < a.rl2;
          }
          if (hit) {
            if (n < max_nb) row[n * 32] = (uint16_t)(slot + 1);
            n++;
          }
        }
      }
    }
  }

  // row length of each particle and each lane's offset inside it
  int incl = n;
#pragma unroll
  for (int o = 1; o < WB; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (sl >= o) incl += y;
  }
  const int nq = __shfl_sync(FULL, incl, qq * WB + WB - 1);
  int *mpre = meta, *mcnt = meta + 32;
  mpre[lane] = incl - n;
  mcnt[lane] = n;
  if (active && sl == 0) {
    a.n_nb[p] = nq;
    if (nq > max_nb) {
      atomicMax(&a.ds->need_max_nb, nq);
      set_error(a.ds, kErrNlistOverflow);
    }
  }
  __syncwarp();

  // write the pass's rows as the pair kernel's row groups (Pp = 32 / Wp
  // particles each; WB <= Wp, so a pass holds whole groups)
  const int lwp = a.w_store_log2, Wp = 1 << lwp, Pp = 32 >> lwp;
  for (int h = 0; h < PB; h += Pp) {
    const int pj = min(Pp, d.nhome - (j * PB + h));
    if (pj <= 0) break;
    const int mine = (active && qq >= h && qq < h + pj) ? min(nq, max_nb) : 0;
    const int mx = (int)__reduce_max_sync(FULL, (unsigned)mine);
    const int T = (mx + Wp - 1) >> lwp;
    const int pg = d.hstart + j * PB + h;
    if (lane == 0) a.nl_tiles[pg] = T;
    uint16_t *out = a.nl + (size_t)pg * (size_t)max_nb;
    const int E = T * pj * Wp;
    const int lpp = 5 - lwp;  // log2 Pp: a full group's tile is 32 entries
    for (int e = lane; e < E; e += 32) {
      const int slp = e & (Wp - 1), rest = e >> lwp;
      const int q2 = pj == Pp ? (rest & (Pp - 1)) : rest % pj;
      const int t = pj == Pp ? (rest >> lpp) : rest / pj;
      const int k = (t << lwp) + slp;
      const int l0 = (h + q2) * WB;  // first lane of the particle's segment
      const int nqb = mpre[l0 + WB - 1] + mcnt[l0 + WB - 1];
      uint16_t v = 0;
      if (k < min(nqb, max_nb)) {
        int sb = 0;
#pragma unroll
        for (int t2 = 1; t2 < WB; t2++)
          if (mpre[l0 + t2] <= k) sb = t2;
        const int off = k - mpre[l0 + sb];
        if (off < max_nb) v = scr[(size_t)off * 32 + (l0 + sb)];
      }
      out[e] = v;
    }
  }
  __syncwarp();
}

// Persistent over bricks b = blockIdx + t G (replicas that do not rebuild are
// skipped); warp w takes the brick's passes w, w + C, ...
template <int WB>
__global__ void __launch_bounds__(kMaxBrickThreads) k_nlist(KArgs a, int cap, int force) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PB = 32 / WB;
  if (!force && !a.ds->rebuild_any) return;  // no replica rebuilds this step
  const long long step = a.ds->step;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the pair kernel runs after this launch has finished (stream order)
    for (int r = 0; r < a.R; r++)
      if (force || a.rebuild[2 * r + (int)(step & 1)]) a.list_ok[r] = 1;
  }
  const BrickSmem M{smem, cap, false};
  const int warp = threadIdx.x >> 5, C = blockDim.x >> 5;
  unsigned char *mine = M.scratch() + (size_t)warp * warp_scratch_bytes(a.max_nb);
  uint16_t *scr = reinterpret_cast<uint16_t *>(mine);
  int *meta = reinterpret_cast<int *>(mine + (size_t)32 * (a.max_nb + 1) * 2);
  const long long G = gridDim.x;
  // the bricks this block builds (rebuilding replicas only)
  auto wanted = [&](long long b) {
    return force || a.rebuild[2 * __ldg(a.brick_rep + b) + (int)(step & 1)] != 0;
  };
  auto next = [&](long long b) {
    while (b < a.n_bricks && !wanted(b)) b += G;
    return b;
  };
  long long bt = next(blockIdx.x);
  if (bt >= a.n_bricks) return;
  long long b1 = next(bt + G);
  if (threadIdx.x < 2) M.pos(threadIdx.x)[0] = make_float4(kFar, kFar, kFar, 0.f);
  desc_fetch(a, bt, M.desc(0));
  if (b1 < a.n_bricks) desc_fetch(a, b1, M.desc(1));
  __syncthreads();
  stage_issue(a, M.desc(0), M.pos(0), nullptr, cap);
  cp_async_wait_all();
  __syncthreads();
  stage_shift_all(a, M.desc(0), M.pos(0), cap);
  __syncthreads();
  constexpr int kDescWords = (int)(sizeof(BrickDesc) / 16);
  for (long long t = 0; bt < a.n_bricks; t++) {
    const bool has1 = b1 < a.n_bricks;
    const long long b2 = has1 ? next(b1 + G) : a.n_bricks;
    const bool has2 = b2 < a.n_bricks;
    if (has1) stage_issue(a, M.desc(t + 1), M.pos(t + 1), nullptr, cap);
    // the descriptor two bricks ahead: loaded now, stored after the work
    // (40 words; a block has at least 32 threads, so two per thread)
    uint4 dv0 = make_uint4(0u, 0u, 0u, 0u), dv1 = dv0;
    const int k0 = threadIdx.x, k1 = threadIdx.x + blockDim.x;
    if (has2) {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.brick_desc + b2);
      if (k0 < kDescWords) dv0 = __ldg(src + k0);
      if (k1 < kDescWords) dv1 = __ldg(src + k1);
    }
    const BrickDesc &d = M.desc(t);
    const int ng = (d.nhome + PB - 1) / PB;
    if (d.off[64] > cap) {
      for (int j = warp; j < ng; j += C) build_pass<WB, true>(a, d, M.pos(t), scr, meta, j);
    } else {
      for (int j = warp; j < ng; j += C) build_pass<WB, false>(a, d, M.pos(t), scr, meta, j);
    }
    if (has2) {
      uint4 *dst = reinterpret_cast<uint4 *>(&M.desc(t + 2));
      if (k0 < kDescWords) dst[k0] = dv0;
      if (k1 < kDescWords) dst[k1] = dv1;
    }
    cp_async_wait_all();
    __syncthreads();
    if (has1) stage_shift_all(a, M.desc(t + 1), M.pos(t + 1), cap);
    __syncthreads();
    bt = b1;
    b1 = b2;
  }
}

// Computing warps that fit beside the stage (each needs its row scratch).
inline int fitting_warps(const KArgs &a, int want) {
  const size_t ring = BrickSmem::bytes(a.stage_cap, false, 0);
  const size_t per = warp_scratch_bytes(a.max_nb);
  const int fit = ring >= 227u * 1024u ? 0 : (int)((227u * 1024u - ring) / per);
  return std::min(want, fit);
}

template <int WB>
cudaError_t launch_w(const KArgs &a, int block, int force, cudaStream_t st) {
  const int C = fitting_warps(a, block / 32);  // large max_nb: fewer warps
  if (C < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = BrickSmem::bytes(a.stage_cap, false, (size_t)C * warp_scratch_bytes(a.max_nb));
  const int threads = 32 * C;
  const int grid = persistent_grid((const void *)k_nlist<WB>, threads, smem, a.n_bricks);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  k_nlist<WB><<<grid, threads, smem, st>>>(a, a.stage_cap, force);
  return cudaGetLastError();
}

template <int WB>
int max_block_w(const KArgs &a) {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_nlist<WB>) != cudaSuccess) return 0;
  return 32 * fitting_warps(a, at.maxThreadsPerBlock / 32);
}

template <int WB>
void allow_smem() {
  cudaFuncSetAttribute(k_nlist<WB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

void nlist_init_attributes() {
  allow_smem<1>(); allow_smem<2>(); allow_smem<4>();
  allow_smem<8>(); allow_smem<16>(); allow_smem<32>();
}

// The build's w never exceeds the pair kernel's (a pass must hold whole row
// groups); a larger request runs at the pair kernel's w.
cudaError_t launch_nlist(const KArgs &a, Launch l, int force, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const int w = std::min(l.w, 1 << a.w_store_log2);
  switch (w) {
    case 1: return launch_w<1>(a, l.block, force, st);
    case 2: return launch_w<2>(a, l.block, force, st);
    case 4: return launch_w<4>(a, l.block, force, st);
    case 8: return launch_w<8>(a, l.block, force, st);
    case 16: return launch_w<16>(a, l.block, force, st);
    case 32: return launch_w<32>(a, l.block, force, st);
    default: return cudaErrorInvalidValue;
  }
}

int max_block_nlist(const KArgs &a, int w) {
  switch (std::min(w, 1 << a.w_store_log2)) {
    case 1: return max_block_w<1>(a);
    case 2: return max_block_w<2>(a);
    case 4: return max_block_w<4>(a);
    case 8: return max_block_w<8>(a);
    case 16: return max_block_w<16>(a);
    case 32: return max_block_w<32>(a);
    default: return 0;
  }
}

}  // namespace mdgb
