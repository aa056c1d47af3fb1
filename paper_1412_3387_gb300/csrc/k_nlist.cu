// Neighbour-list build (Sec. 5.1, Fig. "nlist").
//
// Persistent kernel over brick stages (brick.cuh): while a block's warps work
// on one brick, the next brick's stage is copied into shared memory (bulk
// copies counted on an mbarrier; one block barrier per brick).  A warp
// takes passes of P = 32 / W particles of the brick (W = 2^m <= 32 lanes per
// particle, the paper's threads per particle; the block size is the paper's
// other tuning parameter).  A particle's candidates are the members of the
// 27 cells around its cell: a 3 x 3 x 3 sub-block of the stage, i.e. nine
// contiguous runs of three x-adjacent cells.  Cells keep their members sorted
// by x, so each run is sorted by x at a build: the particle binary-searches
// the part of each run within its reach in x (given its y-z distance to the
// run's row of cells) and skips runs out of reach.  The W lanes of a particle
// split that window into W contiguous parts.  After each block of 32
// candidates (screened in blocks of U = 8) the lanes of a particle take an
// exclusive prefix sum of their hit counts and write their
// hits straight into the row, in the pair kernel's tile layout (brick.cuh);
// rows are then padded with the sentinel up to their group's tile count.
// Rows thus come out compact and in a fixed, deterministic order (block by
// block; within a block, lane by lane, each lane's hits in slot order) with
// no scratch storage.
//
// Half lists (md_set_newton): a pair is kept only in the row of the particle
// with the smaller cell-list position, and the FP64 pair kernel applies
// Newton's third law.
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

// One pass: the brick's particles q0 .. q0 + 32 / WB - 1 (q0 a multiple of
// the pair kernel's group size, so that a pass holds whole row groups).
template <int WB, bool DIRECT>
__device__ __forceinline__ void build_pass(const KArgs &a, const BrickDesc &d, const float4 *spos,
                                           int q0) {
  constexpr int U = 8;
  static_assert(U <= kStagePad, "a block of candidates may read U - 1 slots past a stage");
  const int lane = threadIdx.x & 31;
  const int qq = lane / WB, sl = lane & (WB - 1);
  const int q = q0 + qq;
  const bool active = q < d.nhome;
  const int qe = active ? qq : 0;
  const Rep &rp = a.rep[d.r];
  const bool ident = a.ident[d.r] != 0;
  const HomeSlot hs = home_slot(d, q0 + qe);
  const int p = hs.p;
  const StageSrc<DIRECT> src{a, d, rp, smem_u32(spos), 0u};
  const float4 oi = src.pos((uint32_t)(hs.slot + 1));
  const float lo2 = a.rl2f - rp.band, hi2 = a.rl2f + rp.band;
  // a block with some r^2 in the band [lo2, hi2) goes through the FP64
  // re-test: bthr is the larger exact distance of the rounded band ends from
  // r_list^2, so |r^2 - r_list^2| <= bthr for every r^2 in the band
  const float bthr = fmaxf(a.rl2f - lo2, hi2 - a.rl2f);
  const float rl2f = a.rl2f;  // a local: read in the candidate loop
  const uint64_t oixy = pack2(oi.x, oi.y);
  const int max_nb = a.max_nb;
  // the pair kernel's row layout: groups of Pp = 32 / Wp particles, tiles of
  // Wp entries per particle; the row's entry k sits in tile k / Wp, column k % Wp
  const int lwp = a.w_store_log2, Wp = 1 << lwp, Pp = 32 >> lwp;
  const int Vp = row_depth(Wp);
  const int tcap = max_nb >> lwp;  // tiles a row region holds (a multiple of Vp)
  const int gq = q0 + qe;          // the particle's place in the brick
  const int grp = gq / Pp, q2 = gq - grp * Pp;
  const int pj = min(Pp, d.nhome - grp * Pp);
  uint16_t *gbase = a.nl + (size_t)(d.hstart + grp * Pp) * (size_t)max_nb;
  // row_offset(k, lwp, pj, q2) with the particle's terms hoisted, in
  // unsigned arithmetic (the terms joined by | occupy disjoint bits)
  const unsigned lv = lwp <= 3 ? 2u : 5u - (unsigned)lwp;
  const unsigned pjW = (unsigned)pj << lwp, qW = (unsigned)q2 << lwp;
  auto offs = [&](unsigned k) -> unsigned {
    const unsigned t = k >> lwp;
    return ((((t >> lv) * pjW + qW) | (k & ((unsigned)Wp - 1u))) << lv) | (t & ((1u << lv) - 1u));
  };
  auto put = [&](int k, uint16_t v) {
    if ((k >> lwp) < tcap) gbase[offs((unsigned)k)] = v;
  };
  // the nine runs of the particle's 3 x 3 x 3 stencil: stage cells
  // (hx .. hx + 2, hy + dy, hz + dz) for the home cell (hx + 1, hy + 1, hz + 1)
  const int c0 = (hs.s & 3) - 1 + 4 * (((hs.s >> 2) & 3) - 1) + 16 * ((hs.s >> 4) - 1);
  // x-windows (staged bricks).  At a build every member lies inside its cell
  // and members are sorted by x within a cell, so a run of three x-adjacent
  // cells is sorted by x.  The particle's candidates in a run lie within
  //   |x_j - x_i| <= sqrt(r_list^2 + band - rho^2),
  // rho = its y-z distance to the run's row of cells; a run with rho^2 above
  // r_list^2 + band holds none.  eps (far above the grid rounding of stage
  // coordinates and the drift of the hq-spaced frame faces from the cell
  // faces) keeps the windows conservative.
  const float hy = rp.hq[1], hz = rp.hq[2];
  const float eps = rp.weps;
  const float yb = oi.y - (float)(((hs.s >> 2) & 3) - 2) * hy;  // height above the home row's lower face
  const float zb = oi.z - (float)((hs.s >> 4) - 2) * hz;
  auto xs = [&](int slot) { return lds1(src.spos + 16u * (uint32_t)(slot + 1)); };
  int n = 0;  // row length so far (the same in the particle's WB lanes)
  for (int rr = 0; rr < 9; rr++) {
    const int s = c0 + 4 * (rr % 3) + 16 * (rr / 3);
    int rlo = d.off[s], len = d.off[s + 3] - rlo;
    // cell-list position of a slot of this run (half lists): start of its
    // stage cell (s, s + 1 or s + 2) plus its place in the cell
    const int o1 = d.off[s + 1], o2 = d.off[s + 2];
    const int b0 = d.start[s] - d.off[s], b1 = d.start[s + 1] - o1, b2 = d.start[s + 2] - o2;
    if (!DIRECT) {
      const int dyi = rr % 3, dzi = rr / 3;
      const float ry = fmaxf((dyi == 0 ? yb : dyi == 2 ? hy - yb : 0.f) - eps, 0.f);
      const float rz = fmaxf((dzi == 0 ? zb : dzi == 2 ? hz - zb : 0.f) - eps, 0.f);
      const float rem = hi2 - fmaf(ry, ry, rz * rz);
      if (!(rem >= 0.f)) {
        len = 0;
      } else {
        const float wx = sqrtf(rem) + eps, klo = oi.x - wx, khi = oi.x + wx;
        // first slot with x >= klo (b) and first slot with x > khi (e),
        // searched side by side so that their shared-memory loads overlap; a
        // finished search re-reads its final slot (at most the run's end, a
        // slot of the padded stage) and keeps its result
        int b = rlo, mb = len, e = rlo, me = len;
        while (mb > 0 || me > 0) {
          const int hb = mb >> 1, he = me >> 1;
          const float xb = xs(b + hb), xe = xs(e + he);
          const bool gb = xb < klo, ge = xe <= khi;
          if (mb > 0) {
            b = gb ? b + hb + 1 : b;
            mb = gb ? mb - hb - 1 : hb;
          }
          if (me > 0) {
            e = ge ? e + he + 1 : e;
            me = ge ? me - he - 1 : he;
          }
        }
        rlo = b;
        len = max(e - b, 0);
      }
    }
    // this lane's part of the run; all lanes take part in every run, and the
    // loop runs to the warp's longest part so that the warp-wide vote and the
    // shuffles below see every lane
    const int part = (len + WB - 1) / WB;
    const int beg = rlo + sl * part;
    const int mylen = active ? min(max(len - sl * part, 0), part) : 0;
    const int wlen = (int)__reduce_max_sync(FULL, (unsigned)mylen);
    // One screened block: bit u set iff slot beg + xb + u is a neighbour.
    auto screen = [&](const int xb) -> unsigned {
      // r^2 of the block's candidates (the (x, y) separation as one packed
      // FP32 pair difference)
      float r2u[U];
      if (DIRECT) {
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int slot = beg + xb + u;
          const bool valid = xb + u < mylen && slot != hs.slot;
          const float4 oj = src.pos(valid ? (uint32_t)(slot + 1) : 0u);
          const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
          r2u[u] = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        }
      } else {
        // the whole block is read (up to U - 1 slots past the lane's part,
        // still inside the padded stage) and the slots that are not
        // candidates are masked out below; a lane whose part has ended reads
        // slots 0 .. U - 1
        const uint32_t base = xb < mylen ? src.spos + (uint32_t)(beg + xb + 1) * 16u : src.spos;
        uint64_t xy[U], zw[U];
#pragma unroll
        for (int u = 0; u < U; u++) lds_pairs(base + 16u * u, xy[u], zw[u]);
#pragma unroll
        for (int u = 0; u < U; u++) {
          const float2 dxy = unpack2(sub_f32x2(oixy, xy[u]));
          const float dz = oi.z - unpack2(zw[u]).x;
          r2u[u] = fmaf(dz, dz, fmaf(dxy.y, dxy.y, dxy.x * dxy.x));
        }
      }
      float bmin = 3.0e38f;  // smallest |r^2 - r_list^2| of the block
      unsigned m = 0u;       // bit u: candidate xb + u is a neighbour
#pragma unroll
      for (int u = 0; u < U; u++) {
        bmin = fminf(bmin, fabsf(r2u[u] - rl2f));
        m |= (r2u[u] < lo2 ? 1u : 0u) << u;
      }
      if (__any_sync(FULL, bmin <= bthr)) {
        // rare: decide the block's band candidates in FP64 with the oracle's
        // operation order
        const int32_t i = ident ? p : __ldg(a.cell_idx + p);
        for (int u = 0; u < U; u++) {
          const int slot = beg + xb + u;
          if (!(xb + u < mylen && slot != hs.slot)) continue;
          const float4 oj = src.pos((uint32_t)(slot + 1));
          const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (r2 >= lo2 && r2 < hi2) {
            double dd[3];
            const bool hit = exact_r2(ld_d4(a.pos + i),
                                      ld_d4(a.pos + src.index((uint32_t)(slot + 1), ident)), rp,
                                      dd) < a.rl2;
            m |= (hit ? 1u : 0u) << u;
          }
        }
      }
      if (!DIRECT) {
        // candidates only: slots of this lane's part, not the particle itself
        m &= (1u << min(max(mylen - xb, 0), U)) - 1u;
        const int so = hs.slot - (beg + xb);
        if ((unsigned)so < (unsigned)U) m &= ~(1u << so);
      }
      if (a.half) {
        // half list: a pair stays only in the row of the particle with the
        // smaller cell-list position
        unsigned keep = 0u;
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int slot = beg + xb + u;
          const int g = slot + (slot < o1 ? b0 : slot < o2 ? b1 : b2);
          keep |= (g > p ? 1u : 0u) << u;
        }
        m &= keep;
      }
      return m;
    };
    // Candidates go through the screen in blocks of U and their hits are
    // written in blocks of 4 U = 32: the warp's hit loop runs to its busiest
    // lane, and over 32 candidates that lane's excess over the mean hit count
    // is smaller than over four separate blocks of U (about 2.8 instead of
    // 4.2 iterations per U candidates at the LJ fluid's hit rate).  The
    // blocks of one write block share one copy of the screen's code.
    static_assert(4 * U == 32, "a write block's hits fill one 32-bit mask");
    for (int x0 = 0; x0 < wlen; x0 += 4 * U) {
      unsigned m = 0u;
#pragma unroll 1
      for (int j = 0; j < 4; j++) {
        const int xb = x0 + j * U;
        if (xb >= wlen) break;  // warp-uniform
        m |= screen(xb) << (j * U);
      }
      // compact: this lane's hits follow those of the particle's lower lanes
      const int h = __popc(m);
      int incl = h;
#pragma unroll
      for (int o = 1; o < WB; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (sl >= o) incl += v;
      }
      const int tot = __shfl_sync(FULL, incl, lane | (WB - 1));
      int k = n + incl - h;
      if (k + h <= (tcap << lwp)) {
        // the common case: all of the lane's hits fit the row region
        while (m) {
          const int u = __ffs(m) - 1;
          m &= m - 1u;
          gbase[offs((unsigned)k++)] = (uint16_t)(beg + x0 + u + 1);
        }
      } else {
        while (m) {
          const int u = __ffs(m) - 1;
          m &= m - 1u;
          put(k++, (uint16_t)(beg + x0 + u + 1));
        }
      }
      n += tot;
    }
  }

  // tiles of the particle and of its pair group (Pp particles = Pp * WB
  // aligned lanes of this warp)
  const int tq = active ? (n + Wp - 1) >> lwp : 0;
  int tg = tq;
  const int glanes = Pp * WB;
  for (int o = 1; o < glanes; o <<= 1) tg = max(tg, __shfl_xor_sync(FULL, tg, o));
  tg = min((tg + Vp - 1) / Vp * Vp, tcap);  // whole blocks of Vp tiles
  if (active && sl == 0) {
    a.n_nb[p] = n;
    if (tq > tcap) {
      atomicMax(&a.ds->need_max_nb, tq * Wp);
      set_error(a.ds, kErrNlistOverflow);
    }
  }
  if (active && q2 == 0 && sl == 0) a.nl_tiles[d.hstart + grp * Pp] = tg;
  // sentinel padding of the row up to the group's tile count
  if (active)
    for (int k = n + sl; k < (tg << lwp); k += WB) put(k, 0);
}

// Persistent over bricks b = blockIdx + t G (replicas that do not rebuild are
// skipped); warp w takes the brick's passes w, w + C, ...
template <int WB>
__global__ void __launch_bounds__(kMaxBrickThreads, 1) k_nlist(KArgs a, int cap, int force) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PB = 32 / WB;
  if (!force && !a.ds->rebuild_any) return;  // no replica rebuilds this step
  // After a non-finite position or an over-full cell the step's results are
  // invalid (the host sees the error); skip the build: non-finite positions
  // all bin into one cell, whose stage the build would scan quadratically.
  if (fatal_error(a)) return;
  const long long step = a.ds->step;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the pair kernel runs after this launch has finished (stream order)
    for (int r = 0; r < a.R; r++)
      if (force || a.rebuild[2 * r + (int)(step & 1)]) a.list_ok[r] = 1;
  }
  const BrickSmem M{smem, cap, false};
  const int warp = threadIdx.x >> 5, C = blockDim.x >> 5;
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
  if (threadIdx.x == 0) {
    mbar_init(M.bar(0), 1);
    mbar_init(M.bar(1), 1);
  }
  desc_fetch(a, bt, M.desc(0));
  if (b1 < a.n_bricks) desc_fetch(a, b1, M.desc(1));
  fence_proxy_async();
  __syncthreads();
  stage_issue(a, M.desc(0), M.pos(0), nullptr, M.bar(0), cap);
  bool ok = stage_wait(a, M, 0);
  stage_shift_all(a, M.desc(0), M.pos(0), cap);
  if (!__syncthreads_and(ok)) {
    stage_drain(M, 0);
    return;
  }
  constexpr int kDescWords = (int)(sizeof(BrickDesc) / 16);
  for (long long t = 0; bt < a.n_bricks; t++) {
    const bool has1 = b1 < a.n_bricks;
    const long long b2 = has1 ? next(b1 + G) : a.n_bricks;
    const bool has2 = b2 < a.n_bricks;
    if (has1) stage_issue(a, M.desc(t + 1), M.pos(t + 1), nullptr, M.bar(t + 1), cap);
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
    if (d.off[64] > cap) {
      for (int q0 = warp * PB; q0 < d.nhome; q0 += C * PB) build_pass<WB, true>(a, d, M.pos(t), q0);
    } else {
      // whole rounds of one pass per warp; the rest, when it fits one round of
      // passes at twice the lanes per particle (each lane then scans half a
      // window), is split that way, so that the warps reach the brick barrier
      // together instead of some waiting a whole pass for the others
      const int whole = d.nhome / (C * PB) * (C * PB);
      int q0 = warp * PB;
      for (; q0 < whole; q0 += C * PB) build_pass<WB, false>(a, d, M.pos(t), q0);
      if constexpr (WB < 32) {
        constexpr int PH = PB / 2;
        const int rest = d.nhome - whole;
        if (2 * WB <= (1 << a.w_store_log2) && rest <= C * PH) {
          const int qh = whole + warp * PH;
          if (qh < d.nhome) build_pass<2 * WB, false>(a, d, M.pos(t), qh);
          q0 = d.nhome;
        }
      }
      for (; q0 < d.nhome; q0 += C * PB) build_pass<WB, false>(a, d, M.pos(t), q0);
    }
    if (has2) {
      uint4 *dst = reinterpret_cast<uint4 *>(&M.desc(t + 2));
      if (k0 < kDescWords) dst[k0] = dv0;
      if (k1 < kDescWords) dst[k1] = dv1;
    }
    // brick t + 1's stage: wait for its copies, add the shifts, publish (the
    // barrier also frees brick t's buffer for brick t + 2's copies)
    ok = !has1 || stage_wait(a, M, t + 1);
    if (has1) stage_shift_all(a, M.desc(t + 1), M.pos(t + 1), cap);
    fence_proxy_async();
    if (!__syncthreads_and(ok)) {
      stage_drain(M, t + 1);
      return;
    }
    bt = b1;
    b1 = b2;
  }
}

template <int WB>
cudaError_t launch_w(const KArgs &a, int block, int force, cudaStream_t st) {
  const size_t smem = BrickSmem::bytes(a.stage_cap, false, 0);
  const int grid = persistent_grid((const void *)k_nlist<WB>, block, smem, a.n_bricks);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  k_nlist<WB><<<grid, block, smem, st>>>(a, a.stage_cap, force);
  return cudaGetLastError();
}

template <int WB>
int max_block_w(const KArgs &) {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_nlist<WB>) != cudaSuccess) return 0;
  return at.maxThreadsPerBlock;
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
