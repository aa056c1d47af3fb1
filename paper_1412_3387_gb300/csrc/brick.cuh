// Brick stages shared by the neighbour-list build and the pair kernel.
//
// Cells are grouped into bricks of 2 x 2 x 2 (ceil(nc / 2) bricks per edge,
// the last one thinner when nc is odd).  Bricks follow a Hilbert curve and a
// brick's cells are consecutive in cell-list order (x first, then y, then z),
// so a brick's particles are one contiguous range.
//
// The unit of work of both kernels is a brick.  Its stage is the 4 x 4 x 4
// block of cells around it (stage cell s = sx + 4 sy + 16 sz covers cell
// 2 b - 1 + s per axis, periodically wrapped; on very small grids a cell can
// appear twice, at two periodic images).  Each home cell's 27 neighbour
// cells form a 3 x 3 x 3 sub-block of the stage.  The stage holds the FP32
// positions of all members of the 64 stage cells relative to the brick
// origin: member offset o from its own frame centre (pos4f, kept in
// cell-list order so each cell is a contiguous range) plus the stage cell's
// shift (s - 1.5) hq, plus or minus wq for a cell seen across the periodic
// boundary.  Then
//   x_i - x_j = stage[slot of i] - stage[slot of j]
// for any home particle i and stage particle j of its stencil.
//
// Exactness.  o, hq and wq are multiples of the replica's grid gq (a power of
// two) and every stage coordinate and separation stays below 2^24 gq in
// magnitude, so all of them are computed exactly in FP32: the only error is
// the rounding of each offset to the grid (and of wq), at most 1.5 gq per
// separation component.  A pair's separation seen from i's brick is then
// exactly minus the one seen from j's, and the pair forces the two bricks
// compute are exactly opposite (Newton's third law holds to the last bit,
// so the FP32 forces conserve momentum up to the per-particle sums' rounding).
//
// A persistent block walks bricks b, b + G, b + 2G, ... with two stage
// buffers: while its warps compute brick t, brick t + 1's stage is in flight
// as one bulk copy (cp.async.bulk) per stage cell, issued by one warp and
// counted on the buffer's mbarrier (transaction bytes).  After brick t the
// warps wait for that barrier's phase (bounded: a timeout raises
// kErrTimeout), add the shifts, and a block barrier publishes the stage.  A
// brick's descriptor (stage layout: first slot and cell-list start of each
// stage cell, home cells) is built once per binning (k_brick_desc) and read
// with one coalesced load two bricks ahead.
//
// Stage slot 0 is a sentinel particle far away (its r^2 to anything
// overflows to +inf, never inside a cut-off, and 0 * its offset is 0).  Row
// entries are 1 + the slot index; rows are padded with 0.
//
// Row layout: a brick's particles form groups of P = 32 / W (W = the pair
// kernel's lanes per particle; one group is one warp's work).  Group j
// (particles jP .. jP + Pj - 1, at cell-list positions hstart + jP ...) keeps
// its rows in the list region reserved for those particles, starting at
// (hstart + jP) * max_nb.  Entry k of the group's particle q belongs to tile
// t = k / W and lane l = q W + k % W; V = row_depth(W) consecutive tiles of
// one lane are contiguous:
//   offset(k) = ((t / V) Pj W + l) V + t % V,
// so a lane reads V entries (8 bytes for W <= 8) with one load and a warp
// reads whole 32-byte sectors.  A group's tile count T_j (nl_tiles) is its
// longest row's ceil(length / W) rounded up to a multiple of V; shorter rows
// are padded with the sentinel entry.
//
// A brick whose stage does not fit the buffer (an unusually dense region) is
// "direct": its positions are read from global memory instead.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

constexpr int kStageCells = 64;

// Consecutive tiles of one lane stored together in the row layout.
__host__ __device__ constexpr int row_depth(int W) { return W <= 8 ? 4 : 32 / W; }

// Offset of entry k of the group's particle q from the group's base (row
// layout above); lw = log2 W, pj = particles in the group.
__device__ __forceinline__ int row_offset(int k, int lw, int pj, int q) {
  const int lv = lw <= 3 ? 2 : 5 - lw;  // log2 row_depth(1 << lw)
  const int t = k >> lw;
  return ((((t >> lv) * pj + q) << lw) + (k & ((1 << lw) - 1))) * (1 << lv) + (t & ((1 << lv) - 1));
}
constexpr float kFar = 1e30f;  // sentinel coordinate
constexpr int kMaxBrickThreads = 512;
constexpr int kStagePad = 8;  // slots past a stage that the list build may read (not use)

// Stage layout of one brick (global array, built per binning; copied to
// shared memory by the kernels).  640 bytes.
struct BrickDesc {
  int off[65];    // first slot (0-based, sentinel excluded) of each stage cell; off[64] = total
  int start[64];  // cell-list position of each stage cell's first member
  int r;          // replica
  int hstart;     // cell-list position of the brick's first particle
  int nhome;      // particles in the brick
  int hmask;      // bit p set if the brick's cell p = hx + 2 hy + 4 hz exists
  int hoff[9];    // the brick's particle q lies in its i-th existing cell for hoff[i] <= q < hoff[i+1]
  int hcell[8];   // stage cell of the brick's i-th existing cell
  int hbase[8];   // staged slot of the particle at cell-list position p of that cell: p + hbase[i]
  int bc;         // brick coordinates bx | by << 10 | bz << 20 (periodic images of the stage)
  int pad;
};
static_assert(sizeof(BrickDesc) == 640, "BrickDesc layout");

// Stage cell of the brick's i-th existing cell.
__device__ __forceinline__ int home_stage_cell(int hmask, int i) {
  int p = 0;
  for (int k = 0, seen = 0; k < 8; k++)
    if ((hmask >> k) & 1) {
      if (seen == i) p = k;
      seen++;
    }
  return (1 + (p & 1)) + 4 * (1 + ((p >> 1) & 1)) + 16 * (1 + (p >> 2));
}

// The brick's existing cell holding its particle q.
__device__ __forceinline__ int home_cell_of(const BrickDesc &d, int q) {
  int i = 0;
#pragma unroll
  for (int k = 1; k < 8; k++) i += d.hoff[k] <= q ? 1 : 0;
  return i;
}

// Stage cell holding 0-based slot s (largest k with off[k] <= s).
__device__ __forceinline__ int stage_cell_of(const BrickDesc &d, int s) {
  int k = 0;
#pragma unroll
  for (int step = 32; step >= 1; step >>= 1)
    if (k + step < kStageCells && d.off[k + step] <= s) k += step;
  return k;
}

// Shift of stage cell coordinate s (0..3) along axis ax for a brick at brick
// coordinate b: (s - 1.5) hq, minus wq if the cell is the periodic image
// below the box, plus wq above it.  Both terms are multiples of gq, so the
// shift and its sum with an offset are exact.
__device__ __forceinline__ float stage_shift1(const Rep &rp, int ax, int s, int b) {
  const int c = 2 * b - 1 + s;
  const float w = c < 0 ? -rp.wq[ax] : c >= rp.nc[ax] ? rp.wq[ax] : 0.f;
  return ((float)s - 1.5f) * rp.hq[ax] + w;
}

__device__ __forceinline__ float3 stage_shift(const Rep &rp, int s, int bc) {
  return make_float3(stage_shift1(rp, 0, s & 3, bc & 1023),
                     stage_shift1(rp, 1, (s >> 2) & 3, (bc >> 10) & 1023),
                     stage_shift1(rp, 2, s >> 4, bc >> 20));
}

// ---- asynchronous copies (PTX) ---------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrives once on `bar` and adds `bytes` to the transactions its current
// phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase of `bar` with the given parity to complete, for at most
// about a second (2^31 SM clocks); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// global -> shared, completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Asks the memory system to bring `bytes` (a multiple of 16; address 16-byte
// aligned) of global memory into L2 ahead of use (a hint: no data moves to
// the SM, nothing waits for it).
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory accesses through 32-bit shared-window addresses: one 128-bit
// load per staged particle, whatever the compiler can prove about a pointer.
__device__ __forceinline__ float4 lds4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// A staged particle as two packed FP32 pairs, (x, y) and (z, w).
__device__ __forceinline__ void lds_pairs(uint32_t addr, uint64_t &xy, uint64_t &zw) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(xy), "=l"(zw) : "r"(addr) : "memory");
}

__device__ __forceinline__ uint64_t pack2(float x, float y) {
  uint64_t v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x), "f"(y));
  return v;
}

__device__ __forceinline__ float2 unpack2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// Packed FP32 subtraction (two IEEE round-to-nearest differences in one
// instruction).
__device__ __forceinline__ uint64_t sub_f32x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// 1 / x by the hardware approximation (one instruction; about one ulp of
// relative error, and +inf gives +0).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float lds1(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void sts16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}

// ---- the block's view of its shared memory ---------------------------------

// [3] descriptors, [2] mbarriers (+ pad to 16 B), [2][cap + 1 + pad]
// positions, ([2][cap + 1 + pad] velocities), then scratch.  Slot 0 is the
// sentinel; the pad lets the list build read whole blocks of candidates past
// the end of a stage.
struct BrickSmem {
  unsigned char *base;
  int cap;
  bool vel;
  __host__ __device__ static int pitch(int cap) { return cap + 1 + kStagePad; }
  __host__ __device__ static size_t desc_bytes() { return 3 * sizeof(BrickDesc) + 16; }
  __host__ __device__ static size_t stage_bytes(int cap, bool vel) {
    return (size_t)2 * pitch(cap) * sizeof(float4) * (vel ? 2 : 1);
  }
  __host__ __device__ static size_t bytes(int cap, bool vel, size_t scratch) {
    return desc_bytes() + stage_bytes(cap, vel) + scratch;
  }
  __device__ __forceinline__ BrickDesc &desc(long long t) const {
    return reinterpret_cast<BrickDesc *>(base)[t % 3];
  }
  // the mbarrier counting the copies of the stage buffer of brick t
  __device__ __forceinline__ uint64_t *bar(long long t) const {
    return reinterpret_cast<uint64_t *>(base + 3 * sizeof(BrickDesc)) + (t & 1);
  }
  __device__ __forceinline__ float4 *pos(long long t) const {
    return reinterpret_cast<float4 *>(base + desc_bytes()) + (t & 1) * pitch(cap);
  }
  __device__ __forceinline__ float4 *vel4(long long t) const {
    return reinterpret_cast<float4 *>(base + desc_bytes()) + (2 + (t & 1)) * pitch(cap);
  }
  __device__ __forceinline__ unsigned char *scratch() const {
    return base + desc_bytes() + stage_bytes(cap, vel);
  }
};

// Copies brick descriptor b from global memory into `dst`, cooperatively
// (40 16-byte words).
__device__ __forceinline__ void desc_fetch(const KArgs &a, long long b, BrickDesc &dst) {
  const uint4 *src = reinterpret_cast<const uint4 *>(a.brick_desc + b);
  uint4 *d = reinterpret_cast<uint4 *>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(BrickDesc) / 16); k += blockDim.x) d[k] = __ldg(src + k);
}

// Issues the copies of a brick's stage (positions, and velocities if vel4 is
// given), counted on `bar`: the block's warps share the 64 stage cells (warp
// w takes cells w, w + C, ...), and the two cells of each stage row that
// belong to the brick itself (stage x = 1, 2), adjacent in cell-list order,
// go as one copy.  A brick served from global memory only arrives.  The
// buffer's previous readers and writers fenced and synchronised before this.
// (The arrival may follow some copies' completion: the phase cannot complete
// before its one arrival.)
__device__ __forceinline__ void stage_issue(const KArgs &a, const BrickDesc &d, float4 *pos,
                                            float4 *vel4, uint64_t *bar, int cap) {
  const bool staged = d.off[64] <= cap;
  if (threadIdx.x == 0)
    mbar_arrive_expect_tx(bar, staged ? (uint32_t)d.off[64] * 16u * (vel4 ? 2u : 1u) : 0u);
  if (!staged) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, C = blockDim.x >> 5;
  for (int s = warp + C * lane; s < kStageCells; s += 32 * C) {
    const int sx = s & 3;
    int o = d.off[s], n = d.off[s + 1] - o;
    const int st = d.start[s];
    if (sx == 2 && d.start[s - 1] + (o - d.off[s - 1]) == st) continue;  // sent with its left neighbour
    if (sx == 1 && st + n == d.start[s + 1]) n += d.off[s + 2] - d.off[s + 1];
    if (n > 0) {
      bulk_g2s(pos + 1 + o, a.pos4f + st, 16u * (uint32_t)n, bar);
      if (vel4) bulk_g2s(vel4 + 1 + o, a.vel4f + st, 16u * (uint32_t)n, bar);
    }
  }
}

// Waits for brick t's stage copies (buffer t & 1, its (t >> 1)-th use); on
// timeout raises kErrTimeout and returns false.
__device__ __forceinline__ bool stage_wait(const KArgs &a, const BrickSmem &M, long long t) {
  if (mbar_wait(M.bar(t), (uint32_t)((t >> 1) & 1))) return true;
  if ((threadIdx.x & 31) == 0) set_error(a.ds, kErrTimeout);
  return false;
}

// Leaving after a timed-out wait: the copies of brick t's stage may still be
// writing into this block's shared memory, so wait for them once more (again
// bounded) before the block exits.
__device__ __forceinline__ void stage_drain(const BrickSmem &M, long long t) {
  mbar_wait(M.bar(t), (uint32_t)((t >> 1) & 1));
}

// Kernels that read the neighbour list skip their work once the device error
// word holds a non-finite position or an over-full cell (the step's results
// are invalid; the host sees the error).
__device__ __forceinline__ bool fatal_error(const KArgs &a) {
  return (__ldcg(&a.ds->error) & (kErrNonfinite | kErrCellOverflow)) != 0u;
}

// Adds the stage cells' shifts to their copied offsets (warp w takes stage
// cells w, w + C, ...); the caller has waited for the copies.
__device__ __forceinline__ void stage_shift_all(const KArgs &a, const BrickDesc &d, float4 *pos,
                                                int cap) {
  if (d.off[64] > cap) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, C = blockDim.x >> 5;
  // the brick's twelve shifts, one per lane 4 ax + s (ax = axis, s = stage
  // coordinate), computed once and broadcast to the cells by shuffles
  float tab = 0.f;
  if (lane < 12) {
    const int ax = lane >> 2;
    tab = stage_shift1(a.rep[d.r], ax, lane & 3, (d.bc >> (10 * ax)) & 1023);
  }
  auto shift_of = [&](int s) {
    float3 h;
    h.x = __shfl_sync(0xffffffffu, tab, s & 3);
    h.y = __shfl_sync(0xffffffffu, tab, 4 + ((s >> 2) & 3));
    h.z = __shfl_sync(0xffffffffu, tab, 8 + (s >> 4));
    return h;
  };
  // two cells per pass (s and s + C), both loads ahead of both stores
  float4 *const p1 = pos + 1;
  for (int s = warp; s < kStageCells; s += 2 * C) {
    const int t = s + C < kStageCells ? s + C : s;
    const int oa = d.off[s], na = d.off[s + 1] - oa;
    const int ob = d.off[t], nb = t != s ? d.off[t + 1] - ob : 0;
    const float3 ha = shift_of(s), hb = shift_of(t);
    const int nm = na > nb ? na : nb;
    for (int m = lane; m < nm; m += 32) {
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (m < na) va = p1[oa + m];
      if (m < nb) vb = p1[ob + m];
      if (m < na) p1[oa + m] = make_float4(va.x + ha.x, va.y + ha.y, va.z + ha.z, va.w);
      if (m < nb) p1[ob + m] = make_float4(vb.x + hb.x, vb.y + hb.y, vb.z + hb.z, vb.w);
    }
  }
}

// Where a staged slot's particle lives: the stage, or (direct bricks) global
// memory through the descriptor.  Entries are 1 + slot; entry 0 is the
// far-away sentinel.
template <bool DIRECT>
struct StageSrc {
  const KArgs &a;
  const BrickDesc &d;
  const Rep &rp;
  uint32_t spos, svel;  // shared-window addresses of the stage arrays
  __device__ __forceinline__ float4 pos(uint32_t e) const {
    if (!DIRECT) return lds4(spos + e * 16u);
    if (e == 0u) return make_float4(kFar, kFar, kFar, 0.f);
    const int s = (int)e - 1, k = stage_cell_of(d, s);
    float4 v = __ldg(a.pos4f + d.start[k] + (s - d.off[k]));
    const float3 h = stage_shift(rp, k, d.bc);
    v.x += h.x;
    v.y += h.y;
    v.z += h.z;
    return v;
  }
  __device__ __forceinline__ float4 vel(uint32_t e) const {
    if (!DIRECT) return lds4(svel + e * 16u);
    if (e == 0u) return make_float4(0.f, 0.f, 0.f, 0.f);
    const int s = (int)e - 1, k = stage_cell_of(d, s);
    return __ldg(a.vel4f + d.start[k] + (s - d.off[k]));
  }
  // cell-list position / particle index of the neighbour in entry e (e > 0)
  __device__ __forceinline__ int position(uint32_t e) const {
    const int s = (int)e - 1, k = stage_cell_of(d, s);
    return d.start[k] + (s - d.off[k]);
  }
  __device__ __forceinline__ int32_t index(uint32_t e, bool ident) const {
    const int p = position(e);
    return ident ? p : __ldg(a.cell_idx + p);
  }
};

// The brick's particle q: its cell-list position, stage cell and staged slot.
struct HomeSlot {
  int p, s, slot;
};
__device__ __forceinline__ HomeSlot home_slot(const BrickDesc &d, int q) {
  HomeSlot h;
  const int i = home_cell_of(d, q);
  h.p = d.hstart + q;
  h.s = d.hcell[i];
  h.slot = h.p + d.hbase[i];
  return h;
}

}  // namespace mdgb
