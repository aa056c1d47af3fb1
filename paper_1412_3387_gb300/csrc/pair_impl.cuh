// Pair forces from the neighbour list (Sec. 5.1: W threads per particle stride
// over its row; the W partial forces are combined with warp shuffles).
//
// Persistent kernel over brick stages (brick.cuh): while a block's warps work
// on one brick, the next brick's stage (positions relative to the brick
// centre, plus FP32 velocities for DPD) is copied into shared memory; each
// warp takes whole row groups of the brick (P = 32 / W particles, W lanes
// each), so every neighbour position comes from shared memory and every
// separation is a single FP32 subtraction per component.
//
// Potentials: LJ 12-6 (Sec. 3; benchmarks of Sec. 6, 8.3), DPD in the
// Groot-Warren form with a Philox-4x32-10 pair noise keyed on the global IDs
// (Sec. 9: per-pair generators seeded with global particle IDs), and the
// Gaussian, Morse and Yukawa pairs of Sec. 3's list in their textbook forms.
//
// Precision forms:
//   FP64  -- FP64 distance (fixed-order minimum image) and FP64 force math.
//   mixed -- FP32 separations and force math; each lane sums the forces of a
//            group of U row entries plainly and adds the group sum to
//            Kahan-compensated FP32 per-particle sums, which are merged across
//            the W lanes with error-free two-sums.
// In both forms the cut-off decision r^2 < r_cut^2 is the FP64 one: an FP32
// r^2 inside a proven error band around r_cut^2 is re-tested in FP64.
#pragma once

#include <algorithm>

#include "brick.cuh"

namespace mdgb {

constexpr int kLJ = 0, kDPD = 1, kGauss = 2, kMorse = 3, kYukawa = 4, kTable = 5;

namespace {
constexpr unsigned FULL = 0xffffffffu;

// Kahan accumulation: s - c is the running sum.
struct KSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  // Merge with another lane's (s, c) by an error-free two-sum of the heads.
  __device__ __forceinline__ void merge(float s2, float c2) {
    float t = s + s2;
    float z = t - s;
    float err = (s - (t - z)) + (s2 - z);
    c = (c + c2) - err;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s - c; }
};

template <int W>
__device__ __forceinline__ void seg_merge(KSum &k) {
#pragma unroll
  for (int m = W / 2; m >= 1; m >>= 1) {
    float s2 = __shfl_xor_sync(FULL, k.s, m);
    float c2 = __shfl_xor_sync(FULL, k.c, m);
    k.merge(s2, c2);
  }
}

template <int W>
__device__ __forceinline__ double seg_sum(double v) {
#pragma unroll
  for (int m = W / 2; m >= 1; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
  return v;
}

// FP32 uniform on (0, 1) from a 32-bit random word: ((w >> 9) + 1/2) 2^-23,
// built from the bits (1 + (w >> 9) 2^-23 is the float with those mantissa
// bits; subtracting 1 - 2^-24 is exact), with no integer-to-float conversion.
__device__ __forceinline__ float unit_uniform(uint32_t w) {
  return __uint_as_float(0x3f800000u | (w >> 9)) - 0.99999994039535522f;
}

// Tabulated pair: V and F = -dV/dr linear in r between samples at r_min + j
// dr, held at their r_min values below r_min; segment j = (V_j, F_j,
// V_j+1 - V_j, F_j+1 - F_j).  Returns F / r, V in v.  (A non-finite r^2, the
// sentinel, lands in segment 0; its result is never used.)
__device__ __forceinline__ float table_fr(const PotCoeffF &c, const float4 *tab, float r2,
                                          float &v) {
  const float rinv = rsqrtf(r2), r = r2 * rinv;
  const float x = fmaxf((r - c.c0) * c.c1, 0.f);
  const int k = min((int)x, (int)c.c2);
  const float t = x - (float)k;
  const float4 s = __ldg(tab + __float_as_int(c.c3) + k);
  v = fmaf(t, s.z, s.x);
  return fmaf(t, s.w, s.y) * rinv;
}

__device__ __forceinline__ double table_fr(const PotCoeffD &c, const double4 *tab, double r2,
                                           double &v) {
  const double r = sqrt(r2);
  const double x = fmax((r - c.c0) * c.c1, 0.0);
  const int k = min((int)x, (int)c.c2);
  const double t = x - (double)k;
  const double4 s = ld_d4(tab + (int64_t)c.c3 + k);
  v = s.x + t * s.z;
  return (s.y + t * s.w) / r;
}

// Gaussian V = eps e^(-r^2 / 2 sigma^2), Morse V = D0 (x^2 - 2 x) with
// x = e^(-alpha (r - r0)), Yukawa V = eps e^(-kappa r) / r: the force factor
// fr = -dV/dr / r (f_ij = fr d_ij) at r^2, and V in v.  FP32 (mixed forms).
template <int POT>
__device__ __forceinline__ float pot_fr(const PotCoeffF &c, float r2, float &v) {
  if (POT == kGauss) {
    const float e = __expf(-c.c0 * r2);
    v = c.c2 * e;
    return c.c1 * e;
  } else if (POT == kMorse) {
    const float rinv = rsqrtf(r2), r = r2 * rinv;
    const float x = __expf(-c.c0 * (r - c.c1));
    v = c.c3 * x * (x - 2.f);
    return c.c2 * x * (x - 1.f) * rinv;
  } else {
    const float rinv = rsqrtf(r2), r = r2 * rinv;
    const float e = c.c1 * __expf(-c.c0 * r) * rinv;
    v = e;
    return e * fmaf(c.c0, r, 1.f) * rinv * rinv;
  }
}

// The same in FP64.
template <int POT>
__device__ __forceinline__ double pot_fr(const PotCoeffD &c, double r2, double &v) {
  if (POT == kGauss) {
    const double e = exp(-c.c0 * r2);
    v = c.c2 * e;
    return c.c1 * e;
  } else if (POT == kMorse) {
    const double r = sqrt(r2);
    const double x = exp(-c.c0 * (r - c.c1));
    v = c.c3 * x * (x - 2.0);
    return c.c2 * x * (x - 1.0) / r;
  } else {
    const double r = sqrt(r2);
    const double e = c.c1 * exp(-c.c0 * r) / r;
    v = e;
    return e * (1.0 + c.c0 * r) / r2;
  }
}

// Force on home particle i from the neighbour of entry e (mixed path).  Adds
// to the group sums (gx, gy, gz) and, with ENERGY, to the energy and virial
// Kahan sums.  Nothing happens beyond the cut-off.
template <int POT, bool ENERGY, bool ONE, bool DIRECT>
struct MixedPair {
  const KArgs &a;
  const Rep &rp;
  const StageSrc<DIRECT> &src;
  float4 oi, vi4;
  int ti;
  bool ident;
  int32_t i, tag_i;
  uint64_t step;
  float rc2_lo, rc2_hi, inv_rc;
  LJCoeffF lj0;
  DPDCoeffF dp0;
  PotCoeffF pc0;
  __device__ __forceinline__ void operator()(uint32_t e, float &gx, float &gy, float &gz, KSum &kpe,
                                             KSum *kw) const {
    const float4 oj = src.pos(e);
    const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (!(r2 < rc2_hi)) return;
    if (r2 >= rc2_lo) {
      double d[3];
      if (exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + src.index(e, ident)), rp, d) >= a.rc2) return;
    }
    const int cidx = ti * a.ntypes + cell_type(__float_as_uint(oj.w));
    float fr, v = 0.f;
    if (POT == kLJ) {
      const LJCoeffF c = ONE ? lj0 : reinterpret_cast<const LJCoeffF *>(a.coeff)[cidx];
      const float r2i = rcp_approx(r2);
      const float r6 = r2i * r2i * r2i;
      fr = r2i * r6 * (c.lj1 * r6 - c.lj2);
      if (ENERGY) v = r6 * (c.lj3 * r6 - c.lj4) - c.vshift;
    } else if (POT == kTable) {
      const PotCoeffF c = ONE ? pc0 : reinterpret_cast<const PotCoeffF *>(a.coeff)[cidx];
      float vv;
      fr = table_fr(c, reinterpret_cast<const float4 *>(a.table), r2, vv);
      if (ENERGY) v = vv;
    } else if (POT != kDPD) {
      const PotCoeffF c = ONE ? pc0 : reinterpret_cast<const PotCoeffF *>(a.coeff)[cidx];
      float vv;
      fr = pot_fr<POT>(c, r2, vv);
      if (ENERGY) v = vv - c.vshift;
    } else {
      const DPDCoeffF c = ONE ? dp0 : reinterpret_cast<const DPDCoeffF *>(a.coeff)[cidx];
      const float4 vj = src.vel(e);
      const float rinv = rsqrtf(r2);
      const float rr = r2 * rinv;
      const float w = 1.f - rr * inv_rc;
      const float dot = dx * (vi4.x - vj.x) + dy * (vi4.y - vj.y) + dz * (vi4.z - vj.z);
      const uint32_t word = dpd_word(tag_i, __float_as_int(vj.w), step, a.seed);
      const float uu = unit_uniform(word);
      const float theta = 1.7320508075688772f * (2.f * uu - 1.f);
      const float fmag = c.A * w - c.gamma * w * w * dot * rinv + c.sigma_rdt * w * theta;
      fr = fmag * rinv;
      if (ENERGY) v = 0.5f * c.A * (float)a.r_cut * w * w;
    }
    const float fx = fr * dx, fy = fr * dy, fz = fr * dz;
    gx += fx; gy += fy; gz += fz;
    if (ENERGY) {
      kpe.add(0.5f * v);
      kw[0].add(0.5f * dx * fx); kw[1].add(0.5f * dx * fy); kw[2].add(0.5f * dx * fz);
      kw[3].add(0.5f * dy * fy); kw[4].add(0.5f * dy * fz); kw[5].add(0.5f * dz * fz);
    }
  }
};

// Half lists, Newton's third law: -f_ij on the partner j, and the other half
// of the pair's energy and virial (d and f both change sign).  Out of line,
// so that full-list kernels keep their own instruction schedule.
template <bool ENERGY>
static __device__ __noinline__ void partner_add(double *force, double *virial, int32_t j, double fx,
                                                double fy, double fz, double v, double dx, double dy,
                                                double dz) {
  double *fj = force + 4 * (int64_t)j;
  atomicAdd(fj + 0, -fx);
  atomicAdd(fj + 1, -fy);
  atomicAdd(fj + 2, -fz);
  if (ENERGY) {
    atomicAdd(fj + 3, 0.5 * v);
    double *wj = virial + 6 * (int64_t)j;
    atomicAdd(wj + 0, 0.5 * dx * fx); atomicAdd(wj + 1, 0.5 * dx * fy);
    atomicAdd(wj + 2, 0.5 * dx * fz); atomicAdd(wj + 3, 0.5 * dy * fy);
    atomicAdd(wj + 4, 0.5 * dy * fz); atomicAdd(wj + 5, 0.5 * dz * fz);
  }
}

// Force on home particle i from the neighbour of entry e (FP64 path).
template <int POT, bool ENERGY, bool ONE, bool DIRECT>
struct DoublePair {
  const KArgs &a;
  const Rep &rp;
  const StageSrc<DIRECT> &src;
  float4 oi;
  double4 pi, vi;
  int ti;
  bool ident;
  int32_t tag_i;
  uint64_t step;
  float rc2_hi;
  LJCoeffD lj0;
  DPDCoeffD dp0;
  PotCoeffD pd0;
  bool half;  // half list: the partner receives -f_ij here
  __device__ __forceinline__ void operator()(uint32_t e, double *df, double &dpe, double *dw) const {
    const float4 oj = src.pos(e);
    const float fx32 = oi.x - oj.x, fy32 = oi.y - oj.y, fz32 = oi.z - oj.z;
    const float r2f = fmaf(fz32, fz32, fmaf(fy32, fy32, fx32 * fx32));
    if (!(r2f < rc2_hi)) return;  // FP32 screen: certainly beyond r_cut (or the sentinel)
    const int32_t j = src.index(e, ident);
    double d[3];
    const double r2d = exact_r2(pi, ld_d4(a.pos + j), rp, d);
    if (r2d >= a.rc2) return;
    const int cidx = ti * a.ntypes + cell_type(__float_as_uint(oj.w));
    double fr, v = 0.;
    if (POT == kLJ) {
      const LJCoeffD c = ONE ? lj0 : reinterpret_cast<const LJCoeffD *>(a.coeff)[cidx];
      const double r2i = __drcp_rn(r2d);
      const double r6 = r2i * r2i * r2i;
      fr = r2i * r6 * (c.lj1 * r6 - c.lj2);
      if (ENERGY) v = r6 * (c.lj3 * r6 - c.lj4) - c.vshift;
    } else if (POT == kTable) {
      const PotCoeffD c = ONE ? pd0 : reinterpret_cast<const PotCoeffD *>(a.coeff)[cidx];
      double vv;
      fr = table_fr(c, reinterpret_cast<const double4 *>(a.table), r2d, vv);
      if (ENERGY) v = vv;
    } else if (POT != kDPD) {
      const PotCoeffD c = ONE ? pd0 : reinterpret_cast<const PotCoeffD *>(a.coeff)[cidx];
      double vv;
      fr = pot_fr<POT>(c, r2d, vv);
      if (ENERGY) v = vv - c.vshift;
    } else {
      const DPDCoeffD c = ONE ? dp0 : reinterpret_cast<const DPDCoeffD *>(a.coeff)[cidx];
      const double4 vj = ld_d4(a.vel + j);
      const double rr = sqrt(r2d);
      const double rinv = 1.0 / rr;
      const double w = 1.0 - rr / a.r_cut;
      const double dot = d[0] * (vi.x - vj.x) + d[1] * (vi.y - vj.y) + d[2] * (vi.z - vj.z);
      const uint32_t word = dpd_word(tag_i, a.tag[j], step, a.seed);
      const double uu = ((double)word + 0.5) * 2.3283064365386963e-10;  // 2^-32
      const double theta = 1.7320508075688772 * (2.0 * uu - 1.0);
      const double fmag = c.A * w - c.gamma * w * w * dot * rinv + c.sigma_rdt * w * theta;
      fr = fmag * rinv;
      if (ENERGY) v = 0.5 * c.A * a.r_cut * w * w;
    }
    const double fx = fr * d[0], fy = fr * d[1], fz = fr * d[2];
    df[0] += fx; df[1] += fy; df[2] += fz;
    if (ENERGY) {
      dpe += 0.5 * v;
      dw[0] += 0.5 * d[0] * fx; dw[1] += 0.5 * d[0] * fy; dw[2] += 0.5 * d[0] * fz;
      dw[3] += 0.5 * d[1] * fy; dw[4] += 0.5 * d[1] * fz; dw[5] += 0.5 * d[2] * fz;
    }
    if (half)
      partner_add<ENERGY>(reinterpret_cast<double *>(a.force), reinterpret_cast<double *>(a.virial), j,
                          fx, fy, fz, v, d[0], d[1], d[2]);
  }
};

// V consecutive 16-bit row entries of one lane, loaded with one instruction.
template <int V> struct RowWord;
template <> struct RowWord<4> {
  using T = uint2;
  static __device__ __forceinline__ T load(const uint16_t *p) {
    return __ldcs(reinterpret_cast<const uint2 *>(p));
  }
  static __device__ __forceinline__ T zero() { return make_uint2(0u, 0u); }
  static __device__ __forceinline__ uint32_t get(const T &w, int v) {
    const uint32_t x = v < 2 ? w.x : w.y;
    return (v & 1) ? x >> 16 : x & 0xffffu;
  }
};
template <> struct RowWord<2> {
  using T = uint32_t;
  static __device__ __forceinline__ T load(const uint16_t *p) {
    return __ldcs(reinterpret_cast<const unsigned int *>(p));
  }
  static __device__ __forceinline__ T zero() { return 0u; }
  static __device__ __forceinline__ uint32_t get(const T &w, int v) {
    return (v & 1) ? w >> 16 : w & 0xffffu;
  }
};
template <> struct RowWord<1> {
  using T = uint32_t;
  static __device__ __forceinline__ T load(const uint16_t *p) {
    return (uint32_t)__ldcs(reinterpret_cast<const unsigned short *>(p));
  }
  static __device__ __forceinline__ T zero() { return 0u; }
  static __device__ __forceinline__ uint32_t get(const T &w, int) { return w; }
};

// One row group (P = 32 / W particles of the brick, W lanes each) on one
// warp.  Each lane walks its particle's row in blocks of V entries (one load
// per block, two blocks loaded ahead); a group's rows are padded to whole
// blocks, so every block is processed by the same code.  The mixed forms are
// branch-free: every entry is evaluated (the sentinel's r^2 is +inf) and
// masked by r^2 < r_cut^2; entries whose FP32 r^2 lies in the error band
// around r_cut^2 are settled in FP64 after each pair of blocks.  FULLG: the
// group has all P particles (a block is 32 V entries).
template <int POT, int W, bool MIXED, bool ENERGY, bool ONE, bool DIRECT, bool FULLG>
__device__ __forceinline__ void pair_group(const KArgs &a, const BrickDesc &d, const float4 *spos,
                                           const float4 *svel, int j, uint64_t step) {
  constexpr int P = 32 / W;
  constexpr int V = row_depth(W);
  using RW = RowWord<V>;
  using Word = typename RW::T;
  const int lane = threadIdx.x & 31;
  const int qq = lane / W, sl = lane & (W - 1);
  const int q = j * P + qq;
  const bool active = q < d.nhome;
  const int pj = FULLG ? P : min(P, d.nhome - j * P);
  const int qe = active ? qq : 0;  // idle lanes shadow the group's first particle
  const Rep &rp = a.rep[d.r];
  const bool ident = a.ident[d.r] != 0;
  const HomeSlot hs = home_slot(d, j * P + qe);
  const int p = hs.p;
  const int32_t i = ident ? p : __ldg(a.cell_idx + p);
  const StageSrc<DIRECT> src{a, d, rp, smem_u32(spos), smem_u32(svel)};
  // the home particle's stage coordinates, read once (a volatile load: the
  // compiler keeps the value instead of re-reading it inside the loop)
  const float4 oi = DIRECT ? src.pos((uint32_t)(hs.slot + 1))
                           : lds4(smem_u32(spos) + 16u * (uint32_t)(hs.slot + 1));
  const int pg = d.hstart + j * P;
  const int NB = __ldg(a.nl_tiles + pg) / V;        // blocks of V tiles
  const int bstride = (FULLG ? 32 : pj * W) * V;    // entries per block
  const uint16_t *row = a.nl + (size_t)pg * (size_t)a.max_nb + (qe * W + sl) * V;
  auto ldrow = [&](int b) { return b < NB ? RW::load(row + (size_t)b * bstride) : RW::zero(); };

  KSum kf[3], kpe, kw[6];
  double df[3] = {0., 0., 0.}, dpe = 0., dw[6] = {0., 0., 0., 0., 0., 0.};
  MixedPair<POT, ENERGY, ONE, DIRECT> mp{a, rp, src};
  DoublePair<POT, ENERGY, ONE, DIRECT> dp{a, rp, src};
  if (MIXED) {
    mp.oi = oi;
    mp.ti = cell_type(__float_as_uint(oi.w));
    mp.ident = ident;
    mp.i = i;
    mp.step = step;
    mp.rc2_lo = a.rc2f - rp.band;
    mp.rc2_hi = a.rc2f + rp.band;
    mp.inv_rc = (float)(1.0 / a.r_cut);
    if (ONE) {
      if (POT == kLJ) mp.lj0 = a.lj1f;
      else if (POT == kDPD) mp.dp0 = a.dpd1f;
      else mp.pc0 = a.pot1f;
    }
    if (POT == kDPD) {
      mp.vi4 = src.vel((uint32_t)(hs.slot + 1));
      mp.tag_i = __float_as_int(mp.vi4.w);
    }
  } else {
    dp.oi = oi;
    // idle lanes of a short group shadow its first particle's row: only the
    // lanes of real particles may add to partners
    dp.half = a.half != 0 && active;
    dp.ti = cell_type(__float_as_uint(oi.w));
    dp.ident = ident;
    dp.pi = ld_d4(a.pos + i);
    dp.step = step;
    dp.rc2_hi = a.rc2f + rp.band;
    if (ONE) {
      if (POT == kLJ) dp.lj0 = reinterpret_cast<const LJCoeffD *>(a.coeff)[0];
      else if (POT == kDPD) dp.dp0 = reinterpret_cast<const DPDCoeffD *>(a.coeff)[0];
      else dp.pd0 = reinterpret_cast<const PotCoeffD *>(a.coeff)[0];
    }
    if (POT == kDPD) {
      dp.vi = ld_d4(a.vel + i);
      dp.tag_i = a.tag[i];
    }
  }

  // an entry with r^2 in the band [lo, hi) sends its pair of blocks through
  // the FP64 re-test.  The band's ends are rounded FP32 numbers; bthr is the
  // larger of their exact distances from r_cut^2 (differences of nearby FP32
  // numbers are exact), and |r^2 - r_cut^2| <= bthr holds for every r^2 in
  // [lo, hi), so no band entry escapes the re-test.
  const uint64_t oixy = pack2(oi.x, oi.y);
  const float rc2f = a.rc2f;
  const float lo = mp.rc2_lo;
  const float bthr = fmaxf(rc2f - lo, mp.rc2_hi - rc2f);

  // FP32 separation of the home particle from the neighbour of entry e
  auto sep = [&](uint32_t e, float &dx, float &dy, float &dz, float &ojw) {
    if (DIRECT) {
      const float4 oj = src.pos(e);
      dx = oi.x - oj.x;
      dy = oi.y - oj.y;
      dz = oi.z - oj.z;
      ojw = oj.w;
    } else {
      const float4 oj = spos[e];
      const float2 dxy = unpack2(sub_f32x2(oixy, pack2(oj.x, oj.y)));
      dx = dxy.x;
      dy = dxy.y;
      dz = oi.z - oj.z;
      ojw = oj.w;
    }
  };

  // Everything the hot loop reads is a plain local here: a field read
  // through a reference member of a helper struct (mp.a, src.a) would be a
  // memory load from the parameter buffer inside the loop.
  const LJCoeffF lj = a.lj1f;
  const DPDCoeffF dc = a.dpd1f;
  const PotCoeffF pc = a.pot1f;
  const float4 *table = reinterpret_cast<const float4 *>(a.table);
  const int ntypes = a.ntypes, ti = cell_type(__float_as_uint(oi.w));
  const void *coeff = a.coeff;
  const float inv_rc = (float)(1.0 / a.r_cut), r_cut_f = (float)a.r_cut;
  const uint64_t seed = a.seed;
  const float4 vi4 = MIXED && POT == kDPD ? mp.vi4 : make_float4(0.f, 0.f, 0.f, 0.f);
  const int32_t tag_i = MIXED && POT == kDPD ? mp.tag_i : 0;

  // the V entries of one block, mixed precision: group sums (gx, gy, gz),
  // smallest |r^2 - r_cut^2| in bmin
  auto mixed_block = [&](const Word &w, float &gx, float &gy, float &gz, float &bmin) {
#pragma unroll
    for (int v = 0; v < V; v++) {
      const uint32_t e = RW::get(w, v);
      float dx, dy, dz, ojw;
      sep(e, dx, dy, dz, ojw);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const bool in = r2 < lo;
      bmin = fminf(bmin, fabsf(r2 - rc2f));
      float fr, en = 0.f;
      if (POT == kLJ) {
        const LJCoeffF c = ONE ? lj
                               : reinterpret_cast<const LJCoeffF *>(coeff)[
                                     ti * ntypes + cell_type(__float_as_uint(ojw))];
        const float r2i = rcp_approx(r2);
        const float r6 = r2i * r2i * r2i;
        fr = in ? r2i * r6 * (c.lj1 * r6 - c.lj2) : 0.f;
        if (ENERGY) en = in ? r6 * (c.lj3 * r6 - c.lj4) - c.vshift : 0.f;
      } else if (POT != kDPD) {
        const PotCoeffF c = ONE ? pc
                                : reinterpret_cast<const PotCoeffF *>(coeff)[
                                      ti * ntypes + cell_type(__float_as_uint(ojw))];
        float vv;
        const float f = POT == kTable ? table_fr(c, table, r2, vv) : pot_fr<POT>(c, r2, vv);
        fr = in ? f : 0.f;
        if (ENERGY) en = in ? vv - c.vshift : 0.f;
      } else {
        const DPDCoeffF c = ONE ? dc
                                : reinterpret_cast<const DPDCoeffF *>(coeff)[
                                      ti * ntypes + cell_type(__float_as_uint(ojw))];
        const float4 vj = DIRECT ? src.vel(e) : reinterpret_cast<const float4 *>(svel)[e];
        const float rinv = rsqrtf(r2);
        const float wgt = fmaf(-r2 * rinv, inv_rc, 1.f);
        const float dot = dx * (vi4.x - vj.x) + dy * (vi4.y - vj.y) + dz * (vi4.z - vj.z);
        const uint32_t word = dpd_word(tag_i, __float_as_int(vj.w), step, seed);
        const float uu = unit_uniform(word);
        const float theta = 1.7320508075688772f * (2.f * uu - 1.f);
        const float fmag = c.A * wgt - c.gamma * wgt * wgt * dot * rinv + c.sigma_rdt * wgt * theta;
        fr = in ? fmag * rinv : 0.f;
        if (ENERGY) en = in ? 0.5f * c.A * r_cut_f * wgt * wgt : 0.f;
      }
      gx = fmaf(fr, dx, gx);
      gy = fmaf(fr, dy, gy);
      gz = fmaf(fr, dz, gz);
      if (ENERGY) {
        const float fx = fr * dx, fy = fr * dy, fz = fr * dz;
        kpe.add(0.5f * en);
        kw[0].add(0.5f * dx * fx); kw[1].add(0.5f * dx * fy); kw[2].add(0.5f * dx * fz);
        kw[3].add(0.5f * dy * fy); kw[4].add(0.5f * dy * fz); kw[5].add(0.5f * dz * fz);
      }
    }
  };
  // the block's entries inside the FP32 band: decided in FP64 (rare)
  auto band_block = [&](const Word &w, float &gx, float &gy, float &gz) {
#pragma unroll
    for (int v = 0; v < V; v++) {
      const uint32_t e = RW::get(w, v);
      float dx, dy, dz, ojw;
      sep(e, dx, dy, dz, ojw);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      if (r2 >= mp.rc2_lo && r2 < mp.rc2_hi) mp(e, gx, gy, gz, kpe, kw);
    }
  };
  auto fp64_block = [&](const Word &w) {
#pragma unroll
    for (int v = 0; v < V; v++) {
      const uint32_t e = RW::get(w, v);
      if (e != 0u) dp(e, df, dpe, dw);  // 0: padding
    }
  };

  // two blocks (a Kahan flush and at most one FP64 band pass) per step
  auto two_blocks = [&](const Word &w0, const Word &w1, bool two) {
    if (MIXED) {
      float gx = 0.f, gy = 0.f, gz = 0.f, bmin = 3.0e38f;
      mixed_block(w0, gx, gy, gz, bmin);
      if (two) mixed_block(w1, gx, gy, gz, bmin);
      if (__any_sync(FULL, bmin <= bthr)) {
        band_block(w0, gx, gy, gz);
        if (two) band_block(w1, gx, gy, gz);
      }
      kf[0].add(gx);
      kf[1].add(gy);
      kf[2].add(gz);
    } else {
      fp64_block(w0);
      if (two) fp64_block(w1);
    }
  };
  // four blocks in flight per lane: the row stream is latency-bound, so the
  // bytes a warp keeps in flight set its speed (the next brick's rows are
  // also being prefetched into L2)
  Word q0 = ldrow(0), q1 = ldrow(1), q2 = ldrow(2), q3 = ldrow(3);
  for (int b = 0; b < NB; b += 4) {  // NB is warp-uniform: so are all branches here
    {
      const Word w0 = q0, w1 = q1;
      q0 = ldrow(b + 4);
      q1 = ldrow(b + 5);
      two_blocks(w0, w1, b + 1 < NB);
    }
    if (b + 2 < NB) {
      const Word w0 = q2, w1 = q3;
      q2 = ldrow(b + 6);
      q3 = ldrow(b + 7);
      two_blocks(w0, w1, b + 3 < NB);
    }
  }

  // combine the W partial sums of each particle (intra-warp reduction)
  if (MIXED) {
#pragma unroll
    for (int c = 0; c < 3; c++) seg_merge<W>(kf[c]);
    if (ENERGY) {
      seg_merge<W>(kpe);
#pragma unroll
      for (int c = 0; c < 6; c++) seg_merge<W>(kw[c]);
    }
    if (active && sl == 0) {
      float4 *f = reinterpret_cast<float4 *>(a.force);
      f[i] = make_float4(kf[0].value(), kf[1].value(), kf[2].value(), ENERGY ? kpe.value() : 0.f);
      if (ENERGY) {
        float *vv = reinterpret_cast<float *>(a.virial) + 6 * (int64_t)i;
#pragma unroll
        for (int c = 0; c < 6; c++) vv[c] = kw[c].value();
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; c++) df[c] = seg_sum<W>(df[c]);
    if (ENERGY) {
      dpe = seg_sum<W>(dpe);
#pragma unroll
      for (int c = 0; c < 6; c++) dw[c] = seg_sum<W>(dw[c]);
    }
    if (active && sl == 0 && a.half) {
      // half list: partners add into this particle concurrently
      double *f = reinterpret_cast<double *>(a.force) + 4 * (int64_t)i;
      atomicAdd(f + 0, df[0]);
      atomicAdd(f + 1, df[1]);
      atomicAdd(f + 2, df[2]);
      if (ENERGY) {
        atomicAdd(f + 3, dpe);
        double *vv = reinterpret_cast<double *>(a.virial) + 6 * (int64_t)i;
#pragma unroll
        for (int c = 0; c < 6; c++) atomicAdd(vv + c, dw[c]);
      }
    } else if (active && sl == 0) {
      double2 *f = reinterpret_cast<double2 *>(reinterpret_cast<double4 *>(a.force) + i);
      f[0] = make_double2(df[0], df[1]);
      f[1] = make_double2(df[2], ENERGY ? dpe : 0.);
      if (ENERGY) {
        double *vv = reinterpret_cast<double *>(a.virial) + 6 * (int64_t)i;
#pragma unroll
        for (int c = 0; c < 6; c++) vv[c] = dw[c];
      }
    }
  }
}

// Persistent over bricks b = blockIdx + t G.  Warp w takes the brick's row
// groups w, w + C, ...; the next brick's stage copies run meanwhile.  One
// block barrier per brick.
template <int POT, int W, bool MIXED, bool ENERGY, bool ONE>
__global__ void __launch_bounds__(kMaxBrickThreads) k_pair(KArgs a, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int P = 32 / W;
  constexpr bool VEL = POT == kDPD && MIXED;
  const BrickSmem M{smem, cap, VEL};
  const int warp = threadIdx.x >> 5, C = blockDim.x >> 5;
  const long long G = gridDim.x, b0 = blockIdx.x;
  const uint64_t step = (uint64_t)a.ds->step;
  if (b0 >= a.n_bricks) return;
  if (fatal_error(a)) return;
  // Rows name slots of the binning they were built from: a replica binned
  // again since its last list build (a build skipped after an error, or a
  // binning through the API without a build) has rows that do not match the
  // current stages, and reading them could run past a stage.  Refuse.
  int stale = 0;
  for (int r = threadIdx.x; r < a.R; r += blockDim.x) stale |= __ldcg(a.list_ok + r) == 0;
  if (__syncthreads_or(stale)) {
    if (threadIdx.x == 0) set_error(a.ds, kErrStaleList);
    return;
  }
  if (threadIdx.x < 2) {
    M.pos(threadIdx.x)[0] = make_float4(kFar, kFar, kFar, 0.f);
    if (VEL) M.vel4(threadIdx.x)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (threadIdx.x == 0) {
    mbar_init(M.bar(0), 1);
    mbar_init(M.bar(1), 1);
  }
  desc_fetch(a, b0, M.desc(0));
  if (b0 + G < a.n_bricks) desc_fetch(a, b0 + G, M.desc(1));
  fence_proxy_async();
  __syncthreads();
  stage_issue(a, M.desc(0), M.pos(0), VEL ? M.vel4(0) : nullptr, M.bar(0), cap);
  bool ok = stage_wait(a, M, 0);
  stage_shift_all(a, M.desc(0), M.pos(0), cap);
  if (!__syncthreads_and(ok)) {
    stage_drain(M, 0);
    return;
  }
  constexpr int kDescWords = (int)(sizeof(BrickDesc) / 16);
  for (long long t = 0;; t++) {
    const long long bt = b0 + t * G;
    if (bt >= a.n_bricks) break;
    const bool has1 = bt + G < a.n_bricks, has2 = bt + 2 * G < a.n_bricks;
    if (has1) {
      stage_issue(a, M.desc(t + 1), M.pos(t + 1), VEL ? M.vel4(t + 1) : nullptr, M.bar(t + 1), cap);
      // the next brick's rows into L2 while this brick is computed: per row
      // group, the tiles its list build wrote (a group's tiles are one
      // contiguous run from its base; 16-byte multiples, 64-byte aligned)
      const int lane0 = blockDim.x > 32 ? 32 : 0;
      if ((int)threadIdx.x >= lane0 && (int)threadIdx.x < lane0 + 32) {
        const BrickDesc &dn = M.desc(t + 1);
        const int gn = (dn.nhome + P - 1) / P;
        for (int g = (int)threadIdx.x - lane0; g < gn; g += 32) {
          const int pg = dn.hstart + g * P;
          const uint32_t bytes = (uint32_t)__ldg(a.nl_tiles + pg) *
                                 (uint32_t)(min(P, dn.nhome - g * P) * W) * 2u;
          if (bytes > 0u) prefetch_l2(a.nl + (size_t)pg * (size_t)a.max_nb, (bytes + 15u) & ~15u);
        }
      }
    }
    // the descriptor two bricks ahead: loaded now, stored after the work
    // (40 words; a block has at least 32 threads, so two per thread)
    uint4 dv0 = make_uint4(0u, 0u, 0u, 0u), dv1 = dv0;
    const int k0 = threadIdx.x, k1 = threadIdx.x + blockDim.x;
    if (has2) {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.brick_desc + bt + 2 * G);
      if (k0 < kDescWords) dv0 = __ldg(src + k0);
      if (k1 < kDescWords) dv1 = __ldg(src + k1);
    }
    const BrickDesc &d = M.desc(t);
    const int ng = (d.nhome + P - 1) / P;
    if (d.off[64] > cap) {
      for (int j = warp; j < ng; j += C)
        pair_group<POT, W, MIXED, ENERGY, ONE, true, false>(a, d, M.pos(t), M.vel4(t), j, step);
    } else {
      for (int j = warp; j < ng; j += C) {
        if ((j + 1) * P <= d.nhome)
          pair_group<POT, W, MIXED, ENERGY, ONE, false, true>(a, d, M.pos(t), M.vel4(t), j, step);
        else
          pair_group<POT, W, MIXED, ENERGY, ONE, false, false>(a, d, M.pos(t), M.vel4(t), j, step);
      }
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
  }
}

template <int POT, int W, bool MIXED, bool ENERGY, bool ONE>
cudaError_t go1(const KArgs &a, int block, cudaStream_t st) {
  constexpr bool VEL = POT == kDPD && MIXED;
  const size_t smem = BrickSmem::bytes(a.stage_cap, VEL, 0);
  const auto kern = k_pair<POT, W, MIXED, ENERGY, ONE>;
  const int grid = persistent_grid((const void *)kern, block, smem, a.n_bricks);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  kern<<<grid, block, smem, st>>>(a, a.stage_cap);
  return cudaGetLastError();
}

template <int POT, int W, bool MIXED, bool ENERGY>
cudaError_t go(const KArgs &a, int block, cudaStream_t st) {
  if (a.ntypes == 1) return go1<POT, W, MIXED, ENERGY, true>(a, block, st);
  return go1<POT, W, MIXED, ENERGY, false>(a, block, st);
}

template <int POT, bool MIXED, bool ENERGY>
cudaError_t go_w(const KArgs &a, Launch l, cudaStream_t st) {
  switch (l.w) {
    case 1: return go<POT, 1, MIXED, ENERGY>(a, l.block, st);
    case 2: return go<POT, 2, MIXED, ENERGY>(a, l.block, st);
    case 4: return go<POT, 4, MIXED, ENERGY>(a, l.block, st);
    case 8: return go<POT, 8, MIXED, ENERGY>(a, l.block, st);
    case 16: return go<POT, 16, MIXED, ENERGY>(a, l.block, st);
    case 32: return go<POT, 32, MIXED, ENERGY>(a, l.block, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int POT, int W, bool MIXED, bool ENERGY>
int maxb_w() {
  cudaFuncAttributes a1, a2;
  if (cudaFuncGetAttributes(&a1, k_pair<POT, W, MIXED, ENERGY, true>) != cudaSuccess) return 0;
  if (cudaFuncGetAttributes(&a2, k_pair<POT, W, MIXED, ENERGY, false>) != cudaSuccess) return 0;
  return std::min(a1.maxThreadsPerBlock, a2.maxThreadsPerBlock);
}

template <int POT, bool MIXED, bool ENERGY>
int maxb(int w) {
  switch (w) {
    case 1: return maxb_w<POT, 1, MIXED, ENERGY>();
    case 2: return maxb_w<POT, 2, MIXED, ENERGY>();
    case 4: return maxb_w<POT, 4, MIXED, ENERGY>();
    case 8: return maxb_w<POT, 8, MIXED, ENERGY>();
    case 16: return maxb_w<POT, 16, MIXED, ENERGY>();
    case 32: return maxb_w<POT, 32, MIXED, ENERGY>();
  }
  return 0;
}

template <int POT, int W, bool MIXED, bool ENERGY>
void allow_w() {
  cudaFuncSetAttribute(k_pair<POT, W, MIXED, ENERGY, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_pair<POT, W, MIXED, ENERGY, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <int POT, bool MIXED, bool ENERGY>
void allow_all_w() {
  allow_w<POT, 1, MIXED, ENERGY>(); allow_w<POT, 2, MIXED, ENERGY>();
  allow_w<POT, 4, MIXED, ENERGY>(); allow_w<POT, 8, MIXED, ENERGY>();
  allow_w<POT, 16, MIXED, ENERGY>(); allow_w<POT, 32, MIXED, ENERGY>();
}

}  // namespace

// Entry points of one (potential, precision) form; each form is compiled in
// its own translation unit (k_pair_<form>.cu) to keep builds parallel.
template <int POT, bool MIXED>
cudaError_t launch_pair_form(const KArgs &a, Launch l, int want_virial, cudaStream_t st) {
  return want_virial ? go_w<POT, MIXED, true>(a, l, st) : go_w<POT, MIXED, false>(a, l, st);
}

template <int POT, bool MIXED>
int max_block_pair_form(int w, int want_virial) {
  return want_virial ? maxb<POT, MIXED, true>(w) : maxb<POT, MIXED, false>(w);
}

template <int POT, bool MIXED>
void pair_form_attributes() {
  allow_all_w<POT, MIXED, false>();
  allow_all_w<POT, MIXED, true>();
}

#define MDGB_PAIR_FORM(POT, MIXED)                                                         \
  template cudaError_t launch_pair_form<POT, MIXED>(const KArgs &, Launch, int, cudaStream_t); \
  template int max_block_pair_form<POT, MIXED>(int, int);                                  \
  template void pair_form_attributes<POT, MIXED>();

}  // namespace mdgb
