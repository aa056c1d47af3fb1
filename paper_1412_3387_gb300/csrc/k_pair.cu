// Pair forces from the neighbour list (Sec. 5.1: W threads per particle stride
// over its row; the W partial forces are combined with warp shuffles).
//
// One thread block serves one home cell: it stages the 27 surrounding cells
// (see md_internal.cuh, "cell stage"; positions pre-shifted by their periodic
// image), then each segment of W lanes takes one home particle and walks its
// row of 16-bit stage slots, so every neighbour position comes from shared
// memory and every separation is a single FP32 subtraction per component.
//
// Potentials: LJ 12-6 (Sec. 3; benchmarks of Sec. 6, 8.3) and DPD in the
// Groot-Warren form with a Philox-4x32-10 pair noise keyed on the global IDs
// (Sec. 9: per-pair generators seeded with global particle IDs).
//
// Precision forms:
//   FP64  -- FP64 distance (fixed-order minimum image) and FP64 force math.
//   mixed -- FP32 separations and force math; each lane sums the forces of a
//            group of U row entries plainly and adds the group sum to
//            Kahan-compensated FP32 per-particle sums, which are merged across
//            the W lanes with error-free two-sums.
// In both forms the cut-off decision r^2 < r_cut^2 is the FP64 one: an FP32
// r^2 inside a proven error band around r_cut^2 is re-tested in FP64.
#include <algorithm>

#include "md_internal.cuh"

namespace mdgb {

namespace {

constexpr int kLJ = 0, kDPD = 1;

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
    float s2 = __shfl_xor_sync(0xffffffffu, k.s, m);
    float c2 = __shfl_xor_sync(0xffffffffu, k.c, m);
    k.merge(s2, c2);
  }
}

template <int W>
__device__ __forceinline__ double seg_sum(double v) {
#pragma unroll
  for (int m = W / 2; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Force on home particle i from the neighbour in stage slot sj (mixed path).
// Adds to the group sums (gx, gy, gz) and, with ENERGY, to the energy and
// virial Kahan sums.  Returns nothing when the pair is beyond the cut-off.
template <int POT, bool ENERGY, bool ONE>
struct MixedPair {
  const KArgs &a;
  const Rep &rp;
  float4 oi, vi4;
  int ti;
  int32_t i, tag_i;
  uint64_t step;
  float rc2_lo, rc2_hi, inv_rc;
  LJCoeffF lj0;
  DPDCoeffF dp0;
  const float4 *spos, *svel;
  const int32_t *sidx;
  __device__ __forceinline__ void operator()(int sj, float &gx, float &gy, float &gz, KSum &kpe,
                                             KSum *kw) const {
    const float4 oj = spos[sj];
    const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (r2 >= rc2_hi) return;
    if (r2 > rc2_lo) {
      double d[3];
      if (exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + sidx[sj]), rp, d) >= a.rc2) return;
    }
    const int cidx = ti * a.ntypes + cell_type(__float_as_uint(oj.w));
    float fr, v = 0.f;
    if (POT == kLJ) {
      const LJCoeffF c = ONE ? lj0 : reinterpret_cast<const LJCoeffF *>(a.coeff)[cidx];
      const float r2i = __fdividef(1.0f, r2);
      const float r6 = r2i * r2i * r2i;
      fr = r2i * r6 * (c.lj1 * r6 - c.lj2);
      if (ENERGY) v = r6 * (c.lj3 * r6 - c.lj4) - c.vshift;
    } else {
      const DPDCoeffF c = ONE ? dp0 : reinterpret_cast<const DPDCoeffF *>(a.coeff)[cidx];
      const float4 vj = svel[sj];
      const float rinv = rsqrtf(r2);
      const float rr = r2 * rinv;
      const float w = 1.f - rr * inv_rc;
      const float dot = dx * (vi4.x - vj.x) + dy * (vi4.y - vj.y) + dz * (vi4.z - vj.z);
      const uint32_t word = dpd_word(tag_i, __float_as_int(vj.w), step, a.seed);
      const float uu = ((float)(word >> 8) + 0.5f) * 5.9604644775390625e-08f;  // 2^-24
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

// Force on home particle i from the neighbour in stage slot sj (FP64 path).
template <int POT, bool ENERGY, bool ONE>
struct DoublePair {
  const KArgs &a;
  const Rep &rp;
  float4 oi;
  double4 pi, vi;
  int ti;
  int32_t tag_i;
  uint64_t step;
  float rc2_hi;
  LJCoeffD lj0;
  DPDCoeffD dp0;
  const float4 *spos;
  const int32_t *sidx;
  __device__ __forceinline__ void operator()(int sj, double *df, double &dpe, double *dw) const {
    const float4 oj = spos[sj];
    const float fx32 = oi.x - oj.x, fy32 = oi.y - oj.y, fz32 = oi.z - oj.z;
    const float r2f = fmaf(fz32, fz32, fmaf(fy32, fy32, fx32 * fx32));
    if (r2f >= rc2_hi) return;  // FP32 screen: certainly beyond r_cut
    const int32_t j = sidx[sj];
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
  }
};

template <int POT, int W, bool MIXED, bool ENERGY, bool ONE>
__global__ void k_pair(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int LW = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
  constexpr bool STAGE_VEL = POT == kDPD && MIXED;
  constexpr int U = 8;
  constexpr uint32_t kNone = 0xffffu;
  const int lane = threadIdx.x & 31;
  const int sl = lane & (W - 1), seg = threadIdx.x / W;
  const int segs = blockDim.x / W;
  const int cap = a.stage_cap;
  StageInfo &si = *reinterpret_cast<StageInfo *>(smem);
  float4 *spos = reinterpret_cast<float4 *>(smem + sizeof(StageInfo));
  int32_t *sidx = reinterpret_cast<int32_t *>(spos + cap);
  float4 *svel = reinterpret_cast<float4 *>(sidx + cap);

  const int64_t g = blockIdx.x;  // home cell
  const int cnt = a.cell_count[g];
  if (cnt == 0) return;
  const int r = a.chunk_rep[g / kChunkCells];
  const Rep &rp = a.rep[r];
  const int start = a.cell_start[g];
  stage_info(a, rp, g, si);
  __syncthreads();
  const bool ident = a.ident[r] != 0;
  const int total = si.off[27];
  const bool single = total <= cap;
  if (single) {
    stage_fill(a, si, 0, total, ident, spos, sidx, STAGE_VEL ? svel : nullptr);
    __syncthreads();
  }
  const size_t pitch = ((size_t)a.n_pad) << LW;
  const uint64_t step = (uint64_t)a.ds->step;

  for (int q0 = 0; q0 < cnt; q0 += segs) {
    const int q = q0 + seg;
    const bool active = q < cnt;
    const int p = start + (active ? q : 0);
    const int32_t i = a.cell_idx[p];
    const float4 oi = __ldg(a.pos4f + i);
    const int nn = active ? min(a.n_nb[p], a.max_nb) : 0;
    const int nmine = nn > sl ? (nn - sl + W - 1) / W : 0;  // entries k = t W + sl
    const uint16_t *row = a.nl + ((size_t)p << LW) + sl;
    KSum kf[3], kpe, kw[6];
    double df[3] = {0., 0., 0.}, dpe = 0., dw[6] = {0., 0., 0., 0., 0., 0.};

    MixedPair<POT, ENERGY, ONE> mp{a, rp};
    DoublePair<POT, ENERGY, ONE> dp{a, rp};
    if (MIXED) {
      mp.oi = oi;
      mp.ti = cell_type(__float_as_uint(oi.w));
      mp.i = i;
      mp.step = step;
      mp.rc2_lo = a.rc2f - rp.band;
      mp.rc2_hi = a.rc2f + rp.band;
      mp.inv_rc = (float)(1.0 / a.r_cut);
      mp.spos = spos; mp.svel = svel; mp.sidx = sidx;
      if (ONE) {
        if (POT == kLJ) mp.lj0 = reinterpret_cast<const LJCoeffF *>(a.coeff)[0];
        else mp.dp0 = reinterpret_cast<const DPDCoeffF *>(a.coeff)[0];
      }
      if (POT == kDPD) {
        mp.vi4 = __ldg(a.vel4f + i);
        mp.tag_i = __float_as_int(mp.vi4.w);
      }
    } else {
      dp.oi = oi;
      dp.ti = cell_type(__float_as_uint(oi.w));
      dp.pi = ld_d4(a.pos + i);
      dp.step = step;
      dp.rc2_hi = a.rc2f + rp.band;
      dp.spos = spos; dp.sidx = sidx;
      if (ONE) {
        if (POT == kLJ) dp.lj0 = reinterpret_cast<const LJCoeffD *>(a.coeff)[0];
        else dp.dp0 = reinterpret_cast<const DPDCoeffD *>(a.coeff)[0];
      }
      if (POT == kDPD) {
        dp.vi = ld_d4(a.vel + i);
        dp.tag_i = a.tag[i];
      }
    }

    if (single) {
      // rows are read U entries at a time, one group ahead of use
      const int iters = __reduce_max_sync(FULL, (unsigned)nmine);
      uint32_t ebuf[U];
      const uint16_t *rp_next = row;
#pragma unroll
      for (int u = 0; u < U; u++) {
        ebuf[u] = u < nmine ? (uint32_t)__ldcs(rp_next) : kNone;
        rp_next += pitch;
      }
      for (int t0 = 0; t0 < iters; t0 += U) {
        uint32_t ecur[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          ecur[u] = ebuf[u];
          ebuf[u] = t0 + U + u < nmine ? (uint32_t)__ldcs(rp_next) : kNone;
          rp_next += pitch;
        }
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (MIXED && POT == kLJ) {
          // straight-line LJ: every entry is evaluated and masked; entries in
          // the FP64 tie-break band are settled after the group
          bool band = false;
#pragma unroll
          for (int u = 0; u < U; u++) {
            const bool valid = ecur[u] < (uint32_t)total;
            const float4 oj = spos[valid ? ecur[u] : 0];
            const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const bool in = valid & (r2 < mp.rc2_lo);
            band |= valid & (r2 >= mp.rc2_lo) & (r2 < mp.rc2_hi);
            const LJCoeffF c = ONE ? mp.lj0
                                   : reinterpret_cast<const LJCoeffF *>(a.coeff)[
                                         mp.ti * a.ntypes + cell_type(__float_as_uint(oj.w))];
            const float r2i = __fdividef(1.0f, r2);
            const float r6 = r2i * r2i * r2i;
            const float fr = in ? r2i * r6 * (c.lj1 * r6 - c.lj2) : 0.f;
            gx = fmaf(fr, dx, gx);
            gy = fmaf(fr, dy, gy);
            gz = fmaf(fr, dz, gz);
            if (ENERGY) {
              const float v = in ? r6 * (c.lj3 * r6 - c.lj4) - c.vshift : 0.f;
              const float fx = fr * dx, fy = fr * dy, fz = fr * dz;
              kpe.add(0.5f * v);
              kw[0].add(0.5f * dx * fx); kw[1].add(0.5f * dx * fy); kw[2].add(0.5f * dx * fz);
              kw[3].add(0.5f * dy * fy); kw[4].add(0.5f * dy * fz); kw[5].add(0.5f * dz * fz);
            }
          }
          if (__any_sync(FULL, band)) {
#pragma unroll
            for (int u = 0; u < U; u++) {
              if (ecur[u] >= (uint32_t)total) continue;
              const float4 oj = spos[ecur[u]];
              const float dx = oi.x - oj.x, dy = oi.y - oj.y, dz = oi.z - oj.z;
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              if (r2 >= mp.rc2_lo && r2 < mp.rc2_hi) mp((int)ecur[u], gx, gy, gz, kpe, kw);
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; u++) {
            if (ecur[u] >= (uint32_t)total) continue;  // no entry (or not a slot)
            if (MIXED) mp((int)ecur[u], gx, gy, gz, kpe, kw);
            else dp((int)ecur[u], df, dpe, dw);
          }
        }
        if (MIXED) {
          kf[0].add(gx);
          kf[1].add(gy);
          kf[2].add(gz);
        }
      }
    } else {
      // dense neighbourhood: windows of the stage, rows ascend through them
      int t = 0;
      for (int w0 = 0; w0 < total; w0 += cap) {
        const int mw = min(cap, total - w0);
        __syncthreads();
        stage_fill(a, si, w0, mw, ident, spos, sidx, STAGE_VEL ? svel : nullptr);
        __syncthreads();
        while (t < nmine) {
          const uint32_t v = __ldcs(row + (size_t)t * pitch);
          if (v - (uint32_t)w0 >= (uint32_t)mw) break;  // beyond this window
          t++;
          float gx = 0.f, gy = 0.f, gz = 0.f;
          if (MIXED) {
            mp((int)(v - w0), gx, gy, gz, kpe, kw);
            kf[0].add(gx);
            kf[1].add(gy);
            kf[2].add(gz);
          } else {
            dp((int)(v - w0), df, dpe, dw);
          }
        }
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
      if (active && sl == 0) {
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
}

template <int POT, int W, bool MIXED, bool ENERGY>
cudaError_t go(const KArgs &a, int block, cudaStream_t st) {
  constexpr bool SV = POT == kDPD && MIXED;
  const unsigned grid = (unsigned)a.n_cells;  // one block per home cell
  const size_t smem = stage_bytes(a.stage_cap, SV);
  if (a.ntypes == 1) k_pair<POT, W, MIXED, ENERGY, true><<<grid, block, smem, st>>>(a);
  else k_pair<POT, W, MIXED, ENERGY, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
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
int maxb_w(int cap) {
  constexpr bool SV = POT == kDPD && MIXED;
  cudaFuncAttributes a1, a2;
  if (cudaFuncGetAttributes(&a1, k_pair<POT, W, MIXED, ENERGY, true>) != cudaSuccess) return 0;
  if (cudaFuncGetAttributes(&a2, k_pair<POT, W, MIXED, ENERGY, false>) != cudaSuccess) return 0;
  (void)cap;
  (void)SV;
  return std::min(a1.maxThreadsPerBlock, a2.maxThreadsPerBlock);
}

template <int POT, bool MIXED, bool ENERGY>
int maxb(int w, int cap) {
  switch (w) {
    case 1: return maxb_w<POT, 1, MIXED, ENERGY>(cap);
    case 2: return maxb_w<POT, 2, MIXED, ENERGY>(cap);
    case 4: return maxb_w<POT, 4, MIXED, ENERGY>(cap);
    case 8: return maxb_w<POT, 8, MIXED, ENERGY>(cap);
    case 16: return maxb_w<POT, 16, MIXED, ENERGY>(cap);
    case 32: return maxb_w<POT, 32, MIXED, ENERGY>(cap);
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

void pair_init_attributes() {
  allow_all_w<kLJ, true, false>(); allow_all_w<kLJ, true, true>();
  allow_all_w<kLJ, false, false>(); allow_all_w<kLJ, false, true>();
  allow_all_w<kDPD, true, false>(); allow_all_w<kDPD, true, true>();
  allow_all_w<kDPD, false, false>(); allow_all_w<kDPD, false, true>();
}

cudaError_t launch_pair(const KArgs &a, Launch l, int want_virial, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const bool m = a.mixed != 0;
  if (a.pair == kLJ) {
    if (m) return want_virial ? go_w<kLJ, true, true>(a, l, st) : go_w<kLJ, true, false>(a, l, st);
    return want_virial ? go_w<kLJ, false, true>(a, l, st) : go_w<kLJ, false, false>(a, l, st);
  }
  if (m) return want_virial ? go_w<kDPD, true, true>(a, l, st) : go_w<kDPD, true, false>(a, l, st);
  return want_virial ? go_w<kDPD, false, true>(a, l, st) : go_w<kDPD, false, false>(a, l, st);
}

int max_block_pair(const KArgs &a, int w, int want_virial) {
  const bool m = a.mixed != 0;
  const int cap = a.stage_cap;
  if (a.pair == kLJ) {
    if (m) return want_virial ? maxb<kLJ, true, true>(w, cap) : maxb<kLJ, true, false>(w, cap);
    return want_virial ? maxb<kLJ, false, true>(w, cap) : maxb<kLJ, false, false>(w, cap);
  }
  if (m) return want_virial ? maxb<kDPD, true, true>(w, cap) : maxb<kDPD, true, false>(w, cap);
  return want_virial ? maxb<kDPD, false, true>(w, cap) : maxb<kDPD, false, false>(w, cap);
}

}  // namespace mdgb
