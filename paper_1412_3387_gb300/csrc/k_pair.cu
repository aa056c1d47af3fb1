// Pair forces from the neighbour list (Sec. 5.1: W threads per particle stride
// over its row; the W partial forces are combined with warp shuffles).
//
// Potentials: LJ 12-6 (Sec. 3; benchmarks of Sec. 6, 8.3) and DPD in the
// Groot-Warren form with a Philox-4x32-10 pair noise keyed on the global IDs
// (Sec. 9: per-pair generators seeded with global particle IDs).
//
// Precision forms:
//   FP64  -- FP64 distance (fixed-order minimum image) and FP64 force math.
//   mixed -- separations from FP32 frame-relative offsets plus the FP32 shift
//            of the neighbouring cell named by the entry's code; FP32 force
//            math; each lane sums the forces of a group of U entries plainly
//            and adds the group sum to Kahan-compensated FP32 per-particle
//            sums, which are merged across the W lanes with error-free
//            two-sums.
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

template <int POT, int W, bool MIXED, bool ENERGY, bool ONE>
__global__ void k_pair(KArgs a) {
  extern __shared__ float4 sh_shift[];  // [replicas spanned][27]
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int LW = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : W == 16 ? 4 : 5;
  const int lane = threadIdx.x & 31;
  const int sl = lane & (W - 1);
  const int per_block = blockDim.x / W;
  const int64_t first = (int64_t)blockIdx.x * per_block;
  const int64_t i = first + threadIdx.x / W;
  const bool valid = i < a.n;

  // periodic-image shifts of the 27 neighbouring cells, per replica spanned
  const int r0 = replica_of(a, first);
  const int64_t last = min(first + per_block, a.n) - 1;
  const int r1 = replica_of(a, last);
  for (int t = threadIdx.x; t < (r1 - r0 + 1) * 27; t += blockDim.x) {
    const Rep &rp = a.rep[r0 + t / 27];
    int s = t % 27;
    sh_shift[t] = make_float4((float)(s % 3 - 1) * rp.hf[0], (float)((s / 3) % 3 - 1) * rp.hf[1],
                              (float)(s / 9 - 1) * rp.hf[2], 0.f);
  }
  __syncthreads();

  const int r = valid ? replica_of(a, i) : r0;
  const Rep &rp = a.rep[r];
  const float4 *shift = sh_shift + (r - r0) * 27;
  const float rc2_lo = a.rc2f - rp.band, rc2_hi = a.rc2f + rp.band;
  const float4 oi = valid ? a.pos4f[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int ti = cell_type(__float_as_uint(oi.w));
  const int nn = valid ? min(a.n_nb[i], a.max_nb) : 0;  // an overflowed row keeps max_nb entries
  const int64_t step = a.ds->step;
  const float inv_rc = (float)(1.0 / a.r_cut);

  float4 vi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  double4 pi = make_double4(0., 0., 0., 0.), vi = pi;
  int32_t tag_i = 0;
  if (!MIXED && valid) pi = ld_d4(a.pos + i);
  if (POT == kDPD && valid) {
    if (MIXED) { vi4 = __ldg(a.vel4f + i); tag_i = __float_as_int(vi4.w); }
    else { vi = ld_d4(a.vel + i); tag_i = a.tag[i]; }
  }

  // single-type systems (ONE) keep the pair coefficients in registers
  constexpr bool one_type = ONE;
  LJCoeffF ljf0{};
  LJCoeffD ljd0{};
  DPDCoeffF dpf0{};
  DPDCoeffD dpd0{};
  if (one_type) {
    if (POT == kLJ) {
      if (MIXED) ljf0 = reinterpret_cast<const LJCoeffF *>(a.coeff)[0];
      else ljd0 = reinterpret_cast<const LJCoeffD *>(a.coeff)[0];
    } else {
      if (MIXED) dpf0 = reinterpret_cast<const DPDCoeffF *>(a.coeff)[0];
      else dpd0 = reinterpret_cast<const DPDCoeffD *>(a.coeff)[0];
    }
  }

  // accumulators
  KSum kf[3], kpe, kw[6];
  double df[3] = {0., 0., 0.}, dpe = 0., dw[6] = {0., 0., 0., 0., 0., 0.};

  // Lane sl handles entries k = t W + sl, t < mine.  Entries are fetched U at a
  // time, one group ahead of use (double buffer in registers), and the U
  // position gathers of a group are independent, so each lane keeps several
  // list loads and gathers in flight.
  constexpr int U = 4;
  constexpr uint32_t kNone = 0xffffffffu;  // code 31: no entry
  const int mine = nn > sl ? (nn - sl + W - 1) / W : 0;
  const int iters = __reduce_max_sync(FULL, (unsigned)mine);
  const uint32_t *row = a.nl + (((size_t)i) << LW) + sl;
  const size_t pitch = ((size_t)a.n_pad) << LW;
  uint32_t ebuf[U];
  const uint32_t *rp_next = row;
#pragma unroll
  for (int u = 0; u < U; u++) {
    ebuf[u] = u < mine ? __ldcs(rp_next) : kNone;
    rp_next += pitch;
  }
  for (int t0 = 0; t0 < iters; t0 += U) {
    uint32_t ecur[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      ecur[u] = ebuf[u];
      ebuf[u] = t0 + U + u < mine ? __ldcs(rp_next) : kNone;
      rp_next += pitch;
    }
    // forces of this group are summed plainly, then added to the running
    // Kahan-compensated per-particle sums (one compensated add per group)
    float gx = 0.f, gy = 0.f, gz = 0.f;
    float4 ojs[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      ojs[u] = ecur[u] != kNone ? __ldg(a.pos4f + (ecur[u] & kIdxMask)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint32_t e = ecur[u];
      if (e == kNone) continue;
      const int32_t j = (int32_t)(e & kIdxMask);
      const float4 oj = ojs[u];
      const float4 sh = shift[e >> kIdxBits];
      const float dx = (oi.x - oj.x) - sh.x;
      const float dy = (oi.y - oj.y) - sh.y;
      const float dz = (oi.z - oj.z) - sh.z;
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      if (r2 >= rc2_hi) continue;
      const int tj = cell_type(__float_as_uint(oj.w));
      const int cidx = ti * a.ntypes + tj;
      if (MIXED) {
        if (r2 > rc2_lo) {
          double d[3];
          if (exact_r2(ld_d4(a.pos + i), ld_d4(a.pos + j), rp, d) >= a.rc2) continue;
        }
        float fr, v = 0.f;
        if (POT == kLJ) {
          const LJCoeffF c = one_type ? ljf0 : reinterpret_cast<const LJCoeffF *>(a.coeff)[cidx];
          const float r2i = __fdividef(1.0f, r2);
          const float r6 = r2i * r2i * r2i;
          fr = r2i * r6 * (c.lj1 * r6 - c.lj2);
          if (ENERGY) v = r6 * (c.lj3 * r6 - c.lj4) - c.vshift;
        } else {
          const DPDCoeffF c = one_type ? dpf0 : reinterpret_cast<const DPDCoeffF *>(a.coeff)[cidx];
          const float4 vj = __ldg(a.vel4f + j);
          const float rinv = rsqrtf(r2);
          const float rr = r2 * rinv;
          const float w = 1.f - rr * inv_rc;
          const float dot = dx * (vi4.x - vj.x) + dy * (vi4.y - vj.y) + dz * (vi4.z - vj.z);
          const uint32_t word = dpd_word(tag_i, __float_as_int(vj.w), (uint64_t)step, a.seed);
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
      } else {
        double d[3];
        const double r2d = exact_r2(pi, ld_d4(a.pos + j), rp, d);
        if (r2d >= a.rc2) continue;
        double fr, v = 0.;
        if (POT == kLJ) {
          const LJCoeffD c = one_type ? ljd0 : reinterpret_cast<const LJCoeffD *>(a.coeff)[cidx];
          const double r2i = __drcp_rn(r2d);
          const double r6 = r2i * r2i * r2i;
          fr = r2i * r6 * (c.lj1 * r6 - c.lj2);
          if (ENERGY) v = r6 * (c.lj3 * r6 - c.lj4) - c.vshift;
        } else {
          const DPDCoeffD c = one_type ? dpd0 : reinterpret_cast<const DPDCoeffD *>(a.coeff)[cidx];
          const double4 vj = ld_d4(a.vel + j);
          const double rr = sqrt(r2d);
          const double rinv = 1.0 / rr;
          const double w = 1.0 - rr / a.r_cut;
          const double dot = d[0] * (vi.x - vj.x) + d[1] * (vi.y - vj.y) + d[2] * (vi.z - vj.z);
          const uint32_t word = dpd_word(tag_i, a.tag[j], (uint64_t)step, a.seed);
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
    }
    if (MIXED) {
      kf[0].add(gx);
      kf[1].add(gy);
      kf[2].add(gz);
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
    if (valid && sl == 0) {
      float4 *f = reinterpret_cast<float4 *>(a.force);
      f[i] = make_float4(kf[0].value(), kf[1].value(), kf[2].value(), ENERGY ? kpe.value() : 0.f);
      if (ENERGY) {
        float *vv = reinterpret_cast<float *>(a.virial) + 6 * i;
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
    if (valid && sl == 0) {
      double2 *f = reinterpret_cast<double2 *>(reinterpret_cast<double4 *>(a.force) + i);
      f[0] = make_double2(df[0], df[1]);
      f[1] = make_double2(df[2], ENERGY ? dpe : 0.);
      if (ENERGY) {
        double *vv = reinterpret_cast<double *>(a.virial) + 6 * i;
#pragma unroll
        for (int c = 0; c < 6; c++) vv[c] = dw[c];
      }
    }
  }
}

template <int POT, int W, bool MIXED, bool ENERGY>
cudaError_t go(const KArgs &a, int block, int span, cudaStream_t st) {
  int per_block = block / W;
  unsigned grid = (unsigned)((a.n + per_block - 1) / per_block);
  size_t smem = (size_t)span * 27 * sizeof(float4);
  if (a.ntypes == 1) k_pair<POT, W, MIXED, ENERGY, true><<<grid, block, smem, st>>>(a);
  else k_pair<POT, W, MIXED, ENERGY, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

template <int POT, bool MIXED, bool ENERGY>
cudaError_t go_w(const KArgs &a, Launch l, int span, cudaStream_t st) {
  switch (l.w) {
    case 1: return go<POT, 1, MIXED, ENERGY>(a, l.block, span, st);
    case 2: return go<POT, 2, MIXED, ENERGY>(a, l.block, span, st);
    case 4: return go<POT, 4, MIXED, ENERGY>(a, l.block, span, st);
    case 8: return go<POT, 8, MIXED, ENERGY>(a, l.block, span, st);
    case 16: return go<POT, 16, MIXED, ENERGY>(a, l.block, span, st);
    case 32: return go<POT, 32, MIXED, ENERGY>(a, l.block, span, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int POT, int W, bool MIXED, bool ENERGY>
int maxb_w() {
  cudaFuncAttributes a1, a2;
  if (cudaFuncGetAttributes(&a1, k_pair<POT, W, MIXED, ENERGY, true>) != cudaSuccess) return 0;
  if (cudaFuncGetAttributes(&a2, k_pair<POT, W, MIXED, ENERGY, false>) != cudaSuccess) return 0;
  return a1.maxThreadsPerBlock < a2.maxThreadsPerBlock ? a1.maxThreadsPerBlock : a2.maxThreadsPerBlock;
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

}  // namespace

// Host-side helper: replicas spanned by any block of `per_block` particles.
int pair_span(const int64_t *off, int R, int64_t n, int per_block) {
  int span = 1;
  int r = 0;
  for (int64_t b0 = 0; b0 < n; b0 += per_block) {
    int64_t b1 = std::min<int64_t>(b0 + per_block, n) - 1;
    while (off[r + 1] <= b0) r++;
    int r1 = r;
    while (off[r1 + 1] <= b1) r1++;
    span = std::max(span, r1 - r + 1);
  }
  return span;
}

cudaError_t launch_pair_span(const KArgs &a, Launch l, int want_virial, int span, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const bool m = a.mixed != 0;
  if (a.pair == kLJ) {
    if (m) return want_virial ? go_w<kLJ, true, true>(a, l, span, st) : go_w<kLJ, true, false>(a, l, span, st);
    return want_virial ? go_w<kLJ, false, true>(a, l, span, st) : go_w<kLJ, false, false>(a, l, span, st);
  }
  if (m) return want_virial ? go_w<kDPD, true, true>(a, l, span, st) : go_w<kDPD, true, false>(a, l, span, st);
  return want_virial ? go_w<kDPD, false, true>(a, l, span, st) : go_w<kDPD, false, false>(a, l, span, st);
}

int max_block_pair(const KArgs &a, int w, int want_virial) {
  const bool m = a.mixed != 0;
  if (a.pair == kLJ) {
    if (m) return want_virial ? maxb<kLJ, true, true>(w) : maxb<kLJ, true, false>(w);
    return want_virial ? maxb<kLJ, false, true>(w) : maxb<kLJ, false, false>(w);
  }
  if (m) return want_virial ? maxb<kDPD, true, true>(w) : maxb<kDPD, true, false>(w);
  return want_virial ? maxb<kDPD, false, true>(w) : maxb<kDPD, false, false>(w);
}

}  // namespace mdgb
