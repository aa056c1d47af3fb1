// Velocity-Verlet integration with the fused half-buffer rebuild check,
// harmonic bonds, thermo reductions and small utility kernels.
#include "brick.cuh"

namespace mdgb {

namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ double4 ld_force(const KArgs &a, int64_t i) {
  if (a.mixed) {
    float4 f = reinterpret_cast<const float4 *>(a.force)[i];
    return make_double4(f.x, f.y, f.z, f.w);
  }
  return ld_d4(reinterpret_cast<const double4 *>(a.force) + i);
}

// Force without the energy word (integration needs three components only).
__device__ __forceinline__ double3 ld_force3(const KArgs &a, int64_t i) {
  if (a.mixed) {
    const float4 f = reinterpret_cast<const float4 *>(a.force)[i];
    return make_double3(f.x, f.y, f.z);
  }
  const double4 f = ld_d4(reinterpret_cast<const double4 *>(a.force) + i);
  return make_double3(f.x, f.y, f.z);
}

__device__ __forceinline__ double4 ld_d4_plain(const double4 *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 x = q[0], y = q[1];
  return make_double4(x.x, x.y, y.x, y.y);
}

__device__ __forceinline__ void st_d4(double4 *p, const double4 &v) {
  double2 *q = reinterpret_cast<double2 *>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}

// One coordinate of the first velocity-Verlet half (Sec. 3): kick, drift and
// wrap into [0, L) counting image crossings.  Kick and drift are one fused
// multiply-add each (FP64 instructions are scarce on GB300); the oracle
// multiplies and adds separately, a difference of at most one rounding per
// step.
// A crossing moves x by k L with k = floor(x / L) (k = +-1 for any sane time
// step, where this equals the oracle's single subtraction); the fix-ups
// absorb rounding at the box edge.  Non-finite x is left alone (and flagged
// by the caller), so no loop depends on the value of x.
// On GB300 FP64 instructions are scarce (a few per clock per SM), so the box
// test uses the IEEE bit patterns: for x >= 0 and L > 0 the ordering of the
// doubles is the ordering of their bits as signed 64-bit integers, and x < 0
// (or -0) is the sign bit.  Finite <=> exponent bits not all ones.
__device__ __forceinline__ bool outside_box(double x, long long Lbits) {
  const long long b = __double_as_longlong(x);
  return b < 0 || b >= Lbits;
}
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ void wrap_coord(double &x, int &img, double L) {
  if (outside_box(x, __double_as_longlong(L)) && finite_bits(x)) {
    double k = floor(x / L);
    k = fmin(fmax(k, -1e9), 1e9);
    x = __dsub_rn(x, __dmul_rn(k, L));
    img += (int)k;
    if (x >= L) { x = __dsub_rn(x, L); img++; }
    if (x < 0.0) { x = __dadd_rn(x, L); img--; }
  }
}

__device__ __forceinline__ void kick_drift(double &x, double &v, int &img, double f, double hk,
                                           double dt, double L) {
  v = fma(hk, f, v);
  x = fma(dt, v, x);
  wrap_coord(x, img, L);
}

// Langevin BAOAB, first part, one coordinate: kick (B), half drift (A),
// Ornstein-Uhlenbeck step v = c v + sig theta (O), half drift (A), wrap.
__device__ __forceinline__ void baoab_coord(double &x, double &v, int &img, double f, double hk,
                                            double hdt, double c, double sig, double theta,
                                            double L) {
  v = fma(hk, f, v);
  x = fma(hdt, v, x);
  v = fma(c, v, sig * theta);
  x = fma(hdt, v, x);
  wrap_coord(x, img, L);
}

// Langevin noise of one particle for time step `step`: theta_k = sqrt(3)
// (2 u_k - 1), u_k = (w_k + 1/2) 2^-32, words 0..2 of Philox-4x32-10 with
// counter (tag, 0xFFFFFFFF, step lo, step hi) and key (seed lo, seed hi).
// Every operation after the integer generator is exact in FP64.
__device__ __forceinline__ void langevin_theta(int32_t tag, uint64_t step, uint64_t seed,
                                               double th[3]) {
  const U4 c{(uint32_t)tag, 0xFFFFFFFFu, (uint32_t)step, (uint32_t)(step >> 32)};
  const U4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  th[0] = 1.7320508075688772 * (2.0 * (((double)w.x + 0.5) * 2.3283064365386963e-10) - 1.0);
  th[1] = 1.7320508075688772 * (2.0 * (((double)w.y + 0.5) * 2.3283064365386963e-10) - 1.0);
  th[2] = 1.7320508075688772 * (2.0 * (((double)w.z + 0.5) * 2.3283064365386963e-10) - 1.0);
}

// Velocity Verlet, first half, fused with the frame refresh of the FP32
// positions and the rebuild check of Sec. 4.2 (a particle moved more than half
// the buffer since the last build -> raise the replica's flag).  The last
// block to finish advances the step counter and decides the sorts.
// hk = dt / (2m); or dt / m when the previous step's second half-kick was
// left out (inside a run): v(t - 1/2) -> v(t + 1/2) = v(t - 1/2) + dt F(t) / m,
// the same velocity-Verlet step written as one kick.
// The FP32 velocity copy of mixed-precision DPD.  Out of line, so that other
// systems do not issue its conversions under a predicate.
static __device__ __noinline__ void store_vel4f(const KArgs &a, int64_t p, const double4 &v, int64_t i) {
  a.vel4f[p] = make_float4((float)v.x, (float)v.y, (float)v.z, __int_as_float(a.tag[i]));
}

// Grid-stride: a bounded grid keeps the end-of-kernel ticket (one fenced
// atomic per block) cheap.
// One instance per integrator (INTEG = md_integrator), so the plain
// velocity-Verlet form carries no thermostat registers: at most 64 registers
// (4 blocks of 256 threads per SM) keep enough loads in flight.
template <int INTEG>
__global__ void __launch_bounds__(256, 4) k_integrate1(KArgs a, double hk) {
  __shared__ int is_last;
  const int64_t t = a.ds->step;
  const int par = (int)((t + 1) & 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = replica_of(a, i);
    const Rep &rp = a.rep[r];
    double4 x = ld_d4_plain(a.pos + i);
    double4 v = ld_d4_plain(a.vel + i);
    const double3 f = ld_force3(a, i);
    int4 img = a.image[i];
    const int4 img0 = img;
    if (INTEG == MD_NOSE_HOOVER) {
      // the thermostat's half steps at the end of the previous step and at
      // the start of this one, in that order
      const double s1 = a.nh[kNhFields * r + 3], s2 = a.nh[kNhFields * r + 2];
      v.x = (v.x * s1) * s2;
      v.y = (v.y * s1) * s2;
      v.z = (v.z * s1) * s2;
    }
    if (INTEG == MD_LANGEVIN) {
      double th[3];
      langevin_theta(a.tag[i], (uint64_t)(t + 1), a.t_seed, th);
      const double hdt = 0.5 * a.dt;
      baoab_coord(x.x, v.x, img.x, f.x, hk, hdt, a.t_c, a.t_sig, th[0], rp.L[0]);
      baoab_coord(x.y, v.y, img.y, f.y, hk, hdt, a.t_c, a.t_sig, th[1], rp.L[1]);
      baoab_coord(x.z, v.z, img.z, f.z, hk, hdt, a.t_c, a.t_sig, th[2], rp.L[2]);
    } else {
      kick_drift(x.x, v.x, img.x, f.x, hk, a.dt, rp.L[0]);
      kick_drift(x.y, v.y, img.y, f.y, hk, a.dt, rp.L[1]);
      kick_drift(x.z, v.z, img.z, f.z, hk, a.dt, rp.L[2]);
    }
    st_d4(a.pos + i, x);
    st_d4(a.vel + i, v);
    if (img.x != img0.x || img.y != img0.y || img.z != img0.z) a.image[i] = img;
    // the frame (cell and type in .w) is the one of the last build
    const float4 ref = a.oref[i];
    float4 o = ref;
    const uint32_t w = __float_as_uint(ref.w);
    o.x = frame_offset(x.x, cell_centre(a, rp, 0, cell_x(w)), rp.cq[0], rp.Lf[0], rp.L[0]);
    o.y = frame_offset(x.y, cell_centre(a, rp, 1, cell_y(w)), rp.cq[1], rp.Lf[1], rp.L[1]);
    o.z = frame_offset(x.z, cell_centre(a, rp, 2, cell_z(w)), rp.cq[2], rp.Lf[2], rp.L[2]);
    // the FP32 copies are kept in cell-list order
    const int64_t p = __ldg(a.ident + r) ? i : (int64_t)a.cellpos[i];
    a.pos4f[p] = o;
    const float ex = o.x - ref.x, ey = o.y - ref.y, ez = o.z - ref.z;
    const float d2 = ex * ex + ey * ey + ez * ez;
    if (!(d2 <= a.disp2_f)) a.rebuild[2 * r + par] = 1;  // NaN also triggers
    // a non-finite position, or a finite one the wrap could not bring into
    // the box (more than 1e9 box lengths out): the step is invalid
    if (outside_box(x.x, __double_as_longlong(rp.L[0])) ||
        outside_box(x.y, __double_as_longlong(rp.L[1])) ||
        outside_box(x.z, __double_as_longlong(rp.L[2]))) {
      if (atomicOr(&a.ds->error, kErrNonfinite) == 0u) a.ds->error_detail = i;
    }
    if (a.vel4f) store_vel4f(a, p, v, i);
  }
  // Block barrier, then one fence + ticket per block (release of every
  // thread's flag store through the barrier).
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&a.ds->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  int any = 0;
  for (int r = threadIdx.x; r < a.R; r += blockDim.x) {
    const int rb = __ldcg(a.rebuild + 2 * r + par);
    any |= rb;
    int now = 0;
    if (a.sort_period > 0 && rb && (t + 1 - __ldcg(a.last_sort + r)) >= a.sort_period) {
      now = 1;
      a.last_sort[r] = t + 1;
    }
    a.sort_now[r] = now;
    a.rebuild[2 * r + (int)(t & 1)] = 0;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    a.ds->blocks_done = 0u;
    a.ds->rebuild_any = any;
    a.ds->step = t + 1;
  }
}

// Velocity Verlet, second half: v += dt/2 F/m (one fused multiply-add per
// component, as in the first half).
__global__ void k_integrate2(KArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double4 v = ld_d4_plain(a.vel + i);
  const double3 f = ld_force3(a, i);
  const double hk = a.half_dt_m;
  v.x = fma(hk, f.x, v.x);
  v.y = fma(hk, f.y, v.y);
  v.z = fma(hk, f.z, v.z);
  st_d4(a.vel + i, v);
}

// One Nose-Hoover half step (the factor exp(iL_T dt/2) of the Trotter
// splitting) from the kinetic energy KE of a replica's g = 3N - 3 degrees of
// freedom; returns the velocity scale and updates KE, xi, eta.
__device__ __forceinline__ double nh_half(const KArgs &a, double g, double &KE, double &xi,
                                          double &eta) {
  xi += 0.25 * a.dt * ((2.0 * KE / g) / a.t_kT - 1.0) / (a.t_tau * a.t_tau);
  const double sc = exp(-0.5 * a.dt * xi);
  eta += 0.5 * a.dt * xi;
  KE *= sc * sc;
  xi += 0.25 * a.dt * ((2.0 * KE / g) / a.t_kT - 1.0) / (a.t_tau * a.t_tau);
  return sc;
}

// Nose-Hoover: second half-kick (kick = 1) or none (kick = 0: the start of a
// sequence of steps) and the kinetic-energy sum, one block per thermo chunk
// (fixed assignment and tree: bitwise reproducible).  The last block takes,
// per replica, the thermostat's half step at the end of this step (its scale
// s1 stays pending: the velocities in memory are the unscaled ones) and the
// one at the start of the next step (s2); the next first half applies both.
__global__ void __launch_bounds__(256) k_nh_kick_sum(KArgs a, int kick) {
  __shared__ double sh[256];
  __shared__ int is_last;
  const int64_t ch = blockIdx.x;
  const int r = a.tchunk_rep[ch];
  const Rep &rp = a.rep[r];
  const int64_t p0 = rp.p0 + (ch - rp.tchunk0) * kThermoChunk;
  const int64_t p1 = min(p0 + kThermoChunk, rp.p1);
  const double hk = a.half_dt_m;
  double ke = 0.0;
  for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
    double4 v = ld_d4_plain(a.vel + i);
    if (kick) {
      const double3 f = ld_force3(a, i);
      v.x = fma(hk, f.x, v.x);
      v.y = fma(hk, f.y, v.y);
      v.z = fma(hk, f.z, v.z);
      st_d4(a.vel + i, v);
    }
    ke += 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
  }
  sh[threadIdx.x] = ke;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.nh_part[ch] = sh[0];
    __threadfence();
    is_last = atomicAdd(&a.ds->nh_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int q = threadIdx.x; q < a.R; q += blockDim.x) {
    const Rep &rq = a.rep[q];
    const double g = 3.0 * (double)(rq.p1 - rq.p0) - 3.0;
    if (!(g > 0.0)) continue;
    double KE = 0.0;
    for (int c = 0; c < rq.ntchunk; c++) KE += __ldcg(a.nh_part + rq.tchunk0 + c);
    double *st = a.nh + kNhFields * q;
    double xi = st[0], eta = st[1];
    const double s1 = kick ? nh_half(a, g, KE, xi, eta) : st[3];
    // the state between steps (after this step's end half step) is the one
    // reported; the next step starts from its start half step
    st[4] = xi;
    st[5] = eta;
    const double s2 = nh_half(a, g, KE, xi, eta);
    st[0] = xi;
    st[1] = eta;
    st[2] = s2;
    st[3] = s1;
  }
  if (threadIdx.x == 0) a.ds->nh_done = 0u;
}

// Applies the pending end-of-step scale s1 to the velocities (the state after
// a completed step); k_nh_flush_end then clears it.
__global__ void k_nh_flush(KArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double s1 = a.nh[kNhFields * replica_of(a, i) + 3];
  double4 v = ld_d4_plain(a.vel + i);
  v.x *= s1;
  v.y *= s1;
  v.z *= s1;
  st_d4(a.vel + i, v);
}

__global__ void k_nh_flush_end(KArgs a) {
  for (int q = threadIdx.x; q < a.R; q += blockDim.x) {
    // the start-of-next-step scale was computed from the scaled energy
    a.nh[kNhFields * q + 3] = 1.0;
  }
}

__global__ void k_nh_reset(KArgs a) {
  for (int q = threadIdx.x; q < a.R; q += blockDim.x) {
    double *st = a.nh + kNhFields * q;
    st[0] = st[1] = st[4] = st[5] = 0.0;
    st[2] = st[3] = 1.0;
  }
}

// Harmonic bonds (Sec. 4.3.4: a bond is an unordered pair of particle IDs):
// each particle sums the bonds it belongs to, so no atomics are needed.
// V = K/2 (r - r0)^2, F_i = -K (r - r0) (x_i - x_j) / r.
template <bool ENERGY>
__global__ void k_bonds(KArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int r = replica_of(a, i);
  const Rep &rp = a.rep[r];
  const int32_t ti = a.tag[i];
  const double4 pi = ld_d4(a.pos + i);
  double f[3] = {0., 0., 0.}, pe = 0., w[6] = {0., 0., 0., 0., 0., 0.};
  bool any = false;
  for (int b = 0; b < a.max_bonds; b++) {
    const int32_t p = a.btab[(int64_t)ti * a.max_bonds + b];
    if (p < 0) break;
    any = true;
    const int32_t j = a.rtag[p];
    double d[3];
    const double r2 = exact_r2(pi, ld_d4(a.pos + j), rp, d);
    double fr, v = 0.0;
    if (a.bond_style == MD_BOND_FENE) {
      // FENE: V = -K R0^2 / 2 ln(1 - q), q = (r / R0)^2; -dV/dr / r = -K / (1 - q)
      const double q = r2 / (a.bond_r0 * a.bond_r0);
      if (!(q < 1.0)) {
        if (atomicOr(&a.ds->error, kErrBond) == 0u) a.ds->error_detail = i;
        continue;
      }
      fr = -a.bond_K / (1.0 - q);
      if (ENERGY) v = -0.5 * a.bond_K * a.bond_r0 * a.bond_r0 * log(1.0 - q);
    } else if (a.bond_r0 == 0.0) {
      fr = -a.bond_K;
      if (ENERGY) v = 0.5 * a.bond_K * r2;
    } else {
      const double dr = sqrt(r2);
      fr = dr > 0.0 ? -a.bond_K * (dr - a.bond_r0) / dr : 0.0;
      if (ENERGY) v = 0.5 * a.bond_K * (dr - a.bond_r0) * (dr - a.bond_r0);
    }
    const double fx = fr * d[0], fy = fr * d[1], fz = fr * d[2];
    f[0] += fx; f[1] += fy; f[2] += fz;
    if (ENERGY) {
      pe += 0.5 * v;
      w[0] += 0.5 * d[0] * fx; w[1] += 0.5 * d[0] * fy; w[2] += 0.5 * d[0] * fz;
      w[3] += 0.5 * d[1] * fy; w[4] += 0.5 * d[1] * fz; w[5] += 0.5 * d[2] * fz;
    }
  }
  // harmonic angles this particle takes part in (as an end or the vertex):
  // V = K/2 (theta - theta0)^2 with theta the angle at the vertex b between
  // u = x_a - x_b and w = x_c - x_b; with c = cos theta, s = sin theta and
  // g = K (theta - theta0) / s:
  //   F_a = g (w / (|u| |w|) - c u / |u|^2), F_c likewise, F_b = -(F_a + F_c);
  // each particle takes a third of V and of the virial u (x) F_a + w (x) F_c
  for (int q = 0; q < a.max_angles; q++) {
    const int32_t *e = a.atab + ((int64_t)ti * a.max_angles + q) * 3;
    if (e[0] < 0) break;
    any = true;
    const double4 pa = ld_d4(a.pos + a.rtag[e[0]]);
    const double4 pb = ld_d4(a.pos + a.rtag[e[1]]);
    const double4 pc = ld_d4(a.pos + a.rtag[e[2]]);
    double u[3], wv[3];
    const double uu = exact_r2(pa, pb, rp, u);
    const double ww = exact_r2(pc, pb, rp, wv);
    const double ru = sqrt(uu), rw = sqrt(ww);
    double cs = (u[0] * wv[0] + u[1] * wv[1] + u[2] * wv[2]) / (ru * rw);
    cs = fmin(fmax(cs, -1.0), 1.0);
    const double th = acos(cs);
    const double sn = fmax(sqrt(1.0 - cs * cs), 1e-12);
    const double g = a.angle_K * (th - a.angle_th0) / sn;
    double fa[3], fc[3];
    for (int k = 0; k < 3; k++) {
      fa[k] = g * (wv[k] / (ru * rw) - cs * u[k] / uu);
      fc[k] = g * (u[k] / (ru * rw) - cs * wv[k] / ww);
    }
    const int role = ti == e[0] ? 0 : ti == e[1] ? 1 : 2;
    for (int k = 0; k < 3; k++)
      f[k] += role == 0 ? fa[k] : role == 2 ? fc[k] : -(fa[k] + fc[k]);
    if (ENERGY) {
      pe += 0.5 * a.angle_K * (th - a.angle_th0) * (th - a.angle_th0) / 3.0;
      w[0] += (u[0] * fa[0] + wv[0] * fc[0]) / 3.0; w[1] += (u[0] * fa[1] + wv[0] * fc[1]) / 3.0;
      w[2] += (u[0] * fa[2] + wv[0] * fc[2]) / 3.0; w[3] += (u[1] * fa[1] + wv[1] * fc[1]) / 3.0;
      w[4] += (u[1] * fa[2] + wv[1] * fc[2]) / 3.0; w[5] += (u[2] * fa[2] + wv[2] * fc[2]) / 3.0;
    }
  }
  if (!any) return;
  if (a.mixed) {
    float4 *F = reinterpret_cast<float4 *>(a.force) + i;
    float4 g = *F;
    g.x += (float)f[0]; g.y += (float)f[1]; g.z += (float)f[2];
    if (ENERGY) g.w += (float)pe;
    *F = g;
    if (ENERGY) {
      float *vv = reinterpret_cast<float *>(a.virial) + 6 * i;
      for (int c = 0; c < 6; c++) vv[c] += (float)w[c];
    }
  } else {
    double4 *F = reinterpret_cast<double4 *>(a.force) + i;
    double4 g = ld_d4_plain(F);
    g.x += f[0]; g.y += f[1]; g.z += f[2];
    if (ENERGY) g.w += pe;
    st_d4(F, g);
    if (ENERGY) {
      double *vv = reinterpret_cast<double *>(a.virial) + 6 * i;
      for (int c = 0; c < 6; c++) vv[c] += w[c];
    }
  }
}

// Thermo reduction, stage 1: one block per chunk of <= kThermoChunk particles
// of one replica.  Fixed assignment of particles to threads and a fixed
// shared-memory tree: the result is bitwise reproducible.
__global__ void __launch_bounds__(256) k_thermo_part(KArgs a) {
  __shared__ double sh[8][256];
  const int64_t ch = blockIdx.x;
  const int r = a.tchunk_rep[ch];
  const Rep &rp = a.rep[r];
  const int64_t p0 = rp.p0 + (ch - rp.tchunk0) * kThermoChunk;
  const int64_t p1 = min(p0 + kThermoChunk, rp.p1);
  double acc[8] = {0., 0., 0., 0., 0., 0., 0., 0.};  // ke, pe, w, px, py, pz
  for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
    const double4 v = ld_d4(a.vel + i);
    const double4 f = ld_force(a, i);
    acc[0] += 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
    acc[1] += f.w;
    if (a.mixed) {
      const float *vv = reinterpret_cast<const float *>(a.virial) + 6 * i;
      acc[2] += (double)vv[0] + (double)vv[3] + (double)vv[5];
    } else {
      const double *vv = reinterpret_cast<const double *>(a.virial) + 6 * i;
      acc[2] += vv[0] + vv[3] + vv[5];
    }
    acc[3] += a.mass * v.x;
    acc[4] += a.mass * v.y;
    acc[5] += a.mass * v.z;
  }
  for (int k = 0; k < 8; k++) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 6; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6) a.tpart[ch * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// Stage 2: one thread per replica sums its chunks in order and derives
// P = (2 KE + W) / (3 V) and T = 2 KE / (3 N - 3).
__global__ void k_thermo_final(KArgs a, double *out, int from_run) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  const Rep &rp = a.rep[r];
  double s[6] = {0., 0., 0., 0., 0., 0.};
  for (int c = 0; c < rp.ntchunk; c++)
    for (int k = 0; k < 6; k++) s[k] += a.tpart[(rp.tchunk0 + c) * 8 + k];
  double *o = out;
  if (from_run) {
    // row = number of multiples of the period in (run_base, step], minus one
    const DevState *ds = a.ds;
    if (ds->thermo_out == nullptr) return;
    const int64_t p = ds->thermo_period;
    const int64_t row = ds->step / p - ds->run_base / p - 1;
    if (row < 0 || row >= ds->thermo_rows) return;
    o = ds->thermo_out + row * (int64_t)a.R * 8;
  }
  if (a.integ == MD_NOSE_HOOVER) {
    // the velocities lack the thermostat's pending end-of-step scale
    const double sc = a.nh[kNhFields * r + 3];
    s[0] *= sc * sc;
    s[3] *= sc;
    s[4] *= sc;
    s[5] *= sc;
  }
  const double n = (double)(rp.p1 - rp.p0);
  double *q = o + 8 * r;
  q[0] = s[0];
  q[1] = s[1];
  q[2] = s[2];
  q[3] = (2.0 * s[0] + s[2]) / (3.0 * rp.volume);
  q[4] = n > 1.0 ? 2.0 * s[0] / (3.0 * n - 3.0) : 0.0;
  q[5] = s[3];
  q[6] = s[4];
  q[7] = s[5];
}

// Frames of the FP32 positions from the current FP64 positions, without
// building cells (used once at creation so that md_integrate is defined
// before the first build).
__global__ void k_init_frames(KArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const Rep &rp = a.rep[replica_of(a, i)];
  const double4 x = ld_d4(a.pos + i);
  const int cx = cell_coord(x.x, rp.inv_h[0], rp.nc[0]);
  const int cy = cell_coord(x.y, rp.inv_h[1], rp.nc[1]);
  const int cz = cell_coord(x.z, rp.inv_h[2], rp.nc[2]);
  float4 o;
  o.x = frame_offset(x.x, cell_centre(a, rp, 0, cx), rp.cq[0], rp.Lf[0], rp.L[0]);
  o.y = frame_offset(x.y, cell_centre(a, rp, 1, cy), rp.cq[1], rp.Lf[1], rp.L[1]);
  o.z = frame_offset(x.z, cell_centre(a, rp, 2, cz), rp.cq[2], rp.Lf[2], rp.L[2]);
  // tags must be a permutation of 0..N-1 and types lie in [0, ntypes): both
  // index tables later, so out-of-range values are refused here
  const int32_t tg = a.tag[i], ty = a.type[i];
  const bool ok = tg >= 0 && tg < a.n && ty >= 0 && ty < a.ntypes;
  if (!ok) set_error(a.ds, kErrBadInput);
  o.w = __uint_as_float(pack_cell(cx, cy, cz, ok ? ty : 0));
  a.pos4f[i] = o;
  a.oref[i] = o;
  a.cell_idx[i] = (int32_t)i;
  a.cellpos[i] = (int32_t)i;
  if (ok) a.rtag[tg] = (int32_t)i;
  if (a.vel4f) {
    const double4 v = ld_d4(a.vel + i);
    a.vel4f[i] = make_float4((float)v.x, (float)v.y, (float)v.z, __int_as_float(a.tag[i]));
  }
}

__global__ void k_set_step(KArgs a, int64_t step) { a.ds->step = step; }

__global__ void k_run_begin(KArgs a, double *out, int64_t period, int64_t rows) {
  a.ds->run_base = a.ds->step;
  a.ds->thermo_out = out;
  a.ds->thermo_period = period > 0 ? period : 1;
  a.ds->thermo_rows = rows;
}

__global__ void k_export_forces(KArgs a, double *f, double *v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double4 g = ld_force(a, i);
  f[4 * i] = g.x; f[4 * i + 1] = g.y; f[4 * i + 2] = g.z; f[4 * i + 3] = g.w;
  if (v) {
    for (int c = 0; c < 6; c++)
      v[6 * i + c] = a.mixed ? (double)reinterpret_cast<const float *>(a.virial)[6 * i + c]
                             : reinterpret_cast<const double *>(a.virial)[6 * i + c];
  }
}

// One warp per brick: decode each row's stage slots into particle indices and
// write them, compacted, at the particle's own row (rows in the tile layout
// can hold sentinel gaps).
__global__ void k_export_nlist(KArgs a, int32_t *counts, int32_t *rows) {
  const int lane = threadIdx.x & 31;
  const int64_t b = blockIdx.x;
  const BrickDesc &d = a.brick_desc[b];
  const int lw = a.w_store_log2, W = 1 << lw, P = 32 >> lw;
  for (int q = 0; q < d.nhome; q++) {
    const int p = d.hstart + q;
    const int32_t i = a.cell_idx[p];
    const int jg = q / P, q2 = q % P, pj = min(P, d.nhome - jg * P);
    const uint16_t *grp = a.nl + (size_t)(d.hstart + jg * P) * (size_t)a.max_nb;
    const int T = a.nl_tiles[d.hstart + jg * P];
    if (lane == 0) counts[i] = a.n_nb[p];
    int n = 0;  // entries written so far (the same in every lane)
    for (int k0 = 0; k0 < T * W; k0 += 32) {
      const int k = k0 + lane;
      int e = 0;
      if (k < T * W) e = grp[row_offset(k, lw, pj, q2)];
      const unsigned m = __ballot_sync(0xffffffffu, e > 0);
      if (e > 0) {
        const int at = n + __popc(m & ((1u << lane) - 1u));
        const int s = e - 1, c = stage_cell_of(d, s);
        if (at < a.max_nb) rows[(int64_t)i * a.max_nb + at] = a.cell_idx[d.start[c] + (s - d.off[c])];
      }
      n += __popc(m);
    }
    for (int k = n + lane; k < a.max_nb; k += 32) rows[(int64_t)i * a.max_nb + k] = -1;
  }
}

__global__ void k_export_cells(KArgs a, int32_t *start, int32_t *count, int32_t *idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_cells) {
    start[i] = a.cell_start[i];
    count[i] = a.cell_count[i];
  }
  if (i < a.n) idx[i] = a.cell_idx[i];
}

__global__ void k_philox(const uint32_t *in, uint32_t *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t *q = in + 6 * i;
  U4 c = philox4x32_10(U4{q[0], q[1], q[2], q[3]}, q[4], q[5]);
  out[4 * i] = c.x; out[4 * i + 1] = c.y; out[4 * i + 2] = c.z; out[4 * i + 3] = c.w;
}

}  // namespace

cudaError_t launch_integrate1(const KArgs &a, cudaStream_t st, bool fold_kick) {
  // the step counter must advance even for an empty system; one wave of 4
  // blocks per SM (152 SMs), grid-stride beyond that
  const unsigned need = blocks_for(a.n > 0 ? a.n : 1, 256);
  const unsigned grid = need < 152u * 4u ? need : 152u * 4u;
  const double hk = fold_kick ? 2.0 * a.half_dt_m : a.half_dt_m;
  if (a.integ == MD_LANGEVIN) k_integrate1<MD_LANGEVIN><<<grid, 256, 0, st>>>(a, hk);
  else if (a.integ == MD_NOSE_HOOVER) k_integrate1<MD_NOSE_HOOVER><<<grid, 256, 0, st>>>(a, hk);
  else k_integrate1<MD_NVE><<<grid, 256, 0, st>>>(a, hk);
  return cudaGetLastError();
}

cudaError_t launch_integrate2(const KArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.integ == MD_NOSE_HOOVER) {
    if (a.n_tchunks > 0) k_nh_kick_sum<<<(unsigned)a.n_tchunks, 256, 0, st>>>(a, 1);
  } else {
    k_integrate2<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_nh_begin(const KArgs &a, cudaStream_t st) {
  if (a.n_tchunks > 0) k_nh_kick_sum<<<(unsigned)a.n_tchunks, 256, 0, st>>>(a, 0);
  return cudaGetLastError();
}

cudaError_t launch_nh_flush(const KArgs &a, cudaStream_t st) {
  if (a.n > 0) k_nh_flush<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  k_nh_flush_end<<<1, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nh_reset(const KArgs &a, cudaStream_t st) {
  k_nh_reset<<<1, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bonds(const KArgs &a, int want_virial, cudaStream_t st) {
  if (a.n == 0 || a.max_bonds == 0) return cudaSuccess;
  if (want_virial) k_bonds<true><<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  else k_bonds<false><<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_thermo(const KArgs &a, double *out, int from_run, cudaStream_t st) {
  if (a.n_tchunks > 0) k_thermo_part<<<(unsigned)a.n_tchunks, 256, 0, st>>>(a);
  k_thermo_final<<<blocks_for(a.R, 64), 64, 0, st>>>(a, out, from_run);
  return cudaGetLastError();
}

cudaError_t launch_set_step(const KArgs &a, int64_t step, cudaStream_t st) {
  k_set_step<<<1, 1, 0, st>>>(a, step);
  return cudaGetLastError();
}

cudaError_t launch_run_begin(const KArgs &a, double *out, int64_t period, int64_t rows,
                             cudaStream_t st) {
  k_run_begin<<<1, 1, 0, st>>>(a, out, period, rows);
  return cudaGetLastError();
}

cudaError_t launch_init_frames(const KArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_init_frames<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_export_forces(const KArgs &a, double *f, double *v, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  k_export_forces<<<blocks_for(a.n, 256), 256, 0, st>>>(a, f, v);
  return cudaGetLastError();
}

cudaError_t launch_export_nlist(const KArgs &a, int32_t *counts, int32_t *rows, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.n_bricks > 0) k_export_nlist<<<(unsigned)a.n_bricks, 32, 0, st>>>(a, counts, rows);
  return cudaGetLastError();
}

cudaError_t launch_export_cells(const KArgs &a, int32_t *start, int32_t *count, int32_t *idx,
                                cudaStream_t st) {
  int64_t m = a.n_cells > a.n ? a.n_cells : a.n;
  if (m == 0) return cudaSuccess;
  k_export_cells<<<blocks_for(m, 256), 256, 0, st>>>(a, start, count, idx);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_philox<<<blocks_for(n, 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace mdgb
