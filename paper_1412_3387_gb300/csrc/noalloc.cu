// md_lj_forces_noalloc: FP64 LJ forces of one small periodic system for
// callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: plugins whose host program owns
// every device allocation (a fixed memory pool), real-time loops in which an
// allocation's implicit device synchronisation is not acceptable, and code
// that runs where the allocator is locked down.  This entry point needs no
// workspace from them: its scratch (a cell list) lives in one file-scope
// device array that every process loading the library holds on each device it
// uses, until exit.
//
// The computation is the cell-list variant of the pair-force kernel: bin the
// particles into cells at least r_cut wide, then each particle sums the LJ
// force of every particle within r_cut in the 27 surrounding cells (FP64,
// minimum image).  No neighbour list, no sort.
#include <cmath>
#include <mutex>

#include "md_internal.cuh"

namespace {

// Scratch: cell counts and starts [ncell each], then cell members, slots and
// cells of the particles [n each].  4 MiB.
constexpr int64_t kScratchInts = 1 << 20;
static __device__ __align__(256) int32_t g_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t *g_addr[kMaxDevices] = {};

// Host code cannot use g_scratch's name as a device address (the name stands
// for a host-side shadow).  Look the address up once per device, with that
// device current, and pass it to the kernels.
md_status scratch_for_current_device(int32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MD_ERR_CUDA;
    g_addr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_addr[dev];
  return MD_OK;
}

struct Grid {
  int nc[3];
  double L[3], inv_L[3], inv_h[3];
  int64_t ncell;
};

// Cell of coordinate x: x is first wrapped into [0, L) (callers need not
// wrap their positions), then binned; the clamp only absorbs the rounding of
// the wrap and of x / h at the box edge.
__device__ __forceinline__ int cell_of(double x, double L, double inv_L, double inv_h, int nc) {
  x -= L * floor(x * inv_L);
  int c = (int)floor(x * inv_h);
  c = c >= nc ? nc - 1 : c;
  return c < 0 ? 0 : c;
}

__global__ void k_na_zero(int32_t *count, int64_t ncell) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) count[c] = 0;  // the previous call's counts are still here
}

__global__ void k_na_count(const double4 *pos, int64_t n, Grid g, int32_t *count, int32_t *slot,
                           int32_t *pcell) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4 x = pos[i];
  int cx = cell_of(x.x, g.L[0], g.inv_L[0], g.inv_h[0], g.nc[0]);
  int cy = cell_of(x.y, g.L[1], g.inv_L[1], g.inv_h[1], g.nc[1]);
  int cz = cell_of(x.z, g.L[2], g.inv_L[2], g.inv_h[2], g.nc[2]);
  int32_t c = cx + g.nc[0] * (cy + g.nc[1] * cz);
  pcell[i] = c;
  slot[i] = atomicAdd(count + c, 1);
}

// One block: exclusive scan of the counts into starts.
__global__ void k_na_scan(const int32_t *count, int32_t *start, int64_t ncell) {
  __shared__ int32_t warp_sum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < ncell; base += blockDim.x) {
    int64_t c = base + threadIdx.x;
    int32_t v = c < ncell ? count[c] : 0;
    int32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int32_t t = lane < nw ? warp_sum[lane] : 0, ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      if (lane < nw) warp_sum[lane] = ti - t;
    }
    __syncthreads();
    if (c < ncell) start[c] = carry + warp_sum[wid] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_sum[wid] + incl;
    __syncthreads();
  }
}

__global__ void k_na_scatter(int64_t n, const int32_t *start, const int32_t *slot,
                             const int32_t *pcell, int32_t *members) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  members[start[pcell[i]] + slot[i]] = (int32_t)i;
}

// Compensated (Neumaier) FP64 sum: the per-particle forces of a dense,
// nearly cancelling neighbourhood stay within a few ulps of the exact sum.
struct NSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double get() const { return s + c; }
};

__global__ void k_na_forces(const double4 *pos, int64_t n, Grid g, double rc2, double lj1,
                            double lj2, double lj3, double lj4, const int32_t *count,
                            const int32_t *start, const int32_t *members, const int32_t *pcell,
                            double *force) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4 xi = pos[i];
  const int32_t c = pcell[i];
  const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
  NSum f0, f1, f2, pe;
  for (int s = 0; s < 27; s++) {
    int nx = (cx + s % 3 - 1 + g.nc[0]) % g.nc[0];
    int ny = (cy + (s / 3) % 3 - 1 + g.nc[1]) % g.nc[1];
    int nz = (cz + s / 9 - 1 + g.nc[2]) % g.nc[2];
    int32_t nb = nx + g.nc[0] * (ny + g.nc[1] * nz);
    for (int32_t k = start[nb], e = start[nb] + count[nb]; k < e; k++) {
      int32_t j = members[k];
      if (j == i) continue;
      double4 xj = pos[j];
      // minimum image and r^2 rounded step by step (no fused multiply-add),
      // as in the regular path's exact distance: with a fused L rint(d / L)
      // a separation across the boundary would move by up to an ulp of L
      double d[3] = {__dsub_rn(xi.x, xj.x), __dsub_rn(xi.y, xj.y), __dsub_rn(xi.z, xj.z)};
      for (int a = 0; a < 3; a++)
        d[a] = __dsub_rn(d[a], __dmul_rn(g.L[a], rint(__dmul_rn(d[a], g.inv_L[a]))));
      double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                            __dmul_rn(d[2], d[2]));
      if (r2 >= rc2) continue;
      double r2i = 1.0 / r2, r6 = r2i * r2i * r2i;
      double fr = r2i * r6 * (lj1 * r6 - lj2);
      f0.add(fr * d[0]);
      f1.add(fr * d[1]);
      f2.add(fr * d[2]);
      pe.add(0.5 * r6 * (lj3 * r6 - lj4));
    }
  }
  force[4 * i] = f0.get();
  force[4 * i + 1] = f1.get();
  force[4 * i + 2] = f2.get();
  force[4 * i + 3] = pe.get();
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

extern "C" md_status md_lj_forces_noalloc(const double *dev_pos, int64_t n, const double *box,
                                          double r_cut, double epsilon, double sigma,
                                          double *dev_force, md_stream stream_) {
  if (n < 0 || !box || (n > 0 && (!dev_pos || !dev_force))) return MD_ERR_INVALID_ARG;
  if (!(r_cut > 0) || !(sigma > 0) || !(epsilon >= 0) || !std::isfinite(r_cut))
    return MD_ERR_INVALID_ARG;
  if (((uintptr_t)dev_pos & 15) != 0) return MD_ERR_INVALID_ARG;
  Grid g{};
  for (int d = 0; d < 3; d++) {
    if (!(box[d] > 0) || !std::isfinite(box[d])) return MD_ERR_INVALID_ARG;
    // cells at least r_cut (1 + 1e-12) wide: when the box is an exact multiple
    // of r_cut, a cell exactly r_cut wide could let the rounding of x / h put
    // two particles closer than r_cut two cells apart
    double m = floor(box[d] / (r_cut * (1.0 + 1e-12)));
    if (m < 3.0) return MD_ERR_CELL_GRID;
    if (m > 1024.0) m = 1024.0;
    g.nc[d] = (int)m;
    g.L[d] = box[d];
    g.inv_L[d] = 1.0 / box[d];
    g.inv_h[d] = m / box[d];
  }
  g.ncell = (int64_t)g.nc[0] * g.nc[1] * g.nc[2];
  if (2 * g.ncell + 3 * n > kScratchInts) return MD_ERR_WORKSPACE_TOO_SMALL;  // size limit
  if (n == 0) return MD_OK;
  int32_t *scratch = nullptr;
  md_status st = scratch_for_current_device(&scratch);
  if (st != MD_OK) return st;
  int32_t *count = scratch, *start = count + g.ncell, *members = start + g.ncell;
  int32_t *slot = members + n, *pcell = slot + n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  const double4 *pos = reinterpret_cast<const double4 *>(dev_pos);
  const double s6 = pow(sigma, 6);
  k_na_zero<<<nblk(g.ncell, 256), 256, 0, s>>>(count, g.ncell);
  k_na_count<<<nblk(n, 256), 256, 0, s>>>(pos, n, g, count, slot, pcell);
  k_na_scan<<<1, 1024, 0, s>>>(count, start, g.ncell);
  k_na_scatter<<<nblk(n, 256), 256, 0, s>>>(n, start, slot, pcell, members);
  k_na_forces<<<nblk(n, 128), 128, 0, s>>>(pos, n, g, r_cut * r_cut, 48 * epsilon * s6 * s6,
                                            24 * epsilon * s6, 4 * epsilon * s6 * s6,
                                            4 * epsilon * s6, count, start, members, pcell,
                                            dev_force);
  return cudaGetLastError() == cudaSuccess ? MD_OK : MD_ERR_CUDA;
}
