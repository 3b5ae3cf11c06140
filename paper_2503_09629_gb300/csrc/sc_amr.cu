// sc_amr.cu -- refinement-boundary kernels (prolongation of the parent's
// y_n and stage vectors, dense-output ghost fill, restriction), periodic ghost copy,
// analytic initial data, box pack/unpack and the finiteness check.
//
// Every kernel works on one level's dense FP64 array (one array per field,
// x fastest) through precomputed int32 offset lists.
#include <math.h>

#include "sc_device.cuh"

namespace sc {
namespace {

constexpr int kThreads = 256;

inline int grid_for(long work, int threads) {
  long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > sm_count() * 64L) b = sm_count() * 64L;  // grid-stride beyond 64 blocks per SM
  return (int)b;
}

// Stand-alone kernels over the device-function bodies of sc_device.cuh
// (one launch covers a whole work list; the persistent coarse-step kernel
// runs the same bodies phase by phase).
__global__ void __launch_bounds__(kThreads) amr_prolong_kernel(
    const double* __restrict__ yn, const double* __restrict__ k1, const double* __restrict__ k2,
    const double* __restrict__ k3, const double* __restrict__ k4, long pfs, int psy, int psz,
    const AmrCell* __restrict__ cells, int first, int ncells, double* __restrict__ store, int F, Weights w, int nvec) {
  amr_prolong_cells_body(yn, k1, k2, k3, k4, pfs, psy, psz, cells, first, ncells, store, F, w, nvec, blockIdx.x,
                         gridDim.x);
}

__global__ void __launch_bounds__(256) amr_prolong_tile_kernel(
    const double* __restrict__ yn, const double* __restrict__ k1, const double* __restrict__ k2,
    const double* __restrict__ k3, const double* __restrict__ k4, long pfs, int psy, int psz,
    const AmrTile* __restrict__ tiles, int ntiles, const int32_t* __restrict__ slots, int ncells,
    double* __restrict__ store, int F, Weights w, int nvec) {
  __shared__ double sm[2 * kProlongSmemPerGroup];
  amr_prolong_tiles_body(yn, k1, k2, k3, k4, pfs, psy, psz, tiles, ntiles, slots, ncells, store, F, w, nvec,
                         blockIdx.x, gridDim.x, sm, 2);
}

__global__ void __launch_bounds__(kThreads) amr_apply_kernel(double* __restrict__ vec, long fs, int F,
                                                            const AmrCell* __restrict__ cells, int ncells,
                                                            const double* __restrict__ store, double c1,
                                                            double c2, double c3, double c4, int nk) {
  amr_apply_body(vec, fs, F, cells, ncells, store, c1, c2, c3, c4, nk, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads) restrict_kernel(double* __restrict__ parent, long pfs,
                                                           const double* __restrict__ fine, long ffs, int fsy,
                                                           int fsz, const RestrictCell* __restrict__ cells,
                                                           int ncells, int F, Weights w) {
  restrict_cells_body(parent, pfs, fine, ffs, fsy, fsz, cells, ncells, F, w, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(128) restrict_block_kernel(double* __restrict__ parent, long pfs, int psy,
                                                            int psz, const double* __restrict__ fine, long ffs,
                                                            int fsy, int fsz,
                                                            const RestrictBlock* __restrict__ blocks, int nblocks,
                                                            int F, Weights w) {
  __shared__ double sm[2 * kRestrictSmemPerGroup];
  restrict_blocks_body(parent, pfs, psy, psz, fine, ffs, fsy, fsz, blocks, nblocks, F, w, blockIdx.x, gridDim.x, sm,
                       2);
}

__global__ void __launch_bounds__(kThreads) periodic_copy_kernel(double* __restrict__ vec, long fs, int F,
                                                                const int2* __restrict__ pairs, int npairs) {
  periodic_copy_body(vec, fs, F, pairs, npairs, blockIdx.x, gridDim.x);
}

struct IdParams {
  double p[8];
};

// Analytic initial data at every element of a level array.
__global__ void __launch_bounds__(kThreads) initial_data_kernel(double* __restrict__ vec, Geom g, int F,
                                                               int system, int kind, IdParams ip) {
  const long ncell = (long)g.ext[0] * g.ext[1] * g.ext[2];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < ncell; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.ext[0]);
    const int j = (int)((idx / g.ext[0]) % g.ext[1]);
    const int k = (int)(idx / ((long)g.ext[0] * g.ext[1]));
    const long o = ((long)k * g.ext[1] + j) * g.pitch + i;
    const double x = g.x0[0] + i * g.h, y = g.x0[1] + j * g.h, z = g.x0[2] + k * g.h;
    const double* p = ip.p;
    if (system == SC_WAVE) {
      double u = 0.0, pi = 0.0;
      if (kind == SC_ID_STANDING_WAVE) {
        const double tp = 2.0 * M_PI;
        u = p[0] * sin(tp * p[1] * x) * sin(tp * p[2] * y) * sin(tp * p[3] * z);
      } else if (kind == SC_ID_GAUSSIAN) {
        const double dx = x - p[2], dy = y - p[3], dz = z - p[4];
        u = p[0] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * p[1] * p[1]));
      } else if (kind == SC_ID_SPHERICAL_GAUSSIAN) {
        const double dx = x - p[3], dy = y - p[4], dz = z - p[5];
        const double r = sqrt(dx * dx + dy * dy + dz * dz), t = p[2], s2 = p[1] * p[1];
        const double fm = p[0] * exp(-(t - r) * (t - r) / (2.0 * s2));
        const double fp = p[0] * exp(-(t + r) * (t + r) / (2.0 * s2));
        u = (fm - fp) / r;
        pi = -(fm * (t - r) - fp * (t + r)) / (s2 * r);
      }
      vec[o] = u;
      vec[g.fs + o] = pi;
    } else {
      double s = 0.0;
      if (kind == SC_ID_BRILL_LINDQUIST || kind == SC_ID_BRILL_LINDQUIST_AVG_LAPSE) {
        for (int q = 0; q < 2; ++q) {
          const double dx = x - p[4 * q + 1], dy = y - p[4 * q + 2], dz = z - p[4 * q + 3];
          s += p[4 * q] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
        }
      }
      const double psi = 1.0 + s;
      const double ipsi2 = 1.0 / (psi * psi);
      // lapse: psi^-2, or the averaged form (1 + (1 - s)/(1 + s))/2 of Sec. III.B
      const double lapse = kind == SC_ID_BRILL_LINDQUIST_AVG_LAPSE ? 0.5 * (1.0 + (1.0 - s) / (1.0 + s)) : ipsi2;
      for (int f = 0; f < F; ++f) vec[(long)f * g.fs + o] = 0.0;
      vec[(long)ZW * g.fs + o] = ipsi2;
      vec[(long)(ZG + 0) * g.fs + o] = 1.0;
      vec[(long)(ZG + 3) * g.fs + o] = 1.0;
      vec[(long)(ZG + 5) * g.fs + o] = 1.0;
      vec[(long)ZAL * g.fs + o] = lapse;
    }
  }
}

// Copy a box region of one field between a level array and a contiguous
// x-fastest buffer (unpack = 0: array -> buffer; 1: buffer -> array).
// Regrid: copy the state of cells that stay interior from the old level
// array (pairs: x = destination offset, y = source offset).
__global__ void __launch_bounds__(kThreads) transfer_copy_kernel(double* __restrict__ dst, long dfs,
                                                                const double* __restrict__ src, long sfs,
                                                                const int2* __restrict__ pairs, int n, int F) {
  const long total = (long)n * F;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int a = (int)(idx % n);
    const int f = (int)(idx / n);
    const int2 p = pairs[a];
    dst[(long)f * dfs + p.x] = src[(long)f * sfs + p.y];
  }
}

// Regrid: new interior cells take the quintic prolongation of the parent's
// state (the same stencil as the refinement-boundary ghosts).
__global__ void __launch_bounds__(kThreads) prolong_state_kernel(double* __restrict__ dst, long dfs,
                                                                const double* __restrict__ parent, long pfs,
                                                                int psy, int psz, const AmrCell* __restrict__ cells,
                                                                int n, int F, Weights w) {
  const long total = (long)n * F;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int a = (int)(idx % n);
    const int f = (int)(idx / n);
    const AmrCell c = cells[a];
    const double* wx = w.prolong[c.parity & 1];
    const double* wy = w.prolong[(c.parity >> 1) & 1];
    const double* wz = w.prolong[(c.parity >> 2) & 1];
    const double* p = parent + (long)f * pfs + c.pbase;
    double sz = 0.0;
#pragma unroll
    for (int kz = 0; kz < kPN; ++kz) {
      double sy = 0.0;
#pragma unroll
      for (int ky = 0; ky < kPN; ++ky) {
        const double* row = p + (long)kz * psz + (long)ky * psy;
        double sx = 0.0;
#pragma unroll
        for (int kx = 0; kx < kPN; ++kx) sx = fma(wx[kx], __ldg(row + kx), sx);
        sy = fma(wy[ky], sx, sy);
      }
      sz = fma(wz[kz], sy, sz);
    }
    dst[(long)f * dfs + c.dst] = sz;
  }
}

// Field values at arbitrary points: quintic tensor Lagrange interpolation of
// 6x6x6 cells of a level array with per-point weights computed on the host.
__global__ void __launch_bounds__(kThreads) interpolate_kernel(const InterpPoint* __restrict__ pts, int n,
                                                              double* __restrict__ out) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    const InterpPoint q = pts[a];
    double sz = 0.0;
    for (int kz = 0; kz < kPN; ++kz) {
      double sy = 0.0;
      for (int ky = 0; ky < kPN; ++ky) {
        const double* row = q.base + (long)kz * q.sz + (long)ky * q.sy;
        double sx = 0.0;
        for (int kx = 0; kx < kPN; ++kx) sx = fma(q.w[kx], row[kx], sx);
        sy = fma(q.w[kPN + ky], sx, sy);
      }
      sz = fma(q.w[2 * kPN + kz], sy, sz);
    }
    out[a] = sz;
  }
}

// Gamma-driver damping profile of Sec. III.A at every element of a level array.
__global__ void __launch_bounds__(kThreads) eta_profile_kernel(double* __restrict__ eta, Geom g, double ec, double es,
                                                              double eo) {
  const long ncell = (long)g.ext[0] * g.ext[1] * g.ext[2];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < ncell; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.ext[0]);
    const int j = (int)((idx / g.ext[0]) % g.ext[1]);
    const int k = (int)(idx / ((long)g.ext[0] * g.ext[1]));
    const double x = g.x0[0] + i * g.h, y = g.x0[1] + j * g.h, z = g.x0[2] + k * g.h;
    const double q = (x * x + y * y + z * z) / (es * es);  // (r / eta_s)^2
    eta[((long)k * g.ext[1] + j) * g.pitch + i] = (ec - eo) * exp(-q * q) + eo;
  }
}

__global__ void __launch_bounds__(kThreads) pack_kernel(double* __restrict__ vec, int pitch, int ey, int i0,
                                                       int j0, int k0, int nx, int ny, int nz,
                                                       double* __restrict__ buf, int unpack) {
  const long n = (long)nx * ny * nz;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nx);
    const int j = (int)((idx / nx) % ny);
    const int k = (int)(idx / ((long)nx * ny));
    const long o = ((long)(k0 + k) * ey + (j0 + j)) * pitch + (i0 + i);
    if (unpack) vec[o] = buf[idx];
    else buf[idx] = vec[o];
  }
}

// All F fields of one box region: field f of the region is the f-th block of
// nx*ny*nz values in buf (unpack = 0: array -> buffer; 1: buffer -> array).
// One warp per row of nx values (a row index covers field, z and y), lanes
// along x: both sides are read and written in contiguous runs, and the index
// arithmetic is done once per row.  buf may be device memory or page-locked
// host memory mapped into the device address space (read and written over
// the CPU-GPU link directly).
__global__ void __launch_bounds__(kThreads) pack_fields_kernel(double* __restrict__ vec, long fs, int F, int pitch,
                                                              int ey, int i0, int j0, int k0, int nx, int ny,
                                                              int nz, double* __restrict__ buf, int unpack) {
  const long rows = (long)F * nz * ny;
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long r = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int j = (int)(r % ny);
    const long fk = r / ny;
    const int k = (int)(fk % nz);
    const int f = (int)(fk / nz);
    double* v = vec + (long)f * fs + ((long)(k0 + k) * ey + (j0 + j)) * pitch + i0;
    double* b = buf + r * nx;
    if (unpack)
      for (int i = lane; i < nx; i += 32) v[i] = b[i];
    else
      for (int i = lane; i < nx; i += 32) b[i] = v[i];
  }
}

__global__ void __launch_bounds__(kThreads) nonfinite_kernel(const double* __restrict__ vec, long fs, int F,
                                                            const Tile* __restrict__ tiles, int ntiles,
                                                            int sy, int sz, int* flag) {
  nonfinite_body(vec, fs, F, tiles, ntiles, sy, sz, flag, blockIdx.x, gridDim.x);
}

int g_sm_count[64];  // per device; 0 = not queried yet

}  // namespace

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  int& n = g_sm_count[dev & 63];
  if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 152;
  return n;
}

cudaError_t launch_amr_prolong(const double* yn, const double* k1, const double* k2, const double* k3,
                               const double* k4, long pfs, int psy, int psz, const AmrCell* cells, int first,
                               int ncells, double* store, int F, const Weights& w, cudaStream_t s, int nvec) {
  if (ncells <= first) return cudaSuccess;
  amr_prolong_kernel<<<grid_for((long)(ncells - first) * F, kThreads), kThreads, 0, s>>>(
      yn, k1, k2, k3, k4, pfs, psy, psz, cells, first, ncells, store, F, w, nvec);
  return cudaGetLastError();
}

cudaError_t launch_amr_prolong_tiles(const double* yn, const double* k1, const double* k2, const double* k3,
                                     const double* k4, long pfs, int psy, int psz, const AmrTile* tiles, int ntiles,
                                     const int32_t* slots, int ncells, double* store, int F, const Weights& w,
                                     cudaStream_t s, int nvec) {
  if (ntiles == 0) return cudaSuccess;
  const long items = (long)ntiles * ((nvec * F + 1) / 2);
  const long cap = sm_count() * 6L * 8;
  const int grid = (int)(items < cap ? items : cap);
  amr_prolong_tile_kernel<<<grid, 256, 0, s>>>(yn, k1, k2, k3, k4, pfs, psy, psz, tiles, ntiles, slots, ncells, store,
                                               F, w, nvec);
  return cudaGetLastError();
}

cudaError_t launch_amr_apply(double* vec, long fs, int F, const AmrCell* cells, int ncells, const double* store,
                             const double* c4, cudaStream_t s, int nk) {
  if (ncells == 0) return cudaSuccess;
  amr_apply_kernel<<<grid_for((long)ncells * F, kThreads), kThreads, 0, s>>>(vec, fs, F, cells, ncells, store, c4[0],
                                                                            c4[1], c4[2], c4[3], nk);
  return cudaGetLastError();
}

cudaError_t launch_restrict(double* parent, long pfs, const double* fine, long ffs, int fsy, int fsz,
                            const RestrictCell* cells, int ncells, int F, const Weights& w, cudaStream_t s) {
  if (ncells == 0) return cudaSuccess;
  restrict_kernel<<<grid_for((long)ncells * F, kThreads), kThreads, 0, s>>>(parent, pfs, fine, ffs, fsy, fsz, cells,
                                                                           ncells, F, w);
  return cudaGetLastError();
}

cudaError_t launch_restrict_blocks(double* parent, long pfs, int psy, int psz, const double* fine, long ffs, int fsy,
                                   int fsz, const RestrictBlock* blocks, int nblocks, int F, const Weights& w,
                                   cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  const long pairs = ((long)nblocks * F + 1) / 2;
  const long cap = sm_count() * 10L;
  const int grid = (int)(pairs < cap ? pairs : cap);
  restrict_block_kernel<<<grid, 128, 0, s>>>(parent, pfs, psy, psz, fine, ffs, fsy, fsz, blocks, nblocks, F, w);
  return cudaGetLastError();
}

cudaError_t launch_periodic_copy(double* vec, long fs, int F, const int2* pairs, int npairs, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  periodic_copy_kernel<<<grid_for((long)npairs * F, kThreads), kThreads, 0, s>>>(vec, fs, F, pairs, npairs);
  return cudaGetLastError();
}

cudaError_t launch_initial_data(double* vec, const Geom& g, int F, int system, int kind, const double* params,
                                int nparams, cudaStream_t s) {
  IdParams ip;
  for (int i = 0; i < 8; ++i) ip.p[i] = (i < nparams) ? params[i] : 0.0;
  const long n = (long)g.ext[0] * g.ext[1] * g.ext[2];
  initial_data_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(vec, g, F, system, kind, ip);
  return cudaGetLastError();
}

cudaError_t launch_transfer_copy(double* dst, long dfs, const double* src, long sfs, const int2* pairs, int n, int F,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  transfer_copy_kernel<<<grid_for((long)n * F, kThreads), kThreads, 0, s>>>(dst, dfs, src, sfs, pairs, n, F);
  return cudaGetLastError();
}

cudaError_t launch_prolong_state(double* dst, long dfs, const double* parent, long pfs, int psy, int psz,
                                 const AmrCell* cells, int n, int F, const Weights& w, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  prolong_state_kernel<<<grid_for((long)n * F, kThreads), kThreads, 0, s>>>(dst, dfs, parent, pfs, psy, psz, cells, n,
                                                                           F, w);
  return cudaGetLastError();
}

cudaError_t launch_interpolate(const InterpPoint* pts, int n, double* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  interpolate_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(pts, n, out);
  return cudaGetLastError();
}

cudaError_t launch_eta_profile(double* eta, const Geom& g, double eta_c, double eta_s, double eta_o, cudaStream_t s) {
  const long n = (long)g.ext[0] * g.ext[1] * g.ext[2];
  eta_profile_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(eta, g, eta_c, eta_s, eta_o);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* vec, const Geom& g, const int* lo, const int* n, double* dst, cudaStream_t s) {
  const long cnt = (long)n[0] * n[1] * n[2];
  pack_kernel<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(const_cast<double*>(vec), g.pitch, g.ext[1],
                                                          lo[0] - g.org[0], lo[1] - g.org[1], lo[2] - g.org[2],
                                                          n[0], n[1], n[2], dst, 0);
  return cudaGetLastError();
}

cudaError_t launch_unpack(double* vec, const Geom& g, const int* lo, const int* n, const double* src, cudaStream_t s) {
  const long cnt = (long)n[0] * n[1] * n[2];
  pack_kernel<<<grid_for(cnt, kThreads), kThreads, 0, s>>>(vec, g.pitch, g.ext[1], lo[0] - g.org[0],
                                                          lo[1] - g.org[1], lo[2] - g.org[2], n[0], n[1], n[2],
                                                          const_cast<double*>(src), 1);
  return cudaGetLastError();
}

cudaError_t launch_pack_fields(double* vec, long fs, int F, const Geom& g, const int* lo, const int* n, double* buf,
                               int unpack, cudaStream_t s) {
  const long rows = (long)n[1] * n[2] * F;
  if (rows == 0 || n[0] == 0) return cudaSuccess;
  const long warps_per_block = kThreads / 32;
  long blocks = (rows + warps_per_block - 1) / warps_per_block;
  if (blocks > sm_count() * 16L) blocks = sm_count() * 16L;
  pack_fields_kernel<<<(int)blocks, kThreads, 0, s>>>(vec, fs, F, g.pitch, g.ext[1], lo[0] - g.org[0], lo[1] - g.org[1],
                                                      lo[2] - g.org[2], n[0], n[1], n[2], buf, unpack);
  return cudaGetLastError();
}

cudaError_t launch_nonfinite_check(const double* vec, long fs, int F, const Tile* tiles, int ntiles, int sy, int sz,
                                   int* flag, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  nonfinite_kernel<<<ntiles < sm_count() * 8 ? ntiles : sm_count() * 8, kThreads, 0, s>>>(vec, fs, F, tiles, ntiles, sy, sz, flag);
  return cudaGetLastError();
}

}  // namespace sc
