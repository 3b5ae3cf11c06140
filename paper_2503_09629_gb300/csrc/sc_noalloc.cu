// sc_noalloc.cu -- Z4c constraints of one caller-supplied box without any
// device allocation.
//
// Some callers cannot allocate device memory themselves or through this
// library: a solver plugged into a host application that owns every byte of
// device memory and forbids other allocations, a process whose memory pool is
// fixed at start-up, or a latency-critical loop in which cudaMalloc/cudaFree
// would implicitly synchronise the device and stall unrelated work.  For them
// this file provides sc_z4c_constraints_noalloc: the derivative and
// constraint kernels of sc_get_constraints (4th-order centred differences on 3
// ghost layers, whatever order a context evolves with), with the derivative
// scratch and the tile list held in file-scope static device arrays instead of
// memory a context allocated.
//
// Limits and sharing rules (also stated in include/subcyc.h):
//   * the scratch holds 154 derivative values per ghosted cell for at most
//     kNoallocMaxCells = 32768 ghosted cells (e.g. a 26^3 interior), i.e.
//     40,370,176 bytes, plus a tile list of at most 8192 entries; every GPU
//     that loads this library holds these arrays until the process exits;
//   * every call shares the arrays; calls that overlap on the GPU (different
//     streams, or different host threads on the same device) race and must
//     be serialised by the caller;
//   * nothing in the arrays needs to start at zero: each call first writes
//     its tile list on the device, and the derivative pass writes every
//     scratch value the constraint pass then reads.
//   * the call makes no host-to-device copy: the tile list is generated by a
//     kernel from the box extents, so the call returns without waiting for
//     the stream's earlier work.
#include <stdio.h>

#include <mutex>

#include "sc_internal.h"

namespace {

constexpr long kNoallocMaxCells = 32768;  // ghosted cells of the largest accepted box
constexpr int kNoallocScratchSlots = 154;  // derivative values per cell (scratch layout of sc_z4c.cu)
constexpr int kNoallocMaxTiles = 8192;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchSlots * kNoallocMaxCells];
static __device__ __align__(256) sc::Tile g_noalloc_tiles[kNoallocMaxTiles];

constexpr int kTileX = 32, kTileY = 4, kTileZ = 2;  // the tile shape sc_get_constraints uses

// Interior tiles of an nx x ny x nz box with 3 ghost layers, x fastest, in
// the order sc_get_constraints builds them; written straight into the static
// tile array (device code may name it directly).
__global__ void noalloc_tiles_kernel(int nx, int ny, int nz, int tx, int ty, int nt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const int ix = t % tx, iy = (t / tx) % ty, iz = t / (tx * ty);
    sc::Tile T;
    T.x0 = ix * kTileX + sc::kGhost;
    T.y0 = iy * kTileY + sc::kGhost;
    T.z0 = iz * kTileZ + sc::kGhost;
    T.nx = nx - ix * kTileX < kTileX ? nx - ix * kTileX : kTileX;
    T.ny = ny - iy * kTileY < kTileY ? ny - iy * kTileY : kTileY;
    T.nz = nz - iz * kTileZ < kTileZ ? nz - iz * kTileZ : kTileZ;
    g_noalloc_tiles[t] = T;
  }
}

struct DeviceSymbols {
  bool ready = false;
  double* scratch = nullptr;
  sc::Tile* tiles = nullptr;
};

std::mutex g_setup_mutex;
DeviceSymbols g_symbols[kMaxDevices];

sc_status noalloc_fail(sc_status code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess) snprintf(buf, sizeof(buf), "sc_z4c_constraints_noalloc: %s: %s", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof(buf), "sc_z4c_constraints_noalloc: %s", msg);
  return sc::set_last_error(code, buf);
}

// Device addresses of the static arrays on the current device.  Host code
// must not pass the arrays' names to a kernel (in host code they are only
// host-side stand-ins), so the addresses are looked up once per device, with
// that device current, and cached.
sc_status device_symbols(DeviceSymbols** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SC_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSymbols& s = g_symbols[dev];
  if (!s.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "cudaGetSymbolAddress(scratch)", e);
    s.scratch = static_cast<double*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
    if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "cudaGetSymbolAddress(tiles)", e);
    s.tiles = static_cast<sc::Tile*>(p);
    s.ready = true;
  }
  *out = &s;
  return SC_OK;
}

}  // namespace

extern "C" sc_status sc_z4c_constraints_noalloc(const double* dev_state, double* dev_out, const int* n, double h,
                                                void* cuda_stream) {
  if (!dev_state || !dev_out || !n) return noalloc_fail(SC_EINVAL, "null argument");
  if (n[0] < 1 || n[1] < 1 || n[2] < 1 || !(h > 0)) return noalloc_fail(SC_EINVAL, "box extents and spacing must be positive");
  // each extent alone is bounded before the volume is formed, so the product cannot overflow
  for (int d = 0; d < 3; ++d)
    if (n[d] > kNoallocMaxCells)
      return noalloc_fail(SC_EINVAL, "box too large: at most 32768 cells including 3 ghost layers per side");
  const long ext[3] = {n[0] + 2L * sc::kGhost, n[1] + 2L * sc::kGhost, n[2] + 2L * sc::kGhost};
  const long vol = ext[0] * ext[1] * ext[2];
  if (vol > kNoallocMaxCells)
    return noalloc_fail(SC_EINVAL, "box too large: at most 32768 cells including 3 ghost layers per side");
  // interior tiles of the box, in the shape the context uses (32 x 4 x 2)
  const int tx = (n[0] + kTileX - 1) / kTileX, ty = (n[1] + kTileY - 1) / kTileY, tz = (n[2] + kTileZ - 1) / kTileZ;
  const long nt = (long)tx * ty * tz;
  if (nt > kNoallocMaxTiles) return noalloc_fail(SC_EINVAL, "box too thin: more than 8192 tiles");
  DeviceSymbols* sym = nullptr;
  sc_status st = device_symbols(&sym);
  if (st != SC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  noalloc_tiles_kernel<<<(int)((nt + 127) / 128), 128, 0, s>>>(n[0], n[1], n[2], tx, ty, (int)nt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "tile kernel", e);
  const long fs = vol;  // state: field stride = ghosted box volume
  const int sy = (int)ext[0], sz = (int)(ext[0] * ext[1]);
  e = sc::launch_z4c_derivs(dev_state, sym->scratch, fs, sy, sz, sym->tiles, (int)nt, s);
  if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "derivative kernel", e);
  const int lo[3] = {sc::kGhost, sc::kGhost, sc::kGhost};
  const sc::Z4cParams p{0.0, 0.0, 0.0, 0.0};  // the constraints do not depend on the damping/gauge parameters
  e = sc::launch_z4c_constraints(dev_state, sym->scratch, dev_out, fs, sy, sz, p, sc::deriv_scales(4, h), sym->tiles, (int)nt,
                                 (long)n[0] * n[1] * n[2], lo, n, s);
  if (e != cudaSuccess) return noalloc_fail(SC_ECUDA, "constraint kernel", e);
  return SC_OK;
}
