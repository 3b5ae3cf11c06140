// sc_wave.cu -- fused RK4 stage for the scalar wave (Sec. IV.A) and the
// radiative outer-boundary stage shared by both systems.
//
// One launch covers every interior tile of a level: k_i = f(Y_i) with the
// centred Laplacian (4th or 8th order), then the stage update
//   Y_{i+1} = y_n + c_{i+1} dt k_i                 (Eqs. rk2-rk4 stage vectors)
//   y_{n+1} = y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4)   (RK4's last stage, Eq. rk5)
// or the last-stage combinations of RK3 (y_n + dt/4 k1 + 3dt/4 k3) and RK2
// (y_n + dt k2), or no update (RK3's k4 = f(y_{n+1})).  k_i is stored because
// finer levels need it for dense output.
#include "sc_device.cuh"

namespace sc {
namespace {

constexpr int kThreads = 256;

template <int ORD>
__global__ void __launch_bounds__(kThreads) wave_stage_kernel(StageArgs a, const Tile* __restrict__ tiles,
                                                             int ntiles, FmaK K, ApplyArgs fill) {
  wave_stage_body<ORD>(a, tiles, ntiles, K, blockIdx.x, gridDim.x);
  if (fill.ncells)
    amr_apply_body(fill.vec, fill.fs, fill.F, fill.cells, fill.ncells, fill.store, fill.c[0], fill.c[1], fill.c[2],
                   fill.c[3], fill.nk, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads) radiative_stage_kernel(StageArgs a, const int32_t* __restrict__ cells,
                                                                  int ncells, int F, Geom g, int system) {
  radiative_stage_body(a, cells, ncells, F, g, system, blockIdx.x, gridDim.x);
}

}  // namespace

cudaError_t launch_wave_stage(const StageArgs& a, const Tile* tiles, int ntiles, cudaStream_t s, int order,
                              const ApplyArgs* fill) {
  ApplyArgs f{};
  if (fill) f = *fill;
  const long fill_blocks = ((long)f.ncells * f.F + kThreads - 1) / kThreads;
  long work = ntiles > fill_blocks ? ntiles : fill_blocks;
  if (work == 0) return cudaSuccess;
  const int grid = (int)(work < sm_count() * 16L ? work : sm_count() * 16L);
  const FmaK K{1.0, -1.0, -0.0};
  if (order == 8) wave_stage_kernel<8><<<grid, kThreads, 0, s>>>(a, tiles, ntiles, K, f);
  else wave_stage_kernel<4><<<grid, kThreads, 0, s>>>(a, tiles, ntiles, K, f);
  return cudaGetLastError();
}

cudaError_t launch_radiative_stage(const StageArgs& a, const int32_t* cells, int ncells, int F, const Geom& g,
                                   int system, cudaStream_t s) {
  if (ncells == 0) return cudaSuccess;
  const long work = (long)ncells * F;
  long grid = (work + kThreads - 1) / kThreads;
  if (grid > sm_count() * 32L) grid = sm_count() * 32L;
  radiative_stage_kernel<<<(int)grid, kThreads, 0, s>>>(a, cells, ncells, F, g, system);
  return cudaGetLastError();
}

}  // namespace sc
