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
#include "sc_internal.h"

namespace sc {
namespace {

constexpr int kThreads = 256;

template <int ORD>
__global__ void __launch_bounds__(kThreads) wave_stage_kernel(StageArgs a, const Tile* __restrict__ tiles,
                                                             int ntiles, FmaK K) {
  const double inv12h2 = ORD == 4 ? 1.0 / (12.0 * a.h * a.h) : 1.0 / (5040.0 * a.h * a.h);
  const long sy = a.sy, sz = a.sz;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = tiles[t];
    const int n = T.nx * T.ny * T.nz;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int i = q % T.nx;
      const int j = (q / T.nx) % T.ny;
      const int k = q / (T.nx * T.ny);
      const long o = (T.z0 + k) * sz + (T.y0 + j) * sy + (T.x0 + i);
      const double* u = a.Y;
      const double u0 = u[o];
      // 4th order: -1, 16, -30, 16, -1 over offsets -2..2 in each dimension, / (12 h^2);
      // 8th order: -9, 128, -1008, 8064, -14350, ... over -4..4, / (5040 h^2)
      // sm = sum over the 6 neighbours at distance m, in FMA form (bitwise the plain sums)
      auto ring = [&](int m) {
        return fadd(fadd(fadd(u[o - m], u[o + m], K), fadd(u[o - m * sy], u[o + m * sy], K), K),
                    fadd(u[o - m * sz], u[o + m * sz], K), K);
      };
      const double s1 = ring(1), s2 = ring(2);
      double lap;
      if (ORD == 4) {
        lap = fmul(fma(-90.0, u0, fma(16.0, s1, -s2)), inv12h2, K);
      } else {
        const double s3 = ring(3), s4 = ring(4);
        lap = fmul(fma(-43050.0, u0, fma(8064.0, s1, fma(-1008.0, s2, fma(128.0, s3, fmul(-9.0, s4, K))))), inv12h2,
                   K);
      }
      const double ku = a.Y[a.fs + o];  // d_t u = Pi
      const double kp = lap;            // d_t Pi = Laplacian u
      a.k[o] = ku;
      a.k[a.fs + o] = kp;
      if (a.form == kStageSingle) {
        a.out[o] = fma(a.cdt, ku, a.yn[o]);
        a.out[a.fs + o] = fma(a.cdt, kp, a.yn[a.fs + o]);
      } else if (a.form == kStageRk4) {
        const double su = fadd(fma(2.0, a.k3[o], fma(2.0, a.k2[o], a.k1[o])), ku, K);
        const double sp = fadd(fma(2.0, a.k3[a.fs + o], fma(2.0, a.k2[a.fs + o], a.k1[a.fs + o])), kp, K);
        a.out[o] = fma(a.cdt, su, a.yn[o]);
        a.out[a.fs + o] = fma(a.cdt, sp, a.yn[a.fs + o]);
      } else if (a.form == kStageTwo) {
        a.out[o] = fma(a.cdt, ku, fma(a.c1dt, a.k1[o], a.yn[o]));
        a.out[a.fs + o] = fma(a.cdt, kp, fma(a.c1dt, a.k1[a.fs + o], a.yn[a.fs + o]));
      }
    }
  }
}

// Outgoing radiative condition on the outer ghost shell of a radiative
// level 0 (the boundary cells are evolved with their own right-hand side):
//   d_t u = -(x^i / r) d_i u - (u - u_inf) / r
// with 2nd-order differences, centred where both neighbours exist in the
// array and one-sided inwards on its outermost layer; u_inf = 1 for W,
// alpha and the diagonal of gt, 0 otherwise.
__global__ void __launch_bounds__(kThreads) radiative_stage_kernel(StageArgs a, const int32_t* __restrict__ cells,
                                                                  int ncells, int F, Geom g, int system) {
  const double inv2h = 1.0 / (2.0 * a.h);
  const long str[3] = {1, (long)a.sy, (long)a.sz};
  const long total = (long)ncells * F;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % ncells);
    const int f = (int)(idx / ncells);
    const long o = cells[c];
    const int ijk[3] = {(int)(o % g.pitch), (int)((o / g.pitch) % g.ext[1]), (int)(o / ((long)g.pitch * g.ext[1]))};
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = g.x0[d] + ijk[d] * g.h;
    const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const double ir = rsqrt(r2);
    const double* p = a.Y + (long)f * a.fs;
    double adv = 0.0;
    for (int d = 0; d < 3; ++d) {
      const long s = str[d];
      double der;
      if (ijk[d] == 0) der = (-3.0 * p[o] + 4.0 * p[o + s] - p[o + 2 * s]) * inv2h;
      else if (ijk[d] == g.ext[d] - 1) der = (3.0 * p[o] - 4.0 * p[o - s] + p[o - 2 * s]) * inv2h;
      else der = (p[o + s] - p[o - s]) * inv2h;
      adv = fma(x[d], der, adv);
    }
    double uinf = 0.0;
    if (system == SC_Z4C && (f == ZW || f == ZAL || f == ZG + 0 || f == ZG + 3 || f == ZG + 5)) uinf = 1.0;
    const double kv = -(adv + (p[o] - uinf)) * ir;
    const long fo = (long)f * a.fs + o;
    a.k[fo] = kv;
    if (a.form == kStageSingle) {
      a.out[fo] = fma(a.cdt, kv, a.yn[fo]);
    } else if (a.form == kStageRk4) {
      const double s = fma(2.0, a.k3[fo], fma(2.0, a.k2[fo], a.k1[fo])) + kv;
      a.out[fo] = fma(a.cdt, s, a.yn[fo]);
    } else if (a.form == kStageTwo) {
      a.out[fo] = fma(a.cdt, kv, fma(a.c1dt, a.k1[fo], a.yn[fo]));
    }
  }
}

}  // namespace

cudaError_t launch_wave_stage(const StageArgs& a, const Tile* tiles, int ntiles, cudaStream_t s, int order) {
  if (ntiles == 0) return cudaSuccess;
  const int grid = ntiles < 152 * 16 ? ntiles : 152 * 16;
  const FmaK K{1.0, -1.0, -0.0};
  if (order == 8) wave_stage_kernel<8><<<grid, kThreads, 0, s>>>(a, tiles, ntiles, K);
  else wave_stage_kernel<4><<<grid, kThreads, 0, s>>>(a, tiles, ntiles, K);
  return cudaGetLastError();
}

cudaError_t launch_radiative_stage(const StageArgs& a, const int32_t* cells, int ncells, int F, const Geom& g,
                                   int system, cudaStream_t s) {
  if (ncells == 0) return cudaSuccess;
  const long work = (long)ncells * F;
  long grid = (work + kThreads - 1) / kThreads;
  if (grid > 152 * 32) grid = 152 * 32;
  radiative_stage_kernel<<<(int)grid, kThreads, 0, s>>>(a, cells, ncells, F, g, system);
  return cudaGetLastError();
}

}  // namespace sc
