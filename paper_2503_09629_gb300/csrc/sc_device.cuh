// sc_device.cuh -- bodies of the refinement-boundary, ghost-copy and wave
// stage kernels as device functions over an explicit worker range.
//
// Each body distributes its work over `nb` workers (thread blocks) of which
// this block is number `bid`, with the block's threads as lanes.  The
// stand-alone kernels call them with (blockIdx.x, gridDim.x); the persistent
// coarse-step kernel calls the same functions, phase after phase, with its
// own block range, so both forms execute identical arithmetic per value.
#pragma once

#include "sc_internal.h"

namespace sc {

// Sec. II step 2, per-cell form: tensor-product quintic Lagrange prolongation
// of y_n and the stage vectors the dense output reads (the first nvec of yn,
// k1..k4) from 6x6x6 parent cells to refinement-boundary ghost cells
// [first, ncells); results go to store[(v * F + f) * ncells + cell].
__device__ __forceinline__ void amr_prolong_cells_body(const double* __restrict__ yn, const double* __restrict__ k1,
                                                       const double* __restrict__ k2, const double* __restrict__ k3,
                                                       const double* __restrict__ k4, long pfs, int psy, int psz,
                                                       const AmrCell* __restrict__ cells, int first, int ncells,
                                                       double* __restrict__ store, int F, const Weights& w, int nvec,
                                                       int bid, int nb) {
  const int nc = ncells - first;
  const long total = (long)nc * F;
  for (long idx = bid * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)nb * blockDim.x) {
    const int a = first + (int)(idx % nc);
    const int f = (int)(idx / nc);
    const AmrCell c = cells[a];
    const double* wx = w.prolong[c.parity & 1];
    const double* wy = w.prolong[(c.parity >> 1) & 1];
    const double* wz = w.prolong[(c.parity >> 2) & 1];
    const double* src[5] = {yn, k1, k2, k3, k4};
#pragma unroll 1
    for (int v = 0; v < nvec; ++v) {
      const double* p = src[v] + (long)f * pfs + c.pbase;
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
      store[((long)v * F + f) * ncells + a] = sz;
    }
  }
}

// Offset of the first stencil node of fine position i along one axis from
// the first node of a tile's parent region, for a tile whose first fine
// position has parity p0 (parity 0: the fine centre sits at -1/4 parent cell
// and uses nodes c-3..c+2; parity 1: +1/4 and c-2..c+3).
__device__ __forceinline__ int tile_node_offset(int p0, int i) { return ((p0 + i) >> 1) + ((p0 + i) & 1) - p0; }

// Shared-memory doubles the tile-separable prolongation needs per group of
// 128 threads: the parent region (at most 10 x 10 x 8 nodes), the x sums (at
// most 8 x 10 x 8) and the y sums (at most 8 x 8 x 8).
constexpr int kTileRegion = 800, kTileXSums = 640, kTileYSums = 512;
constexpr int kProlongSmemPerGroup = kTileRegion + kTileXSums + kTileYSums;

// Separable form of the same interpolation for the slab tiles of a ghost
// shell: one group of 128 threads per (tile, vector, field) stages the
// tile's parent region in shared memory and interpolates along x, then y,
// then z.  Each value is the same chain of fused multiply-adds as in the
// per-cell form (x sums over six nodes from zero, then y sums of those, then
// z sums), so both give identical results.  Along the thin axis of a slab
// tile (the ghost width) the sums shrink 7-8 nodes to 3-4 values, so a ghost
// value costs about 20-40 FMAs instead of the 216 + 42 of the per-cell form.
// ngrp groups of 128 threads (threads beyond them idle); sm: ngrp *
// kProlongSmemPerGroup doubles.  Every thread of the block must call this
// function (it synchronises the block).
__device__ __forceinline__ void amr_prolong_tiles_body(const double* __restrict__ yn, const double* __restrict__ k1,
                                                       const double* __restrict__ k2, const double* __restrict__ k3,
                                                       const double* __restrict__ k4, long pfs, int psy, int psz,
                                                       const AmrTile* __restrict__ tiles, int ntiles,
                                                       const int32_t* __restrict__ slots, int ncells,
                                                       double* __restrict__ store, int F, const Weights& w, int nvec,
                                                       int bid, int nb, double* sm, int ngrp) {
  const int grp = threadIdx.x >> 7, t = threadIdx.x & 127;
  double* sR = sm + grp * kProlongSmemPerGroup;
  double* sX = sR + kTileRegion;
  double* sY = sX + kTileXSums;
  const int combos = nvec * F;
  const int ngroups = (combos + ngrp - 1) / ngrp;
  const long items = (long)ntiles * ngroups;
  for (long item = bid; item < items; item += nb) {
    const int b = (int)(item / ngroups);
    const int combo = (int)(item % ngroups) * ngrp + grp;
    const bool active = grp < ngrp && combo < combos;
    const AmrTile T = tiles[b];
    const int ex = T.ext[0], ey = T.ext[1], ez = T.ext[2];
    const int px = T.par & 1, py = (T.par >> 1) & 1, pz = (T.par >> 2) & 1;
    const int Nx = tile_node_offset(px, ex - 1) + kPN, Ny = tile_node_offset(py, ey - 1) + kPN;
    const int Nz = tile_node_offset(pz, ez - 1) + kPN;
    const int v = active ? combo / F : 0, f = active ? combo % F : 0;
    if (active) {
      const double* base = (v == 0 ? yn : v == 1 ? k1 : v == 2 ? k2 : v == 3 ? k3 : k4) + (long)f * pfs + T.pbase;
      for (int q = t; q < Nx * Ny * Nz; q += 128) {
        const int x = q % Nx, r = q / Nx;
        sR[q] = __ldg(base + (long)(r / Ny) * psz + (long)(r % Ny) * psy + x);  // [z][y][x]
      }
    }
    __syncthreads();
    if (active) {  // x: each (y, z) row of nodes to the tile's ex fine positions
      for (int q = t; q < ex * Ny * Nz; q += 128) {
        const int i = q % ex, r = q / ex;
        const int p = (px + i) & 1;
        const double* row = sR + r * Nx + tile_node_offset(px, i);
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < kPN; ++m) s = fma(w.prolong[p][m], row[m], s);
        sX[q] = s;  // [z][y][i]
      }
    }
    __syncthreads();
    if (active) {  // y
      for (int q = t; q < ex * ey * Nz; q += 128) {
        const int i = q % ex, j = (q / ex) % ey, z = q / (ex * ey);
        const int p = (py + j) & 1;
        const double* col = sX + (z * Ny + tile_node_offset(py, j)) * ex + i;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < kPN; ++m) s = fma(w.prolong[p][m], col[m * ex], s);
        sY[q] = s;  // [z][j][i]
      }
    }
    __syncthreads();
    if (active) {  // z, then store the claimed positions
      for (int q = t; q < ex * ey * ez; q += 128) {
        const int ij = q % (ex * ey), k = q / (ex * ey);
        const int p = (pz + k) & 1;
        const double* col = sY + tile_node_offset(pz, k) * ex * ey + ij;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < kPN; ++m) s = fma(w.prolong[p][m], col[m * ex * ey], s);
        const int slot = slots[T.slot_base + q];
        if (slot >= 0) store[((long)v * F + f) * ncells + slot] = s;
      }
    }
    __syncthreads();
  }
}

// Sec. II steps 3/5: ghost value = P[y_n] + sum_j c_j P[k_j] over the nk
// prolonged stage vectors in the store (4 for RK4, 3 for RK3, 2 for RK2, 0
// for a plain prolonged value); the coefficients encode dense output (Eqs.
// denseoutput1/2) and the Taylor stage formulas (Eqs. Y1-Y4) for one stage of
// one fine substep.
__device__ __forceinline__ void amr_apply_body(double* __restrict__ vec, long fs, int F,
                                               const AmrCell* __restrict__ cells, int ncells,
                                               const double* __restrict__ store, double c1, double c2, double c3,
                                               double c4, int nk, int bid, int nb) {
  const long total = (long)ncells * F;
  for (long idx = bid * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)nb * blockDim.x) {
    const int a = (int)(idx % ncells);
    const int f = (int)(idx / ncells);
    const long n = ncells;
    const double* s = store + (long)f * n + a;
    const long vs = (long)F * n;
    double v = s[0];
    if (nk > 0) v = fma(c1, s[vs], v);
    if (nk > 1) v = fma(c2, s[2 * vs], v);
    if (nk > 2) v = fma(c3, s[3 * vs], v);
    if (nk > 3) v = fma(c4, s[4 * vs], v);
    vec[(long)f * fs + cells[a].dst] = v;
  }
}

// Periodic images: ghost cell <- the wrapped interior cell (pairs: x =
// destination offset, y = source offset).
__device__ __forceinline__ void periodic_copy_body(double* __restrict__ vec, long fs, int F,
                                                   const int2* __restrict__ pairs, int npairs, int bid, int nb) {
  const long total = (long)npairs * F;
  for (long idx = bid * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)nb * blockDim.x) {
    const int a = (int)(idx % npairs);
    const int f = (int)(idx / npairs);
    const int2 p = pairs[a];
    vec[(long)f * fs + p.x] = vec[(long)f * fs + p.y];
  }
}

// Sec. II step 7, per-cell form: every parent cell whose eight children are
// fine interior cells takes the tensor-product quintic interpolant of the
// 6x6x6 fine cells centred on it.
__device__ __forceinline__ void restrict_cells_body(double* __restrict__ parent, long pfs,
                                                    const double* __restrict__ fine, long ffs, int fsy, int fsz,
                                                    const RestrictCell* __restrict__ cells, int ncells, int F,
                                                    const Weights& w, int bid, int nb) {
  const long total = (long)ncells * F;
  for (long idx = bid * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)nb * blockDim.x) {
    const int a = (int)(idx % ncells);
    const int f = (int)(idx / ncells);
    const RestrictCell c = cells[a];
    const double* p = fine + (long)f * ffs + c.fbase;
    double sz = 0.0;
#pragma unroll
    for (int kz = 0; kz < kRN; ++kz) {
      double sy = 0.0;
#pragma unroll
      for (int ky = 0; ky < kRN; ++ky) {
        const double* row = p + (long)kz * fsz + (long)ky * fsy;
        double sx = 0.0;
#pragma unroll
        for (int kx = 0; kx < kRN; ++kx) sx = fma(w.restrict_w[kx], __ldg(row + kx), sx);
        sy = fma(w.restrict_w[ky], sx, sy);
      }
      sz = fma(w.restrict_w[kz], sy, sz);
    }
    parent[(long)f * pfs + c.dst] = sz;
  }
}

// Shared-memory doubles the block-separable restriction needs per group.
constexpr int kRestrictSmemPerGroup = 1728 + 576 + 192;

// Separable form of the same restriction for 4x4x4 parent blocks: one group
// of 64 threads per (block, field) stages the 12x12x12 fine region in shared
// memory and sums along x, then y, then z (78 FMAs per parent cell instead of
// 216).  Each parent value is the same chain of fused multiply-adds as in the
// per-cell form (x sums, then y, then z, each from zero in stencil order), so
// both give identical results.  ngrp groups of 64 threads (threads beyond
// them idle); sm: ngrp * kRestrictSmemPerGroup doubles.  Every thread of the
// block must call this function (it synchronises the block).
__device__ __forceinline__ void restrict_blocks_body(double* __restrict__ parent, long pfs, int psy, int psz,
                                                     const double* __restrict__ fine, long ffs, int fsy, int fsz,
                                                     const RestrictBlock* __restrict__ blocks, int nblocks, int F,
                                                     const Weights& w, int bid, int nb, double* sm, int ngrp) {
  const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
  double* sF = sm + grp * 1728;
  double* sX = sm + ngrp * 1728 + grp * 576;
  double* sY = sm + ngrp * 2304 + grp * 192;
  const long items = (long)nblocks * F;
  const long chunks = (items + ngrp - 1) / ngrp;
  for (long it = bid; it < chunks; it += nb) {
    const long item = it * ngrp + grp;
    const bool active = grp < ngrp && item < items;
    const int b = active ? (int)(item / F) : 0, f = active ? (int)(item % F) : 0;
    const RestrictBlock B = blocks[b];
    if (active) {
      const double* src = fine + (long)f * ffs + B.fbase;
      for (int q = t; q < 1728; q += 64) {
        const int z = q / 144, y = (q / 12) % 12, x = q % 12;
        sF[q] = __ldg(src + (long)z * fsz + (long)y * fsy + x);
      }
    }
    __syncthreads();
    if (active) {  // x: row (z, y) of the fine region, parent px
      for (int q = t; q < 576; q += 64) {
        const int z = q / 48, y = (q / 4) % 12, px = q % 4;
        const double* row = &sF[(z * 12 + y) * 12 + 2 * px];
        double sx = 0.0;
#pragma unroll
        for (int m = 0; m < kRN; ++m) sx = fma(w.restrict_w[m], row[m], sx);
        sX[q] = sx;  // [z][y][px]
      }
    }
    __syncthreads();
    if (active) {  // y: fine z, parent (py, px)
      for (int q = t; q < 192; q += 64) {
        const int z = q / 16, py = (q / 4) % 4, px = q % 4;
        double sy = 0.0;
#pragma unroll
        for (int m = 0; m < kRN; ++m) sy = fma(w.restrict_w[m], sX[(z * 12 + 2 * py + m) * 4 + px], sy);
        sY[q] = sy;  // [z][py][px]
      }
    }
    __syncthreads();
    if (active && ((B.mask >> t) & 1ull)) {  // z: parent cell t = px + 4 py + 16 pz
      const int pz = t >> 4, py = (t >> 2) & 3, px = t & 3;
      double sz = 0.0;
#pragma unroll
      for (int m = 0; m < kRN; ++m) sz = fma(w.restrict_w[m], sY[((2 * pz + m) * 4 + py) * 4 + px], sz);
      parent[(long)f * pfs + B.pbase + (long)pz * psz + (long)py * psy + px] = sz;
    }
    __syncthreads();
  }
}

// Scalar-wave stage (Sec. IV.A): k_i = f(Y_i) with the centred Laplacian (4th
// or 8th order), then the stage update of StageArgs (Eqs. rk2-rk5 for RK4,
// the last-stage combinations of RK3/RK2, or k only).  One tile per worker
// at a time, the block's threads over its cells.
template <int ORD>
__device__ __forceinline__ void wave_stage_body(const StageArgs& a, const Tile* __restrict__ tiles, int ntiles,
                                                const FmaK& K, int bid, int nb) {
  const double inv12h2 = ORD == 4 ? 1.0 / (12.0 * a.h * a.h) : 1.0 / (5040.0 * a.h * a.h);
  const long sy = a.sy, sz = a.sz;
  for (int t = bid; t < ntiles; t += nb) {
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
__device__ __forceinline__ void radiative_stage_body(const StageArgs& a, const int32_t* __restrict__ cells,
                                                     int ncells, int F, const Geom& g, int system, int bid, int nb) {
  const double inv2h = 1.0 / (2.0 * a.h);
  const long str[3] = {1, (long)a.sy, (long)a.sz};
  const long total = (long)ncells * F;
  for (long idx = bid * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)nb * blockDim.x) {
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

// Non-finite scan of the interior tiles of one level array: sets bit
// kStatusNonFinite of *flag when any value is NaN or infinite.
__device__ __forceinline__ void nonfinite_body(const double* __restrict__ vec, long fs, int F,
                                               const Tile* __restrict__ tiles, int ntiles, int sy, int sz, int* flag,
                                               int bid, int nb) {
  for (int t = bid; t < ntiles; t += nb) {
    const Tile T = tiles[t];
    const int n = T.nx * T.ny * T.nz;
    for (int q = threadIdx.x; q < n * F; q += blockDim.x) {
      const int f = q / n, c = q % n;
      const int i = c % T.nx, j = (c / T.nx) % T.ny, k = c / (T.nx * T.ny);
      const double v = vec[(long)f * fs + (long)(T.z0 + k) * sz + (long)(T.y0 + j) * sy + T.x0 + i];
      if (!isfinite(v)) atomicOr(flag, kStatusNonFinite);
    }
  }
}

}  // namespace sc
