// sc_z4c.cu -- Z4c right-hand side (Sec. III.A, vacuum, puncture gauge with
// constant eta), Kreiss-Oliger dissipation (Sec. III.C, r = 4) and the fused
// RK4 stage update, plus the constraint evaluation.
//
// Two passes per stage, both over the interior tiles of a level:
//   1. the derivative pass computes the centred first derivatives of every
//      field, the second derivatives of W, gt_ij, alpha and beta^i, and the
//      KO sum sum_d delta_d^6 u, and stores them in a scratch array indexed
//      like the level array: scratch[q * fs + cell].  The stored values are
//      the stencils' integer-weight sums, without their 1/h and 1/h^2
//      factors (see DerivScales): a multiplication issues at the slower of
//      the two FP64 rates, and the consumers fold the factors into FMA
//      constants they evaluate anyway.
//   2. z4c_stage_kernel: one thread per cell reads the 22 fields and their
//      derivatives, evaluates the right-hand side, adds dissipation and
//      performs the RK4 stage update.
// FP64 is the scarce resource on this GPU (the FP64 pipe issues 1/64 of the
// FP32 rate), so the arithmetic is arranged to minimise FP64 operations:
// shared pair sums/differences in the stencils, fused multiply-adds, one
// division for 1/det(gt) and one for 1/W, and the quadratic Christoffel
// terms of the Ricci tensor contracted through one raised-index array.
#include "sc_internal.h"

namespace sc {
namespace {

constexpr int kThreads = 256;

// scratch slots
constexpr int Q_D1 = 0;    // 3 * f + d: first derivative of field f along d
constexpr int Q_D2 = 66;   // 6 * s + p: second derivative, s = slot (W, gt x6, alpha, beta x3), p = xx,xy,xz,yy,yz,zz
constexpr int Q_KO = 132;  // f: sum_d delta_d^6 u_f (unscaled)

// slot of field f among the fields with second derivatives, -1 if none
__host__ __device__ inline int d2_slot(int f) {
  if (f == ZW) return 0;
  if (f >= ZG && f < ZG + 6) return 1 + (f - ZG);
  if (f == ZAL) return 7;
  if (f >= ZB && f < ZB + 3) return 8 + (f - ZB);
  return -1;
}

// One-kernel form of the derivative pass (4th order): one thread per (cell,
// field), mixed derivatives from the direct 16-point product stencil.
// Stored scales as the two-kernel form: 12 h d_i u, 12 h^2 d_i^2 u,
// 144 h^2 d_i d_j u, and the raw Kreiss-Oliger sum.
__global__ void __launch_bounds__(kThreads) z4c_derivs_kernel(const double* __restrict__ Y, double* __restrict__ S,
                                                             long fs, int sy_, int sz_,
                                                             const Tile* __restrict__ tiles, int ntiles) {
  const long st[3] = {1, (long)sy_, (long)sz_};
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = tiles[t];
    const int n = T.nx * T.ny * T.nz;
    for (int q = threadIdx.x; q < n * kNZ4c; q += blockDim.x) {
      const int f = q / n;
      const int c = q - f * n;
      const int i = c % T.nx;
      const int j = (c / T.nx) % T.ny;
      const int k = c / (T.nx * T.ny);
      const long o = (T.z0 + k) * st[2] + (T.y0 + j) * st[1] + (T.x0 + i);
      const double* u = Y + (long)f * fs + o;
      const double u0 = u[0];
      double p1[3], p2[3], P3 = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const long s = st[d];
        const double a1 = u[-s], b1 = u[s], a2 = u[-2 * s], b2 = u[2 * s];
        p1[d] = a1 + b1;
        p2[d] = a2 + b2;
        P3 += u[-3 * s] + u[3 * s];
        // 12 h u' = u_-2 - 8 u_-1 + 8 u_1 - u_2
        S[(long)(Q_D1 + 3 * f + d) * fs + o] = fma(8.0, b1 - a1, a2 - b2);
      }
      // Kreiss-Oliger: sum_d (u_-3 - 6 u_-2 + 15 u_-1 - 20 u_0 + 15 u_1 - 6 u_2 + u_3)
      const double P1 = p1[0] + p1[1] + p1[2], P2 = p2[0] + p2[1] + p2[2];
      S[(long)(Q_KO + f) * fs + o] = fma(15.0, P1, fma(-6.0, P2, fma(-60.0, u0, P3)));
      const int sl = d2_slot(f);
      if (sl < 0) continue;
      double* d2 = S + (long)(Q_D2 + 6 * sl) * fs + o;
      // pure: 12 h^2 u'' = -u_-2 + 16 u_-1 - 30 u_0 + 16 u_1 - u_2
      d2[0 * fs] = fma(-30.0, u0, fma(16.0, p1[0], -p2[0]));
      d2[3 * fs] = fma(-30.0, u0, fma(16.0, p1[1], -p2[1]));
      d2[5 * fs] = fma(-30.0, u0, fma(16.0, p1[2], -p2[2]));
      // mixed: 144 h^2 d_i d_j u, the product of the two first-derivative stencils
      const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2}, slot[3] = {1, 2, 4};
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const long sa = st[pa[m]], sb = st[pb[m]];
        double D[4];
        const int offs[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const double* v = u + offs[r] * sb;
          D[r] = fma(8.0, v[sa] - v[-sa], v[-2 * sa] - v[2 * sa]);
        }
        d2[slot[m] * fs] = fma(8.0, D[2] - D[1], D[0] - D[3]);
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Evolution form of the derivative pass, in two kernels.  The mixed second
// derivatives are the product of two first-derivative stencils, so
//   d_x d_y u = D_y (D_x u),  d_x d_z u = D_z (D_x u),  d_y d_z u = D_z (D_y u)
// exactly (the same 16-point stencil, summed in another order).  The first
// kernel stores D_x u and D_y u of the 11 fields with second derivatives on
// row segments covering the interior and its 2-cell extension in y and z
// (D_x) or in z (D_y); the second kernel computes everything else per
// interior cell and differentiates the stored first derivatives for the
// mixed terms: 4 FP64 operations per mixed derivative instead of 16.

// field of Hessian slot s (W, gt x6, alpha, beta x3): slots 0..6 -> fields 0..6, 7..10 -> 18..21
__device__ __forceinline__ int d2_field(int s) { return s <= 6 ? s : s + 11; }

// The stencil sums are arranged for the FP64 issue rates of this GPU: a
// fused multiply-add whose multiplier is not +-1 and whose addend is not zero
// issues about 1.2x as fast as an addition (or a unit-multiplier FMA, or a
// multiplication).  So every weighted value enters through a general FMA, and
// only values of unit weight are added; pair sums v_m + v_-m are formed only
// where two sums share them.  lo[m] = v_-(m+1), hi[m] = v_(m+1).

// Centred first derivative as the integer-weight sum: 4th order
// 8 (v_1 - v_-1) - (v_2 - v_-2) (= 12 h u'), one addition and two FMAs;
// 8th order 672 d1 - 168 d2 + 32 d3 - 3 d4 (= 840 h u'), dm = v_m - v_-m.
template <int ORD, class KT>
__device__ __forceinline__ double dfirst(const double* lo, const double* hi, const KT& K) {
  if (ORD == 4) return fma(8.0, hi[0], fma(-8.0, lo[0], fsub(lo[1], hi[1], K)));
  return fma(672.0, hi[0],
             fma(-672.0, lo[0],
                 fma(-168.0, hi[1],
                     fma(168.0, lo[1], fma(32.0, hi[2], fma(-32.0, lo[2], fmul(3.0, fsub(lo[3], hi[3], K), K)))))));
}
// The same first derivative from the differences dm = v_m - v_-m, m = 1..R.
template <int ORD, class KT>
__device__ __forceinline__ double dfirst_d(const double* d, const KT& K) {
  if (ORD == 4) return fma(8.0, d[0], -d[1]);
  return fma(672.0, d[0], fma(-168.0, d[1], fma(32.0, d[2], fmul(-3.0, d[3], K))));
}
// Centred second derivative from the pair sums pm = v_m + v_-m, as the
// integer-weight sum: 4th order 16 p1 - p2 - 30 u0 (= 12 h^2 u''), 8th order
// 8064 p1 - 1008 p2 + 128 p3 - 9 p4 - 14350 u0 (= 5040 h^2 u'').
template <int ORD, class KT>
__device__ __forceinline__ double dsecond(const double* p, double u0, const KT& K) {
  if (ORD == 4) return fma(16.0, p[0], fma(-30.0, u0, -p[1]));
  return fma(-14350.0, u0, fma(8064.0, p[0], fma(-1008.0, p[1], fma(128.0, p[2], fmul(-9.0, p[3], K)))));
}

template <int ORD, class KT = FmaK>
__global__ void __launch_bounds__(128) z4c_dxy_kernel(const double* __restrict__ Y, double* __restrict__ S, long fs,
                                                     int sy_, const RowSeg* __restrict__ segs, int nsegs, KT K) {
  constexpr int R = ORD / 2;
  const long sy = sy_;
  for (int sgi = blockIdx.x; sgi < nsegs; sgi += gridDim.x) {
    const RowSeg sg = segs[sgi];
    for (int q = threadIdx.x; q < sg.n * 11; q += blockDim.x) {
      const int slot = q / sg.n;
      const long o = sg.off + (q - slot * sg.n);
      const int f = d2_field(slot);
      const double* u = Y + (long)f * fs + o;
      double lo[R], hi[R];
      if (sg.which & 1) {
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          lo[m - 1] = u[-m];
          hi[m - 1] = u[m];
        }
        S[(long)(Q_D1 + 3 * f + 0) * fs + o] = dfirst<ORD>(lo, hi, K);
      }
      if (sg.which & 2) {
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          lo[m - 1] = u[-m * sy];
          hi[m - 1] = u[m * sy];
        }
        S[(long)(Q_D1 + 3 * f + 1) * fs + o] = dfirst<ORD>(lo, hi, K);
      }
    }
  }
}

template <int ORD, class KT = FmaK>
__global__ void __launch_bounds__(kThreads, 2) z4c_derivs_split_kernel(const double* __restrict__ Y,
                                                                      double* __restrict__ S, long fs, int sy_,
                                                                      int sz_, const Tile* __restrict__ tiles, int ntiles,
                                                                      int max_cols, KT K) {
  // One thread per (x, y, field) column of a tile, walking z with sliding
  // windows: u at z-W..z+W (W = max(R, 3), R = ORD/2 the derivative radius,
  // 3 the Kreiss-Oliger radius) and, for the Hessian fields, the stored
  // D_x, D_y at z-R..z+R, so each step loads one new z value per window.
  // Work is dealt out in units of (tile, chunk of blockDim (field, column)
  // pairs), U chunks per tile (max_cols = the largest tile's columns), so
  // the persistent blocks end together whatever the tile count.
  constexpr int R = ORD / 2;
  constexpr int WR = R > 3 ? R : 3;
  constexpr int NW = 2 * WR + 1;
  constexpr int ND = 2 * R + 1;
  const long sy = sy_, sz = sz_;
  const int U = (max_cols * kNZ4c + blockDim.x - 1) / blockDim.x;
  for (long u = blockIdx.x; u < (long)ntiles * U; u += gridDim.x) {
    const int t = (int)(u / U);
    const Tile T = tiles[t];
    const int ncol = T.nx * T.ny;
    const int q = (int)(u - (long)t * U) * blockDim.x + threadIdx.x;
    if (q < ncol * kNZ4c) {
      const int f = q / ncol;
      const int c = q - f * ncol;
      const int i = c % T.nx;
      const int j = c / T.nx;
      const long o0 = (long)T.z0 * sz + (T.y0 + j) * sy + (T.x0 + i);
      const double* u = Y + (long)f * fs + o0;
      const int sl = d2_slot(f);
      double w[NW];  // u at z-WR..z+WR
#pragma unroll
      for (int m = 0; m < NW; ++m) w[m] = u[(m - WR) * sz];
      const double* Dx = S + (long)(Q_D1 + 3 * f + 0) * fs + o0;
      const double* Dy = S + (long)(Q_D1 + 3 * f + 1) * fs + o0;
      double wx[ND], wy[ND];  // D_x, D_y at z-R..z+R (Hessian fields)
      if (sl >= 0) {
#pragma unroll
        for (int m = 0; m < ND; ++m) {
          wx[m] = Dx[(m - R) * sz];
          wy[m] = Dy[(m - R) * sz];
        }
      }
      // 4th order: two z steps in flight (2.4% faster than one, measured); the
      // 8th-order windows leave no registers for that
#pragma unroll(ORD == 4 ? 2 : 1)
      for (int k = 0; k < T.nz; ++k) {
        const long o = o0 + k * sz;
        const double* v = u + k * sz;
        if (ORD == 4) {
          // 4th order: every weighted value through a general FMA (see dfirst)
          const double u0 = w[WR];
          // u along x and y from memory, along z from the window
          double lo[3][WR], hi[3][WR];
#pragma unroll
          for (int m = 1; m <= WR; ++m) {
            lo[0][m - 1] = v[-m];
            hi[0][m - 1] = v[m];
            lo[1][m - 1] = v[-m * sy];
            hi[1][m - 1] = v[m * sy];
            lo[2][m - 1] = w[WR - m];
            hi[2][m - 1] = w[WR + m];
          }
          // Kreiss-Oliger (r = 4): sum_d (u_-3 - 6 u_-2 + 15 u_-1 - 20 u_0 + 15 u_1 - 6 u_2 + u_3)
          double ko;
          if (sl < 0) {
#pragma unroll
            for (int dim = 0; dim < 3; ++dim) S[(long)(Q_D1 + 3 * f + dim) * fs + o] = dfirst<ORD>(lo[dim], hi[dim], K);
            ko = fma(-60.0, u0, lo[0][2]);
            ko = fadd(ko, hi[0][2], K);
#pragma unroll
            for (int dim = 1; dim < 3; ++dim) ko = fadd(fadd(ko, lo[dim][2], K), hi[dim][2], K);
#pragma unroll
            for (int dim = 0; dim < 3; ++dim)
              ko = fma(15.0, hi[dim][0], fma(15.0, lo[dim][0], fma(-6.0, hi[dim][1], fma(-6.0, lo[dim][1], ko))));
          } else {
            // Hessian fields: the pair sums of the second derivatives, shared with the KO sum
            double p[3][2];
#pragma unroll
            for (int dim = 0; dim < 3; ++dim)
#pragma unroll
              for (int m = 0; m < 2; ++m) p[dim][m] = fadd(lo[dim][m], hi[dim][m], K);
            double* d2 = S + (long)(Q_D2 + 6 * sl) * fs + o;
            d2[0 * fs] = dsecond<ORD>(p[0], u0, K);
            d2[3 * fs] = dsecond<ORD>(p[1], u0, K);
            d2[5 * fs] = dsecond<ORD>(p[2], u0, K);
            ko = fma(-60.0, u0, lo[0][2]);
            ko = fadd(ko, hi[0][2], K);
#pragma unroll
            for (int dim = 1; dim < 3; ++dim) ko = fadd(fadd(ko, lo[dim][2], K), hi[dim][2], K);
            // D_z from the pair sums: 16 v_1 - 8 p1 - 2 v_2 + p2 = 8 (v_1 - v_-1) - (v_2 - v_-2)
            S[(long)(Q_D1 + 3 * f + 2) * fs + o] =
                fma(16.0, hi[2][0], fma(-8.0, p[2][0], fma(-2.0, hi[2][1], p[2][1])));
#pragma unroll
            for (int dim = 0; dim < 3; ++dim) ko = fma(15.0, p[dim][0], fma(-6.0, p[dim][1], ko));
            // mixed: the first-derivative stencil applied to the stored D_x (along y and z) and D_y (along z)
            double ml[R], mh[R];
            const double* dxk = Dx + k * sz;
#pragma unroll
            for (int m = 1; m <= R; ++m) {
              ml[m - 1] = dxk[-m * sy];
              mh[m - 1] = dxk[m * sy];
            }
            d2[1 * fs] = dfirst<ORD>(ml, mh, K);  // D_y D_x
#pragma unroll
            for (int m = 1; m <= R; ++m) {
              ml[m - 1] = wx[R - m];
              mh[m - 1] = wx[R + m];
            }
            d2[2 * fs] = dfirst<ORD>(ml, mh, K);  // D_z D_x
#pragma unroll
            for (int m = 1; m <= R; ++m) {
              ml[m - 1] = wy[R - m];
              mh[m - 1] = wy[R + m];
            }
            d2[4 * fs] = dfirst<ORD>(ml, mh, K);  // D_z D_y
          }
          S[(long)(Q_KO + f) * fs + o] = ko;
        } else {
          // 8th order: differences and pair sums formed first (the 4th-order
          // arrangement ran 6% slower at radius 4, with or without spills)
          const double u0 = w[WR];
          double p[3][4], d[4];
          // x and y from memory, z from the window
#pragma unroll
          for (int dim = 0; dim < 2; ++dim) {
            const long s = dim == 0 ? 1 : sy;
#pragma unroll
            for (int m = 1; m <= WR; ++m) p[dim][m - 1] = fadd(v[-m * s], v[m * s], K);
            if (sl < 0) {
#pragma unroll
              for (int m = 1; m <= R; ++m) d[m - 1] = fsub(v[m * s], v[-m * s], K);
              S[(long)(Q_D1 + 3 * f + dim) * fs + o] = dfirst_d<ORD>(d, K);
            }
          }
#pragma unroll
          for (int m = 1; m <= WR; ++m) p[2][m - 1] = fadd(w[WR - m], w[WR + m], K);
#pragma unroll
          for (int m = 1; m <= R; ++m) d[m - 1] = fsub(w[WR + m], w[WR - m], K);
          S[(long)(Q_D1 + 3 * f + 2) * fs + o] = dfirst_d<ORD>(d, K);
          // Kreiss-Oliger (r = 4): sum_d (u_-3 - 6 u_-2 + 15 u_-1 - 20 u_0 + 15 u_1 - 6 u_2 + u_3)
          const double P1 = fadd(fadd(p[0][0], p[1][0], K), p[2][0], K);
          const double P2 = fadd(fadd(p[0][1], p[1][1], K), p[2][1], K);
          const double P3 = fadd(fadd(p[0][2], p[1][2], K), p[2][2], K);
          S[(long)(Q_KO + f) * fs + o] = fma(15.0, P1, fma(-6.0, P2, fma(-60.0, u0, P3)));
          if (sl >= 0) {
            double* d2 = S + (long)(Q_D2 + 6 * sl) * fs + o;
            d2[0 * fs] = dsecond<ORD>(p[0], u0, K);
            d2[3 * fs] = dsecond<ORD>(p[1], u0, K);
            d2[5 * fs] = dsecond<ORD>(p[2], u0, K);
            const double* dxk = Dx + k * sz;
#pragma unroll
            for (int m = 1; m <= R; ++m) d[m - 1] = fsub(dxk[m * sy], dxk[-m * sy], K);
            d2[1 * fs] = dfirst_d<ORD>(d, K);  // D_y D_x
#pragma unroll
            for (int m = 1; m <= R; ++m) d[m - 1] = fsub(wx[R + m], wx[R - m], K);
            d2[2 * fs] = dfirst_d<ORD>(d, K);  // D_z D_x
#pragma unroll
            for (int m = 1; m <= R; ++m) d[m - 1] = fsub(wy[R + m], wy[R - m], K);
            d2[4 * fs] = dfirst_d<ORD>(d, K);  // D_z D_y
          }
        }
        if (k + 1 < T.nz) {  // slide the windows one cell up in z
#pragma unroll
          for (int m = 0; m < NW - 1; ++m) w[m] = w[m + 1];
          w[NW - 1] = v[(WR + 1) * sz];
          if (sl >= 0) {
#pragma unroll
            for (int m = 0; m < ND - 1; ++m) {
              wx[m] = wx[m + 1];
              wy[m] = wy[m + 1];
            }
            wx[ND - 1] = Dx[(k + 1 + R) * sz];
            wy[ND - 1] = Dy[(k + 1 + R) * sz];
          }
        }
      }
    }
  }
}

// symmetric index helpers: xx xy xz yy yz zz
__device__ __forceinline__ int sidx(int i, int j) {
  return (i == j) ? (i == 0 ? 0 : (i == 1 ? 3 : 5)) : (i + j == 1 ? 1 : (i + j == 2 ? 2 : 4));
}

// Right-hand side of the Z4c system at one cell (Sec. III.A; vacuum, so the
// matter terms vanish).  u: fields; S + o: derivatives in scratch.  Sums,
// differences and products that do not fuse with a neighbour are written as
// fadd, fsub, fmul: FMAs with the run-time unit constants of an FmaK
// (measured faster than plain DADD/DMUL in this kernel), or the DADD/DMUL of
// a PlainK in the op-class build.
// The stored derivatives are stencil sums (DerivScales).  Their scales ride
// on factors formed once per cell where several terms share them (the 1/2 of
// the Christoffel symbols on the metric that raises their index, alpha, W,
// beta, Gamt and second-derivative coefficients) or on kernel-parameter
// constants of the FMAs that use them, so that each term stays one FMA and
// every equation accumulates in one chain.
template <bool kDiag, class KT>
__device__ __forceinline__ void z4c_rhs_point(const double* __restrict__ Y, const double* __restrict__ S, long fs,
                                              long o, const Z4cParams& P, double eta, const DerivScales& ds,
                                              double* rhs, double* diag, const KT& K) {
#define FLD(f) Y[(long)(f) * fs + o]
#define D1(f, d) S[(long)(Q_D1 + 3 * (f) + (d)) * fs + o]
#define D2(sl, p) S[(long)(Q_D2 + 6 * (sl) + (p)) * fs + o]
  const double W = FLD(ZW);
  double g[6], A[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    g[s] = FLD(ZG + s);
    A[s] = FLD(ZA + s);
  }
  const double Kh = FLD(ZK), Th = FLD(ZTH), al = FLD(ZAL);
  const double Gam[3] = {FLD(ZGAM), FLD(ZGAM + 1), FLD(ZGAM + 2)};
  const double be[3] = {FLD(ZB), FLD(ZB + 1), FLD(ZB + 2)};

  // inverse conformal metric
  double gu[6];
  gu[0] = fma(g[3], g[5], fmul(-g[4], g[4], K));
  gu[1] = fma(g[2], g[4], fmul(-g[1], g[5], K));
  gu[2] = fma(g[1], g[4], fmul(-g[2], g[3], K));
  gu[3] = fma(g[0], g[5], fmul(-g[2], g[2], K));
  gu[4] = fma(g[1], g[2], fmul(-g[0], g[4], K));
  gu[5] = fma(g[0], g[3], fmul(-g[1], g[1], K));
  const double det = fma(g[0], gu[0], fma(g[1], gu[1], fmul(g[2], gu[2], K)));
  const double rdw = 1.0 / fmul(det, W, K);  // one division for 1/det and 1/W
  const double idet = fmul(W, rdw, K);
  const double iW = fmul(det, rdw, K);
#pragma unroll
  for (int s = 0; s < 6; ++s) gu[s] = fmul(gu[s], idet, K);
  // trace weights: gt^ij X_ij = sum_s gw[s] X[s] over the 6 symmetric slots
  double gw[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) gw[s] = (s == 1 || s == 2 || s == 4) ? fmul(2.0, gu[s], K) : gu[s];

  // first derivatives of the metric (stencil sums), Christoffel symbols
  double dg[6][3];
#pragma unroll
  for (int s = 0; s < 6; ++s)
#pragma unroll
    for (int d = 0; d < 3; ++d) dg[s][d] = D1(ZG + s, d);
  // Gamma_{k,ij} = (d_i g_jk + d_j g_ik - d_k g_ij) / 2 = hs1 * Gs[k][s(ij)],
  // Gs the combination of stored sums; where k is i or j two of the three
  // terms cancel (k = i: d_j g_ii; k = j: d_i g_jj), where i = j != k two
  // coincide (2 d_i g_ik - d_k g_ii).
  double Gs[3][6], Gu[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        double v;
        if (k == i) v = dg[sidx(i, i)][j];
        else if (k == j) v = dg[sidx(j, j)][i];
        else if (i == j) v = fma(2.0, dg[sidx(i, k)][i], -dg[sidx(i, i)][k]);
        else v = fsub(fadd(dg[sidx(j, k)][i], dg[sidx(i, k)][j], K), dg[sidx(i, j)][k], K);
        Gs[k][sidx(i, j)] = v;
      }
  // the factor hs1 of Gamma_{k,ij} carried by the metric that raises its index
  double gus[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) gus[s] = fmul(gu[s], ds.hs1, K);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s)
      Gu[k][s] = fma(gus[sidx(k, 0)], Gs[0][s], fma(gus[sidx(k, 1)], Gs[1][s], fmul(gus[sidx(k, 2)], Gs[2][s], K)));
  // (Gamma_d)^k = gt^ij Gamma^k_ij
  double Gd[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    Gd[k] = fma(2.0, fma(gu[1], Gu[k][1], fma(gu[2], Gu[k][2], fmul(gu[4], Gu[k][4], K))),
                fma(gu[0], Gu[k][0], fma(gu[3], Gu[k][3], fmul(gu[5], Gu[k][5], K))));

  // U[j][k][l] = gt^{lm} Gamma_{j,km}
  double U[3][3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        U[j][k][l] = fma(gus[sidx(l, 0)], Gs[j][sidx(k, 0)],
                         fma(gus[sidx(l, 1)], Gs[j][sidx(k, 1)], fmul(gus[sidx(l, 2)], Gs[j][sidx(k, 2)], K)));

  const double dW[3] = {fmul(D1(ZW, 0), ds.s1, K), fmul(D1(ZW, 1), ds.s1, K), fmul(D1(ZW, 2), ds.s1, K)};
  const double dal[3] = {fmul(D1(ZAL, 0), ds.s1, K), fmul(D1(ZAL, 1), ds.s1, K), fmul(D1(ZAL, 2), ds.s1, K)};
  // gt^{kl} d_l W and |dW|^2, gt^{kl} d_l W d_k alpha
  double gudW[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    gudW[k] = fma(gu[sidx(k, 0)], dW[0], fma(gu[sidx(k, 1)], dW[1], fmul(gu[sidx(k, 2)], dW[2], K)));
  const double dWdW = fma(gudW[0], dW[0], fma(gudW[1], dW[1], fmul(gudW[2], dW[2], K)));
  const double dWdal = fma(gudW[0], dal[0], fma(gudW[1], dal[1], fmul(gudW[2], dal[2], K)));

  // Ricci tensor R_ij = R^W_ij + Rt_ij, and D_i D_j alpha
  double R[6], DDal[6];
  {
    double DDW[6];
    double trDDW;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const double s2 = (s == 0 || s == 3 || s == 5) ? ds.s2p : ds.s2m;
      DDW[s] = fma(D2(0, s), s2, -fma(Gu[0][s], dW[0], fma(Gu[1][s], dW[1], fmul(Gu[2][s], dW[2], K))));
      trDDW = s == 0 ? fmul(gw[0], DDW[0], K) : fma(gw[s], DDW[s], trDDW);
    }
    // hs1 d_j Gamt^k, and the scales of the second-derivative terms carried by gt^lm
    double dGh[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) dGh[k][j] = fmul(D1(ZGAM + k, j), ds.hs1, K);
    double guS[6];  // -1/2 s2p gt^ll (pure), -s2m gt^lm (mixed: the pair lm, ml counted once)
#pragma unroll
    for (int s = 0; s < 6; ++s) guS[s] = fmul(gu[s], (s == 0 || s == 3 || s == 5) ? -ds.hs2p : -ds.s2m, K);
    double Gdq[3];  // (Gamma_d)^k hs1 / 2
#pragma unroll
    for (int k = 0; k < 3; ++k) Gdq[k] = fmul(Gd[k], ds.qs1, K);
    const double m2WiW = fmul(fmul(fmul(-2.0, dWdW, K), iW, K), iW, K);  // -2 |dW|^2 / W^2
    // Every term of R_ij below is accumulated in one chain of FMAs.
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int s = sidx(i, j);
        // gt^lm (2 Gamma^k_l(i Gamma_j)km + Gamma^k_im Gamma_klj) = T_ij + T_ji + t3,
        // T_ij = Gamma^k_li U[j][k][l], t3 = Gamma^k_im U[k][j][m]
        double r;
        if (i == j) {
          double t = fmul(Gu[0][sidx(0, i)], U[i][0][0], K);
#pragma unroll
          for (int q = 1; q < 9; ++q) t = fma(Gu[q / 3][sidx(q % 3, i)], U[i][q / 3][q % 3], t);
          r = fmul(Gu[0][sidx(i, 0)], U[0][j][0], K);
#pragma unroll
          for (int q = 1; q < 9; ++q) r = fma(Gu[q / 3][sidx(i, q % 3)], U[q / 3][j][q % 3], r);
          r = fma(2.0, t, r);
        } else {
          r = fmul(Gu[0][sidx(i, 0)], U[0][j][0], K);
#pragma unroll
          for (int q = 1; q < 9; ++q) r = fma(Gu[q / 3][sidx(i, q % 3)], U[q / 3][j][q % 3], r);
#pragma unroll
          for (int q = 0; q < 9; ++q)
            r = fma(Gu[q / 3][sidx(q % 3, i)], U[j][q / 3][q % 3], fma(Gu[q / 3][sidx(q % 3, j)], U[i][q / 3][q % 3], r));
        }
        // -1/2 gt^lm d_l d_m gt_ij
#pragma unroll
        for (int q = 0; q < 6; ++q) r = fma(guS[q], D2(1 + s, q), r);
        // gt_k(i d_j) Gamt^k
#pragma unroll
        for (int k = 0; k < 3; ++k) r = fma(g[sidx(k, i)], dGh[k][j], fma(g[sidx(k, j)], dGh[k][i], r));
        // (Gamma_d)^k Gamma_(ij)k
#pragma unroll
        for (int k = 0; k < 3; ++k) r = fma(Gdq[k], Gs[i][sidx(j, k)], fma(Gdq[k], Gs[j][sidx(i, k)], r));
        // R^W_ij = (D_i D_j W + gt_ij D^l D_l W) / W - 2 gt_ij |dW|^2 / W^2
        r = fma(g[s], m2WiW, r);
        R[s] = fma(fma(g[s], trDDW, DDW[s]), iW, r);
        // D_i D_j alpha with Gamma^k_ij - (delta^k_i d_j W + delta^k_j d_i W - gt_ij gt^kl d_l W) / W
        const double gd = fma(Gu[0][s], dal[0], fma(Gu[1][s], dal[1], fmul(Gu[2][s], dal[2], K)));
        const double wt = fma(dW[j], dal[i], fma(dW[i], dal[j], fmul(-g[s], dWdal, K)));
        const double s2 = (s == 0 || s == 3 || s == 5) ? ds.s2p : ds.s2m;
        DDal[s] = fma(D2(7, s), s2, -fma(-wt, iW, gd));
      }
  }
  double trR = fmul(gw[0], R[0], K), trDDal = fmul(gw[0], DDal[0], K);
#pragma unroll
  for (int s = 1; s < 6; ++s) {
    trR = fma(gw[s], R[s], trR);
    trDDal = fma(gw[s], DDal[s], trDDal);
  }
  const double W2 = fmul(W, W, K);
  const double Rsc = fmul(W2, trR, K);
  const double DiDial = fmul(W2, trDDal, K);

  // At with raised indices: Am[i][j] = At^i_j, Auu = At^ij
  double Am[3][3], Auu[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Am[i][j] = fma(gu[sidx(i, 0)], A[sidx(0, j)],
                     fma(gu[sidx(i, 1)], A[sidx(1, j)], fmul(gu[sidx(i, 2)], A[sidx(2, j)], K)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      Auu[sidx(i, j)] =
          fma(Am[i][0], gu[sidx(0, j)], fma(Am[i][1], gu[sidx(1, j)], fmul(Am[i][2], gu[sidx(2, j)], K)));
  const double AA = fma(2.0, fma(A[1], Auu[1], fma(A[2], Auu[2], fmul(A[4], Auu[4], K))),
                        fma(A[0], Auu[0], fma(A[3], Auu[3], fmul(A[5], Auu[5], K))));

  double dbe[3][3];  // dbe[i][j] = d_j beta^i
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) dbe[i][j] = fmul(D1(ZB + i, j), ds.s1, K);
  const double divb = fadd(fadd(dbe[0][0], dbe[1][1], K), dbe[2][2], K);
  const double Kt = fma(2.0, Th, Kh);
  const double third = 1.0 / 3.0, twothird = 2.0 / 3.0;

  // advection beta^i d_i f added onto x, the scale s1 carried by beta
  const double bes[3] = {fmul(be[0], ds.s1, K), fmul(be[1], ds.s1, K), fmul(be[2], ds.s1, K)};
#define ADV_ON(f, x) fma(bes[0], D1(f, 0), fma(bes[1], D1(f, 1), fma(bes[2], D1(f, 2), (x))))
#define ADV(f) fma(bes[0], D1(f, 0), fma(bes[1], D1(f, 1), fmul(bes[2], D1(f, 2), K)))
  // W
  rhs[ZW] = ADV_ON(ZW, fmul(fmul(third, W, K), fma(al, Kt, -divb), K));
  // gt_ij and At_ij
  double X[6], trX;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    X[s] = fma(al, R[s], -DDal[s]);
    trX = s == 0 ? fmul(gw[0], X[0], K) : fma(gw[s], X[s], trX);
  }
  const double alKt = fmul(al, Kt, K);
  const double m2al = fmul(-2.0, al, K);
  const double m23divb = fmul(-twothird, divb, K);
  const double m13trX = fmul(-third, trX, K);
  const double cA = fadd(alKt, m23divb, K);  // (alpha Kt - 2/3 div beta), the coefficient of At_ij
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int s = sidx(i, j);
      // gt_k(i d_j) beta^k and At_k(i d_j) beta^k accumulated onto the terms
      // in gt_ij and At_ij; At_ik At^k_j
      double lg = fmul(m23divb, g[s], K), la = fmul(cA, A[s], K), aa = fmul(Am[0][i], A[sidx(0, j)], K);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        lg = fma(g[sidx(k, i)], dbe[k][j], fma(g[sidx(k, j)], dbe[k][i], lg));
        la = fma(A[sidx(k, i)], dbe[k][j], fma(A[sidx(k, j)], dbe[k][i], la));
        if (k > 0) aa = fma(Am[k][i], A[sidx(k, j)], aa);
      }
      rhs[ZG + s] = ADV_ON(ZG + s, fma(m2al, A[s], lg));
      const double tf = fma(m13trX, g[s], X[s]);
      rhs[ZA + s] = ADV_ON(ZA + s, fma(W2, tf, fma(m2al, aa, la)));
    }
  // Khat
  rhs[ZK] = fma(al, fma(fmul(third, Kt, K), Kt, AA),
                fma(fmul(al, P.kappa1 * (1.0 - P.kappa2), K), Th, ADV_ON(ZK, -DiDial)));
  // Gamt^i
  {
    const double dKh[3] = {D1(ZK, 0), D1(ZK, 1), D1(ZK, 2)};
    const double dTh[3] = {D1(ZTH, 0), D1(ZTH, 1), D1(ZTH, 2)};
    double dd[3];  // d_j (2 Khat + Theta), stencil sums (times s1 below)
#pragma unroll
    for (int j = 0; j < 3; ++j) dd[j] = fma(2.0, dKh[j], dTh[j]);
    // d_j d_k beta^k for each j (the k = j term a pure second derivative)
    double ddivb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      ddivb[j] = fma(D2(8, sidx(j, 0)), j == 0 ? ds.s2p : ds.s2m,
                     fma(D2(9, sidx(j, 1)), j == 1 ? ds.s2p : ds.s2m,
                         fmul(D2(10, sidx(j, 2)), j == 2 ? ds.s2p : ds.s2m, K)));
    const double m3iW = fmul(-3.0, iW, K);
    const double twoal = fmul(2.0, al, K);
    const double twothirddivb = fmul(twothird, divb, K);
    const double m2k1al = fmul(-2.0 * P.kappa1, al, K);
    const double cGd = fsub(twothirddivb, m2k1al, K);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      // Gamt^i_jk At^jk
      double br = fma(2.0, fma(Gu[i][1], Auu[1], fma(Gu[i][2], Auu[2], fmul(Gu[i][4], Auu[4], K))),
                      fma(Gu[i][0], Auu[0], fma(Gu[i][3], Auu[3], fmul(Gu[i][5], Auu[5], K))));
      const double au0 = Auu[sidx(i, 0)], gu0 = gu[sidx(i, 0)];
      double sA = fmul(au0, dal[0], K);     // At^ij d_j alpha
      double sW = fmul(au0, dW[0], K);      // At^ij d_j W
      double sD = fmul(gu0, dd[0], K);      // gt^ij d_j (2 Khat + Theta)
      double sL = fmul(gu0, ddivb[0], K);   // gt^ij d_j d_k beta^k
      double r = fmul(-Gd[0], dbe[i][0], K);
#pragma unroll
      for (int j = 1; j < 3; ++j) {
        const double auij = Auu[sidx(i, j)], guij = gu[sidx(i, j)];
        sA = fma(auij, dal[j], sA);
        sW = fma(auij, dW[j], sW);
        sD = fma(guij, dd[j], sD);
        sL = fma(guij, ddivb[j], sL);
        r = fma(-Gd[j], dbe[i][j], r);
      }
      r = fma(-2.0, sA, r);
      br = fma(m3iW, sW, br);
      br = fma(-ds.ts1, sD, br);
      r = fma(twoal, br, r);
      // 1/3 gt^ij d_j d_k beta^k + gt^jk d_j d_k beta^i
      r = fma(ds.ts2m, fma(gu[1], D2(8 + i, 1), fma(gu[2], D2(8 + i, 2), fmul(gu[4], D2(8 + i, 4), K))), r);
      r = fma(ds.s2p, fma(gu[0], D2(8 + i, 0), fma(gu[3], D2(8 + i, 3), fmul(gu[5], D2(8 + i, 5), K))), r);
      r = fma(third, sL, r);
      // 2/3 (Gamma_d)^i div beta - 2 kappa1 alpha (Gamt^i - (Gamma_d)^i)
      r = fma(Gd[i], cGd, fma(m2k1al, Gam[i], r));
      rhs[ZGAM + i] = ADV_ON(ZGAM + i, r);
    }
  }
  // Theta
  rhs[ZTH] = fma(fmul(0.5, al, K), fma(fmul(twothird, Kt, K), Kt, fsub(Rsc, AA, K)),
                 fma(fmul(-al, P.kappa1 * (2.0 + P.kappa2), K), Th, ADV(ZTH)));
  // lapse (1+log) and shift (Gamma-driver)
  rhs[ZAL] = fma(m2al, Kh, ADV(ZAL));
#pragma unroll
  for (int i = 0; i < 3; ++i) rhs[ZB + i] = ADV_ON(ZB + i, fma(0.75, Gam[i], fmul(-eta, be[i], K)));
  if (kDiag) {
    diag[0] = Rsc;
    diag[1] = AA;
    diag[2] = Kt;
  }
#undef ADV_ON
#undef ADV
#undef FLD
#undef D1
#undef D2
}

// FORM: the stage update of StageArgs (kStageSingle, kStageRk4, kStageTwo,
// kStageNone), fixed at compile time so the update adds no registers to the
// RHS.  BPS: warps per scheduler the build is constrained to (the register
// budget of BPS 128-thread blocks per SM), a choice of sc_autotune: 3 (at
// most 168 registers; the RHS then spills about 1 KB per thread, written back
// to DRAM, which the FP64-bound kernel can afford, while 3 warps per
// scheduler instead of 2 hide the FP64 dependency latency better) or 2 (255
// registers, a few spills).  Blocks of 128 threads over 128-cell tiles, or
// of 64 threads over 64-cell tiles (twice as many per SM) on large levels,
// where the finer split balances the SMs (the host picks per level).
template <int FORM, int BPS, class KT = FmaK>
__global__ void __launch_bounds__(128, BPS) z4c_stage_kernel(StageArgs a, const double* __restrict__ S, Z4cParams P,
                                                            const Tile* __restrict__ tiles, int ntiles, KT K) {
  const double ko = P.ko_sigma / (64.0 * a.h);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = tiles[t];
    const int n = T.nx * T.ny * T.nz;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int i = q % T.nx;
      const int j = (q / T.nx) % T.ny;
      const int k = q / (T.nx * T.ny);
      const long o = (long)(T.z0 + k) * a.sz + (long)(T.y0 + j) * a.sy + (T.x0 + i);
      double rhs[kNZ4c];
      z4c_rhs_point<false>(a.Y, S, a.fs, o, P, a.eta ? a.eta[o] : P.eta, a.ds, rhs, nullptr, K);
#pragma unroll
      for (int f = 0; f < kNZ4c; ++f) {
        const long fo = (long)f * a.fs + o;
        const double kv = fma(ko, S[(long)(Q_KO + f) * a.fs + o], rhs[f]);
        a.k[fo] = kv;
        if (FORM == kStageSingle) {
          a.out[fo] = fma(a.cdt, kv, a.yn[fo]);
        } else if (FORM == kStageRk4) {
          const double s = fadd(fma(2.0, a.k3[fo], fma(2.0, a.k2[fo], a.k1[fo])), kv, K);
          a.out[fo] = fma(a.cdt, s, a.yn[fo]);
        } else if (FORM == kStageTwo) {
          a.out[fo] = fma(a.cdt, kv, fma(a.c1dt, a.k1[fo], a.yn[fo]));
        }
      }
    }
  }
}

// Constraints at the interior cells of one box:
//   H   = R + 2/3 (Khat + 2 Theta)^2 - At_ij At^ij      (R the Ricci scalar of gamma)
//   M^i = d_j At^ij + Gamt^i_jk At^jk - 3 At^ij d_j W / W - 2/3 gt^ij d_j (Khat + 2 Theta)
//   G^i = Gamt^i - gt^jk Gamt^i_jk
// out[c * out_stride + cell], cells numbered x-fastest within the box.
__global__ void __launch_bounds__(128) z4c_constraints_kernel(const double* __restrict__ Y,
                                                             const double* __restrict__ S, double* __restrict__ out,
                                                             long fs, int sy, int sz, Z4cParams P, DerivScales ds,
                                                             const Tile* __restrict__ tiles, int ntiles,
                                                             long out_stride, int bx, int by, int bz, int nbx,
                                                             int nby, FmaK K) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = tiles[t];
    const int n = T.nx * T.ny * T.nz;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int ax = T.x0 + q % T.nx, ay = T.y0 + (q / T.nx) % T.ny, az = T.z0 + q / (T.nx * T.ny);
      const long o = (long)az * sz + (long)ay * sy + ax;
      const long cell = ((long)(az - bz) * nby + (ay - by)) * nbx + (ax - bx);
#define FLD(f) Y[(long)(f) * fs + o]
#define D1(f, d) (ds.s1 * S[(long)(Q_D1 + 3 * (f) + (d)) * fs + o])
      double rhs[kNZ4c], diag[3];
      z4c_rhs_point<true>(Y, S, fs, o, P, P.eta, ds, rhs, diag, K);
      out[cell] = diag[0] + (2.0 / 3.0) * diag[2] * diag[2] - diag[1];
      double g[6], A[6], gu[6];
      for (int s = 0; s < 6; ++s) {
        g[s] = FLD(ZG + s);
        A[s] = FLD(ZA + s);
      }
      gu[0] = fma(g[3], g[5], -g[4] * g[4]);
      gu[1] = fma(g[2], g[4], -g[1] * g[5]);
      gu[2] = fma(g[1], g[4], -g[2] * g[3]);
      gu[3] = fma(g[0], g[5], -g[2] * g[2]);
      gu[4] = fma(g[1], g[2], -g[0] * g[4]);
      gu[5] = fma(g[0], g[3], -g[1] * g[1]);
      const double idet = 1.0 / fma(g[0], gu[0], fma(g[1], gu[1], g[2] * gu[2]));
      for (int s = 0; s < 6; ++s) gu[s] *= idet;
      const double iW = 1.0 / FLD(ZW);
      double Gu[3][6];
      for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b) {
            double v = 0.0;
            for (int l = 0; l < 3; ++l)
              v += gu[sidx(k, l)] * 0.5 * (D1(ZG + sidx(b, l), a) + D1(ZG + sidx(a, l), b) - D1(ZG + sidx(a, b), l));
            Gu[k][sidx(a, b)] = v;
          }
      double Auu[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double v = 0.0;
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) v += gu[sidx(a, c)] * gu[sidx(b, d)] * A[sidx(c, d)];
          Auu[a][b] = v;
        }
      double dgu[3][6];  // d_m gt^{ab} = -gt^{ac} gt^{bd} d_m gt_cd
      for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b) {
            double v = 0.0;
            for (int c = 0; c < 3; ++c)
              for (int d = 0; d < 3; ++d) v -= gu[sidx(a, c)] * gu[sidx(b, d)] * D1(ZG + sidx(c, d), m);
            dgu[m][sidx(a, b)] = v;
          }
      for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int j = 0; j < 3; ++j)  // d_j At^{aj}
          for (int m = 0; m < 3; ++m)
            for (int p = 0; p < 3; ++p)
              v += dgu[j][sidx(a, m)] * gu[sidx(j, p)] * A[sidx(m, p)] +
                   gu[sidx(a, m)] * dgu[j][sidx(j, p)] * A[sidx(m, p)] +
                   gu[sidx(a, m)] * gu[sidx(j, p)] * D1(ZA + sidx(m, p), j);
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c) v += Gu[a][sidx(b, c)] * Auu[b][c];
        for (int b = 0; b < 3; ++b) {
          v -= 3.0 * Auu[a][b] * D1(ZW, b) * iW;
          v -= (2.0 / 3.0) * gu[sidx(a, b)] * (D1(ZK, b) + 2.0 * D1(ZTH, b));
        }
        out[(1 + a) * out_stride + cell] = v;
        double gd = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c) gd += gu[sidx(b, c)] * Gu[a][sidx(b, c)];
        out[(4 + a) * out_stride + cell] = FLD(ZGAM + a) - gd;
      }
#undef FLD
#undef D1
    }
  }
}

// Persistent grids: each Z4c kernel is launched with (SMs x resident blocks
// per SM) blocks at most, looping over its tiles, so a level's work is spread
// evenly over the whole GPU instead of leaving a partial last wave.
struct GridCaps {
  int ready = 0;
  int stage[4] = {304, 304, 304, 456};  // 128-thread blocks, by warps per scheduler of the build (2 or 3)
  int derivs = 1216, dxy = 2432;
};
GridCaps g_caps[64];

inline const GridCaps& caps() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_caps[dev & 63];
}

}  // namespace

cudaError_t z4c_init_launch_config() {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  GridCaps& c = g_caps[dev & 63];
  if (c.ready) return cudaSuccess;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, z4c_stage_kernel<kStageSingle, 2>, 128, 0)) !=
      cudaSuccess)
    return e;
  c.stage[2] = nsm * (occ > 0 ? occ : 1);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, z4c_stage_kernel<kStageSingle, 3>, 128, 0)) !=
      cudaSuccess)
    return e;
  c.stage[3] = nsm * (occ > 0 ? occ : 1);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, z4c_derivs_split_kernel<8>, kThreads, 0)) != cudaSuccess)
    return e;
  c.derivs = nsm * (occ > 0 ? occ : 1);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, z4c_dxy_kernel<8>, 128, 0)) != cudaSuccess) return e;
  c.dxy = nsm * (occ > 0 ? occ : 1);
  c.ready = 1;
  return cudaSuccess;
}

cudaError_t launch_z4c_derivs(const double* Y, double* scratch, long fs, int sy, int sz, const Tile* tiles,
                              int ntiles, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const int grid = ntiles < sm_count() * 16 ? ntiles : sm_count() * 16;
  z4c_derivs_kernel<<<grid, kThreads, 0, s>>>(Y, scratch, fs, sy, sz, tiles, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_z4c_dxy(const double* Y, double* scratch, long fs, int sy, const RowSeg* segs, int nsegs,
                           cudaStream_t s, int order, bool op_class) {
  if (nsegs == 0) return cudaSuccess;
  const int grid = nsegs < caps().dxy ? nsegs : caps().dxy;
  const FmaK K{1.0, -1.0, -0.0};
  if (op_class) {
    if (order == 8) z4c_dxy_kernel<8, PlainK><<<grid, 128, 0, s>>>(Y, scratch, fs, sy, segs, nsegs, PlainK{});
    else z4c_dxy_kernel<4, PlainK><<<grid, 128, 0, s>>>(Y, scratch, fs, sy, segs, nsegs, PlainK{});
  } else if (order == 8) {
    z4c_dxy_kernel<8><<<grid, 128, 0, s>>>(Y, scratch, fs, sy, segs, nsegs, K);
  } else {
    z4c_dxy_kernel<4><<<grid, 128, 0, s>>>(Y, scratch, fs, sy, segs, nsegs, K);
  }
  return cudaGetLastError();
}

cudaError_t launch_z4c_derivs_split(const double* Y, double* scratch, long fs, int sy, int sz,
                                    const Tile* tiles, int ntiles, cudaStream_t s, int order, int max_cols,
                                    bool op_class) {
  if (ntiles == 0) return cudaSuccess;
  if (max_cols < 1) return cudaErrorInvalidValue;
  const long units = (long)ntiles * ((max_cols * kNZ4c + kThreads - 1) / kThreads);
  const int grid = units < caps().derivs ? (int)units : caps().derivs;
  const FmaK K{1.0, -1.0, -0.0};
  if (op_class) {
    if (order == 8)
      z4c_derivs_split_kernel<8, PlainK><<<grid, kThreads, 0, s>>>(Y, scratch, fs, sy, sz, tiles, ntiles, max_cols,
                                                                   PlainK{});
    else
      z4c_derivs_split_kernel<4, PlainK><<<grid, kThreads, 0, s>>>(Y, scratch, fs, sy, sz, tiles, ntiles, max_cols,
                                                                   PlainK{});
  } else if (order == 8) {
    z4c_derivs_split_kernel<8><<<grid, kThreads, 0, s>>>(Y, scratch, fs, sy, sz, tiles, ntiles, max_cols, K);
  } else {
    z4c_derivs_split_kernel<4><<<grid, kThreads, 0, s>>>(Y, scratch, fs, sy, sz, tiles, ntiles, max_cols, K);
  }
  return cudaGetLastError();
}

namespace {

template <int BPS>
void launch_stage_bps(const StageArgs& a, const double* scratch, const Z4cParams& p, const Tile* tiles, int ntiles,
                      int grid, int threads, cudaStream_t s, const FmaK& K, bool op_class) {
  if (op_class)
    z4c_stage_kernel<kStageSingle, BPS, PlainK><<<grid, threads, 0, s>>>(a, scratch, p, tiles, ntiles, PlainK{});
  else if (a.form == kStageRk4) z4c_stage_kernel<kStageRk4, BPS><<<grid, threads, 0, s>>>(a, scratch, p, tiles, ntiles, K);
  else if (a.form == kStageTwo) z4c_stage_kernel<kStageTwo, BPS><<<grid, threads, 0, s>>>(a, scratch, p, tiles, ntiles, K);
  else if (a.form == kStageNone)
    z4c_stage_kernel<kStageNone, BPS><<<grid, threads, 0, s>>>(a, scratch, p, tiles, ntiles, K);
  else z4c_stage_kernel<kStageSingle, BPS><<<grid, threads, 0, s>>>(a, scratch, p, tiles, ntiles, K);
}

}  // namespace

cudaError_t launch_z4c_stage(const StageArgs& a, const double* scratch, const Z4cParams& p, const Tile* tiles,
                             int ntiles, cudaStream_t s, int bps, int threads, bool op_class) {
  if (ntiles == 0) return cudaSuccess;
  if (bps != 2 && bps != 3) return cudaErrorInvalidValue;
  if (threads != 64 && threads != 128) return cudaErrorInvalidValue;
  if (op_class && a.form != kStageSingle) return cudaErrorInvalidValue;
  // persistent grid: the resident blocks (twice as many at 64 threads, whose
  // registers per block are half)
  const int cap = caps().stage[bps] * (128 / threads);
  const int grid = ntiles < cap ? ntiles : cap;
  const FmaK K{1.0, -1.0, -0.0};
  if (bps == 2) launch_stage_bps<2>(a, scratch, p, tiles, ntiles, grid, threads, s, K, op_class);
  else launch_stage_bps<3>(a, scratch, p, tiles, ntiles, grid, threads, s, K, op_class);
  return cudaGetLastError();
}

cudaError_t launch_z4c_constraints(const double* Y, const double* scratch, double* out, long fs, int sy, int sz,
                                   const Z4cParams& p, const DerivScales& ds, const Tile* tiles, int ntiles,
                                   long out_stride, const int* box_lo, const int* box_n, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const int grid = ntiles < sm_count() * 16 ? ntiles : sm_count() * 16;
  z4c_constraints_kernel<<<grid, 128, 0, s>>>(Y, scratch, out, fs, sy, sz, p, ds, tiles, ntiles, out_stride, box_lo[0],
                                              box_lo[1], box_lo[2], box_n[0], box_n[1], FmaK{1.0, -1.0, -0.0});
  return cudaGetLastError();
}

}  // namespace sc
