// oracle.cpp -- plain single-threaded FP64 CPU oracle for RK4 subcycling in
// time with dense-output ghost filling (arXiv:2503.09629, Sec. II).
//
// TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
// benchmark's CPU-baseline leg, never by the product path.  Shares no code
// with the CUDA library.  Built with -O2 -ffp-contract=off.
//
// Layout: every level is a list of boxes; every box stores each field as its
// own array over the box interior plus g ghost cells per side (3 for 4th-order
// differences, 4 for 8th order), x fastest.
// Ghost cells are classified once: copied from a sibling box interior (same
// level, periodic wrap included), filled from the parent level by dense output
// and prolongation (refinement boundary), or physical (outer boundary).
//
// Parity status of each part (what pins it) is listed in the test suite: the
// puncture gauge (Eqs. punclapse/puncshift) by 4th-order convergence to the
// equations evaluated with exact derivatives on data that varies in every
// field (a reversed sign in any term fails); the radiative outer boundary by
// exact outgoing spherical waves; KO dissipation by its closed form on plane
// waves; the rest by closed forms, polynomial exactness, exact solutions
// (gauge wave, flat space in moving coordinates) and convergence.

#include "oracle.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {


// ---------------------------------------------------------------------------
// Operation counter (used once, to count the flops of the Z4c formulation).
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
double g_ops[4];  // add/sub, mul, div, other
inline Cnt operator+(Cnt a, Cnt b) { g_ops[0]++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops[0]++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops[1]++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops[2]++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }

// ---------------------------------------------------------------------------
// Dense output (Eq. denseoutput1 and its theta-derivatives, Eq. denseoutput2):
// b1 = t - 3/2 t^2 + 2/3 t^3, b2 = b3 = t^2 - 2/3 t^3, b4 = -1/2 t^2 + 2/3 t^3.
void dense_b(double t, int m, double* b) {
  if (m == 0) {
    b[0] = t - 1.5 * t * t + (2.0 / 3.0) * t * t * t;
    b[1] = t * t - (2.0 / 3.0) * t * t * t;
    b[2] = b[1];
    b[3] = -0.5 * t * t + (2.0 / 3.0) * t * t * t;
  } else if (m == 1) {
    b[0] = 1.0 - 3.0 * t + 2.0 * t * t;
    b[1] = 2.0 * t - 2.0 * t * t;
    b[2] = b[1];
    b[3] = -t + 2.0 * t * t;
  } else if (m == 2) {
    b[0] = -3.0 + 4.0 * t;
    b[1] = 2.0 - 4.0 * t;
    b[2] = b[1];
    b[3] = -1.0 + 4.0 * t;
  } else if (m == 3) {
    b[0] = 4.0; b[1] = -4.0; b[2] = -4.0; b[3] = 4.0;
  } else {
    b[0] = b[1] = b[2] = b[3] = 0.0;
  }
}

// Value of a refinement-boundary ghost cell on the fine level, from the
// parent's state y_n and stage vectors k1..k4 over the parent step H
// (already prolonged to the ghost cell).  The fine substep starts at progress
// theta0 of the parent step and has step h = H/2.
//   which = 1..4: fine stage state Y_which (Eqs. Y1-Y4), with y, y', y'', y'''
//                 from dense output at theta0 (Eqs. denseoutput1/2) and
//                 f_y y'' = 4 (k3 - k2) / H^2;
//   which = 0:    state at the end of the substep, dense output at theta0+1/2.
double amr_value(double y, const double* k, double H, double theta0, int which) {
  double b[4];
  if (which == 0) {
    dense_b(theta0 + 0.5, 0, b);
    return y + H * (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]);
  }
  const double h = 0.5 * H;
  dense_b(theta0, 0, b);
  const double y0 = y + H * (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]);
  dense_b(theta0, 1, b);
  const double y1 = b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3];
  dense_b(theta0, 2, b);
  const double y2 = (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]) / H;
  dense_b(theta0, 3, b);
  const double y3 = (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]) / (H * H);
  const double fyy = 4.0 * (k[2] - k[1]) / (H * H);
  switch (which) {
    case 1: return y0;
    case 2: return y0 + 0.5 * h * y1;
    case 3: return y0 + 0.5 * h * y1 + 0.25 * h * h * y2 + (h * h * h / 16.0) * (y3 - fyy);
    case 4: return y0 + h * y1 + 0.5 * h * h * y2 + (h * h * h / 8.0) * (y3 + fyy);
  }
  return NAN;
}

// RK2 and RK3 subcycling (the extension the paper's Sec. V names as future
// work).  The paper fixes neither method; the oracle uses
//   RK2: explicit midpoint, Y2 = y + h/2 k1, y_{n+1} = y + h k2;
//   RK3: Heun's third-order method, Y2 = y + h/3 k1, Y3 = y + 2h/3 k2,
//        y_{n+1} = y + h/4 (k1 + 3 k3).
// Dense output:
//   RK2: the quadratic continuous extension b1 = theta - theta^2,
//        b2 = theta^2 (second order, like the method);
//   RK3: the cubic Hermite interpolant through y_n, y_{n+1} with slopes k1
//        and k4 = f(y_{n+1}), evaluated once per step on every level that
//        has a finer level: b1 = theta - 5/4 theta^2 + 1/2 theta^3,
//        b2 = 0, b3 = 9/4 theta^2 - 3/2 theta^3, b4 = -theta^2 + theta^3
//        (third order, one order above RK3's own continuous extensions,
//        which leave the subcycled scheme near order 2.5).
// m-th theta-derivatives of the weights, as dense_b for RK4.
void dense_b_rk(int rk, double t, int m, double* b) {
  b[0] = b[1] = b[2] = b[3] = 0.0;
  if (rk == 4) { dense_b(t, m, b); return; }
  if (rk == 2) {
    if (m == 0) { b[0] = t - t * t; b[1] = t * t; }
    else if (m == 1) { b[0] = 1.0 - 2.0 * t; b[1] = 2.0 * t; }
    else if (m == 2) { b[0] = -2.0; b[1] = 2.0; }
    return;
  }
  if (m == 0) {
    b[0] = t - 1.25 * t * t + 0.5 * t * t * t;
    b[2] = 2.25 * t * t - 1.5 * t * t * t;
    b[3] = -t * t + t * t * t;
  } else if (m == 1) {
    b[0] = 1.0 - 2.5 * t + 1.5 * t * t;
    b[2] = 4.5 * t - 4.5 * t * t;
    b[3] = -2.0 * t + 3.0 * t * t;
  } else if (m == 2) {
    b[0] = -2.5 + 3.0 * t;
    b[2] = 4.5 - 9.0 * t;
    b[3] = -2.0 + 6.0 * t;
  } else if (m == 3) {
    b[0] = 3.0; b[2] = -9.0; b[3] = 6.0;
  }
}

// Refinement-boundary ghost value for the RK2 / RK3 fine substep starting at
// theta0 (step h = H/2).  The fine stage states follow from expanding the
// method's stages about the substep start, to the order the method needs:
//   RK2: Y1 = y, Y2 = y + h/2 y';
//   RK3: Y1 = y, Y2 = y + h/3 y', Y3 = y + 2h/3 y' + 2h^2/9 y''
// (exact when f is linear), with y, y', y'' from the dense output at theta0.
// which = 0: the state at the end of the substep (dense output at theta0+1/2).
double amr_value_rk(int rk, double y, const double* k, double H, double theta0, int which) {
  if (rk == 4) return amr_value(y, k, H, theta0, which);
  double b[4];
  if (which == 0) {
    dense_b_rk(rk, theta0 + 0.5, 0, b);
    return y + H * (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]);
  }
  const double h = 0.5 * H;
  dense_b_rk(rk, theta0, 0, b);
  const double y0 = y + H * (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]);
  dense_b_rk(rk, theta0, 1, b);
  const double y1 = b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3];
  dense_b_rk(rk, theta0, 2, b);
  const double y2 = (b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3]) / H;
  if (rk == 2) {
    switch (which) {
      case 1: return y0;
      case 2: return y0 + 0.5 * h * y1;
    }
    return NAN;
  }
  switch (which) {
    case 1: return y0;
    case 2: return y0 + (h / 3.0) * y1;
    case 3: return y0 + (2.0 * h / 3.0) * y1 + (2.0 * h * h / 9.0) * y2;
  }
  return NAN;
}

// ---------------------------------------------------------------------------
// Hierarchy.

enum { V_Y = 0, V_YOLD = 1, V_STAGE = 2, V_K1 = 3, V_NVEC = 7 };

struct BoxData {
  int g = 3;  // ghost width: 3 for 4th-order differences, 4 for 8th order
  int lo[3], hi[3];
  int n[3], N[3];
  long vol;
  std::vector<double> v[V_NVEC];
  // ghost classification
  std::vector<long> sib_dst, sib_src;
  std::vector<int> sib_box;
  std::vector<long> amr_cell;       // local offsets of refinement-boundary ghosts
  std::vector<int> amr_glob;        // 3 ints per amr cell: wrapped global fine index
  std::vector<double> amr_P;        // prolonged parent vectors: [cell][5][F]
  std::vector<long> phys_cell;      // outer-boundary ghost cells
  long off(int i, int j, int k) const {
    return ((long)(k + g) * N[1] + (j + g)) * N[0] + (i + g);
  }
};

struct Level {
  std::vector<BoxData> boxes;
  int ext[3];
  double h, dt, t;
};

struct Hier {
  int system, F, nlev, bc, subcycle;
  int order;  // finite-difference order of the right-hand sides: 4 or 8 (Sec. III.C)
  int rk;     // Runge-Kutta method: 4 (Sec. II), 3 or 2 (see dense_b_rk)
  double cfl, h0, origin[3];
  int ncells0[3];
  double kappa1, kappa2, eta, sigma;
  bool eta_profile;                 // Sec. III.A eta(r) instead of the constant eta
  double eta_c, eta_s, eta_o;
  std::vector<Level> lev;
  double t;
  double zu_finest, zu_actual;
  orc_bc_fn cb;
  void* cb_user;
};

char g_err[256];
int fail(int code, const char* msg) {
  std::strncpy(g_err, msg, sizeof(g_err) - 1);
  return code;
}

int wrapi(int g, int n) { int r = g % n; return r < 0 ? r + n : r; }

// Box of level l whose interior holds global cell g (wrapped when periodic);
// -1 if none.  On success li[] is the local index in that box.
int find_interior(const Hier& H, int l, const int* g_in, int* li) {
  const Level& L = H.lev[l];
  int g[3];
  for (int d = 0; d < 3; ++d) {
    g[d] = g_in[d];
    if (H.bc == ORC_BC_PERIODIC) g[d] = wrapi(g[d], L.ext[d]);
    else if (g[d] < 0 || g[d] >= L.ext[d]) return -1;
  }
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const BoxData& B = L.boxes[b];
    if (g[0] >= B.lo[0] && g[0] <= B.hi[0] && g[1] >= B.lo[1] && g[1] <= B.hi[1] &&
        g[2] >= B.lo[2] && g[2] <= B.hi[2]) {
      for (int d = 0; d < 3; ++d) li[d] = g[d] - B.lo[d];
      return (int)b;
    }
  }
  return -1;
}

// Box of level l whose ghosted array holds global cell g (interior preferred).
int find_ghosted(const Hier& H, int l, const int* g, int* li) {
  int b = find_interior(H, l, g, li);
  if (b >= 0) return b;
  const Level& L = H.lev[l];
  for (size_t bb = 0; bb < L.boxes.size(); ++bb) {
    const BoxData& B = L.boxes[bb];
    bool ok = true;
    int loc[3];
    for (int d = 0; d < 3 && ok; ++d) {
      bool found = false;
      for (int m = -1; m <= 1 && !found; ++m) {
        if (m != 0 && H.bc != ORC_BC_PERIODIC) continue;
        int gg = g[d] + m * L.ext[d];
        if (gg >= B.lo[d] - B.g && gg <= B.hi[d] + B.g) { loc[d] = gg - B.lo[d]; found = true; }
      }
      ok = found;
    }
    if (ok) { for (int d = 0; d < 3; ++d) li[d] = loc[d]; return (int)bb; }
  }
  return -1;
}

// Lagrange basis weights for nodes x[0..n-1] evaluated at point p.
void lagrange(const double* x, int n, double p, double* w) {
  for (int m = 0; m < n; ++m) {
    double num = 1.0, den = 1.0;
    for (int q = 0; q < n; ++q) {
      if (q == m) continue;
      num *= (p - x[q]);
      den *= (x[m] - x[q]);
    }
    w[m] = num / den;
  }
}

// Stencil points of prolongation and restriction: quintic Lagrange in each
// dimension.  The paper does not name the spatial transfer operators; with
// cubic ones the refinement boundary limits the scalar-wave convergence to
// about 3rd order (the Laplacian differentiates the O(h^4) transfer error
// twice), quintic ones restore the 4th order the paper reports (Fig. 2).
const int g_pn = 6, g_rn = 6;

// Prolongation stencil along one dimension for fine cell f (cell-centred,
// refinement 2): the PN parent cells nearest to the fine centre and their
// Lagrange weights.
void prolong_stencil_1d(int f, int* nodes, double* w) {
  const int c = (f >= 0) ? f / 2 : -((-f + 1) / 2);
  // fine centre in parent-cell units relative to the centre of parent cell c
  const double p = (f - 2 * c == 1) ? 0.25 : -0.25;
  const int half = g_pn / 2;
  const int first = (p > 0) ? c - half + 1 : c - half;
  double x[8];
  for (int m = 0; m < g_pn; ++m) { nodes[m] = first + m; x[m] = (double)(first + m - c); }
  lagrange(x, g_pn, p, w);
}

// Restriction stencil along one dimension for parent cell C: the RN fine
// cells centred on the parent centre and their Lagrange weights there.
void restrict_stencil_1d(int C, int* nodes, double* w) {
  double x[8];
  const int half = g_rn / 2;
  for (int m = 0; m < g_rn; ++m) { nodes[m] = 2 * C - half + 1 + m; x[m] = -(half - 0.5) + m; }
  lagrange(x, g_rn, 0.0, w);
}

// ---------------------------------------------------------------------------
// Right-hand sides.

// Centred derivative stencils.  4th order over offsets -2..2:
const double D1W[5] = {1.0, -8.0, 0.0, 8.0, -1.0};       // / (12 h)
const double D2W[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};   // / (12 h^2)
// 8th order over offsets -4..4 (the paper's production differences, Sec. III.C):
const double D1W8[9] = {3.0, -32.0, 168.0, -672.0, 0.0, 672.0, -168.0, 32.0, -3.0};              // / (840 h)
const double D2W8[9] = {-9.0, 128.0, -1008.0, 8064.0, -14350.0, 8064.0, -1008.0, 128.0, -9.0};  // / (5040 h^2)

// Scalar wave (Sec. IV.A): d_t u = Pi, d_t Pi = Laplacian u; centred differences of the chosen order.
void wave_rhs_cell(const BoxData& B, const double* Y, double* K, int i, int j, int k, double h, int order) {
  const long c = B.off(i, j, k);
  const long s[3] = {1, (long)B.N[0], (long)B.N[0] * B.N[1]};
  const double* u = Y;
  const double* pi = Y + B.vol;
  double lap = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (order == 8) {
      double acc = 0.0;
      for (int m = 0; m < 9; ++m) acc += D2W8[m] * u[c + (m - 4) * s[d]];
      lap += acc / (5040.0 * h * h);
    } else {
      lap += (-u[c - 2 * s[d]] + 16.0 * u[c - s[d]] - 30.0 * u[c] + 16.0 * u[c + s[d]] - u[c + 2 * s[d]]) /
             (12.0 * h * h);
    }
  }
  K[c] = pi[c];
  K[B.vol + c] = lap;
}

const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
const int SYMI[6] = {0, 0, 0, 1, 1, 2};
const int SYMJ[6] = {0, 1, 2, 1, 2, 2};
// Z4c field order: W, gt(6), Khat, At(6), Gamt(3), Theta, alpha, beta(3).
enum { FW = 0, FG = 1, FK = 7, FA = 8, FGAM = 14, FTH = 17, FAL = 18, FB = 19, NZ4C = 22 };

// Z4c evolution equations (Sec. III.A), vacuum, with the puncture gauge
// (Eqs. punclapse, puncshift) at constant eta.  u: fields at the cell;
// du[f][k] = d_k u_f; dd[f][s] = second derivative of u_f for symmetric pair s.
template <class T>
void z4c_point(const T* u, const T (*du)[3], const T (*dd)[6], T* rhs, double kappa1,
               double kappa2, double eta, T* diag = nullptr) {
  const T W = u[FW];
  T g[3][3], A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) { g[i][j] = u[FG + SYM[i][j]]; A[i][j] = u[FA + SYM[i][j]]; }
  const T Kh = u[FK], Th = u[FTH], al = u[FAL];
  T Gam[3], be[3];
  for (int i = 0; i < 3; ++i) { Gam[i] = u[FGAM + i]; be[i] = u[FB + i]; }
  // derivatives
  T dW[3], dal[3], dKh[3], dTh[3], ddW[3][3], ddal[3][3];
  T dg[3][3][3];       // dg[k][i][j] = d_k gt_ij
  T ddg[3][3][3][3];   // ddg[i][j][l][m] = d_l d_m gt_ij
  T dGam[3][3];        // dGam[i][j] = d_j Gamt^i
  T dbe[3][3];         // dbe[i][j] = d_j beta^i
  T ddbe[3][3][3];     // ddbe[i][j][k] = d_j d_k beta^i
  for (int k = 0; k < 3; ++k) {
    dW[k] = du[FW][k]; dal[k] = du[FAL][k]; dKh[k] = du[FK][k]; dTh[k] = du[FTH][k];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ddW[i][j] = dd[FW][SYM[i][j]];
      ddal[i][j] = dd[FAL][SYM[i][j]];
      dGam[i][j] = du[FGAM + i][j];
      dbe[i][j] = du[FB + i][j];
      for (int k = 0; k < 3; ++k) {
        dg[k][i][j] = du[FG + SYM[i][j]][k];
        ddbe[i][j][k] = dd[FB + i][SYM[j][k]];
        for (int m = 0; m < 3; ++m) ddg[i][j][k][m] = dd[FG + SYM[i][j]][SYM[k][m]];
      }
    }
  // inverse conformal metric
  const T det = g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
                g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
                g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
  T gu[3][3];
  gu[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / det;
  gu[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / det;
  gu[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / det;
  gu[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / det;
  gu[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / det;
  gu[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / det;
  gu[1][0] = gu[0][1]; gu[2][0] = gu[0][2]; gu[2][1] = gu[1][2];
  // Christoffel symbols of gt: first kind Gl[k][i][j] = Gamma_{k ij}, second kind Gu
  T Gl[3][3][3], Gu[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Gl[k][i][j] = T(0.5) * (dg[i][j][k] + dg[j][i][k] - dg[k][i][j]);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T s = T(0.0);
        for (int l = 0; l < 3; ++l) s += gu[k][l] * Gl[l][i][j];
        Gu[k][i][j] = s;
      }
  // (Gamma_d)^i = gt^{jk} Gamma^i_{jk}
  T Gd[3];
  for (int i = 0; i < 3; ++i) {
    T s = T(0.0);
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += gu[j][k] * Gu[i][j][k];
    Gd[i] = s;
  }
  // Ricci tensor R_ij = R^W_ij + Rt_ij
  T R[3][3];
  T DDW[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = ddW[i][j];
      for (int k = 0; k < 3; ++k) s -= Gu[k][i][j] * dW[k];
      DDW[i][j] = s;
    }
  T trDDW = T(0.0), dWdW = T(0.0);
  for (int l = 0; l < 3; ++l)
    for (int m = 0; m < 3; ++m) { trDDW += gu[l][m] * DDW[l][m]; dWdW += gu[l][m] * dW[l] * dW[m]; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T rt = T(0.0);
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) rt -= T(0.5) * gu[l][m] * ddg[i][j][l][m];
      for (int k = 0; k < 3; ++k) rt += T(0.5) * (g[k][i] * dGam[k][j] + g[k][j] * dGam[k][i]);
      for (int k = 0; k < 3; ++k) rt += Gd[k] * T(0.5) * (Gl[i][j][k] + Gl[j][i][k]);
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m)
          for (int k = 0; k < 3; ++k)
            rt += gu[l][m] * (Gu[k][l][i] * Gl[j][k][m] + Gu[k][l][j] * Gl[i][k][m] + Gu[k][i][m] * Gl[k][l][j]);
      const T rw = (DDW[i][j] + g[i][j] * trDDW) / W - T(2.0) * g[i][j] * dWdW / (W * W);
      R[i][j] = rw + rt;
    }
  T trR = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trR += gu[i][j] * R[i][j];
  const T Rsc = W * W * trR;
  // D_i D_j alpha with the physical Christoffel symbols
  T gudW[3];
  for (int k = 0; k < 3; ++k) {
    T s = T(0.0);
    for (int l = 0; l < 3; ++l) s += gu[k][l] * dW[l];
    gudW[k] = s;
  }
  T DDal[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = ddal[i][j];
      for (int k = 0; k < 3; ++k) {
        T Gphys = Gu[k][i][j] - ((k == i ? dW[j] : T(0.0)) + (k == j ? dW[i] : T(0.0)) - g[i][j] * gudW[k]) / W;
        s -= Gphys * dal[k];
      }
      DDal[i][j] = s;
    }
  T trDDal = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trDDal += gu[i][j] * DDal[i][j];
  trDDal = W * W * trDDal;
  // At with raised indices
  T Amix[3][3], Auu[3][3];  // Amix[i][j] = At^i_j, Auu = At^{ij}
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s += gu[i][k] * A[k][j];
      Amix[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s += Amix[i][k] * gu[k][j];
      Auu[i][j] = s;
    }
  T AA = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += A[i][j] * Auu[i][j];
  const T divb = dbe[0][0] + dbe[1][1] + dbe[2][2];
  const T Kt = Kh + T(2.0) * Th;
  T adv[NZ4C];
  for (int f = 0; f < NZ4C; ++f) adv[f] = be[0] * du[f][0] + be[1] * du[f][1] + be[2] * du[f][2];

  rhs[FW] = adv[FW] + T(1.0 / 3.0) * W * (al * Kt - divb);
  T X[3][3], trX = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = -DDal[i][j] + al * R[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trX += gu[i][j] * X[i][j];
  for (int s = 0; s < 6; ++s) {
    const int i = SYMI[s], j = SYMJ[s];
    T r = adv[FG + s] - T(2.0) * al * A[i][j] - T(2.0 / 3.0) * g[i][j] * divb;
    for (int k = 0; k < 3; ++k) r += g[k][i] * dbe[k][j] + g[k][j] * dbe[k][i];
    rhs[FG + s] = r;
    T ra = adv[FA + s] + W * W * (X[i][j] - T(1.0 / 3.0) * g[i][j] * trX) + al * Kt * A[i][j] -
           T(2.0 / 3.0) * A[i][j] * divb;
    for (int k = 0; k < 3; ++k) ra += A[k][i] * dbe[k][j] + A[k][j] * dbe[k][i] - T(2.0) * al * Amix[k][i] * A[k][j];
    rhs[FA + s] = ra;
  }
  rhs[FK] = adv[FK] - trDDal + al * (AA + T(1.0 / 3.0) * Kt * Kt) + al * T(kappa1 * (1.0 - kappa2)) * Th;
  for (int i = 0; i < 3; ++i) {
    T r = adv[FGAM + i];
    T br = T(0.0);
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) br += Gu[i][j][k] * Auu[j][k];
    for (int j = 0; j < 3; ++j) {
      r -= T(2.0) * Auu[i][j] * dal[j];
      br -= T(3.0) * Auu[i][j] * dW[j] / W;
      br -= T(1.0 / 3.0) * gu[i][j] * (T(2.0) * dKh[j] + dTh[j]);
    }
    r += T(2.0) * al * br;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        r += gu[j][k] * ddbe[i][j][k];
        r += T(1.0 / 3.0) * gu[i][j] * ddbe[k][j][k];
      }
    for (int j = 0; j < 3; ++j) r -= Gd[j] * dbe[i][j];
    r += T(2.0 / 3.0) * Gd[i] * divb;
    r -= T(2.0 * kappa1) * al * (Gam[i] - Gd[i]);
    rhs[FGAM + i] = r;
  }
  rhs[FTH] = adv[FTH] + T(0.5) * al * (Rsc - AA + T(2.0 / 3.0) * Kt * Kt) - al * T(kappa1 * (2.0 + kappa2)) * Th;
  rhs[FAL] = adv[FAL] - T(2.0) * al * Kh;
  for (int i = 0; i < 3; ++i) rhs[FB + i] = adv[FB + i] + T(0.75) * Gam[i] - T(eta) * be[i];
  if (diag) { diag[0] = Rsc; diag[1] = AA; diag[2] = Kt; }
}

// Kreiss-Oliger with r = 4 (Sec. III.C): Q u = sigma / (64 h) sum_d delta_d^6 u.
const double KOW[7] = {1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0};

template <class T>
void z4c_derivs(const BoxData& B, const double* Y, long c, double h, T (*u)[1], T (*du)[3], T (*dd)[6], T* ko,
                int order = 4) {
  const long s[3] = {1, (long)B.N[0], (long)B.N[0] * B.N[1]};
  const int R = order / 2;  // reach of the derivative stencils
  const double* w1 = order == 8 ? D1W8 : D1W;
  const double* w2 = order == 8 ? D2W8 : D2W;
  const double n1 = order == 8 ? 840.0 : 12.0, n2 = order == 8 ? 5040.0 : 12.0;
  for (int f = 0; f < NZ4C; ++f) {
    const double* p = Y + (long)f * B.vol;
    u[f][0] = T(p[c]);
    for (int d = 0; d < 3; ++d) {
      T acc = T(0.0);
      for (int m = 0; m <= 2 * R; ++m) acc += T(w1[m]) * T(p[c + (m - R) * s[d]]);
      du[f][d] = acc / T(n1 * h);
    }
    for (int q = 0; q < 6; ++q) {
      const int a = SYMI[q], b = SYMJ[q];
      T acc = T(0.0);
      if (a == b) {
        for (int m = 0; m <= 2 * R; ++m) acc += T(w2[m]) * T(p[c + (m - R) * s[a]]);
        dd[f][q] = acc / T(n2 * h * h);
      } else {
        // mixed: product of the two first-derivative stencils
        for (int m = 0; m <= 2 * R; ++m)
          for (int n = 0; n <= 2 * R; ++n) {
            if (w1[m] == 0.0 || w1[n] == 0.0) continue;
            acc += T(w1[m] * w1[n]) * T(p[c + (m - R) * s[a] + (n - R) * s[b]]);
          }
        dd[f][q] = acc / T(n1 * n1 * h * h);
      }
    }
    T k = T(0.0);
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < 7; ++m) k += T(KOW[m]) * T(p[c + (m - 3) * s[d]]);
    ko[f] = k;
  }
}

void z4c_rhs_cell(const Hier& H, const BoxData& B, const double* Y, double* K, int i, int j, int k, double h,
                  const double* x);

// Gamma-driver damping: the constant eta, or the profile of Sec. III.A,
// eta(r) = (eta_c - eta_o) exp(-(r / eta_s)^4) + eta_o, r the coordinate radius.
double eta_at(const Hier& H, const double* x) {
  if (!H.eta_profile) return H.eta;
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  return (H.eta_c - H.eta_o) * std::exp(-std::pow(r / H.eta_s, 4.0)) + H.eta_o;
}

void z4c_rhs_cell(const Hier& H, const BoxData& B, const double* Y, double* K, int i, int j, int k, double h,
                  const double* x) {
  const long c = B.off(i, j, k);
  double u[NZ4C][1], du[NZ4C][3], dd[NZ4C][6], ko[NZ4C], uu[NZ4C], rhs[NZ4C];
  z4c_derivs<double>(B, Y, c, h, u, du, dd, ko, H.order);
  for (int f = 0; f < NZ4C; ++f) uu[f] = u[f][0];
  z4c_point<double>(uu, du, dd, rhs, H.kappa1, H.kappa2, eta_at(H, x));
  for (int f = 0; f < NZ4C; ++f) K[(long)f * B.vol + c] = rhs[f] + H.sigma / (64.0 * h) * ko[f];
}

// Outgoing radiative condition on the outer ghost cells of level 0:
// d_t u = -(x^i/r) d_i u - (u - u_inf)/r, unit speed; 2nd-order differences,
// centred where both neighbours exist in the array, one-sided inwards on the
// outermost layer.
double u_inf(const Hier& H, int f) {
  if (H.system != ORC_Z4C) return 0.0;
  if (f == FW || f == FAL || f == FG + 0 || f == FG + 3 || f == FG + 5) return 1.0;
  return 0.0;
}

void radiative_rhs_cell(const Hier& H, const BoxData& B, const double* Y, double* K, int i, int j, int k,
                        double h, const double* x) {
  const long c = B.off(i, j, k);
  const long s[3] = {1, (long)B.N[0], (long)B.N[0] * B.N[1]};
  const int li[3] = {i, j, k};
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  for (int f = 0; f < H.F; ++f) {
    const double* p = Y + (long)f * B.vol;
    double adv = 0.0;
    for (int d = 0; d < 3; ++d) {
      double der;
      if (li[d] == -B.g) der = (-3.0 * p[c] + 4.0 * p[c + s[d]] - p[c + 2 * s[d]]) / (2.0 * h);
      else if (li[d] == B.n[d] + B.g - 1) der = (3.0 * p[c] - 4.0 * p[c - s[d]] + p[c - 2 * s[d]]) / (2.0 * h);
      else der = (p[c + s[d]] - p[c - s[d]]) / (2.0 * h);
      adv += (x[d] / r) * der;
    }
    K[(long)f * B.vol + c] = -adv - (p[c] - u_inf(H, f)) / r;
  }
}

void cell_centre(const Hier& H, int l, const BoxData& B, int i, int j, int k, double* x) {
  const double h = H.lev[l].h;
  x[0] = H.origin[0] + (B.lo[0] + i + 0.5) * h;
  x[1] = H.origin[1] + (B.lo[1] + j + 0.5) * h;
  x[2] = H.origin[2] + (B.lo[2] + k + 0.5) * h;
}

bool is_interior(const BoxData& B, int i, int j, int k) {
  return i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1] && k >= 0 && k < B.n[2];
}

bool evolves_shell(const Hier& H, int l) { return l == 0 && H.bc == ORC_BC_RADIATIVE; }

// k = f(Y) on the evolved cells of one box.
void rhs_box(const Hier& H, int l, const BoxData& B, const double* Y, double* K) {
  const double h = H.lev[l].h;
  for (int k = -B.g; k < B.n[2] + B.g; ++k)
    for (int j = -B.g; j < B.n[1] + B.g; ++j)
      for (int i = -B.g; i < B.n[0] + B.g; ++i) {
        if (is_interior(B, i, j, k)) {
          if (H.system == ORC_WAVE) {
            wave_rhs_cell(B, Y, K, i, j, k, h, H.order);
          } else {
            double x[3];
            cell_centre(H, l, B, i, j, k, x);
            z4c_rhs_cell(H, B, Y, K, i, j, k, h, x);
          }
        } else if (evolves_shell(H, l)) {
          double x[3];
          cell_centre(H, l, B, i, j, k, x);
          radiative_rhs_cell(H, B, Y, K, i, j, k, h, x);
        }
      }
}

// Apply fn(local offset) over the evolved cells of a box.
template <class Fn>
void for_evolved(const Hier& H, int l, const BoxData& B, Fn fn) {
  for (int k = -B.g; k < B.n[2] + B.g; ++k)
    for (int j = -B.g; j < B.n[1] + B.g; ++j)
      for (int i = -B.g; i < B.n[0] + B.g; ++i)
        if (is_interior(B, i, j, k) || evolves_shell(H, l)) fn(B.off(i, j, k));
}

// ---------------------------------------------------------------------------
// Ghost filling.

void copy_siblings(Hier& H, int l, int vec) {
  Level& L = H.lev[l];
  for (BoxData& B : L.boxes) {
    for (size_t q = 0; q < B.sib_dst.size(); ++q) {
      const BoxData& S = L.boxes[B.sib_box[q]];
      for (int f = 0; f < H.F; ++f) B.v[vec][(long)f * B.vol + B.sib_dst[q]] = S.v[vec][(long)f * S.vol + B.sib_src[q]];
    }
  }
}


// Parent-level location of the tensor stencil nodes[d][0..n-1]: if the whole
// block lies inside one box interior (the usual case) return that box and the
// local index of the first node, else -1 (callers then look up point by point).
int find_block(const Hier& H, int l, int (*nodes)[8], int n, int* li0) {
  const int g0[3] = {nodes[0][0], nodes[1][0], nodes[2][0]};
  const int g1[3] = {nodes[0][n - 1], nodes[1][n - 1], nodes[2][n - 1]};
  int a[3], b[3];
  const int ba = find_interior(H, l, g0, a);
  const int bb = find_interior(H, l, g1, b);
  if (ba < 0 || ba != bb) return -1;
  for (int d = 0; d < 3; ++d)
    if (b[d] - a[d] != n - 1) return -1;  // wrapped across the periodic seam
  for (int d = 0; d < 3; ++d) li0[d] = a[d];
  return ba;
}

// Offset of stencil node (cx, cy, cz) in the parent level: fast path through
// the block found by find_block, else a point lookup.
long node_offset(const Hier& H, int l, int (*nodes)[8], int blk, const int* li0, int cx, int cy, int cz,
                 int* box) {
  if (blk >= 0) {
    *box = blk;
    return H.lev[l].boxes[blk].off(li0[0] + cx, li0[1] + cy, li0[2] + cz);
  }
  const int pg[3] = {nodes[0][cx], nodes[1][cy], nodes[2][cz]};
  int li[3];
  *box = find_interior(H, l, pg, li);
  return H.lev[l].boxes[*box].off(li[0], li[1], li[2]);
}

int rk_stages_of(const Hier& H) { return H.rk; }
// Stage vectors the dense output reads: k1..k4 (RK3: k4 = f(y_{n+1})), k1..k2 for RK2.
int dense_vectors_of(const Hier& H) { return H.rk == 2 ? 2 : 4; }

// Step 2 of the algorithm: prolong the parent's y_n and k1..k_s to the
// refinement-boundary ghost cells of level l (tensor-product quintic Lagrange).
void prolong_parent_vectors(Hier& H, int l) {
  Level& L = H.lev[l];
  const int src_vec[5] = {V_YOLD, V_K1, V_K1 + 1, V_K1 + 2, V_K1 + 3};
  for (BoxData& B : L.boxes) {
    const size_t na = B.amr_cell.size();
    B.amr_P.assign(na * 5 * H.F, 0.0);
    for (size_t a = 0; a < na; ++a) {
      int nodes[3][8];
      double w[3][8];
      for (int d = 0; d < 3; ++d) prolong_stencil_1d(B.amr_glob[3 * a + d], nodes[d], w[d]);
      int li0[3];
      const int blk = find_block(H, l - 1, nodes, g_pn, li0);
      for (int cz = 0; cz < g_pn; ++cz)
        for (int cy = 0; cy < g_pn; ++cy)
          for (int cx = 0; cx < g_pn; ++cx) {
            int pb;
            const long po = node_offset(H, l - 1, nodes, blk, li0, cx, cy, cz, &pb);
            const BoxData& P = H.lev[l - 1].boxes[pb];
            const double ww = w[0][cx] * w[1][cy] * w[2][cz];
            for (int v = 0; v <= dense_vectors_of(H); ++v)
              for (int f = 0; f < H.F; ++f)
                B.amr_P[(a * 5 + v) * H.F + f] += ww * P.v[src_vec[v]][(long)f * P.vol + po];
          }
    }
  }
}

// Unsubcycled variant: prolong one parent vector directly into the AMR ghosts.
void prolong_direct(Hier& H, int l, int parent_vec, int dst_vec) {
  Level& L = H.lev[l];
  for (BoxData& B : L.boxes) {
    for (size_t a = 0; a < B.amr_cell.size(); ++a) {
      int nodes[3][8];
      double w[3][8];
      for (int d = 0; d < 3; ++d) prolong_stencil_1d(B.amr_glob[3 * a + d], nodes[d], w[d]);
      for (int f = 0; f < H.F; ++f) B.v[dst_vec][(long)f * B.vol + B.amr_cell[a]] = 0.0;
      int li0[3];
      const int blk = find_block(H, l - 1, nodes, g_pn, li0);
      for (int cz = 0; cz < g_pn; ++cz)
        for (int cy = 0; cy < g_pn; ++cy)
          for (int cx = 0; cx < g_pn; ++cx) {
            int pb;
            const long po = node_offset(H, l - 1, nodes, blk, li0, cx, cy, cz, &pb);
            const BoxData& P = H.lev[l - 1].boxes[pb];
            const double ww = w[0][cx] * w[1][cy] * w[2][cz];
            for (int f = 0; f < H.F; ++f)
              B.v[dst_vec][(long)f * B.vol + B.amr_cell[a]] += ww * P.v[parent_vec][(long)f * P.vol + po];
          }
    }
  }
}

// Step 3 / 5: refinement-boundary ghosts of vector vec from the prolonged
// parent vectors, for the fine substep starting at theta0.
void fill_amr(Hier& H, int l, int vec, double theta0, int which) {
  Level& L = H.lev[l];
  const double Hp = H.lev[l - 1].dt;
  for (BoxData& B : L.boxes) {
    for (size_t a = 0; a < B.amr_cell.size(); ++a)
      for (int f = 0; f < H.F; ++f) {
        const double* P = &B.amr_P[a * 5 * H.F];
        const double y = P[f];
        const double k[4] = {P[H.F + f], P[2 * H.F + f], P[3 * H.F + f], P[4 * H.F + f]};
        B.v[vec][(long)f * B.vol + B.amr_cell[a]] = amr_value_rk(H.rk, y, k, Hp, theta0, which);
      }
  }
}

void fill_physical_callback(Hier& H, int vec, int which, double t_n, double dt) {
  if (H.bc != ORC_BC_CALLBACK || !H.cb) return;
  Level& L = H.lev[0];
  for (BoxData& B : L.boxes) {
    const int np = (int)B.phys_cell.size();
    if (np == 0) continue;
    std::vector<double> xyz(3 * (size_t)np), out((size_t)H.F * np);
    for (int p = 0; p < np; ++p) {
      long o = B.phys_cell[p];
      const int i = (int)(o % B.N[0]) - B.g;
      const int j = (int)((o / B.N[0]) % B.N[1]) - B.g;
      const int k = (int)(o / ((long)B.N[0] * B.N[1])) - B.g;
      cell_centre(H, 0, B, i, j, k, &xyz[3 * (size_t)p]);
    }
    H.cb(H.cb_user, which, t_n, dt, np, xyz.data(), out.data());
    for (int p = 0; p < np; ++p)
      for (int f = 0; f < H.F; ++f) B.v[vec][(long)f * B.vol + B.phys_cell[p]] = out[(size_t)f * np + p];
  }
}

// All ghosts of vector vec on level l for stage `which` (0 = end of step).
void fill_ghosts(Hier& H, int l, int vec, double theta0, int which, double t_n, double dt) {
  if (l > 0) fill_amr(H, l, vec, theta0, which);
  if (l == 0) fill_physical_callback(H, vec, which, t_n, dt);
  copy_siblings(H, l, vec);
}

// Step 7: restrict level l onto level l-1 (vector y): every parent cell whose
// 8 children are fine interior cells takes the tensor-product quintic
// interpolant of the 6^3 fine cells around its centre.
void restrict_level(Hier& H, int l) {
  Level& P = H.lev[l - 1];
  for (BoxData& PB : P.boxes) {
    for (int k = 0; k < PB.n[2]; ++k)
      for (int j = 0; j < PB.n[1]; ++j)
        for (int i = 0; i < PB.n[0]; ++i) {
          const int C[3] = {PB.lo[0] + i, PB.lo[1] + j, PB.lo[2] + k};
          bool covered = true;
          for (int q = 0; q < 8 && covered; ++q) {
            const int fg[3] = {2 * C[0] + (q & 1), 2 * C[1] + ((q >> 1) & 1), 2 * C[2] + ((q >> 2) & 1)};
            int li[3];
            covered = find_interior(H, l, fg, li) >= 0;
          }
          if (!covered) continue;
          int nodes[3][8];
          double w[3][8];
          for (int d = 0; d < 3; ++d) restrict_stencil_1d(C[d], nodes[d], w[d]);
          const long po = PB.off(i, j, k);
          for (int f = 0; f < H.F; ++f) PB.v[V_Y][(long)f * PB.vol + po] = 0.0;
          for (int cz = 0; cz < g_rn; ++cz)
            for (int cy = 0; cy < g_rn; ++cy)
              for (int cx = 0; cx < g_rn; ++cx) {
                const int fg[3] = {nodes[0][cx], nodes[1][cy], nodes[2][cz]};
                int li[3];
                const int fb = find_ghosted(H, l, fg, li);
                const BoxData& FB = H.lev[l].boxes[fb];
                const long fo = FB.off(li[0], li[1], li[2]);
                const double ww = w[0][cx] * w[1][cy] * w[2][cz];
                for (int f = 0; f < H.F; ++f) PB.v[V_Y][(long)f * PB.vol + po] += ww * FB.v[V_Y][(long)f * FB.vol + fo];
              }
        }
  }
  copy_siblings(H, l - 1, V_Y);
}

// ---------------------------------------------------------------------------
// Time stepping (Sec. II).

const double RK_C[3] = {0.5, 0.5, 1.0};

// Stages of the method and the multiplier of k_{s-1} in stage input s >= 2
// (every method here builds stage s from y_n and k_{s-1} alone).
int rk_stages(const Hier& H) { return rk_stages_of(H); }
double rk_stage_c(const Hier& H, int s) {
  if (H.rk == 4) return RK_C[s - 2];
  if (H.rk == 3) return s == 2 ? 1.0 / 3.0 : 2.0 / 3.0;
  return 0.5;
}

// Stage input s of level l from y_n (V_YOLD) and k_{s-1}.
void stage_input(Hier& H, int l, BoxData& B, int s, double dt) {
  if (s == 1) {
    B.v[V_STAGE] = B.v[V_YOLD];
    return;
  }
  const double c = rk_stage_c(H, s) * dt;
  for (int f = 0; f < H.F; ++f) {
    const long fo = (long)f * B.vol;
    const std::vector<double>& kp = B.v[V_K1 + s - 2];
    for_evolved(H, l, B, [&](long o) { B.v[V_STAGE][fo + o] = B.v[V_YOLD][fo + o] + c * kp[fo + o]; });
  }
}

// y_{n+1} from y_n and the stage vectors: Eq. rk5 for RK4; midpoint and
// Heun's third-order combinations for RK2 and RK3.
void final_update(Hier& H, int l, BoxData& B, double dt) {
  for (int f = 0; f < H.F; ++f) {
    const long fo = (long)f * B.vol;
    const std::vector<double>& y0 = B.v[V_YOLD];
    const std::vector<double>& k1 = B.v[V_K1];
    const std::vector<double>& k2 = B.v[V_K1 + 1];
    const std::vector<double>& k3 = B.v[V_K1 + 2];
    const std::vector<double>& k4 = B.v[V_K1 + 3];
    std::vector<double>& y = B.v[V_Y];
    if (H.rk == 4)
      for_evolved(H, l, B, [&](long o) {
        y[fo + o] = y0[fo + o] + dt / 6.0 * (k1[fo + o] + 2.0 * k2[fo + o] + 2.0 * k3[fo + o] + k4[fo + o]);
      });
    else if (H.rk == 3)
      for_evolved(H, l, B, [&](long o) { y[fo + o] = y0[fo + o] + dt * (0.25 * k1[fo + o] + 0.75 * k3[fo + o]); });
    else
      for_evolved(H, l, B, [&](long o) { y[fo + o] = y0[fo + o] + dt * k2[fo + o]; });
  }
}

// One RK step of level l (Eqs. rk1-rk5 for RK4).  For l >= 1 the step is the
// fine substep starting at progress theta0 of the parent step; its
// refinement-boundary ghosts come from the parent's dense output.  The stage
// vectors k_i are kept.
void step_level(Hier& H, int l, double theta0) {
  Level& L = H.lev[l];
  const double dt = L.dt;
  const double t_n = L.t;
  for (BoxData& B : L.boxes) B.v[V_YOLD] = B.v[V_Y];
  for (int s = 1; s <= rk_stages(H); ++s) {
    for (BoxData& B : L.boxes) stage_input(H, l, B, s, dt);
    fill_ghosts(H, l, V_STAGE, theta0, s, t_n, dt);
    for (BoxData& B : L.boxes) rhs_box(H, l, B, B.v[V_STAGE].data(), B.v[V_K1 + s - 1].data());
  }
  for (BoxData& B : L.boxes) final_update(H, l, B, dt);
  fill_ghosts(H, l, V_Y, theta0, 0, t_n, dt);
  // RK3 dense output: k4 = f(y_{n+1}) on levels that have a finer level
  if (H.rk == 3 && l + 1 < H.nlev)
    for (BoxData& B : L.boxes) rhs_box(H, l, B, B.v[V_Y].data(), B.v[V_K1 + 3].data());
  L.t = t_n + dt;
}

// Steps 2-7 below level l: two fine substeps of level l+1 at theta0 = 0 and
// 1/2 with recursion after each, then restriction onto level l.
void advance_children(Hier& H, int l) {
  prolong_parent_vectors(H, l + 1);
  for (int s = 0; s < 2; ++s) {
    step_level(H, l + 1, 0.5 * s);
    if (l + 2 < H.nlev) advance_children(H, l + 1);
  }
  restrict_level(H, l + 1);
}

void coarse_step_subcycled(Hier& H) {
  step_level(H, 0, 0.0);
  if (H.nlev > 1) advance_children(H, 0);
}

// Uniform time step on all levels (the comparison mode): the levels advance
// stage by stage in lockstep, refinement-boundary ghosts are the prolonged
// parent stage state of the same stage.
void global_step_uniform(Hier& H, double dt) {
  const double t_n = H.lev[0].t;
  for (int l = 0; l < H.nlev; ++l)
    for (BoxData& B : H.lev[l].boxes) B.v[V_YOLD] = B.v[V_Y];
  for (int s = 1; s <= rk_stages(H); ++s) {
    for (int l = 0; l < H.nlev; ++l) {
      for (BoxData& B : H.lev[l].boxes) stage_input(H, l, B, s, dt);
      if (l > 0) prolong_direct(H, l, V_STAGE, V_STAGE);
      if (l == 0) fill_physical_callback(H, V_STAGE, s, t_n, dt);
      copy_siblings(H, l, V_STAGE);
      for (BoxData& B : H.lev[l].boxes) rhs_box(H, l, B, B.v[V_STAGE].data(), B.v[V_K1 + s - 1].data());
    }
  }
  for (int l = 0; l < H.nlev; ++l)
    for (BoxData& B : H.lev[l].boxes) final_update(H, l, B, dt);
  // ghosts of the new state first (restriction reads fine ghosts next to the
  // fine interior), from the parent's new state, then restriction.
  for (int l = 0; l < H.nlev; ++l) {
    if (l > 0) prolong_direct(H, l, V_Y, V_Y);
    if (l == 0) fill_physical_callback(H, V_Y, 0, t_n, dt);
    copy_siblings(H, l, V_Y);
    H.lev[l].t = t_n + dt;
  }
  for (int l = H.nlev - 1; l >= 1; --l) restrict_level(H, l);
}

// ---------------------------------------------------------------------------
// Construction: ghost classification and the nesting checks.

int classify(Hier& H) {
  for (int l = 0; l < H.nlev; ++l) {
    Level& L = H.lev[l];
    for (size_t b = 0; b < L.boxes.size(); ++b) {
      BoxData& B = L.boxes[b];
      for (int k = -B.g; k < B.n[2] + B.g; ++k)
        for (int j = -B.g; j < B.n[1] + B.g; ++j)
          for (int i = -B.g; i < B.n[0] + B.g; ++i) {
            if (is_interior(B, i, j, k)) continue;
            const long o = B.off(i, j, k);
            int g[3] = {B.lo[0] + i, B.lo[1] + j, B.lo[2] + k};
            bool outside = false;
            for (int d = 0; d < 3; ++d) {
              if (H.bc == ORC_BC_PERIODIC) g[d] = wrapi(g[d], L.ext[d]);
              else if (g[d] < 0 || g[d] >= L.ext[d]) outside = true;
            }
            if (outside) {
              if (l != 0) return fail(-4, "fine level reaches the outer boundary");
              B.phys_cell.push_back(o);
              continue;
            }
            int li[3];
            const int sb = find_interior(H, l, g, li);
            if (sb >= 0) {
              B.sib_dst.push_back(o);
              B.sib_box.push_back(sb);
              B.sib_src.push_back(L.boxes[sb].off(li[0], li[1], li[2]));
              continue;
            }
            if (l == 0) return fail(-4, "level 0 does not cover the domain");
            // refinement boundary: the prolongation stencil must lie in the parent interior
            for (int d = 0; d < 3; ++d) B.amr_glob.push_back(g[d]);
            B.amr_cell.push_back(o);
            int nodes[3][8];
            double w[3][8];
            for (int d = 0; d < 3; ++d) prolong_stencil_1d(g[d], nodes[d], w[d]);
            for (int cz = 0; cz < g_pn; ++cz)
              for (int cy = 0; cy < g_pn; ++cy)
                for (int cx = 0; cx < g_pn; ++cx) {
                  const int pg[3] = {nodes[0][cx], nodes[1][cy], nodes[2][cz]};
                  if (find_interior(H, l - 1, pg, li) < 0)
                    return fail(-4, "prolongation stencil leaves the parent interior (proper nesting)");
                }
          }
    }
  }
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.

extern "C" {

int orc_create(int system, int nlevels, const int* nboxes, const int* boxes, const int* ncells0,
               const double* origin, double h0, int bc, double cfl, int subcycle, const double* params,
               void** out) {
  return orc_create_ex(system, nlevels, nboxes, boxes, ncells0, origin, h0, bc, cfl, subcycle, params, 4, 4, out);
}

int orc_create_ex(int system, int nlevels, const int* nboxes, const int* boxes, const int* ncells0,
                  const double* origin, double h0, int bc, double cfl, int subcycle, const double* params,
                  int fd_order, int rk_order, void** out) {
  if (fd_order != 4 && fd_order != 8) return fail(-1, "fd_order must be 4 or 8");
  if (rk_order < 2 || rk_order > 4) return fail(-1, "rk_order must be 2, 3 or 4");
  if (!out || nlevels < 1 || !nboxes || !boxes || !ncells0 || !origin) return fail(-1, "bad arguments");
  if (system != ORC_WAVE && system != ORC_Z4C) return fail(-1, "unknown system");
  Hier* H = new Hier();
  H->system = system;
  H->F = (system == ORC_WAVE) ? 2 : NZ4C;
  H->nlev = nlevels;
  H->bc = bc;
  H->subcycle = subcycle;
  H->order = fd_order;
  H->rk = rk_order;
  H->cfl = cfl;
  H->h0 = h0;
  for (int d = 0; d < 3; ++d) { H->origin[d] = origin[d]; H->ncells0[d] = ncells0[d]; }
  H->kappa1 = params ? params[0] : 0.02;
  H->kappa2 = params ? params[1] : 0.0;
  H->eta = params ? params[2] : 2.0;
  H->sigma = params ? params[3] : 0.3;
  H->t = 0.0;
  H->zu_finest = H->zu_actual = 0.0;
  H->cb = nullptr;
  H->cb_user = nullptr;
  H->eta_profile = false;
  H->eta_c = H->eta_s = H->eta_o = 0.0;
  H->lev.resize(nlevels);
  int bi = 0;
  for (int l = 0; l < nlevels; ++l) {
    Level& L = H->lev[l];
    L.h = h0 / std::pow(2.0, l);
    L.dt = cfl * L.h;
    L.t = 0.0;
    for (int d = 0; d < 3; ++d) L.ext[d] = ncells0[d] << l;
    if (nboxes[l] < 1) { delete H; return fail(-1, "empty level"); }
    for (int b = 0; b < nboxes[l]; ++b, ++bi) {
      BoxData B;
      B.g = fd_order == 8 ? 4 : 3;
      for (int d = 0; d < 3; ++d) {
        B.lo[d] = boxes[6 * bi + d];
        B.hi[d] = boxes[6 * bi + 3 + d];
        if (B.hi[d] < B.lo[d] || B.lo[d] < 0 || B.hi[d] >= L.ext[d]) { delete H; return fail(-1, "box outside level"); }
        if (l > 0 && ((B.lo[d] & 1) || !(B.hi[d] & 1))) { delete H; return fail(-4, "fine box not aligned to parent cells"); }
        B.n[d] = B.hi[d] - B.lo[d] + 1;
        B.N[d] = B.n[d] + 2 * B.g;
      }
      B.vol = (long)B.N[0] * B.N[1] * B.N[2];
      for (int v = 0; v < V_NVEC; ++v) B.v[v].assign((size_t)H->F * B.vol, 0.0);
      L.boxes.push_back(B);
    }
    // boxes of one level must not overlap
    for (size_t a = 0; a < L.boxes.size(); ++a)
      for (size_t b = a + 1; b < L.boxes.size(); ++b) {
        bool ov = true;
        for (int d = 0; d < 3; ++d)
          ov = ov && L.boxes[a].lo[d] <= L.boxes[b].hi[d] && L.boxes[b].lo[d] <= L.boxes[a].hi[d];
        if (ov) { delete H; return fail(-1, "overlapping boxes"); }
      }
  }
  if (bc == ORC_BC_RADIATIVE && H->lev[0].boxes.size() != 1) { delete H; return fail(-1, "radiative boundary needs one level-0 box"); }
  const int rc = classify(*H);
  if (rc) { delete H; return rc; }
  *out = H;
  return 0;
}

void orc_destroy(void* h) { delete static_cast<Hier*>(h); }
int orc_nfields(void* h) { return static_cast<Hier*>(h)->F; }

int orc_set_eta_profile(void* h, double eta_c, double eta_s, double eta_o) {
  Hier* H = static_cast<Hier*>(h);
  if (!(eta_s > 0)) return fail(-1, "eta_s must be positive");
  H->eta_profile = true;
  H->eta_c = eta_c;
  H->eta_s = eta_s;
  H->eta_o = eta_o;
  return 0;
}

int orc_set_bc_callback(void* h, orc_bc_fn fn, void* user) {
  Hier* H = static_cast<Hier*>(h);
  H->cb = fn;
  H->cb_user = user;
  return 0;
}

static BoxData* get_box(Hier* H, int l, int b) {
  if (l < 0 || l >= H->nlev || b < 0 || b >= (int)H->lev[l].boxes.size()) return nullptr;
  return &H->lev[l].boxes[b];
}

int orc_set_field(void* h, int l, int b, int f, const double* src) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* B = get_box(H, l, b);
  if (!B || f < 0 || f >= H->F) return fail(-1, "bad index");
  long q = 0;
  for (int k = 0; k < B->n[2]; ++k)
    for (int j = 0; j < B->n[1]; ++j)
      for (int i = 0; i < B->n[0]; ++i) B->v[V_Y][(long)f * B->vol + B->off(i, j, k)] = src[q++];
  return 0;
}

int orc_get_field(void* h, int l, int b, int f, double* dst) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* B = get_box(H, l, b);
  if (!B || f < 0 || f >= H->F) return fail(-1, "bad index");
  long q = 0;
  for (int k = 0; k < B->n[2]; ++k)
    for (int j = 0; j < B->n[1]; ++j)
      for (int i = 0; i < B->n[0]; ++i) dst[q++] = B->v[V_Y][(long)f * B->vol + B->off(i, j, k)];
  return 0;
}

int orc_set_field_ghosted(void* h, int l, int b, int f, const double* src) {
  return orc_debug_set_vector(h, l, b, V_Y, f, src);
}
int orc_get_field_ghosted(void* h, int l, int b, int f, double* dst) {
  return orc_debug_get_vector(h, l, b, V_Y, f, dst);
}

int orc_debug_set_vector(void* h, int l, int b, int vec, int f, const double* src) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* B = get_box(H, l, b);
  if (!B || f < 0 || f >= H->F || vec < 0 || vec >= V_NVEC) return fail(-1, "bad index");
  std::memcpy(&B->v[vec][(long)f * B->vol], src, sizeof(double) * B->vol);
  return 0;
}

int orc_debug_get_vector(void* h, int l, int b, int vec, int f, double* dst) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* B = get_box(H, l, b);
  if (!B || f < 0 || f >= H->F || vec < 0 || vec >= V_NVEC) return fail(-1, "bad index");
  std::memcpy(dst, &B->v[vec][(long)f * B->vol], sizeof(double) * B->vol);
  return 0;
}

int orc_set_initial_data(void* h, int kind, const double* p, int np) {
  Hier* H = static_cast<Hier*>(h);
  for (int l = 0; l < H->nlev; ++l)
    for (BoxData& B : H->lev[l].boxes)
      for (int k = -B.g; k < B.n[2] + B.g; ++k)
        for (int j = -B.g; j < B.n[1] + B.g; ++j)
          for (int i = -B.g; i < B.n[0] + B.g; ++i) {
            double x[3];
            cell_centre(*H, l, B, i, j, k, x);
            const long o = B.off(i, j, k);
            double val[NZ4C];
            for (int f = 0; f < NZ4C; ++f) val[f] = 0.0;
            if (kind == ORC_ID_STANDING_WAVE && H->system == ORC_WAVE && np >= 4) {
              // u = A sin(2 pi kx x) sin(2 pi ky y) sin(2 pi kz z) at t = 0, Pi = 0
              const double tp = 2.0 * M_PI;
              val[0] = p[0] * std::sin(tp * p[1] * x[0]) * std::sin(tp * p[2] * x[1]) * std::sin(tp * p[3] * x[2]);
              val[1] = 0.0;
            } else if (kind == ORC_ID_GAUSSIAN && H->system == ORC_WAVE && np >= 5) {
              // u = A exp(-|x - c|^2 / (2 w^2)), Pi = 0
              const double dx = x[0] - p[2], dy = x[1] - p[3], dz = x[2] - p[4];
              val[0] = p[0] * std::exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * p[1] * p[1]));
              val[1] = 0.0;
            } else if (kind == ORC_ID_SPHERICAL_GAUSSIAN && H->system == ORC_WAVE && np >= 6) {
              // Sec. IV.A: u = (f(t-r) - f(t+r))/r, Pi = -(f(t-r)(t-r) - f(t+r)(t+r))/(sigma^2 r)
              const double A = p[0], sg = p[1], t = p[2];
              const double dx = x[0] - p[3], dy = x[1] - p[4], dz = x[2] - p[5];
              const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
              const double fm = A * std::exp(-(t - r) * (t - r) / (2.0 * sg * sg));
              const double fp = A * std::exp(-(t + r) * (t + r) / (2.0 * sg * sg));
              val[0] = (fm - fp) / r;
              val[1] = -(fm * (t - r) - fp * (t + r)) / (sg * sg * r);
            } else if (((kind == ORC_ID_BRILL_LINDQUIST || kind == ORC_ID_BRILL_LINDQUIST_AVG_LAPSE) && np >= 8) ||
                       kind == ORC_ID_MINKOWSKI) {
              if (H->system != ORC_Z4C) return fail(-1, "initial data needs Z4c");
              double psi = 1.0, s = 0.0;
              if (kind != ORC_ID_MINKOWSKI) {
                for (int q = 0; q < 2; ++q) {
                  const double m = p[4 * q], dx = x[0] - p[4 * q + 1], dy = x[1] - p[4 * q + 2],
                               dz = x[2] - p[4 * q + 3];
                  s += m / (2.0 * std::sqrt(dx * dx + dy * dy + dz * dz));
                }
                psi += s;
              }
              // gamma_ij = psi^4 delta_ij: W = gamma^{-1/6} = psi^-2, gt_ij = delta_ij,
              // K_ij = 0, Theta = 0, Gamt^i = 0, lapse psi^-2, zero shift.
              val[FW] = 1.0 / (psi * psi);
              val[FG + 0] = val[FG + 3] = val[FG + 5] = 1.0;
              val[FAL] = 1.0 / (psi * psi);
              // Sec. III.B: the averaged initial lapse 1/2 (1 + (1 - s) / (1 + s))
              if (kind == ORC_ID_BRILL_LINDQUIST_AVG_LAPSE) val[FAL] = 0.5 * (1.0 + (1.0 - s) / (1.0 + s));
            } else {
              return fail(-1, "unknown initial data");
            }
            for (int f = 0; f < H->F; ++f) B.v[V_Y][(long)f * B.vol + o] = val[f];
          }
  return 0;
}

int orc_advance(void* h, int n) {
  Hier* H = static_cast<Hier*>(h);
  if (n < 0) return fail(-1, "negative step count");
  const int L = H->nlev;
  double ncell[32] = {0};
  for (int l = 0; l < L; ++l)
    for (BoxData& B : H->lev[l].boxes) ncell[l] += (double)B.n[0] * B.n[1] * B.n[2];
  for (int s = 0; s < n; ++s) {
    if (H->subcycle) {
      coarse_step_subcycled(*H);
    } else {
      const int nf = 1 << (L - 1);
      for (int q = 0; q < nf; ++q) global_step_uniform(*H, H->lev[L - 1].dt);
    }
    H->t += H->lev[0].dt;
    for (int l = 0; l < L; ++l) {
      H->lev[l].t = H->t;
      H->zu_finest += (double)(1 << (L - 1)) * ncell[l];
      H->zu_actual += (double)(H->subcycle ? (1 << l) : (1 << (L - 1))) * ncell[l];
    }
  }
  return 0;
}

double orc_time(void* h) { return static_cast<Hier*>(h)->t; }

int orc_zone_updates(void* h, double* finest, double* actual) {
  Hier* H = static_cast<Hier*>(h);
  *finest = H->zu_finest;
  *actual = H->zu_actual;
  return 0;
}

void orc_dense_b(double theta, int m, double* b4) { dense_b(theta, m, b4); }
void orc_dense_b_rk(int rk, double theta, int m, double* b4) { dense_b_rk(rk, theta, m, b4); }
double orc_amr_value_rk(int rk, double y, const double* k4, double H, double theta0, int which) {
  return amr_value_rk(rk, y, k4, H, theta0, which);
}

double orc_amr_value(double y, const double* k4, double H, double theta0, int which) {
  return amr_value(y, k4, H, theta0, which);
}

int orc_rhs_box(void* h, int l, int b, const double* state, double* rhs) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* B = get_box(H, l, b);
  if (!B) return fail(-1, "bad index");
  std::memset(rhs, 0, sizeof(double) * H->F * B->vol);
  rhs_box(*H, l, *B, state, rhs);
  return 0;
}

int orc_debug_prolong(void* h, int l) {
  Hier* H = static_cast<Hier*>(h);
  if (l < 1 || l >= H->nlev) return fail(-1, "bad level");
  prolong_parent_vectors(*H, l);
  return 0;
}

int orc_debug_fill_amr(void* h, int l, int vec, double theta0, int which) {
  Hier* H = static_cast<Hier*>(h);
  if (l < 1 || l >= H->nlev || vec < 0 || vec >= V_NVEC) return fail(-1, "bad level");
  fill_amr(*H, l, vec, theta0, which);
  return 0;
}

int orc_debug_restrict(void* h, int l) {
  Hier* H = static_cast<Hier*>(h);
  if (l < 1 || l >= H->nlev) return fail(-1, "bad level");
  restrict_level(*H, l);
  return 0;
}

int orc_debug_fill_ghosts(void* h) {
  Hier* H = static_cast<Hier*>(h);
  for (int l = 0; l < H->nlev; ++l) copy_siblings(*H, l, V_Y);
  return 0;
}

// Z4c constraints at the interior cells of one box, from the current state
// (ghosts must be valid): out[q * ncell + cell] for q = H, M^x, M^y, M^z,
// G^x, G^y, G^z with
//   H   = R + 2/3 (Khat + 2 Theta)^2 - At_ij At^ij,
//   M^i = d_j At^ij + Gamt^i_jk At^jk - 3 At^ij d_j W / W - 2/3 gt^ij d_j (Khat + 2 Theta),
//   G^i = Gamt^i - gt^jk Gamt^i_jk.
int orc_constraints(void* h, int l, int b, double* out) {
  Hier* H = static_cast<Hier*>(h);
  BoxData* Bp = get_box(H, l, b);
  if (!Bp || H->system != ORC_Z4C) return fail(-1, "bad index or system");
  const BoxData& B = *Bp;
  const double hh = H->lev[l].h;
  const long ncell = (long)B.n[0] * B.n[1] * B.n[2];
  long q = 0;
  const double* Y = B.v[V_Y].data();
  for (int k = 0; k < B.n[2]; ++k)
    for (int j = 0; j < B.n[1]; ++j)
      for (int i = 0; i < B.n[0]; ++i, ++q) {
        const long c = B.off(i, j, k);
        double u[NZ4C][1], du[NZ4C][3], dd[NZ4C][6], ko[NZ4C];
        z4c_derivs<double>(B, Y, c, hh, u, du, dd, ko, H->order);
        double uu[NZ4C], rhs[NZ4C], diag[3];
        for (int f = 0; f < NZ4C; ++f) uu[f] = u[f][0];
        z4c_point<double>(uu, du, dd, rhs, H->kappa1, H->kappa2, H->eta, diag);
        const double Ham = diag[0] + (2.0 / 3.0) * diag[2] * diag[2] - diag[1];
        // momentum constraint and G^i, written out
        const double W = uu[FW];
        double g[3][3], A[3][3], dg[3][3][3], dA[3][3][3];
        for (int a = 0; a < 3; ++a)
          for (int c2 = 0; c2 < 3; ++c2) {
            g[a][c2] = uu[FG + SYM[a][c2]];
            A[a][c2] = uu[FA + SYM[a][c2]];
            for (int m = 0; m < 3; ++m) {
              dg[m][a][c2] = du[FG + SYM[a][c2]][m];
              dA[m][a][c2] = du[FA + SYM[a][c2]][m];
            }
          }
        const double det = g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
                           g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
                           g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
        double gu[3][3];
        gu[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / det;
        gu[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / det;
        gu[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / det;
        gu[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / det;
        gu[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / det;
        gu[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / det;
        gu[1][0] = gu[0][1]; gu[2][0] = gu[0][2]; gu[2][1] = gu[1][2];
        double Gu[3][3][3];
        for (int a = 0; a < 3; ++a)
          for (int i2 = 0; i2 < 3; ++i2)
            for (int j2 = 0; j2 < 3; ++j2) {
              double s = 0.0;
              for (int m = 0; m < 3; ++m) s += gu[a][m] * 0.5 * (dg[i2][j2][m] + dg[j2][i2][m] - dg[m][i2][j2]);
              Gu[a][i2][j2] = s;
            }
        double Auu[3][3];
        for (int a = 0; a < 3; ++a)
          for (int c2 = 0; c2 < 3; ++c2) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m)
              for (int n = 0; n < 3; ++n) s += gu[a][m] * gu[c2][n] * A[m][n];
            Auu[a][c2] = s;
          }
        // d_m gt^{ab} = -gt^{ac} gt^{bd} d_m gt_cd
        double dgu[3][3][3];
        for (int m = 0; m < 3; ++m)
          for (int a = 0; a < 3; ++a)
            for (int c2 = 0; c2 < 3; ++c2) {
              double s = 0.0;
              for (int e = 0; e < 3; ++e)
                for (int f2 = 0; f2 < 3; ++f2) s -= gu[a][e] * gu[c2][f2] * dg[m][e][f2];
              dgu[m][a][c2] = s;
            }
        double dKt[3];
        for (int m = 0; m < 3; ++m) dKt[m] = du[FK][m] + 2.0 * du[FTH][m];
        double Mom[3], Gc[3];
        for (int a = 0; a < 3; ++a) {
          double divA = 0.0;  // d_j At^{aj}
          for (int j2 = 0; j2 < 3; ++j2)
            for (int m = 0; m < 3; ++m)
              for (int n = 0; n < 3; ++n)
                divA += dgu[j2][a][m] * gu[j2][n] * A[m][n] + gu[a][m] * dgu[j2][j2][n] * A[m][n] +
                        gu[a][m] * gu[j2][n] * dA[j2][m][n];
          double s = divA;
          for (int j2 = 0; j2 < 3; ++j2)
            for (int k2 = 0; k2 < 3; ++k2) s += Gu[a][j2][k2] * Auu[j2][k2];
          for (int j2 = 0; j2 < 3; ++j2) {
            s -= 3.0 * Auu[a][j2] * du[FW][j2] / W;
            s -= (2.0 / 3.0) * gu[a][j2] * dKt[j2];
          }
          Mom[a] = s;
          double gd = 0.0;
          for (int j2 = 0; j2 < 3; ++j2)
            for (int k2 = 0; k2 < 3; ++k2) gd += gu[j2][k2] * Gu[a][j2][k2];
          Gc[a] = uu[FGAM + a] - gd;
        }
        out[0 * ncell + q] = Ham;
        for (int a = 0; a < 3; ++a) {
          out[(1 + a) * ncell + q] = Mom[a];
          out[(4 + a) * ncell + q] = Gc[a];
        }
      }
  return 0;
}

// Moving boxes: replace the boxes of levels >= 1.  Every interior cell of
// the new hierarchy that was an interior cell of the same level before keeps
// its state; every other interior cell takes the quintic prolongation of the
// (already regridded) parent's state.  Level 0 must be unchanged.
int orc_regrid(void* h, const int* nboxes, const int* boxes) {
  Hier* H = static_cast<Hier*>(h);
  const int L = H->nlev;
  void* nh = nullptr;
  double prm[4] = {H->kappa1, H->kappa2, H->eta, H->sigma};
  const int rc = orc_create_ex(H->system, L, nboxes, boxes, H->ncells0, H->origin, H->h0, H->bc, H->cfl,
                               H->subcycle, prm, H->order, H->rk, &nh);
  if (rc) return rc;
  Hier* N = static_cast<Hier*>(nh);
  if (N->lev[0].boxes.size() != H->lev[0].boxes.size()) {
    orc_destroy(nh);
    return fail(-1, "regrid keeps level 0 unchanged");
  }
  for (size_t b = 0; b < N->lev[0].boxes.size(); ++b)
    for (int d = 0; d < 3; ++d)
      if (N->lev[0].boxes[b].lo[d] != H->lev[0].boxes[b].lo[d] || N->lev[0].boxes[b].hi[d] != H->lev[0].boxes[b].hi[d]) {
        orc_destroy(nh);
        return fail(-1, "regrid keeps level 0 unchanged");
      }
  N->lev[0].boxes = H->lev[0].boxes;  // level 0 keeps its data
  for (int l = 1; l < L; ++l) {
    for (BoxData& B : N->lev[l].boxes)
      for (int k = 0; k < B.n[2]; ++k)
        for (int j = 0; j < B.n[1]; ++j)
          for (int i = 0; i < B.n[0]; ++i) {
            const int g[3] = {B.lo[0] + i, B.lo[1] + j, B.lo[2] + k};
            const long o = B.off(i, j, k);
            int li[3];
            const int ob = find_interior(*H, l, g, li);
            if (ob >= 0) {
              const BoxData& O = H->lev[l].boxes[ob];
              const long oo = O.off(li[0], li[1], li[2]);
              for (int f = 0; f < N->F; ++f) B.v[V_Y][(long)f * B.vol + o] = O.v[V_Y][(long)f * O.vol + oo];
              continue;
            }
            int nodes[3][8];
            double w[3][8];
            for (int d = 0; d < 3; ++d) prolong_stencil_1d(g[d], nodes[d], w[d]);
            for (int f = 0; f < N->F; ++f) B.v[V_Y][(long)f * B.vol + o] = 0.0;
            for (int cz = 0; cz < g_pn; ++cz)
              for (int cy = 0; cy < g_pn; ++cy)
                for (int cx = 0; cx < g_pn; ++cx) {
                  const int pg[3] = {nodes[0][cx], nodes[1][cy], nodes[2][cz]};
                  int pl[3];
                  const int pb = find_interior(*N, l - 1, pg, pl);
                  if (pb < 0) {
                    orc_destroy(nh);
                    return fail(-4, "regrid: new cell cannot be prolonged from the parent interior");
                  }
                  const BoxData& P = N->lev[l - 1].boxes[pb];
                  const long po = P.off(pl[0], pl[1], pl[2]);
                  const double ww = w[0][cx] * w[1][cy] * w[2][cz];
                  for (int f = 0; f < N->F; ++f) B.v[V_Y][(long)f * B.vol + o] += ww * P.v[V_Y][(long)f * P.vol + po];
                }
          }
  }
  // keep time, counters and options; take the new levels
  N->t = H->t;
  N->zu_finest = H->zu_finest;
  N->zu_actual = H->zu_actual;
  N->cb = H->cb;
  N->cb_user = H->cb_user;
  N->eta_profile = H->eta_profile;
  N->eta_c = H->eta_c;
  N->eta_s = H->eta_s;
  N->eta_o = H->eta_o;
  for (int l = 0; l < L; ++l) N->lev[l].t = H->lev[l].t;
  std::swap(*H, *N);
  orc_destroy(nh);
  return 0;
}

// Field values at points: tensor-product quintic Lagrange interpolation on
// the finest level whose 6x6x6 cell stencil around the point is interior.
int orc_interpolate(void* h, int npts, const double* xyz, int field, double* out) {
  Hier* H = static_cast<Hier*>(h);
  if (field < 0 || field >= H->F) return fail(-1, "bad field");
  for (int a = 0; a < npts; ++a) {
    bool found = false;
    for (int l = H->nlev - 1; l >= 0 && !found; --l) {
      const double hl = H->lev[l].h;
      double s[3], w[3][8];
      int first[3];
      for (int d = 0; d < 3; ++d) {
        s[d] = (xyz[3 * a + d] - H->origin[d]) / hl - 0.5;
        first[d] = (int)std::floor(s[d]) - 2;
        double x[8];
        for (int m = 0; m < g_pn; ++m) x[m] = first[d] + m;
        lagrange(x, g_pn, s[d], w[d]);
      }
      double acc = 0.0;
      bool ok = true;
      for (int cz = 0; cz < g_pn && ok; ++cz)
        for (int cy = 0; cy < g_pn && ok; ++cy)
          for (int cx = 0; cx < g_pn && ok; ++cx) {
            const int g[3] = {first[0] + cx, first[1] + cy, first[2] + cz};
            int li[3];
            const int b = find_interior(*H, l, g, li);
            if (b < 0) {
              ok = false;
              break;
            }
            const BoxData& B = H->lev[l].boxes[b];
            acc += w[0][cx] * w[1][cy] * w[2][cz] * B.v[V_Y][(long)field * B.vol + B.off(li[0], li[1], li[2])];
          }
      if (ok) {
        out[a] = acc;
        found = true;
      }
    }
    if (!found) return fail(-1, "no level holds the interpolation stencil");
  }
  return 0;
}

// Operation counts of one Z4c right-hand side at one cell in this oracle's
// formulation (derivative stencils, KO and the pointwise equations):
// counts[0..3] = add/sub, mul, div, total flops.
void orc_flop_counts(double* counts) {
  for (int q = 0; q < 4; ++q) g_ops[q] = 0.0;
  BoxData B;
  for (int d = 0; d < 3; ++d) { B.lo[d] = 0; B.hi[d] = 0; B.n[d] = 1; B.N[d] = 1 + 2 * B.g; }
  B.vol = (long)B.N[0] * B.N[1] * B.N[2];
  std::vector<double> Y((size_t)NZ4C * B.vol, 1.0);
  Cnt u[NZ4C][1], du[NZ4C][3], dd[NZ4C][6], ko[NZ4C], uu[NZ4C], rhs[NZ4C];
  z4c_derivs<Cnt>(B, Y.data(), B.off(0, 0, 0), 1.0, u, du, dd, ko);
  for (int f = 0; f < NZ4C; ++f) uu[f] = u[f][0];
  z4c_point<Cnt>(uu, du, dd, rhs, 0.02, 0.0, 2.0);
  for (int f = 0; f < NZ4C; ++f) rhs[f] = rhs[f] + Cnt(0.3 / 64.0) * ko[f];
  counts[0] = g_ops[0];
  counts[1] = g_ops[1];
  counts[2] = g_ops[2];
  counts[3] = g_ops[0] + g_ops[1] + g_ops[2];
}

}  // extern "C"
