// sc_host.cu -- host runtime and C ABI of the subcycling library.
//
// Each level is stored as one dense FP64 array per field over the bounding
// box of its boxes (grown by the ghost width: 3 cells, 4 with 8th-order
// differences).  Sibling boxes therefore share
// memory: a ghost cell of one box that is interior to another needs no copy.
// The remaining ghost cells are classified once at creation:
//   * refinement boundary (levels >= 1): filled from the parent's dense
//     output after prolongation (Sec. II steps 2, 3, 5);
//   * periodic images: copied from the wrapped interior cell;
//   * outer boundary of a radiative level 0: evolved by the radiative kernel.
// One coarse step (Sec. II steps 1-7, recursively) is a fixed sequence of
// kernel launches, captured once into a CUDA graph per parity of the level-0
// state buffers and replayed by sc_advance.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sc_internal.h"
#include "sc_persist.h"

using namespace sc;

namespace {

thread_local char g_err[512];

sc_status fail(sc_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

enum CellKind : int8_t { K_UNUSED = 0, K_INTERIOR = 1, K_AMR = 2, K_PERIODIC = 3, K_PHYS = 4 };

// Lagrange basis weights for nodes x[0..n-1] at point p.
void lagrange_weights(const double* x, int n, double p, double* w) {
  for (int m = 0; m < n; ++m) {
    double num = 1.0, den = 1.0;
    for (int q = 0; q < n; ++q)
      if (q != m) {
        num *= p - x[q];
        den *= x[m] - x[q];
      }
    w[m] = num / den;
  }
}

Weights make_weights() {
  Weights w;
  double x[kPN];
  // parity 0: fine centre at -1/4 parent cell, nodes c-3..c+2;
  // parity 1: fine centre at +1/4, nodes c-2..c+3 (offsets from parent c).
  for (int m = 0; m < kPN; ++m) x[m] = -3.0 + m;
  lagrange_weights(x, kPN, -0.25, w.prolong[0]);
  for (int m = 0; m < kPN; ++m) x[m] = -2.0 + m;
  lagrange_weights(x, kPN, 0.25, w.prolong[1]);
  // restriction: fine cells 2C-2..2C+3 at offsets -2.5..2.5 fine cells from the parent centre
  for (int m = 0; m < kRN; ++m) x[m] = -2.5 + m;
  lagrange_weights(x, kRN, 0.0, w.restrict_w);
  return w;
}

// Dense-output weights b_i(theta) and their theta-derivatives (Eqs.
// denseoutput1/2): b1 = t - 3t^2/2 + 2t^3/3, b2 = b3 = t^2 - 2t^3/3,
// b4 = -t^2/2 + 2t^3/3.
void dense_weights(double t, int m, double* b) {
  switch (m) {
    case 0:
      b[0] = t * (1.0 + t * (-1.5 + t * (2.0 / 3.0)));
      b[1] = b[2] = t * t * (1.0 - t * (2.0 / 3.0));
      b[3] = t * t * (-0.5 + t * (2.0 / 3.0));
      break;
    case 1:
      b[0] = 1.0 + t * (-3.0 + 2.0 * t);
      b[1] = b[2] = t * (2.0 - 2.0 * t);
      b[3] = t * (-1.0 + 2.0 * t);
      break;
    case 2:
      b[0] = -3.0 + 4.0 * t;
      b[1] = b[2] = 2.0 - 4.0 * t;
      b[3] = -1.0 + 4.0 * t;
      break;
    default:
      b[0] = 4.0; b[1] = -4.0; b[2] = -4.0; b[3] = 4.0;
  }
}

// Runge-Kutta methods (rk = number of stages = order).  Every method here
// builds stage input s >= 2 from y_n and k_{s-1} alone (RK3 levels with a
// finer level also evaluate k4 = f(y_{n+1}) for their dense output):
//   rk = 4: classic RK4 (Eqs. rk1-rk5), multipliers 1/2, 1/2, 1;
//   rk = 3: Heun's third-order method, multipliers 1/3, 2/3,
//           y_{n+1} = y_n + dt/4 (k1 + 3 k3);
//   rk = 2: explicit midpoint, multiplier 1/2, y_{n+1} = y_n + dt k2.
double stage_mult(int rk, int s) {
  if (rk == 4) return s == 4 ? 1.0 : 0.5;
  if (rk == 3) return s == 2 ? 1.0 / 3.0 : 2.0 / 3.0;
  return 0.5;
}

// Stage vectors the dense output uses, in the order they are prolonged into
// the ghost store: k1..k4 for RK4; k1, k3 and k4 = f(y_{n+1}) for RK3; k1
// and k2 for RK2.
int dense_vectors(int rk, int* idx) {
  if (rk == 4) {
    for (int j = 0; j < 4; ++j) idx[j] = j;
    return 4;
  }
  if (rk == 3) {
    idx[0] = 0;
    idx[1] = 2;
    idx[2] = 3;
    return 3;
  }
  idx[0] = 0;
  idx[1] = 1;
  return 2;
}

int dense_count(int rk) {
  int idx[4];
  return dense_vectors(rk, idx);
}

// Dense-output weights of RK3 and RK2 and their theta-derivatives, per stage
// vector (index 3 = k4 = f(y_{n+1})):
//   RK3: the cubic Hermite interpolant through y_n, y_{n+1} with slopes k1
//        and k4: b1 = t - 5t^2/4 + t^3/2, b3 = 9t^2/4 - 3t^3/2,
//        b4 = -t^2 + t^3 (third order; RK3's own second-order continuous
//        extensions leave the subcycled scheme near order 2.5);
//   RK2: b1 = t - t^2, b2 = t^2 (second order).
void dense_weights_rk(int rk, double t, int m, double* b) {
  if (rk == 4) {
    dense_weights(t, m, b);
    return;
  }
  b[0] = b[1] = b[2] = b[3] = 0.0;
  if (rk == 3) {
    if (m == 0) {
      b[0] = t * (1.0 + t * (-1.25 + 0.5 * t));
      b[2] = t * t * (2.25 - 1.5 * t);
      b[3] = t * t * (-1.0 + t);
    } else if (m == 1) {
      b[0] = 1.0 + t * (-2.5 + 1.5 * t);
      b[2] = t * (4.5 - 4.5 * t);
      b[3] = t * (-2.0 + 3.0 * t);
    } else if (m == 2) {
      b[0] = -2.5 + 3.0 * t;
      b[2] = 4.5 - 9.0 * t;
      b[3] = -2.0 + 6.0 * t;
    } else if (m == 3) {
      b[0] = 3.0;
      b[2] = -9.0;
      b[3] = 6.0;
    }
    return;
  }
  if (m == 0) {
    b[0] = t * (1.0 - t);
    b[1] = t * t;
  } else if (m == 1) {
    b[0] = 1.0 - 2.0 * t;
    b[1] = 2.0 * t;
  } else if (m == 2) {
    b[0] = -2.0;
    b[1] = 2.0;
  }
}

// Coefficients c_j of ghost value = P[y_n] + sum_j c_j P[k_j] for the fine
// substep starting at progress theta0 of a parent step H (fine step
// h = H/2), one per prolonged stage vector (dense_vectors order):
//   which = 1..rk: fine stage input Y_which.  RK4: the Taylor expansions of
//     Eqs. Y1-Y4 with the first three theta-derivatives of the dense output
//     at theta0 (Eqs. denseoutput1/2) and f_y y2 = 4 (k3 - k2) / H^2.
//     RK3: Y1 = y, Y2 = y + h/3 y1, Y3 = y + 2h/3 y1 + 2h^2/9 y2.
//     RK2: Y1 = y, Y2 = y + h/2 y1.  (y1, y2: first and second time
//     derivatives; each formula is exact for linear right-hand sides.)
//   which = 0: state at the end of the substep, dense output at theta0 + 1/2.
void fill_coeffs(int rk, double H, double theta0, int which, double* c) {
  double b0[4], b1[4], b2[4], b3[4], full[4];
  if (which == 0) {
    dense_weights_rk(rk, theta0 + 0.5, 0, b0);
    for (int j = 0; j < 4; ++j) full[j] = H * b0[j];
  } else {
    const double h = 0.5 * H;
    dense_weights_rk(rk, theta0, 0, b0);
    dense_weights_rk(rk, theta0, 1, b1);
    dense_weights_rk(rk, theta0, 2, b2);
    if (rk == 4) dense_weights(theta0, 3, b3);
    const double fyy[4] = {0.0, -4.0, 4.0, 0.0};  // times 1/H^2
    for (int j = 0; j < 4; ++j) {
      const double y0 = H * b0[j], y1 = b1[j], y2 = b2[j] / H;
      if (rk == 4) {
        const double y3 = b3[j] / (H * H), fy = fyy[j] / (H * H);
        switch (which) {
          case 1: full[j] = y0; break;
          case 2: full[j] = y0 + 0.5 * h * y1; break;
          case 3: full[j] = y0 + 0.5 * h * y1 + 0.25 * h * h * y2 + (h * h * h / 16.0) * (y3 - fy); break;
          default: full[j] = y0 + h * y1 + 0.5 * h * h * y2 + (h * h * h / 8.0) * (y3 + fy); break;
        }
      } else if (rk == 3) {
        switch (which) {
          case 1: full[j] = y0; break;
          case 2: full[j] = y0 + (h / 3.0) * y1; break;
          default: full[j] = y0 + (2.0 * h / 3.0) * y1 + (2.0 * h * h / 9.0) * y2; break;
        }
      } else {
        full[j] = which == 1 ? y0 : y0 + 0.5 * h * y1;
      }
    }
  }
  int idx[4];
  const int n = dense_vectors(rk, idx);
  for (int j = 0; j < 4; ++j) c[j] = j < n ? full[idx[j]] : 0.0;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Level {
  std::vector<sc_box> boxes;
  Geom g;
  double dt = 0;
  std::vector<int8_t> kind;  // per array element (host only)
  // device arrays: state pair, two stage buffers, k1..k_rk (unused ones null)
  double* S[2] = {nullptr, nullptr};
  double* A = nullptr;
  double* B = nullptr;
  double* K[4] = {nullptr, nullptr, nullptr, nullptr};
  // work lists (device) and their sizes
  Tile* tiles = nullptr;
  int ntiles = 0;
  int tile_cols = 0;                // largest nx * ny of the tiles
  std::vector<int> box_tile_begin;  // tiles of box b: [box_tile_begin[b], box_tile_begin[b + 1])
  Tile* ptiles = nullptr;           // 32 x ny x 1 tiles for the pointwise Z4c kernel (one cell per thread)
  int nptiles = 0;
  int ptile_threads = 128;          // 32 * ny: the stage kernel's block size on this level
  std::vector<int> box_ptile_begin;
  AmrCell* amr = nullptr;
  int namr = 0;
  AmrTile* atiles = nullptr;  // separable-prolongation tiles and their position -> AMR index map
  int natiles = 0;
  int32_t* aslots = nullptr;
  long tile_fmas = 0;
  RowSeg* dxy = nullptr;
  int ndxy = 0;
  double* eta = nullptr;  // per-element eta(r) (Z4c with the Sec. III.A profile), else null
  std::vector<void*> allocs;  // device buffers owned by this level (freed on regrid)
  int namr_blocked = 0;
  double* amr_store = nullptr;  // (1 + dense vectors) * F * namr prolonged parent vectors
  int2* periodic = nullptr;
  int nperiodic = 0;
  int32_t* phys = nullptr;
  int nphys = 0;
  RestrictCell* restr = nullptr;  // parent cells restricted from this level (per-cell kernel)
  int nrestr = 0;
  RestrictBlock* rblocks = nullptr;  // the rest, in 4x4x4 parent blocks (separable kernel)
  int nrblocks = 0;
  long interior_cells = 0;
  int parity = 0;  // which of S[] holds the current state
};

enum OpKind { OP_PROLONG, OP_FILL, OP_STAGE, OP_RESTRICT, OP_PROLONG_DIRECT, OP_CHECK };

struct Op {
  OpKind kind;
  int level;
  int stage;      // OP_STAGE: 1..4
  double* in;     // stage input / fill target
  double* yn;
  double* out;
  double c[4];    // OP_FILL coefficients
  double cdt;     // OP_STAGE update (StageArgs)
  double c1dt;
  int form;
  bool no_amr;    // OP_FILL: periodic images only (uniform-step mode)
  bool amr_folded;  // OP_FILL: its refinement-boundary part runs in the stage launch before it
  bool fold_fill;   // OP_STAGE: also applies the next op's refinement-boundary fill
  double* fold_vec;
  double fold_c[4];
};

}  // namespace

struct sc_ctx {
  int system = 0, F = 0, nlev = 0, bc = 0;
  int ncells0[3];
  double origin[3], h0 = 0, cfl = 0;
  Z4cParams zp;
  cudaStream_t stream = nullptr;
  sc_allocator alloc{};
  bool has_alloc = false;
  std::vector<Level> lev;
  Weights w;
  double* scratch = nullptr;  // Z4c derivative temporaries
  long scratch_fs = 0;
  double* staging = nullptr;  // pack/unpack buffer
  size_t staging_bytes = 0;
  int* flag = nullptr;         // sc_check_finite's result
  int* status = nullptr;       // per-step device status word (kStatus* bits), read by sc_synchronize
  int finite_check = 0;        // check the state for non-finite values after every coarse step
  std::vector<DevBuf> bufs;
  size_t footprint = 0;
  double t = 0;
  double zu_finest = 0, zu_actual = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_stale[2] = {true, true};  // the schedule changed since graph[p] was built
  long launches_per_step = 0;
  int exec_mode = SC_EXEC_GRAPH;
  int subcycle = 1;
  int order = 4;   // finite-difference order of the right-hand sides (4 or 8)
  int rk = 4;      // Runge-Kutta method: stages = order = 4, 3 or 2
  int ghost = 3;   // ghost layers per box: 3 for 4th order, 4 for 8th
  int tile[3] = {32, 4, 2};  // stencil-kernel tile shape (autotuned on request)
  // Z4c derivative pass: 0 = two kernels (D_x/D_y row pass, then the per-column
  // pass that differentiates them for the mixed derivatives), 1 = one kernel
  // per (cell, field) with direct 16-point mixed stencils (4th order only);
  // stage kernel build: 2 or 3 blocks of 128 threads per SM (autotuned)
  int deriv_form = 0;
  int stage_bps = 3;
  int eta_profile = 0;
  double eta_c = 0, eta_s = 0, eta_o = 0;
  std::vector<Op> plain_ops[2];  // per-box form: the schedule, run directly
  // persistent form (scalar wave): the phase table of each parity (device and
  // host copies), the grid it needs and the barrier of its launches
  POp* pops[2] = {nullptr, nullptr};
  std::vector<POp> host_pops[2];
  long pwork[2] = {0, 0};
  GridBarrier* bar = nullptr;
  // whole-state transfers: mode (SC_XFER_*) and the split timing of the last one
  int xfer_mode = SC_XFER_AUTO;
  cudaEvent_t xev[4] = {nullptr, nullptr, nullptr, nullptr};
  double xfer_copy_ms = 0, xfer_kernel_ms = 0;
  size_t xfer_bytes = 0;
  int xfer_direct = 0;

  void* dalloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (has_alloc) {
      p = alloc.alloc(bytes, alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) {
      bufs.push_back({p, bytes});
      footprint += bytes;
    }
    return p;
  }
  void dfree(void* p) {
    for (size_t i = 0; i < bufs.size(); ++i)
      if (bufs[i].p == p) {
        if (has_alloc) alloc.free(p, alloc.user);
        else cudaFree(p);
        footprint -= bufs[i].bytes;
        bufs.erase(bufs.begin() + i);
        return;
      }
  }
  void release() {
    for (auto& b : bufs) {
      if (has_alloc) alloc.free(b.p, alloc.user);
      else cudaFree(b.p);
    }
    bufs.clear();
    footprint = 0;
  }
};

namespace {

int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Global index of array element (i, j, k).
inline void elem_global(const Geom& g, int i, int j, int k, int* gi) {
  gi[0] = g.org[0] + i;
  gi[1] = g.org[1] + j;
  gi[2] = g.org[2] + k;
}

inline bool in_array(const Geom& g, const int* gi) {
  for (int d = 0; d < 3; ++d)
    if (gi[d] < g.org[d] || gi[d] >= g.org[d] + g.ext[d]) return false;
  return true;
}

inline long elem_index(const Geom& g, const int* gi) {
  return ((long)(gi[2] - g.org[2]) * g.ext[1] + (gi[1] - g.org[1])) * g.ext[0] + (gi[0] - g.org[0]);
}

sc_status validate(const sc_desc* d) {
  if (!d) return fail(SC_EINVAL, "null descriptor");
  if (d->system != SC_WAVE && d->system != SC_Z4C) return fail(SC_EINVAL, "unknown system %d", d->system);
  if (d->nlevels < 1 || d->nlevels > 16) return fail(SC_EINVAL, "nlevels must be 1..16");
  if (!d->nboxes || !d->boxes) return fail(SC_EINVAL, "null box arrays");
  if (d->subcycle != 0 && d->subcycle != 1) return fail(SC_EINVAL, "subcycle must be 0 or 1");
  if (d->fd_order != 0 && d->fd_order != 4 && d->fd_order != 8) return fail(SC_EINVAL, "fd_order must be 4 or 8");
  if (d->rk_order != 0 && (d->rk_order < 2 || d->rk_order > 4)) return fail(SC_EINVAL, "rk_order must be 2, 3 or 4");
  if (d->outer_bc != SC_BC_PERIODIC && d->outer_bc != SC_BC_RADIATIVE) return fail(SC_EINVAL, "unknown outer_bc");
  if (!(d->h0 > 0) || !(d->cfl > 0)) return fail(SC_EINVAL, "h0 and cfl must be positive");
  for (int q = 0; q < 3; ++q)
    if (d->ncells0[q] < 1) return fail(SC_EINVAL, "ncells0 must be positive");
  if (d->outer_bc == SC_BC_RADIATIVE && d->nboxes[0] != 1) return fail(SC_EINVAL, "radiative boundary needs one level-0 box");
  if (d->eta_profile && !(d->eta_s > 0)) return fail(SC_EINVAL, "eta_s must be positive");
  if (d->exec_mode != SC_EXEC_GRAPH && d->exec_mode != SC_EXEC_PER_BOX && d->exec_mode != SC_EXEC_PERSISTENT)
    return fail(SC_EINVAL, "unknown exec_mode %d", d->exec_mode);
  if (d->exec_mode == SC_EXEC_PERSISTENT && d->system != SC_WAVE)
    return fail(SC_EINVAL, "the persistent coarse-step kernel is built for the scalar wave");
  int bi = 0;
  for (int l = 0; l < d->nlevels; ++l) {
    if (d->nboxes[l] < 1) return fail(SC_EINVAL, "level %d has no boxes", l);
    for (int b = 0; b < d->nboxes[l]; ++b, ++bi) {
      const sc_box& B = d->boxes[bi];
      for (int q = 0; q < 3; ++q) {
        const long ext = (long)d->ncells0[q] << l;
        if (B.lo[q] < 0 || B.hi[q] < B.lo[q] || B.hi[q] >= ext)
          return fail(SC_EINVAL, "box %d of level %d outside the level", b, l);
        if (l > 0 && ((B.lo[q] & 1) || !(B.hi[q] & 1)))
          return fail(SC_ENESTING, "box %d of level %d not aligned to parent cells", b, l);
      }
    }
  }
  return SC_OK;
}

// Build geometry, classification and work lists of every level (host side).
struct HostLists {
  std::vector<Tile> tiles;
  std::vector<Tile> ptiles;
  std::vector<AmrCell> amr;
  std::vector<int> amr_gi, amr_gw;  // unwrapped / wrapped global fine index per AMR cell
  std::vector<AmrTile> atiles;      // slab tiles served by the separable kernel
  std::vector<int32_t> aslots;      // per tile position: AMR list index or -1
  long tile_fmas = 0;               // FMAs of the tile kernel per (vector, field)
  std::vector<RowSeg> dxy;          // rows where D_x / D_y of the Hessian fields are stored
  int namr_blocked = 0;             // AMR cells [0, namr_blocked) belong to tiles
  std::vector<int2> periodic;
  std::vector<int32_t> phys;
  std::vector<RestrictCell> restr;   // restricted parent cells outside blocks
  std::vector<RestrictBlock> rblocks;  // 4x4x4 parent blocks for the separable kernel
};

sc_status build_level_geometry(sc_ctx* c, int l, const sc_box* boxes, int nb) {
  Level& L = c->lev[l];
  L.boxes.assign(boxes, boxes + nb);
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  L.interior_cells = 0;
  for (const sc_box& B : L.boxes) {
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], B.lo[q]);
      hi[q] = std::max(hi[q], B.hi[q]);
    }
    L.interior_cells += (long)(B.hi[0] - B.lo[0] + 1) * (B.hi[1] - B.lo[1] + 1) * (B.hi[2] - B.lo[2] + 1);
  }
  Geom& g = L.g;
  g.h = c->h0 / (double)(1L << l);
  for (int q = 0; q < 3; ++q) {
    g.org[q] = lo[q] - c->ghost;
    g.ext[q] = hi[q] - lo[q] + 1 + 2 * c->ghost;
    g.x0[q] = c->origin[q] + (g.org[q] + 0.5) * g.h;
  }
  g.pitch = (g.ext[0] + 7) & ~7;
  const long plane = (long)g.pitch * g.ext[1] * g.ext[2];
  if (plane >= (1L << 31)) return fail(SC_EINVAL, "level %d array too large for 32-bit offsets", l);
  g.fs = (plane + 31) & ~31L;
  L.dt = c->cfl * g.h;
  // overlap check and interior marking
  const long nelem = (long)g.ext[0] * g.ext[1] * g.ext[2];
  L.kind.assign(nelem, K_UNUSED);
  for (const sc_box& B : L.boxes)
    for (int k = B.lo[2]; k <= B.hi[2]; ++k)
      for (int j = B.lo[1]; j <= B.hi[1]; ++j)
        for (int i = B.lo[0]; i <= B.hi[0]; ++i) {
          const int gi[3] = {i, j, k};
          int8_t& e = L.kind[elem_index(g, gi)];
          if (e == K_INTERIOR) return fail(SC_EINVAL, "overlapping boxes on level %d", l);
          e = K_INTERIOR;
        }
  return SC_OK;
}

bool is_interior(const Level& L, const int* gi) {
  if (!in_array(L.g, gi)) return false;
  return L.kind[elem_index(L.g, gi)] == K_INTERIOR;
}

// Summed-volume table of a level's interior cells: S(i,j,k) = number of
// interior array elements with index < (i,j,k) componentwise, so any box of
// elements is counted in O(1) (the proper-nesting check of a ghost cell's
// 6x6x6 prolongation stencil).
struct InteriorCount {
  Geom g;
  std::vector<int32_t> sat;  // (ext0+1) x (ext1+1) x (ext2+1)
  long at(int i, int j, int k) const {
    return sat[((long)k * (g.ext[1] + 1) + j) * (g.ext[0] + 1) + i];
  }
  explicit InteriorCount(const Level& L) : g(L.g) {
    const int X = g.ext[0] + 1, Y = g.ext[1] + 1, Z = g.ext[2] + 1;
    sat.assign((size_t)X * Y * Z, 0);
    for (int k = 1; k < Z; ++k)
      for (int j = 1; j < Y; ++j)
        for (int i = 1; i < X; ++i) {
          const long e = ((long)(k - 1) * g.ext[1] + (j - 1)) * g.ext[0] + (i - 1);
          const int32_t v = L.kind[e] == K_INTERIOR ? 1 : 0;
          sat[((long)k * Y + j) * X + i] = v + at(i - 1, j, k) + at(i, j - 1, k) + at(i, j, k - 1) -
                                           at(i - 1, j - 1, k) - at(i - 1, j, k - 1) - at(i, j - 1, k - 1) +
                                           at(i - 1, j - 1, k - 1);
        }
  }
  // true when every cell of the global box [lo, lo + n) is interior
  bool all_interior(const int* lo, int n) const {
    int a[3], b[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = lo[d] - g.org[d];
      b[d] = a[d] + n;
      if (a[d] < 0 || b[d] > g.ext[d]) return false;
    }
    const long c = at(b[0], b[1], b[2]) - at(a[0], b[1], b[2]) - at(b[0], a[1], b[2]) - at(b[0], b[1], a[2]) +
                   at(a[0], a[1], b[2]) + at(a[0], b[1], a[2]) + at(b[0], a[1], a[2]) - at(a[0], a[1], a[2]);
    return c == (long)n * n * n;
  }
};

// Tile the refinement-boundary ghost cells of level l for the separable
// prolongation.  The ghost shell of every box is cut into six slabs -- the
// low and high z slabs span the whole shell in x and y, the y slabs the
// shell in x and the box in z, the x slabs the box in y and z -- and each
// slab into tiles of at most 8 cells along its two long axes and the ghost
// width along its thin axis.  A tile claims the ghost cells in it that no
// earlier tile claimed and that wrap by the same periodic shift as its first
// one; the kernel computes every position of the tile (its parent region must
// lie in the parent array) and stores the claimed ones.  Claimed cells are
// reordered tile by tile (x fastest within a tile); the others follow and use
// the per-cell kernel.
void build_amr_tiles(sc_ctx* c, int l, HostLists& hl) {
  const Level& L = c->lev[l];
  const Level& P = c->lev[l - 1];
  const Geom& g = L.g;
  const size_t n = hl.amr.size();
  std::vector<int32_t> at((size_t)g.ext[0] * g.ext[1] * g.ext[2], -1);  // AMR index of each array element
  for (size_t a = 0; a < n; ++a) {
    const int gi[3] = {hl.amr_gi[3 * a], hl.amr_gi[3 * a + 1], hl.amr_gi[3 * a + 2]};
    at[elem_index(g, gi)] = (int32_t)a;
  }
  auto shift_of = [&](size_t a, int q) { return hl.amr_gw[3 * a + q] - hl.amr_gi[3 * a + q]; };
  std::vector<char> claimed(n, 0);
  std::vector<AmrCell> fast;
  fast.reserve(n);
  hl.atiles.clear();
  hl.aslots.clear();
  const int G = c->ghost;
  for (const sc_box& B : L.boxes) {
    for (int sl = 0; sl < 6; ++sl) {
      const int ax = 2 - sl / 2;  // thin axis: z, z, y, y, x, x
      const bool high = sl & 1;
      int lo[3], hi[3];
      for (int q = 0; q < 3; ++q) {
        // long axes below the thin one (x for the y slabs, x and y for the z
        // slabs) span the shell, those above it span the box, so the six
        // slabs partition the shell
        const bool span_shell = q < ax;
        lo[q] = span_shell ? B.lo[q] - G : B.lo[q];
        hi[q] = span_shell ? B.hi[q] + G : B.hi[q];
      }
      lo[ax] = high ? B.hi[ax] + 1 : B.lo[ax] - G;
      hi[ax] = high ? B.hi[ax] + G : B.lo[ax] - 1;
      for (int z0 = lo[2]; z0 <= hi[2]; z0 += (ax == 2 ? G : 8))
        for (int y0 = lo[1]; y0 <= hi[1]; y0 += (ax == 1 ? G : 8))
          for (int x0 = lo[0]; x0 <= hi[0]; x0 += (ax == 0 ? G : 8)) {
            const int t0[3] = {x0, y0, z0};
            int ext[3];
            for (int q = 0; q < 3; ++q) ext[q] = std::min(q == ax ? G : 8, hi[q] - t0[q] + 1);
            // first unclaimed ghost cell of the tile fixes its periodic shift
            long first = -1;
            for (int k = 0; k < ext[2] && first < 0; ++k)
              for (int j = 0; j < ext[1] && first < 0; ++j)
                for (int i = 0; i < ext[0] && first < 0; ++i) {
                  const int gi[3] = {x0 + i, y0 + j, z0 + k};
                  const int32_t a = in_array(g, gi) ? at[elem_index(g, gi)] : -1;
                  if (a >= 0 && !claimed[a]) first = a;
                }
            if (first < 0) continue;
            int shift[3], par = 0, r0[3], r1[3];
            for (int q = 0; q < 3; ++q) {
              shift[q] = shift_of(first, q);
              const int wo = t0[q] + shift[q];  // wrapped fine origin
              const int p0 = wo & 1;
              par |= p0 << q;
              r0[q] = (wo >> 1) - 3 + p0;  // first parent node of the region
              const int i = ext[q] - 1;
              r1[q] = r0[q] + ((p0 + i) >> 1) + ((p0 + i) & 1) - p0 + kPN - 1;  // last node
            }
            if (!in_array(P.g, r0) || !in_array(P.g, r1)) continue;
            // the kernel's shared-memory bounds (always met by slabs of
            // extents <= 8 x 8 x 4; checked so that no tile can exceed them)
            const long N[3] = {r1[0] - r0[0] + 1L, r1[1] - r0[1] + 1L, r1[2] - r0[2] + 1L};
            if (N[0] * N[1] * N[2] > 800 || ext[0] * N[1] * N[2] > 640 || (long)ext[0] * ext[1] * N[2] > 512) continue;
            hl.tile_fmas += 6 * (ext[0] * N[1] * N[2] + (long)ext[0] * ext[1] * N[2] + (long)ext[0] * ext[1] * ext[2]);
            AmrTile T;
            T.pbase = (int32_t)P.g.off(r0[0], r0[1], r0[2]);
            T.slot_base = (int32_t)hl.aslots.size();
            for (int q = 0; q < 3; ++q) T.ext[q] = (int8_t)ext[q];
            T.par = (int8_t)par;
            for (int k = 0; k < ext[2]; ++k)
              for (int j = 0; j < ext[1]; ++j)
                for (int i = 0; i < ext[0]; ++i) {
                  const int gi[3] = {x0 + i, y0 + j, z0 + k};
                  const int32_t a = in_array(g, gi) ? at[elem_index(g, gi)] : -1;
                  bool take = a >= 0 && !claimed[a];
                  for (int q = 0; q < 3 && take; ++q) take = shift_of(a, q) == shift[q];
                  if (take) {
                    claimed[a] = 1;
                    hl.aslots.push_back((int32_t)fast.size());
                    fast.push_back(hl.amr[a]);
                  } else {
                    hl.aslots.push_back(-1);
                  }
                }
            hl.atiles.push_back(T);
          }
    }
  }
  hl.namr_blocked = (int)fast.size();
  for (size_t a = 0; a < n; ++a)
    if (!claimed[a]) fast.push_back(hl.amr[a]);
  hl.amr.swap(fast);
}

// Interior tiles of the stencil kernels: per box, tiles of shape tile[0..2]
// clipped to the box (ragged tiles at the high ends).
int max_tile_cols(const std::vector<Tile>& v) {
  int m = 1;
  for (const Tile& t : v) m = std::max(m, t.nx * t.ny);
  return m;
}

void build_stencil_tiles(Level& L, const int* tile, std::vector<Tile>& out) {
  const Geom& g = L.g;
  out.clear();
  L.box_tile_begin.clear();
  for (const sc_box& B : L.boxes) {
    L.box_tile_begin.push_back((int)out.size());
    for (int z = B.lo[2]; z <= B.hi[2]; z += tile[2])
      for (int y = B.lo[1]; y <= B.hi[1]; y += tile[1])
        for (int x = B.lo[0]; x <= B.hi[0]; x += tile[0]) {
          Tile t;
          t.x0 = x - g.org[0];
          t.y0 = y - g.org[1];
          t.z0 = z - g.org[2];
          t.nx = std::min(tile[0], B.hi[0] - x + 1);
          t.ny = std::min(tile[1], B.hi[1] - y + 1);
          t.nz = std::min(tile[2], B.hi[2] - z + 1);
          out.push_back(t);
        }
  }
  L.box_tile_begin.push_back((int)out.size());
  L.tile_cols = max_tile_cols(out);
}

sc_status classify_level(sc_ctx* c, int l, HostLists& hl) {
  Level& L = c->lev[l];
  const Geom& g = L.g;
  const bool periodic = c->bc == SC_BC_PERIODIC;
  int next[3];
  for (int q = 0; q < 3; ++q) next[q] = c->ncells0[q] << l;
  // ghost cells: within c->ghost (per dimension) of a box interior
  const int G = c->ghost;
  for (const sc_box& B : L.boxes)
    for (int k = B.lo[2] - G; k <= B.hi[2] + G; ++k)
      for (int j = B.lo[1] - G; j <= B.hi[1] + G; ++j)
        for (int i = B.lo[0] - G; i <= B.hi[0] + G; ++i) {
          const int gi[3] = {i, j, k};
          const long e = elem_index(g, gi);
          if (L.kind[e] != K_UNUSED) continue;
          int gw[3];
          bool outside = false;
          for (int q = 0; q < 3; ++q) {
            gw[q] = gi[q];
            if (gi[q] < 0 || gi[q] >= next[q]) {
              if (periodic) gw[q] = wrapi(gi[q], next[q]);
              else outside = true;
            }
          }
          if (outside) {
            if (l != 0) return fail(SC_ENESTING, "level %d reaches the outer boundary", l);
            L.kind[e] = K_PHYS;
            continue;
          }
          if ((gw[0] != gi[0] || gw[1] != gi[1] || gw[2] != gi[2]) && is_interior(L, gw)) {
            L.kind[e] = K_PERIODIC;
            continue;
          }
          if (l == 0) return fail(SC_ENESTING, "level 0 does not cover the domain");
          L.kind[e] = K_AMR;
        }
  // work lists
  std::unique_ptr<InteriorCount> pcount;
  if (l > 0) pcount.reset(new InteriorCount(c->lev[l - 1]));
  for (int k = 0; k < g.ext[2]; ++k)
    for (int j = 0; j < g.ext[1]; ++j)
      for (int i = 0; i < g.ext[0]; ++i) {
        int gi[3];
        elem_global(g, i, j, k, gi);
        const int8_t kd = L.kind[elem_index(g, gi)];
        const int32_t off = (int32_t)g.off(gi[0], gi[1], gi[2]);
        if (kd == K_PHYS) {
          hl.phys.push_back(off);
        } else if (kd == K_PERIODIC) {
          int gw[3];
          for (int q = 0; q < 3; ++q) gw[q] = wrapi(gi[q], next[q]);
          hl.periodic.push_back(make_int2(off, (int32_t)g.off(gw[0], gw[1], gw[2])));
        } else if (kd == K_AMR) {
          // wrapped fine index, parent cell and the 6^3 parent stencil
          int gw[3], first[3], par = 0;
          for (int q = 0; q < 3; ++q) {
            gw[q] = periodic ? wrapi(gi[q], next[q]) : gi[q];
            const int pc = gw[q] >> 1;
            const int odd = gw[q] & 1;
            par |= odd << q;
            first[q] = odd ? pc - 2 : pc - 3;
          }
          const Level& P = c->lev[l - 1];
          if (!pcount->all_interior(first, kPN))
            return fail(SC_ENESTING,
                        "level %d: prolongation stencil of ghost cell (%d,%d,%d) leaves the parent interior", l,
                        gi[0], gi[1], gi[2]);
          AmrCell ac;
          ac.dst = off;
          ac.pbase = (int32_t)P.g.off(first[0], first[1], first[2]);
          ac.parity = par;
          hl.amr.push_back(ac);
          for (int q = 0; q < 3; ++q) {
            hl.amr_gi.push_back(gi[q]);
            hl.amr_gw.push_back(gw[q]);
          }
        }
      }
  if (l > 0 && !hl.amr.empty()) build_amr_tiles(c, l, hl);
  build_stencil_tiles(L, c->tile, hl.tiles);
  // Pointwise tiles of the Z4c stage kernel, one cell per thread: 64-cell
  // tiles in 64-thread blocks on levels of at least 2^17 cells (a 64^3
  // level's 4096 tiles split over the 152 SMs to within 0.2%, against 4% for
  // 2048 tiles of 128 cells: 892 instead of 895 ms per step of the 7-level
  // benchmark), 128-cell tiles in 128-thread blocks on smaller ones (requests
  // of that size served concurrently on streams ran 3% slower in total with
  // the smaller blocks: 2.73e8 against 2.82e8 zone-updates/s on the serving
  // ensemble).
  const int pny = L.interior_cells >= (1L << 17) ? 2 : 4;
  L.ptile_threads = 32 * pny;
  L.box_ptile_begin.clear();
  for (const sc_box& B : L.boxes) {
    L.box_ptile_begin.push_back((int)hl.ptiles.size());
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; y += pny)
        for (int x = B.lo[0]; x <= B.hi[0]; x += 32) {
          Tile t;
          t.x0 = x - g.org[0];
          t.y0 = y - g.org[1];
          t.z0 = z - g.org[2];
          t.nx = std::min(32, B.hi[0] - x + 1);
          t.ny = std::min(pny, B.hi[1] - y + 1);
          t.nz = 1;
          hl.ptiles.push_back(t);
        }
  }
  L.box_ptile_begin.push_back((int)hl.ptiles.size());
  // rows where the Z4c evolution stores D_x (interior cells and their 2-cell
  // extension in y or z) and D_y (extension in z) of the Hessian fields
  if (c->system == SC_Z4C) {
    auto interior_at = [&](int i, int j, int k) {
      if (i < 0 || j < 0 || k < 0 || i >= g.ext[0] || j >= g.ext[1] || k >= g.ext[2]) return false;
      return L.kind[((long)k * g.ext[1] + j) * g.ext[0] + i] == K_INTERIOR;
    };
    for (int k = 0; k < g.ext[2]; ++k)
      for (int j = 0; j < g.ext[1]; ++j) {
        int run_start = -1, run_which = 0;
        const int R = c->order / 2;  // reach of the first-derivative stencil
        for (int i = 0; i <= g.ext[0]; ++i) {
          int which = 0;
          if (i < g.ext[0]) {
            bool dz = false, dy = false;
            for (int d = -R; d <= R && !dz; ++d) dz = interior_at(i, j, k + d);
            for (int d = -R; d <= R && !dy; ++d) dy = interior_at(i, j + d, k);
            which = ((dz || dy) ? 1 : 0) | (dz ? 2 : 0);
          }
          if (which != run_which) {
            if (run_which) {
              RowSeg sg;
              sg.off = (int32_t)(((long)k * g.ext[1] + j) * g.pitch + run_start);
              sg.n = i - run_start;
              sg.which = run_which;
              hl.dxy.push_back(sg);
            }
            run_start = i;
            run_which = which;
          }
        }
      }
  }
  // restriction onto the parent: parent cells whose 8 children are interior here
  if (l > 0) {
    std::vector<std::array<int, 3>> rcells;
    const Level& P = c->lev[l - 1];
    const Geom& pg = P.g;
    for (int k = 0; k < pg.ext[2]; ++k)
      for (int j = 0; j < pg.ext[1]; ++j)
        for (int i = 0; i < pg.ext[0]; ++i) {
          int C[3];
          elem_global(pg, i, j, k, C);
          if (P.kind[elem_index(pg, C)] != K_INTERIOR) continue;
          bool covered = true;
          for (int q = 0; q < 8 && covered; ++q) {
            const int fc[3] = {2 * C[0] + (q & 1), 2 * C[1] + ((q >> 1) & 1), 2 * C[2] + ((q >> 2) & 1)};
            covered = is_interior(L, fc);
          }
          if (!covered) continue;
          const int fb[3] = {2 * C[0] - 2, 2 * C[1] - 2, 2 * C[2] - 2};
          const int fe[3] = {2 * C[0] + 3, 2 * C[1] + 3, 2 * C[2] + 3};
          if (!in_array(g, fb) || !in_array(g, fe)) return fail(SC_ENESTING, "restriction stencil outside level %d", l);
          rcells.push_back({C[0], C[1], C[2]});
        }
    // 4x4x4 parent blocks whose 12^3 fine region lies in the fine array go to
    // the separable kernel; the other cells to the per-cell kernel
    std::map<std::array<int, 3>, unsigned long long> blk;
    for (const auto& C : rcells) {
      const std::array<int, 3> key{C[0] >> 2, C[1] >> 2, C[2] >> 2};
      blk[key] |= 1ull << ((C[0] & 3) + 4 * (C[1] & 3) + 16 * (C[2] & 3));
    }
    for (const auto& kv : blk) {
      const int C0[3] = {4 * kv.first[0], 4 * kv.first[1], 4 * kv.first[2]};
      const int fb[3] = {2 * C0[0] - 2, 2 * C0[1] - 2, 2 * C0[2] - 2};
      const int fe[3] = {2 * C0[0] + 9, 2 * C0[1] + 9, 2 * C0[2] + 9};
      if (in_array(g, fb) && in_array(g, fe)) {
        RestrictBlock rb;
        rb.pbase = (int32_t)pg.off(C0[0], C0[1], C0[2]);
        rb.fbase = (int32_t)g.off(fb[0], fb[1], fb[2]);
        rb.mask = kv.second;
        hl.rblocks.push_back(rb);
        continue;
      }
      for (int q = 0; q < 64; ++q) {
        if (!((kv.second >> q) & 1ull)) continue;
        const int C[3] = {C0[0] + (q & 3), C0[1] + ((q >> 2) & 3), C0[2] + (q >> 4)};
        RestrictCell rc;
        rc.dst = (int32_t)pg.off(C[0], C[1], C[2]);
        rc.fbase = (int32_t)g.off(2 * C[0] - 2, 2 * C[1] - 2, 2 * C[2] - 2);
        hl.restr.push_back(rc);
      }
    }
  }
  return SC_OK;
}

// Allocation owned by one level (released when the level is regridded).
void* level_alloc(sc_ctx* c, Level& L, size_t bytes) {
  void* p = c->dalloc(bytes);
  if (p) L.allocs.push_back(p);
  return p;
}

template <class T>
sc_status level_upload(sc_ctx* c, Level& L, const std::vector<T>& v, T** dst) {
  *dst = nullptr;
  if (v.empty()) return SC_OK;
  *dst = (T*)level_alloc(c, L, v.size() * sizeof(T));
  if (!*dst) return fail(SC_ENOMEM, "device allocation of %zu bytes failed", v.size() * sizeof(T));
  CU(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return SC_OK;
}

void free_level(sc_ctx* c, Level& L) {
  for (void* p : L.allocs) c->dfree(p);
  L.allocs.clear();
}

// Stage vectors a level keeps: rk, plus k4 = f(y_{n+1}) on RK3 levels that
// have a finer level.
int level_kvecs(int rk, int l, int nlev) { return rk == 3 && l + 1 < nlev ? 4 : rk; }

// Device side of a level: the state pair, the two stage buffers and the
// stage vectors (zeroed), its work lists, the ghost store and the eta(r) array.
sc_status setup_level_device(sc_ctx* c, int l, HostLists& hl) {
  Level& L = c->lev[l];
  const size_t vbytes = sizeof(double) * (size_t)c->F * L.g.fs;
  double** vecs[8] = {&L.S[0], &L.S[1], &L.A, &L.B, &L.K[0], &L.K[1], &L.K[2], &L.K[3]};
  for (int j = 0; j < 4; ++j) L.K[j] = nullptr;
  for (int q = 0; q < 4 + level_kvecs(c->rk, l, c->nlev); ++q) {
    double** v = vecs[q];
    *v = (double*)level_alloc(c, L, vbytes);
    if (!*v) return fail(SC_ENOMEM, "level %d: allocation of %zu bytes failed", l, vbytes);
    CU(cudaMemsetAsync(*v, 0, vbytes, c->stream));
  }
  sc_status st;
  if ((st = level_upload(c, L, hl.tiles, &L.tiles)) || (st = level_upload(c, L, hl.amr, &L.amr)) ||
      (st = level_upload(c, L, hl.periodic, &L.periodic)) || (st = level_upload(c, L, hl.phys, &L.phys)) ||
      (st = level_upload(c, L, hl.restr, &L.restr)) || (st = level_upload(c, L, hl.rblocks, &L.rblocks)) ||
      (st = level_upload(c, L, hl.atiles, &L.atiles)) || (st = level_upload(c, L, hl.aslots, &L.aslots)) ||
      (st = level_upload(c, L, hl.dxy, &L.dxy)) || (st = level_upload(c, L, hl.ptiles, &L.ptiles)))
    return st;
  L.ntiles = (int)hl.tiles.size();
  L.namr = (int)hl.amr.size();
  L.natiles = (int)hl.atiles.size();
  L.tile_fmas = hl.tile_fmas;
  L.nptiles = (int)hl.ptiles.size();
  L.ndxy = (int)hl.dxy.size();
  L.namr_blocked = hl.namr_blocked;
  L.nperiodic = (int)hl.periodic.size();
  L.nphys = (int)hl.phys.size();
  L.nrestr = (int)hl.restr.size();
  L.nrblocks = (int)hl.rblocks.size();
  L.amr_store = nullptr;
  if (L.namr) {
    int idx[4];
    const int nvec = 1 + dense_vectors(c->rk, idx);
    L.amr_store = (double*)level_alloc(c, L, sizeof(double) * nvec * (size_t)c->F * L.namr);
    if (!L.amr_store) return fail(SC_ENOMEM, "level %d: ghost store allocation failed", l);
  }
  L.eta = nullptr;
  if (c->system == SC_Z4C && c->eta_profile) {
    L.eta = (double*)level_alloc(c, L, sizeof(double) * (size_t)L.g.fs);
    if (!L.eta) return fail(SC_ENOMEM, "level %d: eta profile allocation failed", l);
    CU(launch_eta_profile(L.eta, L.g, c->eta_c, c->eta_s, c->eta_o, c->stream));
  }
  return SC_OK;
}

// ---------------------------------------------------------------- schedule
struct Emitter {
  sc_ctx* c;
  std::vector<Op> ops;
  std::vector<int> par;

  void fill(int l, double* vec, int which, double theta0) {
    Op o{};
    o.kind = OP_FILL;
    o.level = l;
    o.in = vec;
    o.stage = which;
    if (l > 0) fill_coeffs(c->rk, c->lev[l - 1].dt, theta0, which, o.c);
    ops.push_back(o);
  }
  // Update of stage s with step dt: the next stage input, or y_{n+1}.
  void stage_update(Op& o, int s, double dt) {
    const int S = c->rk;
    if (s < S) {
      o.form = kStageSingle;
      o.cdt = stage_mult(S, s + 1) * dt;
    } else if (S == 4) {
      o.form = kStageRk4;
      o.cdt = dt / 6.0;
    } else if (S == 3) {
      o.form = kStageTwo;
      o.c1dt = 0.25 * dt;
      o.cdt = 0.75 * dt;
    } else {
      o.form = kStageSingle;
      o.cdt = dt;
    }
  }
  // One RK step of level l (Eqs. rk1-rk5 for RK4); for l >= 1 the fine
  // substep at progress theta0 of the parent step.
  void level_step(int l, double theta0) {
    Level& L = c->lev[l];
    double* yn = L.S[par[l]];
    double* ynew = L.S[par[l] ^ 1];
    double* in[4] = {yn, L.A, L.B, L.A};
    const int S = c->rk;
    for (int s = 1; s <= S; ++s) {
      fill(l, in[s - 1], s, theta0);
      Op o{};
      o.kind = OP_STAGE;
      o.level = l;
      o.stage = s;
      o.in = in[s - 1];
      o.yn = yn;
      o.out = (s < S) ? in[s] : ynew;
      stage_update(o, s, L.dt);
      ops.push_back(o);
    }
    const bool k4 = S == 3 && l + 1 < c->nlev;
    // end-of-substep ghosts (read by restriction; and by k4 below)
    if (l > 0 || k4) fill(l, ynew, 0, theta0);
    if (k4) {  // RK3 dense output: k4 = f(y_{n+1}), no state update
      Op o{};
      o.kind = OP_STAGE;
      o.level = l;
      o.stage = 4;
      o.in = ynew;
      o.yn = yn;
      o.out = nullptr;
      o.form = kStageNone;
      ops.push_back(o);
    }
    par[l] ^= 1;
  }
  // Steps 2-7 below level l, after level l has taken a step.
  void children(int l) {
    Op p{};
    p.kind = OP_PROLONG;
    p.level = l + 1;
    p.yn = c->lev[l].S[par[l] ^ 1];  // parent's y_n (its state before the step)
    ops.push_back(p);
    for (int s = 0; s < 2; ++s) {
      level_step(l + 1, 0.5 * s);
      if (l + 2 < c->nlev) children(l + 1);
    }
    Op r{};
    r.kind = OP_RESTRICT;
    r.level = l + 1;
    r.in = c->lev[l + 1].S[par[l + 1]];  // fine state at the end of the parent step
    r.out = c->lev[l].S[par[l]];         // parent's new state
    ops.push_back(r);
  }
  void coarse_step() {
    if (!c->subcycle) {
      for (int q = 0; q < (1 << (c->nlev - 1)); ++q) uniform_step();
      return;
    }
    level_step(0, 0.0);
    if (c->nlev > 1) children(0);
  }
  // Uniform time step (the comparison mode of Sec. IV.A): every level steps
  // with the finest dt, stage by stage in lockstep; refinement-boundary
  // ghosts of a stage state are the prolonged parent stage state of the same
  // stage; after the step the new states' ghosts come from the parents' new
  // states, then restriction runs finest to coarsest.
  void prolong_direct(int l, double* parent_vec, double* dst) {
    Op o{};
    o.kind = OP_PROLONG_DIRECT;
    o.level = l;
    o.in = parent_vec;
    o.out = dst;
    ops.push_back(o);
  }
  void periodic_only(int l, double* vec) {
    Op o{};
    o.kind = OP_FILL;
    o.level = l;
    o.in = vec;
    o.no_amr = true;
    ops.push_back(o);
  }
  void uniform_step() {
    const int L = c->nlev;
    const double dt = c->lev[L - 1].dt;
    const int S = c->rk;
    std::vector<std::array<double*, 4>> in(L);
    for (int l = 0; l < L; ++l) in[l] = {c->lev[l].S[par[l]], c->lev[l].A, c->lev[l].B, c->lev[l].A};
    for (int s = 1; s <= S; ++s)
      for (int l = 0; l < L; ++l) {
        if (l > 0) prolong_direct(l, in[l - 1][s - 1], in[l][s - 1]);
        periodic_only(l, in[l][s - 1]);
        Op o{};
        o.kind = OP_STAGE;
        o.level = l;
        o.stage = s;
        o.in = in[l][s - 1];
        o.yn = c->lev[l].S[par[l]];
        o.out = (s < S) ? in[l][s] : c->lev[l].S[par[l] ^ 1];
        stage_update(o, s, dt);
        ops.push_back(o);
      }
    for (int l = 1; l < L; ++l) {
      prolong_direct(l, c->lev[l - 1].S[par[l - 1] ^ 1], c->lev[l].S[par[l] ^ 1]);
      periodic_only(l, c->lev[l].S[par[l] ^ 1]);
    }
    for (int l = L - 1; l >= 1; --l) {
      Op r{};
      r.kind = OP_RESTRICT;
      r.level = l;
      r.in = c->lev[l].S[par[l] ^ 1];
      r.out = c->lev[l - 1].S[par[l - 1] ^ 1];
      ops.push_back(r);
    }
    for (int l = 0; l < L; ++l) par[l] ^= 1;
  }
};

// Sec. II step 2: prolong the parent's y_n and the stage vectors its dense
// output uses to the refinement-boundary ghost cells of level l.
cudaError_t prolong_parent(sc_ctx* c, int l, const double* yn, cudaStream_t s) {
  Level& L = c->lev[l];
  const Level& P = c->lev[l - 1];
  int idx[4];
  const int nk = dense_vectors(c->rk, idx);
  const double* v[4] = {yn, yn, yn, yn};
  for (int j = 0; j < nk; ++j) v[j] = P.K[idx[j]];
  const int psy = P.g.pitch, psz = P.g.pitch * P.g.ext[1];
  cudaError_t e = launch_amr_prolong_tiles(yn, v[0], v[1], v[2], v[3], P.g.fs, psy, psz, L.atiles, L.natiles, L.aslots,
                                           L.namr,
                                            L.amr_store, c->F, c->w, s, 1 + nk);
  if (e != cudaSuccess) return e;
  return launch_amr_prolong(yn, v[0], v[1], v[2], v[3], P.g.fs, psy, psz, L.amr, L.namr_blocked, L.namr, L.amr_store,
                            c->F, c->w, s, 1 + nk);
}

sc_status run_op(sc_ctx* c, const Op& o, cudaStream_t s) {
  Level& L = c->lev[o.level];
  const Geom& g = L.g;
  switch (o.kind) {
    case OP_PROLONG:
      CU(prolong_parent(c, o.level, o.yn, s));
      break;
    case OP_PROLONG_DIRECT: {
      // one vector through the separable block kernel into the ghost store,
      // then an apply with zero k coefficients (exactly the prolonged value)
      const Level& P = c->lev[o.level - 1];
      const int psy = P.g.pitch, psz = P.g.pitch * P.g.ext[1];
      CU(launch_amr_prolong_tiles(o.in, o.in, o.in, o.in, o.in, P.g.fs, psy, psz, L.atiles, L.natiles, L.aslots, L.namr,
                                   L.amr_store, c->F, c->w, s, 1));
      CU(launch_amr_prolong(o.in, o.in, o.in, o.in, o.in, P.g.fs, psy, psz, L.amr, L.namr_blocked, L.namr, L.amr_store,
                            c->F, c->w, s, 1));
      const double zero[4] = {0.0, 0.0, 0.0, 0.0};
      CU(launch_amr_apply(o.out, g.fs, c->F, L.amr, L.namr, L.amr_store, zero, s, 0));
      break;
    }
    case OP_FILL:
      if (o.level > 0 && !o.no_amr && !o.amr_folded)
        CU(launch_amr_apply(o.in, g.fs, c->F, L.amr, L.namr, L.amr_store, o.c, s, dense_count(c->rk)));
      CU(launch_periodic_copy(o.in, g.fs, c->F, L.periodic, L.nperiodic, s));
      break;
    case OP_STAGE: {
      StageArgs a{};
      a.Y = o.in;
      a.yn = o.yn;
      a.k = L.K[o.stage - 1];
      a.out = o.out;
      a.k1 = L.K[0];
      a.k2 = L.K[1];
      a.k3 = L.K[2];
      a.cdt = o.cdt;
      a.c1dt = o.c1dt;
      a.form = o.form;
      a.stage = o.stage;
      a.fs = g.fs;
      a.sy = g.pitch;
      a.sz = g.pitch * g.ext[1];
      a.h = g.h;
      a.ds = deriv_scales(c->order, g.h);
      a.eta = L.eta;
      // graph form: one launch over the tiles of all boxes; per-box form: one per box
      const int nparts = c->exec_mode == SC_EXEC_PER_BOX ? (int)L.boxes.size() : 1;
      ApplyArgs fold{};
      if (o.fold_fill) {
        fold.vec = o.fold_vec;
        fold.fs = g.fs;
        fold.F = c->F;
        fold.cells = L.amr;
        fold.ncells = L.namr;
        fold.store = L.amr_store;
        for (int j = 0; j < 4; ++j) fold.c[j] = o.fold_c[j];
        fold.nk = dense_count(c->rk);
      }
      const ApplyArgs* foldp = (o.fold_fill && nparts == 1) ? &fold : nullptr;
      const bool one_pass = c->deriv_form == 1 && c->order == 4;
      if (c->system == SC_Z4C && !one_pass)
        CU(launch_z4c_dxy(a.Y, c->scratch, g.fs, a.sy, L.dxy, L.ndxy, s, c->order));
      for (int b = 0; b < nparts; ++b) {
        const int t0 = nparts == 1 ? 0 : L.box_tile_begin[b];
        const int nt = nparts == 1 ? L.ntiles : L.box_tile_begin[b + 1] - t0;
        if (c->system == SC_WAVE) {
          CU(launch_wave_stage(a, L.tiles + t0, nt, s, c->order, foldp));
        } else {
          const int p0 = nparts == 1 ? 0 : L.box_ptile_begin[b];
          const int np = nparts == 1 ? L.nptiles : L.box_ptile_begin[b + 1] - p0;
          if (one_pass) CU(launch_z4c_derivs(a.Y, c->scratch, g.fs, a.sy, a.sz, L.tiles + t0, nt, s));
          else
            CU(launch_z4c_derivs_split(a.Y, c->scratch, g.fs, a.sy, a.sz, L.tiles + t0, nt, s, c->order,
                                       L.tile_cols));
          CU(launch_z4c_stage(a, c->scratch, c->zp, L.ptiles + p0, np, s, c->stage_bps, L.ptile_threads));
        }
      }
      if (L.nphys) CU(launch_radiative_stage(a, L.phys, L.nphys, c->F, g, c->system, s));
      break;
    }
    case OP_CHECK:
      CU(launch_nonfinite_check(o.in, g.fs, c->F, L.tiles, L.ntiles, g.pitch, g.pitch * g.ext[1], c->status, s));
      break;
    case OP_RESTRICT: {
      const Level& P = c->lev[o.level - 1];
      CU(launch_restrict_blocks(o.out, P.g.fs, P.g.pitch, P.g.pitch * P.g.ext[1], o.in, g.fs, g.pitch,
                                g.pitch * g.ext[1], L.rblocks, L.nrblocks, c->F, c->w, s));
      CU(launch_restrict(o.out, P.g.fs, o.in, g.fs, g.pitch, g.pitch * g.ext[1], L.restr, L.nrestr, c->F, c->w, s));
      break;
    }
  }
  return SC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Graph capture of one coarse step per parity of the level-0 state.

namespace {

// Phase table of the persistent coarse-step kernel from the op list: each op
// becomes the phase(s) that do what run_op launches for it.
void persistent_phases(sc_ctx* c, const std::vector<Op>& ops, std::vector<POp>& out) {
  out.clear();
  int idx[4];
  const int nk = dense_vectors(c->rk, idx);
  for (const Op& o : ops) {
    Level& L = c->lev[o.level];
    const Geom& g = L.g;
    POp p{};
    p.F = c->F;
    p.nk = -1;
    switch (o.kind) {
      case OP_PROLONG:
      case OP_PROLONG_DIRECT: {
        const Level& P = c->lev[o.level - 1];
        p.kind = kPhaseProlong;
        const double* v0 = o.kind == OP_PROLONG ? o.yn : o.in;
        for (int j = 0; j < 5; ++j) p.pv[j] = v0;
        if (o.kind == OP_PROLONG)
          for (int j = 0; j < nk; ++j) p.pv[1 + j] = P.K[idx[j]];
        p.nvec = o.kind == OP_PROLONG ? 1 + nk : 1;
        p.pfs = P.g.fs;
        p.psy = P.g.pitch;
        p.psz = P.g.pitch * P.g.ext[1];
        p.atiles = L.atiles;
        p.natiles = L.natiles;
        p.aslots = L.aslots;
        p.amr = L.amr;
        p.namr = L.namr;
        p.namr_blocked = L.namr_blocked;
        p.store = L.amr_store;
        out.push_back(p);
        if (o.kind == OP_PROLONG_DIRECT) {  // then the prolonged value itself (zero k coefficients)
          POp q{};
          q.kind = kPhaseFill;
          q.F = c->F;
          q.vec = o.out;
          q.fs = g.fs;
          q.amr = L.amr;
          q.namr = L.namr;
          q.store = L.amr_store;
          q.nk = 0;
          out.push_back(q);
        }
        break;
      }
      case OP_FILL:
        p.kind = kPhaseFill;
        p.vec = o.in;
        p.fs = g.fs;
        if (o.level > 0 && !o.no_amr) {
          p.amr = L.amr;
          p.namr = L.namr;
          p.store = L.amr_store;
          for (int j = 0; j < 4; ++j) p.c[j] = o.c[j];
          p.nk = nk;
        }
        p.periodic = L.periodic;
        p.nperiodic = L.nperiodic;
        out.push_back(p);
        break;
      case OP_STAGE:
        p.kind = kPhaseStage;
        p.a.Y = o.in;
        p.a.yn = o.yn;
        p.a.k = L.K[o.stage - 1];
        p.a.out = o.out;
        p.a.k1 = L.K[0];
        p.a.k2 = L.K[1];
        p.a.k3 = L.K[2];
        p.a.cdt = o.cdt;
        p.a.c1dt = o.c1dt;
        p.a.form = o.form;
        p.a.stage = o.stage;
        p.a.fs = g.fs;
        p.a.sy = g.pitch;
        p.a.sz = g.pitch * g.ext[1];
        p.a.h = g.h;
        p.a.eta = L.eta;
        p.tiles = L.tiles;
        p.ntiles = L.ntiles;
        p.order = c->order;
        p.phys = L.phys;
        p.nphys = L.nphys;
        p.system = c->system;
        p.g = g;
        out.push_back(p);
        break;
      case OP_RESTRICT: {
        const Level& P = c->lev[o.level - 1];
        p.kind = kPhaseRestrict;
        p.parent = o.out;
        p.ppfs = P.g.fs;
        p.ppsy = P.g.pitch;
        p.ppsz = P.g.pitch * P.g.ext[1];
        p.fine = o.in;
        p.ffs = g.fs;
        p.fsy = g.pitch;
        p.fsz = g.pitch * g.ext[1];
        p.rblocks = L.rblocks;
        p.nrblocks = L.nrblocks;
        p.rcells = L.restr;
        p.nrcells = L.nrestr;
        out.push_back(p);
        break;
      }
      case OP_CHECK:
        p.kind = kPhaseCheck;
        p.vec = o.in;
        p.fs = g.fs;
        p.tiles = L.tiles;
        p.ntiles = L.ntiles;
        p.a.sy = g.pitch;
        p.a.sz = g.pitch * g.ext[1];
        p.status = c->status;
        out.push_back(p);
        break;
    }
  }
  // Fold a pure refinement-boundary fill (no periodic images) into the stage
  // phase before it when the fill's buffer is not the stage's input: the
  // fill writes ghost cells of the next stage input (or of the new state),
  // which the stage neither reads nor writes, and reads only the ghost store
  // an earlier phase prolonged.  One grid barrier fewer per stage.
  std::vector<POp> merged;
  for (const POp& q : out) {
    if (q.kind == kPhaseFill && q.nk >= 0 && q.nperiodic == 0 && !merged.empty() &&
        merged.back().kind == kPhaseStage && merged.back().nk < 0 && merged.back().a.Y != q.vec &&
        merged.back().a.yn != q.vec) {
      POp& st = merged.back();
      st.vec = q.vec;
      st.fs = q.fs;
      st.amr = q.amr;
      st.namr = q.namr;
      st.store = q.store;
      for (int j = 0; j < 4; ++j) st.c[j] = q.c[j];
      st.nk = q.nk;
      continue;
    }
    merged.push_back(q);
  }
  out.swap(merged);
}

// Build (or refresh) the coarse-step schedule of level-0 parity p: the op
// list for the per-box form, the phase table for the persistent form, else
// one CUDA graph captured from the op list.  An
// existing executable graph is updated in place when the new capture has the
// same topology (the usual case after a regrid: same levels, same phases,
// new work lists and sizes), which is much cheaper than instantiating.
sc_status build_schedule(sc_ctx* c, int p) {
  Emitter em;
  em.c = c;
  em.par.assign(c->nlev, 0);
  em.par[0] = p;
  em.coarse_step();
  if (c->finite_check)
    for (int l = 0; l < c->nlev; ++l) {
      Op o{};
      o.kind = OP_CHECK;
      o.level = l;
      o.in = c->lev[l].S[em.par[l]];
      em.ops.push_back(o);
    }
  if (c->exec_mode == SC_EXEC_PERSISTENT) {
    std::vector<POp>& ph = c->host_pops[p];
    persistent_phases(c, em.ops, ph);
    if (c->pops[p]) c->dfree(c->pops[p]);
    c->pops[p] = (POp*)c->dalloc(sizeof(POp) * ph.size());
    if (!c->pops[p]) return fail(SC_ENOMEM, "phase table allocation failed");
    CU(cudaMemcpyAsync(c->pops[p], ph.data(), sizeof(POp) * ph.size(), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));  // the host vector stays, but keep uploads ordered before use
    long work = 1;
    for (const POp& q : ph) work = std::max(work, phase_work_blocks(q));
    c->pwork[p] = work;
    c->launches_per_step = 1;
    c->graph_stale[p] = false;
    return SC_OK;
  }
  if (c->exec_mode == SC_EXEC_PER_BOX) {
    c->plain_ops[p] = em.ops;
    long n = 0;
    for (const Op& o : em.ops) {
      const Level& L = c->lev[o.level];
      if (o.kind == OP_STAGE)
        n += (long)L.boxes.size() * (c->system == SC_Z4C ? 2 : 1) +
             (c->system == SC_Z4C && !(c->deriv_form == 1 && c->order == 4) ? 1 : 0) + (L.nphys ? 1 : 0);
      else if (o.kind == OP_PROLONG)
        n += (L.natiles ? 1 : 0) + (L.namr > L.namr_blocked ? 1 : 0);
      else if (o.kind == OP_FILL)
        n += (o.level > 0 && L.namr && !o.no_amr ? 1 : 0) + (L.nperiodic ? 1 : 0);
      else if (o.kind == OP_PROLONG_DIRECT)
        n += (L.natiles ? 1 : 0) + (L.namr > L.namr_blocked ? 1 : 0) + (L.namr ? 1 : 0);
      else if (o.kind == OP_CHECK)
        n += L.ntiles ? 1 : 0;
      else
        n += (L.nrestr ? 1 : 0) + (L.nrblocks ? 1 : 0);
    }
    c->launches_per_step = n;
    c->graph_stale[p] = false;
    return SC_OK;
  }
  // Graph form of the scalar wave: fold each refinement-boundary fill into
  // the stage launch before it when the fill writes ghost cells of a buffer
  // that stage neither reads nor writes (the next stage input, or the new
  // state): one launch fewer per fine-level stage.  Not for Z4c, where the
  // fill inside the register-heavy stage kernel ran slower than alone.
  for (size_t i = 0; i + 1 < em.ops.size(); ++i) {
    Op& st = em.ops[i];
    Op& fl = em.ops[i + 1];
    if (c->system == SC_WAVE && st.kind == OP_STAGE && fl.kind == OP_FILL && fl.level == st.level && fl.level > 0 &&
        !fl.no_amr &&
        c->lev[fl.level].namr > 0 && fl.in != st.in && fl.in != st.yn) {
      st.fold_fill = true;
      st.fold_vec = fl.in;
      for (int j = 0; j < 4; ++j) st.fold_c[j] = fl.c[j];
      fl.amr_folded = true;
    }
  }
  cudaStream_t cs;
  CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(SC_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  sc_status st = SC_OK;
  for (const Op& o : em.ops) {
    st = run_op(c, o, cs);
    if (st != SC_OK) break;
  }
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (st != SC_OK) return st;
  if (e != cudaSuccess) return fail(SC_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  size_t nn = 0;
  CU(cudaGraphGetNodes(graph, nullptr, &nn));
  c->launches_per_step = (long)nn;
  bool updated = false;
  if (c->graph[p]) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(c->graph[p], graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();  // a topology change is not an error: instantiate anew
      cudaGraphExecDestroy(c->graph[p]);
      c->graph[p] = nullptr;
    }
  }
  if (!updated) e = cudaGraphInstantiate(&c->graph[p], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(SC_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  c->graph_stale[p] = false;
  return SC_OK;
}

// The schedule changed (creation, regrid, new tile shape): rebuild the
// schedule of the current level-0 parity now (errors surface here), the
// other one at its first use, or now as well when both = true.
sc_status build_graphs(sc_ctx* c, bool both = true) {
  c->graph_stale[0] = c->graph_stale[1] = true;
  const int p = c->lev[0].parity;
  sc_status st = build_schedule(c, p);
  if (st == SC_OK && both) st = build_schedule(c, p ^ 1);
  return st;
}

sc_status check_box(sc_ctx* c, int level, int box, int field) {
  if (!c) return fail(SC_EINVAL, "null context");
  if (level < 0 || level >= c->nlev) return fail(SC_EINVAL, "bad level %d", level);
  if (box < 0 || box >= (int)c->lev[level].boxes.size()) return fail(SC_EINVAL, "bad box %d", box);
  if (field < 0 || field >= c->F) return fail(SC_EINVAL, "bad field %d", field);
  return SC_OK;
}

sc_status ensure_staging(sc_ctx* c, size_t bytes) {
  if (c->staging_bytes >= bytes) return SC_OK;
  if (c->staging) {  // the stream may still read the old buffer
    CU(cudaStreamSynchronize(c->stream));
    c->dfree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
  }
  c->staging = (double*)c->dalloc(bytes);
  if (!c->staging) return fail(SC_ENOMEM, "staging allocation of %zu bytes failed", bytes);
  c->staging_bytes = bytes;
  return SC_OK;
}

// Region of a box (optionally with its ghost layers): lo and extents.
void box_region(const sc_box& B, int ghost_layers, int* lo, int* n) {
  const int g = ghost_layers;
  for (int q = 0; q < 3; ++q) {
    lo[q] = B.lo[q] - g;
    n[q] = B.hi[q] - B.lo[q] + 1 + 2 * g;
  }
}

sc_status copy_field(sc_ctx* c, int level, int box, int field, bool ghosted, const double* src, double* dst,
                     bool host) {
  sc_status st = check_box(c, level, box, field);
  if (st) return st;
  Level& L = c->lev[level];
  int lo[3], n[3];
  box_region(L.boxes[box], ghosted ? c->ghost : 0, lo, n);
  const size_t bytes = sizeof(double) * (size_t)n[0] * n[1] * n[2];
  double* state = L.S[L.parity] + (long)field * L.g.fs;
  if (src) {
    const double* dsrc = src;
    if (host) {
      if ((st = ensure_staging(c, bytes))) return st;
      CU(cudaMemcpyAsync(c->staging, src, bytes, cudaMemcpyHostToDevice, c->stream));
      dsrc = c->staging;
    }
    CU(launch_unpack(state, L.g, lo, n, dsrc, c->stream));
    if (host) CU(cudaStreamSynchronize(c->stream));
  } else {
    double* ddst = dst;
    if (host) {
      if ((st = ensure_staging(c, bytes))) return st;
      ddst = c->staging;
    }
    CU(launch_pack(state, L.g, lo, n, ddst, c->stream));
    if (host) {
      CU(cudaMemcpyAsync(dst, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
    }
  }
  return SC_OK;
}

}  // namespace

sc_status sc::set_last_error(sc_status code, const char* msg) { return fail(code, "%s", msg); }


// ---------------------------------------------------------------------------
// Autotuner: tile shape of the stencil kernels.

namespace {

std::mutex g_tune_mutex;
// per (system, level shapes): tile shape, derivative form, stage blocks per SM
std::map<std::string, std::array<int, 5>> g_tune_cache;

std::string tune_key(const sc_ctx* c) {
  std::string k = std::to_string(c->system) + "/" + std::to_string(c->order);
  for (const Level& L : c->lev) {
    std::vector<std::array<int, 3>> ext;
    for (const sc_box& B : L.boxes) ext.push_back({B.hi[0] - B.lo[0] + 1, B.hi[1] - B.lo[1] + 1, B.hi[2] - B.lo[2] + 1});
    std::sort(ext.begin(), ext.end());
    k += "|";
    for (auto& e : ext) k += std::to_string(e[0]) + "x" + std::to_string(e[1]) + "x" + std::to_string(e[2]) + ",";
  }
  return k;
}

StageArgs tuning_stage_args(const Level& L, int order) {
  const Geom& g = L.g;
  StageArgs a{};
  a.Y = L.A;
  a.yn = L.S[L.parity];
  a.k = L.K[1];
  a.out = L.B;
  a.k1 = L.K[0];
  a.k2 = L.K[1];
  a.k3 = L.K[2];
  a.cdt = 0.5 * L.dt;
  a.form = kStageSingle;
  a.stage = 2;
  a.fs = g.fs;
  a.sy = g.pitch;
  a.sz = g.pitch * g.ext[1];
  a.h = g.h;
  a.ds = deriv_scales(order, g.h);
  a.eta = L.eta;
  return a;
}

// Time one candidate on one level with CUDA events on the context's stream
// (one untimed launch first, then reps): kind 0 = the stencil kernel with the
// given tiles (the wave's fused stage, or the Z4c derivative pass in the form
// deriv_form), kind 1 = the Z4c stage kernel built for bps blocks per SM.
sc_status time_candidate(sc_ctx* c, Level& L, int kind, const Tile* tiles, int ntiles, int cols, int deriv_form,
                         int bps, int reps, double* ms) {
  const Geom& g = L.g;
  const StageArgs a = tuning_stage_args(L, c->order);
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  for (int r = -1; r < reps; ++r) {
    if (r == 0) CU(cudaEventRecord(e0, c->stream));
    if (kind == 1) {
      CU(launch_z4c_stage(a, c->scratch, c->zp, L.ptiles, L.nptiles, c->stream, bps, L.ptile_threads));
    } else if (c->system == SC_WAVE) {
      CU(launch_wave_stage(a, tiles, ntiles, c->stream, c->order));
    } else if (deriv_form == 1) {
      CU(launch_z4c_derivs(a.Y, c->scratch, g.fs, a.sy, a.sz, tiles, ntiles, c->stream));
    } else {
      CU(launch_z4c_dxy(a.Y, c->scratch, g.fs, a.sy, L.dxy, L.ndxy, c->stream, c->order));
      CU(launch_z4c_derivs_split(a.Y, c->scratch, g.fs, a.sy, a.sz, tiles, ntiles, c->stream, c->order, cols));
    }
  }
  CU(cudaEventRecord(e1, c->stream));
  CU(cudaEventSynchronize(e1));
  float t = 0;
  CU(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return SC_OK;
}

sc_status apply_tuning(sc_ctx* c, const int* shape, int deriv_form, int bps) {
  for (int q = 0; q < 3; ++q) c->tile[q] = shape[q];
  c->deriv_form = deriv_form;
  c->stage_bps = bps;
  for (Level& L : c->lev) {
    std::vector<Tile> t;
    build_stencil_tiles(L, c->tile, t);
    Tile* d = nullptr;
    CU(cudaStreamSynchronize(c->stream));  // the old list may still be read by queued work
    sc_status st = level_upload(c, L, t, &d);
    if (st) return st;
    if (L.tiles) {
      c->dfree(L.tiles);
      L.allocs.erase(std::find(L.allocs.begin(), L.allocs.end(), (void*)L.tiles));
    }
    L.tiles = d;
    L.ntiles = (int)t.size();
    L.tile_cols = max_tile_cols(t);
  }
  CU(cudaStreamSynchronize(c->stream));
  return build_graphs(c, false);
}

}  // namespace

// Autotuner (the search space: tile shape x derivative-pass split x stage
// kernel blocks per SM).  On the context's largest level it times every tile
// shape of the stencil kernel (the wave's fused stage, or the Z4c derivative
// pass in its two-kernel form), the one-kernel Z4c derivative pass (4th
// order, default tiles), and the Z4c stage kernel built for 2 and for 3 blocks
// per SM; it keeps the fastest derivative configuration and the faster stage
// build.  All forms compute the same derivatives (the one-kernel form sums the
// mixed stencils in another order, so its results differ by rounding).
extern "C" sc_status sc_autotune(sc_ctx* c, int* tile_out, double* ms_out) {
  if (!c) return fail(SC_EINVAL, "null context");
  const std::string key = tune_key(c);
  std::array<int, 5> best{c->tile[0], c->tile[1], c->tile[2], c->deriv_form, c->stage_bps};
  double best_ms = -1.0;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    int big = 0;
    for (int l = 1; l < c->nlev; ++l)
      if (c->lev[l].interior_cells > c->lev[big].interior_cells) big = l;
    Level& L = c->lev[big];
    static const int cand[][3] = {{32, 4, 2}, {32, 2, 4}, {32, 1, 8}, {32, 4, 4}, {32, 2, 8}, {32, 1, 16},
                                  {16, 4, 8}, {64, 1, 8}, {16, 2, 16}, {32, 1, 32}};
    const int nform = (c->system == SC_Z4C && c->order == 4) ? 2 : 1;
    std::vector<Tile> t;
    Tile* d = nullptr;
    size_t cap = 0;
    std::vector<void*> scratch_lists;
    for (int form = 0; form < nform; ++form)
      for (const auto& cd : cand) {
        if (form == 1 && (cd[0] != 32 || cd[1] != 4 || cd[2] != 2)) continue;  // one-kernel form: default tiles
        build_stencil_tiles(L, cd, t);
        if (t.size() > cap) {
          cap = t.size() * 2;
          d = (Tile*)c->dalloc(cap * sizeof(Tile));
          if (!d) return fail(SC_ENOMEM, "autotune tile buffer");
          scratch_lists.push_back(d);
        }
        CU(cudaMemcpyAsync(d, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
        double ms = 0;
        sc_status st = time_candidate(c, L, 0, d, (int)t.size(), max_tile_cols(t), form, 0, 3, &ms);
        if (st) return st;
        if (best_ms < 0 || ms < best_ms) {
          best_ms = ms;
          best = {cd[0], cd[1], cd[2], form, best[4]};
        }
      }
    if (c->system == SC_Z4C) {
      double ms2 = 0, ms3 = 0;
      sc_status st = time_candidate(c, L, 1, nullptr, 0, 0, 0, 2, 3, &ms2);
      if (!st) st = time_candidate(c, L, 1, nullptr, 0, 0, 0, 3, 3, &ms3);
      if (st) return st;
      best[4] = ms2 < ms3 ? 2 : 3;
    }
    CU(cudaStreamSynchronize(c->stream));
    for (void* p : scratch_lists) c->dfree(p);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  sc_status st = apply_tuning(c, best.data(), best[3], best[4]);
  if (st) return st;
  if (tile_out)
    for (int q = 0; q < 3; ++q) tile_out[q] = best[q];
  if (ms_out) *ms_out = best_ms;
  return SC_OK;
}

extern "C" sc_status sc_get_tuning(sc_ctx* c, int* tile, int* deriv_form, int* stage_blocks_per_sm) {
  if (!c || !tile || !deriv_form || !stage_blocks_per_sm) return fail(SC_EINVAL, "null argument");
  for (int q = 0; q < 3; ++q) tile[q] = c->tile[q];
  *deriv_form = c->deriv_form;
  *stage_blocks_per_sm = c->stage_bps;
  return SC_OK;
}

extern "C" sc_status sc_set_tuning(sc_ctx* c, const int* tile, int deriv_form, int stage_blocks_per_sm) {
  if (!c || !tile) return fail(SC_EINVAL, "null argument");
  for (int q = 0; q < 3; ++q)
    if (tile[q] < 1 || tile[q] > 64) return fail(SC_EINVAL, "tile extents must be 1..64");
  if ((long)tile[0] * tile[1] > 1024) return fail(SC_EINVAL, "tile columns must be at most 1024");
  if (deriv_form != 0 && deriv_form != 1) return fail(SC_EINVAL, "derivative form must be 0 or 1");
  if (deriv_form == 1 && (c->system != SC_Z4C || c->order != 4))
    return fail(SC_EINVAL, "the one-kernel derivative pass exists for Z4c at 4th order");
  if (stage_blocks_per_sm != 2 && stage_blocks_per_sm != 3) return fail(SC_EINVAL, "stage blocks per SM must be 2 or 3");
  return apply_tuning(c, tile, deriv_form, stage_blocks_per_sm);
}

// ---------------------------------------------------------------------------
// Moving boxes: regrid and point interpolation.

namespace {

// Transfer lists of one regridded level: cells that stay interior copy
// from the old array; new interior cells are prolonged from the new parent.
struct Transfer {
  std::vector<int2> copy;
  std::vector<AmrCell> prolong;
};

sc_status build_transfer(sc_ctx* c, int l, const Level& old, Transfer& tr) {
  const Level& L = c->lev[l];
  const Level& P = c->lev[l - 1];
  for (const sc_box& B : L.boxes)
    for (int k = B.lo[2]; k <= B.hi[2]; ++k)
      for (int j = B.lo[1]; j <= B.hi[1]; ++j)
        for (int i = B.lo[0]; i <= B.hi[0]; ++i) {
          const int gi[3] = {i, j, k};
          const int32_t dst = (int32_t)L.g.off(i, j, k);
          if (is_interior(old, gi)) {
            tr.copy.push_back(make_int2(dst, (int32_t)old.g.off(i, j, k)));
            continue;
          }
          int first[3], par = 0;
          for (int q = 0; q < 3; ++q) {
            const int odd = gi[q] & 1;
            par |= odd << q;
            first[q] = odd ? (gi[q] >> 1) - 2 : (gi[q] >> 1) - 3;
          }
          for (int a = 0; a < kPN; ++a)
            for (int b = 0; b < kPN; ++b)
              for (int d = 0; d < kPN; ++d) {
                const int pg[3] = {first[0] + d, first[1] + b, first[2] + a};
                if (!is_interior(P, pg))
                  return fail(SC_ENESTING, "regrid: level %d cell (%d,%d,%d) cannot be prolonged from the parent interior",
                              l, i, j, k);
              }
          AmrCell ac;
          ac.dst = dst;
          ac.pbase = (int32_t)P.g.off(first[0], first[1], first[2]);
          ac.parity = par;
          tr.prolong.push_back(ac);
        }
  return SC_OK;
}

}  // namespace

extern "C" sc_status sc_regrid(sc_ctx* c, const int* nboxes, const sc_box* boxes) {
  if (!c || !nboxes || !boxes) return fail(SC_EINVAL, "null argument");
  sc_desc d{};
  d.system = c->system;
  d.nlevels = c->nlev;
  d.nboxes = nboxes;
  d.boxes = boxes;
  for (int q = 0; q < 3; ++q) {
    d.ncells0[q] = c->ncells0[q];
    d.origin[q] = c->origin[q];
  }
  d.h0 = c->h0;
  d.outer_bc = c->bc;
  d.cfl = c->cfl;
  d.subcycle = 1;
  d.fd_order = c->order;
  d.rk_order = c->rk;
  sc_status st = validate(&d);
  if (st) return st;
  if (nboxes[0] != (int)c->lev[0].boxes.size()) return fail(SC_EINVAL, "regrid keeps level 0 unchanged");
  for (int b = 0; b < nboxes[0]; ++b)
    for (int q = 0; q < 3; ++q)
      if (boxes[b].lo[q] != c->lev[0].boxes[b].lo[q] || boxes[b].hi[q] != c->lev[0].boxes[b].hi[q])
        return fail(SC_EINVAL, "regrid keeps level 0 unchanged");
  // phase 1 (host only): new geometry, classification and transfer lists;
  // on failure the old levels are put back untouched.
  std::vector<Level> old(c->nlev);
  for (int l = 1; l < c->nlev; ++l) old[l] = std::move(c->lev[l]);
  std::vector<HostLists> hls(c->nlev);
  std::vector<Transfer> trs(c->nlev);
  int bi = nboxes[0];
  auto restore = [&]() {
    for (int l = 1; l < c->nlev; ++l) c->lev[l] = std::move(old[l]);
  };
  for (int l = 1; l < c->nlev; ++l) {
    c->lev[l] = Level();
    st = build_level_geometry(c, l, boxes + bi, nboxes[l]);
    if (!st) st = classify_level(c, l, hls[l]);
    if (!st) st = build_transfer(c, l, old[l], trs[l]);
    if (st) {
      restore();
      return st;
    }
    bi += nboxes[l];
  }
  // phase 2 (device): allocate the new levels, transfer the state coarse to
  // fine, release the old levels
  const long old_scratch_fs = c->scratch_fs;
  long maxfs = c->lev[0].g.fs;
  for (int l = 1; l < c->nlev; ++l) {
    st = setup_level_device(c, l, hls[l]);
    if (st) return st;  // device allocation failed: the context is unusable (documented)
    Level& L = c->lev[l];
    maxfs = std::max(maxfs, L.g.fs);
    int2* dcopy = nullptr;
    AmrCell* dpro = nullptr;
    if ((st = level_upload(c, L, trs[l].copy, &dcopy)) || (st = level_upload(c, L, trs[l].prolong, &dpro))) return st;
    CU(launch_transfer_copy(L.S[0], L.g.fs, old[l].S[old[l].parity], old[l].g.fs, dcopy, (int)trs[l].copy.size(), c->F,
                            c->stream));
    const Level& P = c->lev[l - 1];
    CU(launch_prolong_state(L.S[0], L.g.fs, P.S[P.parity], P.g.fs, P.g.pitch, P.g.pitch * P.g.ext[1], dpro,
                            (int)trs[l].prolong.size(), c->F, c->w, c->stream));
  }
  CU(cudaStreamSynchronize(c->stream));
  for (int l = 1; l < c->nlev; ++l) free_level(c, old[l]);
  if (c->system == SC_Z4C && maxfs > old_scratch_fs) {
    c->dfree(c->scratch);
    c->scratch = (double*)c->dalloc(sizeof(double) * 176 * (size_t)maxfs);
    if (!c->scratch) return fail(SC_ENOMEM, "derivative scratch allocation failed");
    c->scratch_fs = maxfs;
  }
  return build_graphs(c, false);
}

extern "C" sc_status sc_interpolate(sc_ctx* c, int npts, const double* xyz, int field, double* out) {
  if (!c || (npts > 0 && (!xyz || !out)) || npts < 0) return fail(SC_EINVAL, "bad argument");
  if (field < 0 || field >= c->F) return fail(SC_EINVAL, "bad field %d", field);
  if (npts == 0) return SC_OK;
  std::vector<InterpPoint> pts(npts);
  for (int a = 0; a < npts; ++a) {
    bool found = false;
    for (int l = c->nlev - 1; l >= 0 && !found; --l) {
      const Level& L = c->lev[l];
      int first[3];
      double s[3];
      for (int q = 0; q < 3; ++q) {
        s[q] = (xyz[3 * a + q] - c->origin[q]) / L.g.h - 0.5;  // position in cell-index units
        first[q] = (int)floor(s[q]) - 2;
      }
      bool ok = true;
      for (int kz = 0; kz < kPN && ok; ++kz)
        for (int ky = 0; ky < kPN && ok; ++ky)
          for (int kx = 0; kx < kPN && ok; ++kx) {
            const int g[3] = {first[0] + kx, first[1] + ky, first[2] + kz};
            ok = is_interior(L, g);
          }
      if (!ok) continue;
      InterpPoint& p = pts[a];
      p.base = L.S[L.parity] + (long)field * L.g.fs + L.g.off(first[0], first[1], first[2]);
      p.sy = L.g.pitch;
      p.sz = (long)L.g.pitch * L.g.ext[1];
      for (int q = 0; q < 3; ++q) {
        double x[kPN];
        for (int m = 0; m < kPN; ++m) x[m] = first[q] + m;
        lagrange_weights(x, kPN, s[q], p.w + q * kPN);
      }
      found = true;
    }
    if (!found) return fail(SC_EINVAL, "point %d: no level holds its interpolation stencil", a);
  }
  const size_t rec = sizeof(InterpPoint) * (size_t)npts, outb = sizeof(double) * (size_t)npts;
  sc_status st = ensure_staging(c, rec + outb + 256);
  if (st) return st;
  InterpPoint* dpts = (InterpPoint*)c->staging;
  double* dout = (double*)((char*)c->staging + ((rec + 255) & ~(size_t)255));
  CU(cudaMemcpyAsync(dpts, pts.data(), rec, cudaMemcpyHostToDevice, c->stream));
  CU(launch_interpolate(dpts, npts, dout, c->stream));
  CU(cudaMemcpyAsync(out, dout, outb, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return SC_OK;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char* sc_last_error(void) { return g_err; }

sc_status sc_footprint_estimate(const sc_desc* d, size_t* bytes) {
  sc_status st = validate(d);
  if (st) return st;
  const int F = d->system == SC_WAVE ? kNWave : kNZ4c;
  const int ghost = d->fd_order == 8 ? 4 : 3;
  const int rk = d->rk_order == 0 ? 4 : d->rk_order;
  size_t total = 0, maxfs = 0;
  int bi = 0;
  for (int l = 0; l < d->nlevels; ++l) {
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    long ghost_cells = 0;
    for (int b = 0; b < d->nboxes[l]; ++b, ++bi) {
      const sc_box& B = d->boxes[bi];
      long inner = 1, outer = 1;
      for (int q = 0; q < 3; ++q) {
        lo[q] = std::min(lo[q], B.lo[q]);
        hi[q] = std::max(hi[q], B.hi[q]);
        inner *= B.hi[q] - B.lo[q] + 1;
        outer *= B.hi[q] - B.lo[q] + 1 + 2 * ghost;
      }
      ghost_cells += outer - inner;
    }
    const long pitch = ((hi[0] - lo[0] + 1 + 2 * ghost) + 7) & ~7;
    const long fs = ((pitch * (hi[1] - lo[1] + 1 + 2 * ghost) * (hi[2] - lo[2] + 1 + 2 * ghost)) + 31) & ~31L;
    total += (4 + level_kvecs(rk, l, d->nlevels)) * (size_t)F * fs * sizeof(double);  // S0, S1, A, B, k's
    if (d->system == SC_Z4C && d->eta_profile) total += (size_t)fs * sizeof(double);
    total += (size_t)ghost_cells * ((1 + dense_count(rk)) * F * sizeof(double) + 32);  // prolonged vectors + lists
    total += (size_t)fs * 4;                                       // tiles and other lists (bound)
    maxfs = std::max(maxfs, (size_t)fs);
  }
  if (d->system == SC_Z4C) total += (size_t)maxfs * 176 * sizeof(double);
  // staging for field copies and constraints (largest ghosted box, 7 values per cell), plus slack
  size_t maxbox = 0;
  for (int b = 0; b < bi; ++b) {
    size_t v = 1;
    for (int q = 0; q < 3; ++q) v *= (size_t)(d->boxes[b].hi[q] - d->boxes[b].lo[q] + 1 + 2 * ghost);
    maxbox = std::max(maxbox, v);
  }
  total += maxbox * 7 * sizeof(double) + (1u << 20);
  *bytes = total;
  return SC_OK;
}

sc_status sc_create(const sc_desc* d, sc_ctx** out) {
  if (!out) return fail(SC_EINVAL, "null output pointer");
  *out = nullptr;
  sc_status st = validate(d);
  if (st) return st;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  CU(z4c_init_launch_config());
  std::unique_ptr<sc_ctx> c(new sc_ctx());
  c->system = d->system;
  c->F = d->system == SC_WAVE ? kNWave : kNZ4c;
  c->nlev = d->nlevels;
  c->bc = d->outer_bc;
  for (int q = 0; q < 3; ++q) {
    c->ncells0[q] = d->ncells0[q];
    c->origin[q] = d->origin[q];
  }
  c->h0 = d->h0;
  c->cfl = d->cfl;
  c->zp = Z4cParams{d->kappa1, d->kappa2, d->eta, d->ko_sigma};
  c->stream = (cudaStream_t)d->cuda_stream;
  c->exec_mode = d->exec_mode;
  c->subcycle = d->subcycle;
  c->order = d->fd_order == 8 ? 8 : 4;
  c->ghost = c->order == 8 ? 4 : 3;
  c->rk = d->rk_order == 0 ? 4 : d->rk_order;
  c->eta_profile = d->eta_profile ? 1 : 0;
  c->eta_c = d->eta_c;
  c->eta_s = d->eta_s;
  c->eta_o = d->eta_o;
  c->finite_check = d->finite_check ? 1 : 0;
  cudaError_t e0 = cudaSuccess;
  if (d->allocator && d->allocator->alloc && d->allocator->free) {
    c->alloc = *d->allocator;
    c->has_alloc = true;
  }
  c->w = make_weights();
  c->lev.resize(c->nlev);
  int bi = 0;
  for (int l = 0; l < c->nlev; ++l) {
    st = build_level_geometry(c.get(), l, d->boxes + bi, d->nboxes[l]);
    if (st) return st;
    bi += d->nboxes[l];
  }
  long maxfs = 0;
  for (int l = 0; l < c->nlev; ++l) {
    HostLists hl;
    st = classify_level(c.get(), l, hl);
    if (st) {
      c->release();
      return st;
    }
    st = setup_level_device(c.get(), l, hl);
    if (st) {
      c->release();
      return st;
    }
    Level& L = c->lev[l];
    maxfs = std::max(maxfs, L.g.fs);
  }
  if (c->system == SC_Z4C) {
    c->scratch_fs = maxfs;
    c->scratch = (double*)c->dalloc(sizeof(double) * 176 * (size_t)maxfs);
    if (!c->scratch) {
      c->release();
      return fail(SC_ENOMEM, "derivative scratch allocation failed");
    }
  }
  c->flag = (int*)c->dalloc(sizeof(int));
  c->status = (int*)c->dalloc(sizeof(int));
  c->bar = (GridBarrier*)c->dalloc(sizeof(GridBarrier));
  if (!c->flag || !c->status || !c->bar) {
    c->release();
    return fail(SC_ENOMEM, "flag allocation failed");
  }
  e0 = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e0 == cudaSuccess) e0 = cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), c->stream);
  if (e0 != cudaSuccess) {
    c->release();
    return fail(SC_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e0));
  }
  // lists are uploaded from pageable host vectors: finish before they go away
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->release();
    return fail(SC_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  }
  st = build_graphs(c.get());
  if (st == SC_OK && d->autotune) st = sc_autotune(c.get(), nullptr, nullptr);
  if (st) {
    c->release();
    return st;
  }
  *out = c.release();
  return SC_OK;
}

void sc_destroy(sc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
  for (auto& e : c->xev)
    if (e) cudaEventDestroy(e);
  c->release();
  delete c;
}

sc_status sc_set_initial_data(sc_ctx* c, int kind, const double* params, int nparams) {
  if (!c) return fail(SC_EINVAL, "null context");
  if (nparams < 0 || nparams > 8 || (nparams > 0 && !params)) return fail(SC_EINVAL, "bad parameters");
  const bool wave_kind = kind == SC_ID_STANDING_WAVE || kind == SC_ID_GAUSSIAN || kind == SC_ID_SPHERICAL_GAUSSIAN;
  const bool z4c_kind = kind == SC_ID_BRILL_LINDQUIST || kind == SC_ID_MINKOWSKI || kind == SC_ID_BRILL_LINDQUIST_AVG_LAPSE;
  if ((c->system == SC_WAVE && !wave_kind) || (c->system == SC_Z4C && !z4c_kind))
    return fail(SC_EINVAL, "initial data kind %d does not match the system", kind);
  const int need[6] = {4, 5, 8, 0, 6, 8};
  if (nparams < need[kind]) return fail(SC_EINVAL, "initial data kind %d needs %d parameters", kind, need[kind]);
  for (Level& L : c->lev) {
    L.parity = 0;
    CU(launch_initial_data(L.S[0], L.g, c->F, c->system, kind, params, nparams, c->stream));
  }
  c->t = 0;
  c->zu_finest = c->zu_actual = 0;
  CU(cudaStreamSynchronize(c->stream));
  return SC_OK;
}

sc_status sc_set_field(sc_ctx* c, int l, int b, int f, const double* src) {
  if (!src) return fail(SC_EINVAL, "null source");
  return copy_field(c, l, b, f, false, src, nullptr, true);
}
sc_status sc_set_field_ghosted(sc_ctx* c, int l, int b, int f, const double* src) {
  if (!src) return fail(SC_EINVAL, "null source");
  return copy_field(c, l, b, f, true, src, nullptr, true);
}
sc_status sc_get_field(sc_ctx* c, int l, int b, int f, double* dst) {
  if (!dst) return fail(SC_EINVAL, "null destination");
  return copy_field(c, l, b, f, false, nullptr, dst, true);
}
sc_status sc_get_field_ghosted(sc_ctx* c, int l, int b, int f, double* dst) {
  if (!dst) return fail(SC_EINVAL, "null destination");
  return copy_field(c, l, b, f, true, nullptr, dst, true);
}
sc_status sc_set_field_device(sc_ctx* c, int l, int b, int f, const double* src) {
  if (!src) return fail(SC_EINVAL, "null source");
  return copy_field(c, l, b, f, false, src, nullptr, false);
}
sc_status sc_get_field_device(sc_ctx* c, int l, int b, int f, double* dst) {
  if (!dst) return fail(SC_EINVAL, "null destination");
  return copy_field(c, l, b, f, false, nullptr, dst, false);
}

namespace {

// Packed whole-state transfer (sc_set_state / sc_get_state).  Direct form
// (page-locked host memory, or SC_XFER_DIRECT): the pack/unpack kernels read
// and write the host buffer through its device mapping, so the data crosses
// the CPU-GPU link once, with no staging buffer.  Staged form: one DMA copy
// between the host buffer and a device staging buffer, and the kernels work
// on the staging buffer.  CUDA events on the context's stream split the time
// into copy (DMA) and kernel parts.
sc_status state_transfer(sc_ctx* c, double* host, int ghosted_level0, bool to_device) {
  if (!c || !host) return fail(SC_EINVAL, "null argument");
  if (ghosted_level0 != 0 && ghosted_level0 != 1) return fail(SC_EINVAL, "ghosted_level0 must be 0 or 1");
  size_t bytes = 0;
  sc_status st = sc_state_bytes(c, ghosted_level0, &bytes);
  if (st) return st;
  double* dhost = nullptr;
  if (c->xfer_mode != SC_XFER_STAGED) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) cudaGetLastError();
    else if (at.type == cudaMemoryTypeHost && at.devicePointer) dhost = static_cast<double*>(at.devicePointer);
    if (c->xfer_mode == SC_XFER_DIRECT && !dhost)
      return fail(SC_EINVAL, "direct state transfer needs page-locked (or registered) host memory");
  }
  if (!dhost && (st = ensure_staging(c, bytes))) return st;
  for (auto& e : c->xev)
    if (!e) CU(cudaEventCreate(&e));
  double* buf = dhost ? dhost : c->staging;
  CU(cudaEventRecord(c->xev[0], c->stream));
  if (!dhost && to_device) CU(cudaMemcpyAsync(c->staging, host, bytes, cudaMemcpyHostToDevice, c->stream));
  CU(cudaEventRecord(c->xev[1], c->stream));
  size_t off = 0;
  for (int l = 0; l < c->nlev; ++l) {
    Level& L = c->lev[l];
    for (const sc_box& B : L.boxes) {
      int lo[3], n[3];
      box_region(B, (l == 0 && ghosted_level0) ? c->ghost : 0, lo, n);
      CU(launch_pack_fields(L.S[L.parity], L.g.fs, c->F, L.g, lo, n, buf + off, to_device ? 1 : 0, c->stream));
      off += (size_t)n[0] * n[1] * n[2] * c->F;
    }
  }
  CU(cudaEventRecord(c->xev[2], c->stream));
  if (!dhost && !to_device) CU(cudaMemcpyAsync(host, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaEventRecord(c->xev[3], c->stream));
  CU(cudaStreamSynchronize(c->stream));
  float t01 = 0, t12 = 0, t23 = 0;
  CU(cudaEventElapsedTime(&t01, c->xev[0], c->xev[1]));
  CU(cudaEventElapsedTime(&t12, c->xev[1], c->xev[2]));
  CU(cudaEventElapsedTime(&t23, c->xev[2], c->xev[3]));
  c->xfer_copy_ms = dhost ? 0.0 : (double)t01 + t23;
  c->xfer_kernel_ms = t12;
  c->xfer_bytes = bytes;
  c->xfer_direct = dhost ? 1 : 0;
  return SC_OK;
}

}  // namespace

sc_status sc_state_bytes(sc_ctx* c, int ghosted_level0, size_t* bytes) {
  if (!c || !bytes) return fail(SC_EINVAL, "null argument");
  if (ghosted_level0 != 0 && ghosted_level0 != 1) return fail(SC_EINVAL, "ghosted_level0 must be 0 or 1");
  size_t v = 0;
  for (int l = 0; l < c->nlev; ++l)
    for (const sc_box& B : c->lev[l].boxes) {
      int lo[3], n[3];
      box_region(B, (l == 0 && ghosted_level0) ? c->ghost : 0, lo, n);
      v += (size_t)n[0] * n[1] * n[2] * c->F;
    }
  *bytes = v * sizeof(double);
  return SC_OK;
}

sc_status sc_set_state(sc_ctx* c, const double* src, int ghosted_level0) {
  return state_transfer(c, const_cast<double*>(src), ghosted_level0, true);
}

sc_status sc_get_state(sc_ctx* c, double* dst, int ghosted_level0) {
  return state_transfer(c, dst, ghosted_level0, false);
}

sc_status sc_set_transfer_mode(sc_ctx* c, int mode) {
  if (!c) return fail(SC_EINVAL, "null context");
  if (mode != SC_XFER_AUTO && mode != SC_XFER_STAGED && mode != SC_XFER_DIRECT)
    return fail(SC_EINVAL, "unknown transfer mode %d", mode);
  c->xfer_mode = mode;
  return SC_OK;
}

sc_status sc_transfer_stats(sc_ctx* c, double* copy_ms, double* kernel_ms, size_t* bytes, int* direct) {
  if (!c || !copy_ms || !kernel_ms || !bytes || !direct) return fail(SC_EINVAL, "null argument");
  *copy_ms = c->xfer_copy_ms;
  *kernel_ms = c->xfer_kernel_ms;
  *bytes = c->xfer_bytes;
  *direct = c->xfer_direct;
  return SC_OK;
}

sc_status sc_advance(sc_ctx* c, int n) {
  if (!c) return fail(SC_EINVAL, "null context");
  if (n < 0) return fail(SC_EINVAL, "negative step count");
  for (int s = 0; s < n; ++s) {
    Level& L0 = c->lev[0];
    if (c->graph_stale[L0.parity]) {
      sc_status st = build_schedule(c, L0.parity);
      if (st != SC_OK) return st;
    }
    if (c->exec_mode == SC_EXEC_PERSISTENT) {
      PBatch b{};
      b.n = 1;
      b.nops = (int)c->host_pops[L0.parity].size();
      b.bar = c->bar;
      b.w = c->w;
      b.ops[0] = c->pops[L0.parity];
      b.status[0] = c->status;
      b.nops_r[0] = b.nops;
      int maxb = 0;
      CU(persistent_max_blocks(&maxb));
      CU(launch_persistent_step(b, (int)std::min<long>(c->pwork[L0.parity], maxb), c->stream));
    } else if (c->exec_mode == SC_EXEC_PER_BOX) {
      for (const Op& o : c->plain_ops[L0.parity]) {
        sc_status st = run_op(c, o, c->stream);
        if (st != SC_OK) return st;
      }
    } else {
      CU(cudaGraphLaunch(c->graph[L0.parity], c->stream));
    }
    sc::persistent_step_done(c);
  }
  return SC_OK;
}

}  // extern "C"

void sc::persistent_step_done(sc_ctx* c) {
  const int L = c->nlev;
  Level& L0 = c->lev[0];
  // level 0 takes one step per coarse step when subcycling, 2^(L-1) otherwise
  if (c->subcycle || L == 1) L0.parity ^= 1;
  c->t += L0.dt;
  for (int l = 0; l < L; ++l) {
    c->zu_finest += (double)(1L << (L - 1)) * (double)c->lev[l].interior_cells;
    c->zu_actual += (double)(c->subcycle ? (1L << l) : (1L << (L - 1))) * (double)c->lev[l].interior_cells;
  }
}

sc_status sc::persistent_view(sc_ctx* c, PersistView* v) {
  if (!c || !v || c->exec_mode != SC_EXEC_PERSISTENT) return fail(SC_EINVAL, "not a persistent-form context");
  const int p = c->lev[0].parity;
  if (c->graph_stale[p]) {
    sc_status st = build_schedule(c, p);
    if (st != SC_OK) return st;
  }
  v->ops = c->pops[p];
  v->host = &c->host_pops[p];
  v->status = c->status;
  v->w = c->w;
  return SC_OK;
}

extern "C" {

// Read and clear the device status word after the stream is idle.
sc_status read_status(sc_ctx* c) {
  int h = 0;
  CU(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (!h) return SC_OK;
  CU(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (h & kStatusTimeout) return fail(SC_ETIMEOUT, "a grid barrier of the persistent coarse-step kernel timed out");
  return fail(SC_ENONFINITE, "non-finite value in the evolved state after a coarse step");
}

sc_status sc_synchronize(sc_ctx* c) {
  if (!c) return fail(SC_EINVAL, "null context");
  CU(cudaStreamSynchronize(c->stream));
  return read_status(c);
}

sc_status sc_synchronize_timeout(sc_ctx* c, double timeout_s) {
  if (!c || !(timeout_s >= 0)) return fail(SC_EINVAL, "bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(SC_ECUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= timeout_s)
      return fail(SC_ETIMEOUT, "the context's stream was still busy after %.3f s", timeout_s);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return read_status(c);
}

sc_status sc_get_constraints(sc_ctx* c, int level, int box, double* dst) {
  sc_status st = check_box(c, level, box, 0);
  if (st) return st;
  if (c->system != SC_Z4C) return fail(SC_EINVAL, "constraints need Z4c");
  if (!dst) return fail(SC_EINVAL, "null destination");
  Level& L = c->lev[level];
  const sc_box& B = L.boxes[box];
  int lo[3], n[3];
  box_region(B, 0, lo, n);
  const long ncell = (long)n[0] * n[1] * n[2];
  const size_t bytes = sizeof(double) * kNCons * (size_t)ncell;
  if ((st = ensure_staging(c, bytes))) return st;
  // tiles of this box only
  std::vector<Tile> tl;
  for (int z = B.lo[2]; z <= B.hi[2]; z += 2)
    for (int y = B.lo[1]; y <= B.hi[1]; y += 4)
      for (int x = B.lo[0]; x <= B.hi[0]; x += 32) {
        Tile t;
        t.x0 = x - L.g.org[0];
        t.y0 = y - L.g.org[1];
        t.z0 = z - L.g.org[2];
        t.nx = std::min(32, B.hi[0] - x + 1);
        t.ny = std::min(4, B.hi[1] - y + 1);
        t.nz = std::min(2, B.hi[2] - z + 1);
        tl.push_back(t);
      }
  Tile* dt = (Tile*)c->dalloc(tl.size() * sizeof(Tile));
  if (!dt) return fail(SC_ENOMEM, "tile list allocation failed");
  CU(cudaMemcpyAsync(dt, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  const double* Y = L.S[L.parity];
  const int sy = L.g.pitch, sz = L.g.pitch * L.g.ext[1];
  const int blo[3] = {B.lo[0] - L.g.org[0], B.lo[1] - L.g.org[1], B.lo[2] - L.g.org[2]};
  if (c->order == 4) {
    CU(launch_z4c_derivs(Y, c->scratch, L.g.fs, sy, sz, dt, (int)tl.size(), c->stream));
  } else {
    CU(launch_z4c_dxy(Y, c->scratch, L.g.fs, sy, L.dxy, L.ndxy, c->stream, c->order));
    CU(launch_z4c_derivs_split(Y, c->scratch, L.g.fs, sy, sz, dt, (int)tl.size(), c->stream, c->order,
                               max_tile_cols(tl)));
  }
  CU(launch_z4c_constraints(Y, c->scratch, c->staging, L.g.fs, sy, sz, c->zp, deriv_scales(c->order, L.g.h), dt, (int)tl.size(), ncell, blo, n,
                            c->stream));
  CU(cudaMemcpyAsync(dst, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->dfree(dt);  // the per-call tile list (the stream is idle)
  return SC_OK;
}

sc_status sc_get_time(sc_ctx* c, double* t) {
  if (!c || !t) return fail(SC_EINVAL, "null argument");
  *t = c->t;
  return SC_OK;
}

sc_status sc_zone_updates(sc_ctx* c, double* finest, double* actual) {
  if (!c || !finest || !actual) return fail(SC_EINVAL, "null argument");
  *finest = c->zu_finest;
  *actual = c->zu_actual;
  return SC_OK;
}

sc_status sc_launches_per_step(sc_ctx* c, long* n) {
  if (!c || !n) return fail(SC_EINVAL, "null argument");
  *n = c->launches_per_step;
  return SC_OK;
}

sc_status sc_time_stage_kernels(sc_ctx* c, int level, int nrep, double* ms) {
  if (!c || !ms || nrep < 1) return fail(SC_EINVAL, "bad argument");
  if (level < 0 || level >= c->nlev) return fail(SC_EINVAL, "bad level %d", level);
  Level& L = c->lev[level];
  const Geom& g = L.g;
  StageArgs a{};
  a.Y = L.A;
  a.yn = L.S[L.parity];
  a.k = L.K[1];
  a.out = L.B;
  a.k1 = L.K[0];
  a.k2 = L.K[1];
  a.k3 = L.K[2];
  a.cdt = 0.5 * L.dt;
  a.form = kStageSingle;
  a.stage = 2;
  a.fs = g.fs;
  a.sy = g.pitch;
  a.sz = g.pitch * g.ext[1];
  a.h = g.h;
  a.ds = deriv_scales(c->order, g.h);
  a.eta = L.eta;
  cudaEvent_t e[3];
  for (auto& x : e) CU(cudaEventCreate(&x));
  float t0 = 0, t1 = 0;
  CU(cudaEventRecord(e[0], c->stream));
  for (int r = 0; r < nrep; ++r) {
    if (c->system == SC_WAVE) CU(launch_wave_stage(a, L.tiles, L.ntiles, c->stream, c->order));
    else if (c->deriv_form == 1 && c->order == 4)
      CU(launch_z4c_derivs(a.Y, c->scratch, g.fs, a.sy, a.sz, L.tiles, L.ntiles, c->stream));
    else {
      CU(launch_z4c_dxy(a.Y, c->scratch, g.fs, a.sy, L.dxy, L.ndxy, c->stream, c->order));
      CU(launch_z4c_derivs_split(a.Y, c->scratch, g.fs, a.sy, a.sz, L.tiles, L.ntiles, c->stream, c->order,
                                 L.tile_cols));
    }
  }
  CU(cudaEventRecord(e[1], c->stream));
  if (c->system == SC_Z4C)
    for (int r = 0; r < nrep; ++r)
      CU(launch_z4c_stage(a, c->scratch, c->zp, L.ptiles, L.nptiles, c->stream, c->stage_bps, L.ptile_threads));
  CU(cudaEventRecord(e[2], c->stream));
  CU(cudaEventSynchronize(e[2]));
  CU(cudaEventElapsedTime(&t0, e[0], e[1]));
  CU(cudaEventElapsedTime(&t1, e[1], e[2]));
  for (auto& x : e) cudaEventDestroy(x);
  ms[0] = t0 / nrep;
  ms[1] = c->system == SC_Z4C ? t1 / nrep : 0.0;
  return SC_OK;
}

sc_status sc_run_op_class_pass(sc_ctx* c, int level) {
  if (!c) return fail(SC_EINVAL, "null context");
  if (c->system != SC_Z4C) return fail(SC_EINVAL, "the op-class pass exists for Z4c only");
  if (level < 0 || level >= c->nlev) return fail(SC_EINVAL, "bad level %d", level);
  Level& L = c->lev[level];
  const Geom& g = L.g;
  const StageArgs a = tuning_stage_args(L, c->order);
  CU(launch_z4c_dxy(a.Y, c->scratch, g.fs, a.sy, L.dxy, L.ndxy, c->stream, c->order, true));
  CU(launch_z4c_derivs_split(a.Y, c->scratch, g.fs, a.sy, a.sz, L.tiles, L.ntiles, c->stream, c->order, L.tile_cols,
                             true));
  CU(launch_z4c_stage(a, c->scratch, c->zp, L.ptiles, L.nptiles, c->stream, c->stage_bps, L.ptile_threads, true));
  CU(cudaStreamSynchronize(c->stream));
  return SC_OK;
}

sc_status sc_check_finite(sc_ctx* c) {
  if (!c) return fail(SC_EINVAL, "null context");
  CU(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  for (Level& L : c->lev)
    CU(launch_nonfinite_check(L.S[L.parity], L.g.fs, c->F, L.tiles, L.ntiles, L.g.pitch, L.g.pitch * L.g.ext[1], c->flag,
                              c->stream));
  int h = 0;
  CU(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (h) return fail(SC_ENONFINITE, "non-finite value in the evolved state");
  return SC_OK;
}

sc_status sc_debug_get_vector(sc_ctx* c, int level, int box, int vec, int field, int ghosted, double* dst) {
  sc_status st = check_box(c, level, box, field);
  if (st) return st;
  if (!dst || vec < 0 || vec > 7) return fail(SC_EINVAL, "bad vector or destination");
  Level& L = c->lev[level];
  double* src[8] = {L.S[L.parity], L.S[L.parity ^ 1], L.A, L.B, L.K[0], L.K[1], L.K[2], L.K[3]};
  if (!src[vec]) return fail(SC_EINVAL, "vector %d is not used by this Runge-Kutta method", vec);
  int lo[3], n[3];
  box_region(L.boxes[box], ghosted ? c->ghost : 0, lo, n);
  const size_t bytes = sizeof(double) * (size_t)n[0] * n[1] * n[2];
  if ((st = ensure_staging(c, bytes))) return st;
  CU(launch_pack(src[vec] + (long)field * L.g.fs, L.g, lo, n, c->staging, c->stream));
  CU(cudaMemcpyAsync(dst, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return SC_OK;
}

sc_status sc_time_ghost_kernels(sc_ctx* c, int level, int nrep, double* ms, long* counts) {
  if (!c || !ms || !counts || nrep < 1) return fail(SC_EINVAL, "bad argument");
  if (level < 1 || level >= c->nlev) return fail(SC_EINVAL, "level must be a refined level");
  Level& L = c->lev[level];
  const Level& P = c->lev[level - 1];
  double coef[4];
  fill_coeffs(c->rk, P.dt, 0.0, 2, coef);
  cudaEvent_t e[3];
  for (auto& x : e) CU(cudaEventCreate(&x));
  CU(cudaEventRecord(e[0], c->stream));
  for (int r = 0; r < nrep; ++r) CU(prolong_parent(c, level, P.S[P.parity], c->stream));
  CU(cudaEventRecord(e[1], c->stream));
  for (int r = 0; r < nrep; ++r)
    CU(launch_amr_apply(L.A, L.g.fs, c->F, L.amr, L.namr, L.amr_store, coef, c->stream, dense_count(c->rk)));
  CU(cudaEventRecord(e[2], c->stream));
  CU(cudaEventSynchronize(e[2]));
  float t0 = 0, t1 = 0;
  CU(cudaEventElapsedTime(&t0, e[0], e[1]));
  CU(cudaEventElapsedTime(&t1, e[1], e[2]));
  for (auto& x : e) cudaEventDestroy(x);
  ms[0] = t0 / nrep;
  ms[1] = t1 / nrep;
  counts[0] = L.namr;
  counts[1] = L.natiles;
  counts[2] = L.namr - L.namr_blocked;
  counts[3] = L.tile_fmas;
  return SC_OK;
}

sc_status sc_footprint(sc_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(SC_EINVAL, "null argument");
  *bytes = c->footprint;
  return SC_OK;
}

}  // extern "C"
