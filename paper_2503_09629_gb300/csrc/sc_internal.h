// sc_internal.h -- shared declarations of the subcycling library (host runtime
// and kernel launchers).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "subcyc.h"

namespace sc {

constexpr int kGhost = 3;   // ghost width of every box
constexpr int kPN = 6;      // prolongation stencil points per dimension (quintic)
constexpr int kRN = 6;      // restriction stencil points per dimension (quintic)
constexpr int kNZ4c = 22;   // Z4c evolved fields
constexpr int kNWave = 2;   // scalar wave fields (u, Pi)
constexpr int kNCons = 7;   // Z4c constraint outputs (H, M^i, G^i)

// Z4c field order: W, gt(xx,xy,xz,yy,yz,zz), Khat, At(6), Gamt(3), Theta, alpha, beta(3).
enum { ZW = 0, ZG = 1, ZK = 7, ZA = 8, ZGAM = 14, ZTH = 17, ZAL = 18, ZB = 19 };

// Geometry of one level's dense array.  The array covers the bounding box of
// the level's box interiors grown by the ghost width; x is fastest.
struct Geom {
  int org[3];     // global cell index of array element (0,0,0)
  int ext[3];     // array extents
  int pitch;      // row pitch (>= ext[0], multiple of 8)
  long fs;        // field stride in doubles (multiple of 32)
  double h;       // grid spacing
  double x0[3];   // physical centre of array element (0,0,0)
  long off(int gx, int gy, int gz) const {
    return ((long)(gz - org[2]) * ext[1] + (gy - org[1])) * pitch + (gx - org[0]);
  }
};

// One interior tile: array coordinates of its first cell and its extents.
struct Tile {
  int x0, y0, z0, nx, ny, nz;
};

// Refinement-boundary ghost cell: destination offset in the fine array,
// offset of the first parent stencil cell in the parent array, parity of
// the fine index per dimension (bit d set: fine centre at +1/4 parent cell).
struct AmrCell {
  int32_t dst;
  int32_t pbase;
  int32_t parity;
};

// A tile of refinement-boundary ghost positions prolonged together by the
// separable kernel: extents ext[3] (at most 8 per axis, at most 4 along its
// thin axis), bit d of par = parity of the wrapped fine index of its first
// position along axis d, pbase = offset of the first parent node of the
// region its stencils cover, and slots[slot_base + (k * ext[1] + j) * ext[0]
// + i] = the store slot (AMR list index) of position (i, j, k), or -1 for a
// position that is computed but not stored.
struct AmrTile {
  int32_t pbase;
  int32_t slot_base;
  int8_t ext[3];
  int8_t par;
};

// Restricted parent cell: its offset in the parent array and the offset of
// the first fine stencil cell (2C-2 per dimension) in the fine array.
struct RestrictCell {
  int32_t dst;
  int32_t fbase;
};

// 4x4x4 parent cells restricted together (aligned to multiples of 4 in the
// parent index space): offset of the block's first parent cell in the parent
// array (may lie outside it; only masked cells are written), offset of the
// first of the 12x12x12 fine cells their stencils cover, and which of the 64
// parent cells (bit x + 4y + 16z) are restricted.
struct RestrictBlock {
  int32_t pbase;
  int32_t fbase;
  unsigned long long mask;
};

// A run of consecutive cells of one array row: offset of the first cell,
// count, and which first derivatives to store there (bit 0: D_x, bit 1: D_y).
struct RowSeg {
  int32_t off;
  int32_t n;
  int32_t which;
};

// One interpolation point: first cell of its 6x6x6 stencil in a level array,
// the array strides, and the quintic weights per dimension (x, y, z).
struct InterpPoint {
  const double* base;
  long sy, sz;
  double w[3 * kPN];
};

struct Weights {
  double prolong[2][kPN];   // [parity][node]
  double restrict_w[kRN];
};

// Factors that turn the Z4c derivative pass's stored integer-weight stencil
// sums into derivatives: first derivatives times s1, pure second derivatives
// times s2p, mixed second derivatives times s2m (4th order: 1/(12h),
// 1/(12h^2), 1/(144h^2); 8th order: 1/(840h), 1/(5040h^2), 1/(840h)^2).
struct DerivScales {
  double s1, s2p, s2m;  // first, pure second and mixed second derivative
  double hs1, ts1, qs1;  // s1 / 2, s1 / 3 and s1 / 4
  double hs2p, ts2m;    // s2p / 2 and 2 s2m
};
// The products are formed on the host so that the kernels take every factor
// as a kernel-parameter operand (no register, no extra instruction).
inline DerivScales deriv_scales(int order, double h) {
  const double w1 = order == 8 ? 840.0 : 12.0, w2 = order == 8 ? 5040.0 : 12.0;
  DerivScales d;
  d.s1 = 1.0 / (w1 * h);
  d.s2p = 1.0 / (w2 * h * h);
  d.s2m = 1.0 / (w1 * h * w1 * h);
  d.hs1 = 0.5 * d.s1;
  d.ts1 = d.s1 / 3.0;
  d.qs1 = 0.25 * d.s1;
  d.hs2p = 0.5 * d.s2p;
  d.ts2m = 2.0 * d.s2m;
  return d;
}

// Arguments of one fused RK4 stage (right-hand side + stage update).
struct StageArgs {
  const double* Y;   // stage input, ghosts valid
  const double* yn;  // state at the start of the step
  double* k;         // k_stage (output)
  double* out;       // next stage input, or y_{n+1} after the last stage
  const double* k1;
  const double* k2;
  const double* k3;
  // Update written to out (kStage* below):
  //   kStageSingle: out = yn + cdt k           (stage inputs; RK2's last stage)
  //   kStageRk4:    out = yn + cdt (k1 + 2 k2 + 2 k3 + k), cdt = dt / 6
  //   kStageTwo:    out = yn + c1dt k1 + cdt k (RK3's last stage)
  //   kStageNone:   k only, out unused (RK3's k4 = f(y_{n+1}))
  double cdt;
  double c1dt;
  int form;
  int stage;         // 1..s
  long fs;
  int sy, sz;        // strides of y and z in doubles
  double h;
  const double* eta; // Z4c: per-cell Gamma-driver damping eta(r), or null for the constant
  DerivScales ds;    // Z4c: scales of the stored derivative sums
};

// Additions, subtractions and scalings that do not fuse are written as fused
// multiply-adds with constants the compiler cannot see (+1, -1, -0 arrive as
// kernel arguments): fma(a, 1, b) = a + b, fma(b, -1, a) = a - b and
// fma(x, y, -0) = x * y exactly, so the results are bitwise those of the
// plain operations.  Measured on this GPU: the Z4c derivative and stage
// kernels run about 5% faster this way than in their op-class build below,
// the same arithmetic with DADD/DSUB/DMUL (ncu on a 262,144-cell level:
// 339 against 358 us and 538 against 564 us), although an isolated chain of
// fma(x, 1, a) issues no faster than DADD (504 G/s; a general DFMA 597 G/s).
struct FmaK {
  double one, mone, mzero;
};
// The op-class form of the same arithmetic (sc_run_op_class_pass): each such
// operation issued as a DADD or DMUL that the compiler never contracts into an
// FMA, so an instruction counter separates the general FMAs (the faster issue
// rate) from the operations that issue at the DADD rate.  Bitwise the same
// results as FmaK.
struct PlainK {};
#ifdef __CUDACC__
__device__ __forceinline__ double fadd(double a, double b, const FmaK& K) { return fma(a, K.one, b); }
__device__ __forceinline__ double fsub(double a, double b, const FmaK& K) { return fma(b, K.mone, a); }
__device__ __forceinline__ double fmul(double a, double b, const FmaK& K) { return fma(a, b, K.mzero); }
__device__ __forceinline__ double fadd(double a, double b, const PlainK&) { return __dadd_rn(a, b); }
__device__ __forceinline__ double fsub(double a, double b, const PlainK&) { return __dsub_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b, const PlainK&) { return __dmul_rn(a, b); }
#endif

enum { kStageSingle = 0, kStageRk4 = 1, kStageTwo = 2, kStageNone = 3 };

// A refinement-boundary ghost fill carried out by a stage launch (ncells = 0:
// none): ghost value = store[0] + sum_j c_j store[j + 1] over nk prolonged
// stage vectors, written to vec at the AMR cells.  The graph form of the
// scalar wave folds the fill of the next stage input into the stage that
// precedes it: the fill writes ghost cells of a buffer that stage neither
// reads nor writes.  (Z4c keeps separate fill launches: inside its stage
// kernel, at 12 warps per SM, the latency-bound fill ran slower than alone
// and lengthened the step.)
struct ApplyArgs {
  double* vec;
  long fs;
  int F;
  const AmrCell* cells;
  int ncells;
  const double* store;
  double c[4];
  int nk;
};

// Bits of a context's device status word (OR-ed by kernels, read and cleared
// by sc_synchronize): a non-finite value after a coarse step, a grid barrier
// of the persistent coarse-step kernel that gave up waiting.
enum { kStatusNonFinite = 1, kStatusTimeout = 2 };

struct Z4cParams {
  double kappa1, kappa2, eta, ko_sigma;
};

// Record a message for sc_last_error() and return code (defined in sc_host.cu).
sc_status set_last_error(sc_status code, const char* msg);

// Streaming multiprocessors of the current device (queried once per device;
// the grid caps of the grid-stride and persistent launches are multiples of
// it).  Defined in sc_amr.cu.
int sm_count();

// ---- kernel launchers (defined in the .cu files) -------------------------
cudaError_t launch_wave_stage(const StageArgs& a, const Tile* tiles, int ntiles, cudaStream_t s, int order = 4,
                              const ApplyArgs* fill = nullptr);

cudaError_t launch_z4c_derivs(const double* Y, double* scratch, long fs, int sy, int sz,
                              const Tile* tiles, int ntiles, cudaStream_t s);
// Occupancy-derived persistent grid sizes of the Z4c kernels (once per device,
// before any graph capture).
cudaError_t z4c_init_launch_config();
// order: finite-difference order of the derivatives, 4 or 8 (Kreiss-Oliger stays r = 4).
// op_class: the PlainK build of the kernel (same results; see PlainK).
cudaError_t launch_z4c_dxy(const double* Y, double* scratch, long fs, int sy, const RowSeg* segs, int nsegs,
                           cudaStream_t s, int order = 4, bool op_class = false);
// max_cols: the largest nx * ny of the tiles (work is dealt out per tile in
// chunks sized by it); cudaErrorInvalidValue if below 1.
cudaError_t launch_z4c_derivs_split(const double* Y, double* scratch, long fs, int sy, int sz,
                                    const Tile* tiles, int ntiles, cudaStream_t s, int order, int max_cols,
                                    bool op_class = false);
// bps: warps per scheduler of the stage kernel's build (the register budget of
// bps 128-thread blocks per SM), 2 or 3 (a tuning choice); threads: block
// size, 128 (tiles of at most 128 cells) or 64 (tiles of at most 64 cells, 2 bps
// blocks per SM); cudaErrorInvalidValue otherwise.  op_class: the PlainK build
// (stage form kStageSingle only, cudaErrorInvalidValue for the others).
cudaError_t launch_z4c_stage(const StageArgs& a, const double* scratch, const Z4cParams& p,
                             const Tile* tiles, int ntiles, cudaStream_t s, int bps, int threads,
                             bool op_class = false);
cudaError_t launch_radiative_stage(const StageArgs& a, const int32_t* cells, int ncells, int F,
                                   const Geom& g, int system, cudaStream_t s);
cudaError_t launch_z4c_constraints(const double* Y, const double* scratch, double* out, long fs, int sy,
                                   int sz, const Z4cParams& p, const DerivScales& ds, const Tile* tiles, int ntiles,
                                   long out_stride, const int* box_lo, const int* box_n, cudaStream_t s);

cudaError_t launch_periodic_copy(double* vec, long fs, int F, const int2* pairs, int npairs, cudaStream_t s);
// per-cell prolongation of AMR cells [first, ncells) of the list (store has ncells slots per vector-field);
// nvec = 1 + the number of stage vectors the dense output reads (5 for RK4, 4 for RK3, 3 for RK2), passed
// in order as k1..k4; nvec = 1 prolongs only the first vector
cudaError_t launch_amr_prolong(const double* yn, const double* k1, const double* k2, const double* k3,
                               const double* k4, long pfs, int psy, int psz, const AmrCell* cells, int first,
                               int ncells, double* store, int F, const Weights& w, cudaStream_t s, int nvec = 5);
// separable prolongation of the ghost cells grouped in slab tiles
cudaError_t launch_amr_prolong_tiles(const double* yn, const double* k1, const double* k2, const double* k3,
                                     const double* k4, long pfs, int psy, int psz, const AmrTile* tiles, int ntiles,
                                     const int32_t* slots, int ncells, double* store, int F, const Weights& w,
                                     cudaStream_t s, int nvec = 5);
cudaError_t launch_amr_apply(double* vec, long fs, int F, const AmrCell* cells, int ncells,
                             const double* store, const double* c4, cudaStream_t s, int nk = 4);
cudaError_t launch_restrict(double* parent, long pfs, const double* fine, long ffs, int fsy, int fsz,
                            const RestrictCell* cells, int ncells, int F, const Weights& w, cudaStream_t s);
// Separable form of the restriction over RestrictBlocks (bitwise the same
// results as launch_restrict for the same cells).
cudaError_t launch_restrict_blocks(double* parent, long pfs, int psy, int psz, const double* fine, long ffs, int fsy,
                                   int fsz, const RestrictBlock* blocks, int nblocks, int F, const Weights& w,
                                   cudaStream_t s);
cudaError_t launch_initial_data(double* vec, const Geom& g, int F, int system, int kind, const double* params,
                                int nparams, cudaStream_t s);
cudaError_t launch_transfer_copy(double* dst, long dfs, const double* src, long sfs, const int2* pairs, int n, int F,
                                 cudaStream_t s);
cudaError_t launch_prolong_state(double* dst, long dfs, const double* parent, long pfs, int psy, int psz,
                                 const AmrCell* cells, int n, int F, const Weights& w, cudaStream_t s);
cudaError_t launch_interpolate(const InterpPoint* pts, int n, double* out, cudaStream_t s);
// eta(r) = (eta_c - eta_o) exp(-(r / eta_s)^4) + eta_o at every element of a level array
cudaError_t launch_eta_profile(double* eta, const Geom& g, double eta_c, double eta_s, double eta_o, cudaStream_t s);
cudaError_t launch_pack(const double* vec, const Geom& g, const int* lo, const int* n, double* dst,
                        cudaStream_t s);
cudaError_t launch_unpack(double* vec, const Geom& g, const int* lo, const int* n, const double* src,
                          cudaStream_t s);
// All F fields (stride fs) of a box region to or from a packed buffer (F
// consecutive x-fastest blocks); unpack = 1 writes the array.
cudaError_t launch_pack_fields(double* vec, long fs, int F, const Geom& g, const int* lo, const int* n, double* buf,
                               int unpack, cudaStream_t s);
cudaError_t launch_nonfinite_check(const double* vec, long fs, int F, const Tile* tiles, int ntiles, int sy,
                                   int sz, int* flag, cudaStream_t s);

}  // namespace sc
