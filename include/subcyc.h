/*
 * subcyc.h -- C ABI of the GB300 (sm_103a) library for RK4 subcycling in time
 * on nested refined boxes with dense-output ghost filling, after
 * "GPU-accelerated Subcycling Time Integration with the Einstein Toolkit"
 * (arXiv:2503.09629).
 *
 * Library: libsubcyc.so.  All arithmetic is FP64 and runs in CUDA kernels on
 * one GPU; there is no CPU fallback: every compute entry point fails with
 * SC_ECUDA when no device is usable.
 *
 * Conventions shared by every call:
 *   - cell-centred grids; level l has spacing h_l = h0 / 2^l and cell index
 *     space [0, ncells0[d] * 2^l) per dimension; cell i of level l has centre
 *     origin + (i + 1/2) h_l;
 *   - refinement factor 2 between levels (Sec. II: h^(l) / h^(l+1) = 2);
 *   - 3 ghost cells around every box (4 with 8th-order differences);
 *   - field arrays exchanged with the caller are x-fastest, contiguous,
 *     FP64, one field at a time;
 *   - every call returns an sc_status (0 = success, negative = error) and
 *     never aborts; sc_last_error() gives a thread-local message;
 *   - the caller owns every descriptor and host buffer it passes; no call
 *     keeps a caller pointer after it returns; the library owns its device
 *     memory, obtained through the caller's allocator when one is given.
 */
#ifndef SUBCYC_H
#define SUBCYC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sc_ctx sc_ctx;
typedef int sc_status;

enum {
  SC_OK = 0,
  SC_EINVAL = -1,      /* bad argument */
  SC_ENOMEM = -2,      /* device allocation failed */
  SC_ECUDA = -3,       /* CUDA error (message in sc_last_error) */
  SC_ENESTING = -4,    /* hierarchy not properly nested or not aligned */
  SC_ENONFINITE = -5,  /* non-finite value found in the evolved state */
  SC_ETIMEOUT = -6,    /* a bounded wait ran out */
  SC_EBUSY = -7        /* request can never fit the memory budget */
};

typedef enum { SC_WAVE = 0, SC_Z4C = 1 } sc_system;
typedef enum { SC_BC_PERIODIC = 0, SC_BC_RADIATIVE = 1 } sc_outer_bc;

/* Initial data kinds for sc_set_initial_data (params in brackets):
 *  SC_ID_STANDING_WAVE  wave: [A, kx, ky, kz]  u = A sin(2 pi kx x) sin(2 pi ky y) sin(2 pi kz z), Pi = 0
 *  SC_ID_GAUSSIAN       wave: [A, w, cx, cy, cz]  u = A exp(-|x - c|^2 / (2 w^2)), Pi = 0
 *  SC_ID_BRILL_LINDQUIST z4c: [m1, x1, y1, z1, m2, x2, y2, z2]  psi = 1 + sum m/(2 r),
 *                       W = psi^-2, gt = delta, alpha = psi^-2, rest 0 (Sec. III.B, lapse psi^-2)
 *  SC_ID_MINKOWSKI      z4c: []  flat space
 *  SC_ID_SPHERICAL_GAUSSIAN wave: [A, sigma, t, cx, cy, cz]  Sec. IV.A exact solution
 *  SC_ID_BRILL_LINDQUIST_AVG_LAPSE z4c: as SC_ID_BRILL_LINDQUIST with the averaged lapse of
 *                       Sec. III.B, alpha = (1 + (1 - s)/(1 + s))/2, s = sum m/(2 r) */
enum { SC_ID_STANDING_WAVE = 0, SC_ID_GAUSSIAN = 1, SC_ID_BRILL_LINDQUIST = 2, SC_ID_MINKOWSKI = 3,
       SC_ID_SPHERICAL_GAUSSIAN = 4, SC_ID_BRILL_LINDQUIST_AVG_LAPSE = 5 };

/* A box: inclusive cell indices in its level's index space. */
typedef struct {
  int lo[3];
  int hi[3];
} sc_box;

/* Device-memory allocator supplied by the caller (e.g. a framework's caching
 * allocator).  alloc returns a device pointer aligned to >= 256 bytes or NULL;
 * free releases it.  NULL allocator -> cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} sc_allocator;

/* Hierarchy description, deep-copied by sc_create.
 *   boxes: all boxes, level 0 first, nboxes[l] of them for level l;
 *   level 0 must cover the domain [0, ncells0) exactly (disjoint boxes);
 *   fine boxes (l >= 1) must start on even and end on odd indices (aligned to
 *   parent cells), must not overlap each other, and every refinement-boundary
 *   ghost cell's prolongation stencil (6 parent cells per dimension) must lie
 *   in the parent level's interior (proper nesting, else SC_ENESTING);
 *   outer_bc: SC_BC_RADIATIVE needs exactly one level-0 box;
 *   cfl: dt_l = cfl * h_l; subcycle = 1: the paper's subcycling; 0: the
 *   uniform-step comparison mode (Sec. IV.A): every level steps with the
 *   finest dt in lockstep, 2^(nlevels-1) steps per coarse step, fine ghosts
 *   from the prolonged parent stage state of the same stage;
 *   kappa1, kappa2, eta, ko_sigma: Z4c damping, Gamma-driver and
 *   Kreiss-Oliger parameters (Sec. III);
 *   cuda_stream: cudaStream_t all work is ordered on (NULL = legacy stream). */
typedef struct {
  int system;
  int nlevels;
  const int* nboxes;
  const sc_box* boxes;
  int ncells0[3];
  double origin[3];
  double h0;
  int outer_bc;
  double cfl;
  int subcycle;
  double kappa1, kappa2, eta, ko_sigma;
  void* cuda_stream;
  const sc_allocator* allocator;
  int exec_mode;  /* SC_EXEC_GRAPH (0, default): one CUDA graph per coarse step, one launch per
                     level and phase covering all boxes; SC_EXEC_PER_BOX (1): the plain form, stage
                     kernels launched box by box directly on the stream, no graph (for comparison);
                     SC_EXEC_PERSISTENT (2, scalar wave only): one cooperative launch per coarse
                     step runs every phase of Sec. II steps 1-7 on all levels (all stages of every
                     substep, ghost fills, prolongation, restriction) with grid-wide barriers
                     between dependent phases; bitwise the same fields as the graph form */
  int autotune;   /* 1: run sc_autotune at creation (cached per system and level shapes) */
  int eta_profile; /* Z4c: 0 = constant eta; 1 = eta(r) = (eta_c - eta_o) exp(-(r/eta_s)^4) + eta_o
                      with r the coordinate radius (Sec. III.A) */
  double eta_c, eta_s, eta_o;
  int fd_order;    /* finite-difference order of the right-hand sides: 4 (0 = default) or 8, the
                      paper's production setting (Sec. III.C); Kreiss-Oliger stays r = 4.  Every box
                      then carries 4 ghost layers instead of 3 (the _ghosted field calls use them). */
  int rk_order;    /* Runge-Kutta method, subcycled with its own dense output: 4 (0 = default), the
                      classic RK4 of Sec. II; 3, Heun's third-order method (stage inputs y + h/3 k1,
                      y + 2h/3 k2; y_{n+1} = y + h/4 (k1 + 3 k3)); 2, the explicit midpoint rule
                      (y + h/2 k1; y_{n+1} = y + h k2).  RK2 and RK3 are the extension the paper
                      (Sec. V) leaves to future work.  Dense outputs: RK3 uses the cubic Hermite
                      interpolant through y_n and y_{n+1} with slopes k1 and k4 = f(y_{n+1}),
                      b1 = t - 5t^2/4 + t^3/2, b3 = 9t^2/4 - 3t^3/2, b4 = -t^2 + t^3 (third
                      order; k4 costs one extra right-hand side per step on every level that
                      has a finer level); RK2 uses b1 = t - t^2, b2 = t^2.  Fine stage inputs at
                      refinement boundaries are the Taylor expansions of the method's stages
                      (RK3: y, y + h/3 y', y + 2h/3 y' + 2h^2/9 y''; RK2: y, y + h/2 y').
                      Other values: SC_EINVAL. */
  int finite_check; /* 1: every coarse step ends with a device scan of every level's state for
                       non-finite values (failure detection of a long evolution; no host
                       synchronisation); the next sc_synchronize reports SC_ENONFINITE */
} sc_desc;

enum { SC_EXEC_GRAPH = 0, SC_EXEC_PER_BOX = 1, SC_EXEC_PERSISTENT = 2 };

/* Build the hierarchy of Sec. II: nested levels with h^(l) / h^(l+1) = 2,
 * each a set of boxes.  Validates nesting and alignment, allocates every
 * level's state, stage and k1..k_s arrays (s = rk_order; the stage vectors
 * the dense output of Eq. denseoutput1 reads are kept on every level that has
 * a finer level), builds the device work lists and the coarse-step CUDA
 * graphs.  *out receives the context (owned by the caller until
 * sc_destroy); on error *out = NULL and nothing stays allocated.
 * Errors: SC_EINVAL, SC_ENESTING, SC_ENOMEM, SC_ECUDA. */
sc_status sc_create(const sc_desc* desc, sc_ctx** out);

/* Release every device allocation of a context made by sc_create
 * (synchronises the context's stream).  NULL is ignored. */
void sc_destroy(sc_ctx* ctx);

/* Fill the state of every level (interior and ghosts) with analytic initial
 * data, on the device (Sec. III.B Brill-Lindquist data; Sec. IV.A scalar
 * waves); resets the time to 0.  params: host array of nparams doubles as
 * listed for each kind above.  Synchronises.  Errors: SC_EINVAL (kind does
 * not match the system, too few parameters), SC_ECUDA. */
sc_status sc_set_initial_data(sc_ctx* ctx, int kind, const double* params, int nparams);

/* Set initial data (Sec. III.B, Sec. IV.A: the paper's initial data are
 * given per grid point) for one field of one box from host memory: src holds
 * the box interior, (hi-lo+1) cells per dimension, x fastest, FP64; fields in
 * the order listed at sc_desc (wave u, Pi; Z4c W, gt_xx..gt_zz, Khat,
 * At_xx..At_zz, Gamt^x..^z, Theta, alpha, beta^x..^z).  Stream-ordered and
 * synchronous with respect to the host buffer (returns after the copy has
 * been consumed).  Errors: SC_EINVAL (level, box, field out of range, NULL
 * src), SC_ENOMEM (staging), SC_ECUDA. */
sc_status sc_set_field(sc_ctx* ctx, int level, int box, int field, const double* host_src);
/* As sc_set_field, including the ghost cells (3 per side, 4 with 8th-order
 * differences): src has (hi-lo+7) or (hi-lo+9) cells per dimension.  Needed for
 * the evolved outer ghost shell of a radiative level 0 and for
 * checkpoint/resume. */
sc_status sc_set_field_ghosted(sc_ctx* ctx, int level, int box, int field, const double* host_src);

/* Read one field of one box (interior, layout as sc_set_field) to host
 * memory: the evolved fields of Sec. III.A / IV.A, e.g. for the
 * convergence and waveform comparisons of Sec. IV.  Synchronises.  Errors as
 * sc_set_field. */
sc_status sc_get_field(sc_ctx* ctx, int level, int box, int field, double* host_dst);
sc_status sc_get_field_ghosted(sc_ctx* ctx, int level, int box, int field, double* host_dst);

/* Device-resident variants (Sec. II keeps the whole state on the GPU): the
 * same copies between the state and a caller-owned device buffer of the
 * same shape; stream-ordered on the context's stream, no host
 * synchronisation.  Errors as sc_set_field. */
sc_status sc_set_field_device(sc_ctx* ctx, int level, int box, int field, const double* dev_src);
sc_status sc_get_field_device(sc_ctx* ctx, int level, int box, int field, double* dev_dst);

/* Whole-state transfer (no counterpart in the paper, which keeps the state on
 * the device; this is the upload/download of a host application that owns
 * its data, and the checkpoint/restart path).  The packed layout
 * concatenates, for every level l (coarse to fine), every box b (creation
 * order) and every field f, the box region x fastest: with its ghost cells on
 * level 0 when ghosted_level0 = 1 (the evolved shell of a radiative boundary
 * lives there), its interior elsewhere.  *bytes = size of that buffer.
 * Two forms, chosen by sc_set_transfer_mode:
 *   direct (the default for page-locked or registered host memory): one
 *     pack/unpack kernel per box reads or writes the host buffer through its
 *     device mapping, so the data crosses the CPU-GPU link once and no
 *     device staging memory is used;
 *   staged (pageable memory, or SC_XFER_STAGED): one DMA copy between the
 *     host buffer and a device staging buffer of the same size (allocated on
 *     first use, kept with the context) plus one kernel per box.
 * Both return after the host buffer has been consumed or filled (they
 * synchronise the context's stream); sc_transfer_stats then gives the
 * split of the last transfer, timed with CUDA events on the stream: DMA
 * milliseconds (0 in the direct form), pack/unpack kernel milliseconds, the
 * bytes moved and whether the direct form ran.  Errors: SC_EINVAL (null
 * pointer, ghosted_level0 not 0/1, SC_XFER_DIRECT with pageable memory),
 * SC_ENOMEM (staging), SC_ECUDA. */
enum { SC_XFER_AUTO = 0, SC_XFER_STAGED = 1, SC_XFER_DIRECT = 2 };
sc_status sc_state_bytes(sc_ctx* ctx, int ghosted_level0, size_t* bytes);
sc_status sc_set_state(sc_ctx* ctx, const double* host_src, int ghosted_level0);
sc_status sc_get_state(sc_ctx* ctx, double* host_dst, int ghosted_level0);
sc_status sc_set_transfer_mode(sc_ctx* ctx, int mode);
sc_status sc_transfer_stats(sc_ctx* ctx, double* copy_ms, double* kernel_ms, size_t* bytes, int* direct);

/* Advance n coarse steps (Sec. II, steps 1-7 per coarse step): level 0
 * takes one RK step storing its stage vectors, every finer level two substeps per
 * parent step with refinement-boundary ghosts from the parent's dense
 * output (theta0 = 0 and 1/2), recursively, then restriction.  Each coarse
 * step is one CUDA graph launch on the context's stream; asynchronous. */
sc_status sc_advance(sc_ctx* ctx, int n_coarse_steps);

/* Block until the context's stream is idle (the coarse steps of
 * sc_advance, Sec. II, have completed).  Returns SC_ECUDA on a device error
 * and SC_ENONFINITE when the per-step finiteness check of a context created
 * with finite_check = 1 found a non-finite value. */
sc_status sc_synchronize(sc_ctx* ctx);
/* As sc_synchronize with a bounded host-side wait: SC_ETIMEOUT (work still
 * queued, the context stays usable) if the stream is not idle after
 * timeout_s seconds. */
sc_status sc_synchronize_timeout(sc_ctx* ctx, double timeout_s);

/* Scan the interior state of every level on the device (the evolved fields
 * of Sec. III.A / IV.A): SC_OK if every value is finite, SC_ENONFINITE
 * otherwise.  Synchronises.  The paper has no counterpart: it is the
 * failure detection of a long evolution. */
sc_status sc_check_finite(sc_ctx* ctx);

/* Z4c constraints of the current state at the interior cells of one box
 * (Sec. IV.B, Fig. 6 plots the L2 norms of H and M_x): H = R + 2/3 (Khat +
 * 2 Theta)^2 - At_ij At^ij, M^i = d_j At^ij + Gamt^i_jk At^jk - 3 At^ij d_j W / W
 * - 2/3 gt^ij d_j (Khat + 2 Theta), G^i = Gamt^i - gt^jk Gamt^i_jk, with the
 * context's finite-difference order.  host_dst: 7 * ncell doubles
 * (constraint-major H, M^x, M^y, M^z, G^x, G^y, G^z; x fastest).
 * Synchronises.  Errors: SC_EINVAL (not Z4c, bad level/box, NULL), SC_ENOMEM,
 * SC_ECUDA. */
sc_status sc_get_constraints(sc_ctx* ctx, int level, int box, double* host_dst);

/* Simulation time of level 0 (Sec. II: dt_l = cfl * h_l, the coarse step
 * advances t by dt_0). */
sc_status sc_get_time(sc_ctx* ctx, double* t);
/* Cell updates done so far: finest-equivalent (every cell counted at the
 * finest time step, "as if no subcycling had been used", Sec. IV.C) and
 * actual (each level's cells times its own steps). */
sc_status sc_zone_updates(sc_ctx* ctx, double* finest_equiv, double* actual);
/* Number of kernel launches one coarse step performs (graph nodes; Sec. II
 * steps 1-7 on every level). */
sc_status sc_launches_per_step(sc_ctx* ctx, long* n);
/* Device bytes held by the context (all levels' state, stage and k
 * vectors of Sec. II, work lists, scratch). */
sc_status sc_footprint(sc_ctx* ctx, size_t* bytes);
/* Footprint a descriptor would need, without allocating (an upper bound of
 * sc_footprint after sc_create; used for admission by the server). */
sc_status sc_footprint_estimate(const sc_desc* desc, size_t* bytes);

/* Measurement (no counterpart in the paper).  Time the kernels of one RK4
 * stage (stage 2, Eq. rk2) of one level outside the graph, with CUDA events recorded on the context's stream, averaged over
 * nrep launches each: ms[0] = Z4c derivative pass (wave: fused stage kernel),
 * ms[1] = Z4c right-hand-side + update pass (wave: 0).  Overwrites only the
 * level's k2 and second stage buffer, which every coarse step recomputes
 * before reading; call between sc_advance calls.  Synchronises. */
sc_status sc_time_stage_kernels(sc_ctx* ctx, int level, int nrep, double* ms);
/* Measurement (no counterpart in the paper; Z4c only, SC_EINVAL for the
 * scalar wave).  Run the kernels that sc_time_stage_kernels times (the
 * derivative pass in its row-segment + per-cell form, then the right-hand
 * side + update pass) once on one level in their op-class build: the same
 * arithmetic, bitwise the same results, with every addition, subtraction and
 * multiplication issued as a DADD or DMUL instead of a unit-constant FMA.  An
 * instruction counter over these launches (their kernel names carry PlainK)
 * then splits the FP64 stream into general FMAs and the operations that issue
 * at the slower DADD rate.  Writes what sc_time_stage_kernels writes, plus the
 * derivative scratch, which every stage recomputes; call between sc_advance
 * calls.  Synchronises. */
sc_status sc_run_op_class_pass(sc_ctx* ctx, int level);

/* Z4c constraints of one box held by the caller, computed without allocating
 * any device memory.  The paper has no counterpart: this entry point serves
 * callers that cannot allocate -- a solver embedded in a host application
 * that owns all device memory and forbids other allocations, a process whose
 * memory pool is fixed at start-up, or a latency-critical loop in which
 * cudaMalloc/cudaFree would implicitly synchronise the device.
 * It computes 4th-order centred differences on 3 ghost layers whatever
 * finite-difference order the caller's evolution uses.
 *   dev_state: device pointer, 22 Z4c fields (field order as in the context),
 *              each a box with 3 ghost layers per side, (n[0]+6)(n[1]+6)(n[2]+6)
 *              doubles, x fastest, fields contiguous one after another;
 *              the ghost layers must hold valid data;
 *   dev_out:   device pointer, 7 * n[0]*n[1]*n[2] doubles, written with
 *              H, M^x, M^y, M^z, G^x, G^y, G^z at the interior cells
 *              (constraint-major, x fastest), as sc_get_constraints;
 *   n:         host pointer, interior extents; h: grid spacing;
 *   cuda_stream: cudaStream_t the work is ordered on (NULL = legacy stream).
 * The derivative scratch is a static device array of this library sized for
 * at most 32,768 cells including ghosts (for example a 26^3 interior), about
 * 40 MB, which every GPU that loads the library holds until the process
 * exits; larger boxes are rejected with SC_EINVAL.  Every call shares that
 * array, so calls that overlap on the GPU race: serialise them (one stream,
 * or wait for the previous call).  The first call on a device looks up the
 * array's device address (with that device current) and caches it; make the
 * first call before any stream capture.  The call makes no host-to-device
 * copy (its tile list is generated on the device) and is asynchronous:
 * dev_out is ready when the stream reaches it.  Errors: SC_EINVAL (NULL
 * pointer, non-positive extent or spacing, box too large), SC_ECUDA.  No
 * cudaMalloc, cudaFree or allocating library routine is called. */
sc_status sc_z4c_constraints_noalloc(const double* dev_state, double* dev_out, const int* n, double h,
                                     void* cuda_stream);

/* Moving boxes (Sec. II: the refined regions follow the punctures and the
 * hierarchy is regridded; Sec. IV.B runs move the box stacks every coarse
 * step): replace the boxes of every refined level (level 0 must stay
 * as it is; layout as in sc_desc: nboxes per level, boxes level by level).
 * Each interior cell of the new layout that was an interior cell of the same
 * level keeps its state; every other interior cell takes the quintic
 * prolongation of its parent's state (the parent already regridded).  The
 * new layout must satisfy the same nesting rules as sc_create (else
 * SC_ENESTING, with the old layout kept).  Rebuilds the work lists and the
 * coarse-step graphs; call between sc_advance calls.  Synchronises.  After a
 * device allocation failure (SC_ENOMEM) the context must be destroyed. */
sc_status sc_regrid(sc_ctx* ctx, const int* nboxes, const sc_box* boxes);

/* Field values at npts points (xyz: 3 doubles per point, physical
 * coordinates; used for puncture tracking, dx_p/dt = -beta(x_p), of the
 * moving boxes) by tensor-product quintic Lagrange interpolation on the finest
 * level whose 6x6x6 cell stencil around the point is interior; SC_EINVAL if
 * no level holds it.  out: npts doubles (host).  Synchronises. */
sc_status sc_interpolate(sc_ctx* ctx, int npts, const double* xyz, int field, double* out);

/* Autotuner (no counterpart in the paper): on the context's largest level,
 * with CUDA events on its stream, time the candidate tile shapes of the
 * stencil kernel (the fused wave stage, or the Z4c derivative pass in its
 * two-kernel form), the one-kernel Z4c derivative pass (4th order) and the
 * Z4c stage kernel built for 2 and for 3 warps per scheduler; keep the fastest
 * derivative configuration and stage build, rebuild the tile lists and the
 * coarse-step graphs.  The choice is cached for the process per
 * (system, box shapes of every level); a cached context skips the timing
 * (*ms_out = -1).  Overwrites only stage/scratch buffers that every coarse
 * step recomputes; call between sc_advance calls.  tile_out: 3 ints or NULL. */
sc_status sc_autotune(sc_ctx* ctx, int* tile_out, double* ms_out);
/* The tuning in effect (no counterpart in the paper): tile = 3 ints (tile
 * shape of the stencil kernels), deriv_form = 0 (Z4c derivative pass as two
 * kernels: D_x/D_y of the Hessian fields on rows, then the per-column pass
 * that differentiates them for the mixed derivatives) or 1 (one kernel per
 * cell and field with direct 16-point mixed stencils; Z4c at 4th order
 * only), stage_blocks_per_sm = 2 or 3 (the Z4c stage kernel's build: the
 * register budget of that many 128-thread blocks per SM, i.e. 2 or 3 warps
 * per scheduler; on levels of 2^17 cells or more it runs as twice as many
 * 64-thread blocks over 64-cell tiles).  sc_set_tuning applies a
 * choice made elsewhere (rebuilds the tile lists and graphs; call between
 * sc_advance calls); SC_EINVAL for values outside those ranges. */
sc_status sc_get_tuning(sc_ctx* ctx, int* tile, int* deriv_form, int* stage_blocks_per_sm);
sc_status sc_set_tuning(sc_ctx* ctx, const int* tile, int deriv_form, int stage_blocks_per_sm);

/* ---- serving: continuous batching of independent evolutions ---------------
 * The paper has no counterpart: this is the serving form of the method, many
 * small independent evolutions (each one hierarchy of Sec. II) sharing one GPU.
 * A server owns max_active slots (one CUDA stream each) and a device-memory
 * budget.  sc_server_submit queues a request (hierarchy, analytic initial
 * data, number of coarse steps); it fails with SC_EBUSY if the request's
 * footprint (sc_footprint_estimate) exceeds the whole budget.  Each
 * sc_server_tick (non-blocking) retires requests whose last step completed,
 * admits queued requests in arrival order while a slot is free and their
 * footprint fits the budget left (allocating their state from a
 * stream-ordered pool on the slot's stream), and launches the next coarse step
 * of every active request with fewer than `depth` steps in flight.  Requests
 * run concurrently on their own streams; a request's result is bitwise the
 * same as when it runs alone.  A finished request keeps its state resident
 * until sc_server_release.  latency = completion seen by a tick - submission. */
typedef struct sc_server sc_server;
sc_status sc_server_create(size_t hbm_budget_bytes, int max_active, int depth, sc_server** out);
sc_status sc_server_submit(sc_server* srv, const sc_desc* desc, int id_kind, const double* id_params, int nparams,
                           int n_coarse_steps, unsigned long long* ticket);
sc_status sc_server_tick(sc_server* srv, int* n_active, int* n_queued, int* n_launched);
/* done = 1 once the request finished; returns the request's status: SC_OK,
 * or SC_ENOMEM when its state could not be allocated while no other request
 * was running (it then holds nothing; release it). */
sc_status sc_server_poll(sc_server* srv, unsigned long long ticket, int* done, double* latency_s);
/* Tick and poll until the request is done or timeout_s seconds have passed
 * (SC_ETIMEOUT; the request keeps running).  Host-side wait, bounded. */
sc_status sc_server_wait(sc_server* srv, unsigned long long ticket, double timeout_s, double* latency_s);
/* Merged form (on = 1; off by default): scalar-wave requests run in the
 * persistent coarse-step form (SC_EXEC_PERSISTENT) and each tick launches the
 * next coarse step of all of them as one cooperative kernel on the server's
 * batch stream (phase i of every request between the same two grid
 * barriers); Z4c requests keep one graph per step on their own stream.
 * on = 0 (the default, measured faster on GB300): every request runs its own
 * graph on its own stream.  Applies to requests admitted afterwards; results
 * are bitwise the same either way. */
sc_status sc_server_set_merge(sc_server* srv, int on);
/* Host-side fault injection for tests of the admission path: the k-th device
 * allocation the server makes from now on fails as if the pool were
 * exhausted (k = 0 disables).  A request whose allocation fails is retried
 * after running requests free memory, or fails with SC_ENOMEM when none is
 * running. */
sc_status sc_server_inject_alloc_failure(sc_server* srv, long k);
sc_status sc_server_read(sc_server* srv, unsigned long long ticket, int level, int box, int field, double* host_dst);
sc_status sc_server_release(sc_server* srv, unsigned long long ticket);
sc_status sc_server_stats(sc_server* srv, double* zu_finest_done, double* zu_actual_done, long* launches,
                          size_t* bytes_in_use);
sc_status sc_server_destroy(sc_server* srv);

/* Read any of a level's internal vectors for one box and field (inspection
 * and testing): vec 0 = current state, 1 = the other state buffer (after a
 * step: the state at the start of the level's last step, with the ghost
 * values its first stage used), 2/3 = stage buffers, 4..7 = k1..k4 of the
 * level's last step (SC_EINVAL for k's the Runge-Kutta method does not have).
 * ghosted: include the ghost cells (3 or 4 per side).  Synchronises. */
sc_status sc_debug_get_vector(sc_ctx* ctx, int level, int box, int vec, int field, int ghosted, double* host_dst);

/* Time the refinement-boundary kernels of one refined level outside the
 * graph, with CUDA events on the context's stream, averaged over nrep:
 * ms[0] = prolongation of the parent's y_n and the stage vectors its dense
 * output uses (k1..k4 for RK4) to the level's ghost cells
 * (tile-separable kernel plus per-cell fallback), ms[1] = one dense-output
 * ghost fill.  counts (4 longs): [0] ghost cells, [1] slab tiles of the
 * separable kernel, [2] ghost cells on the per-cell fallback, [3] FMAs the
 * separable kernel executes per (vector, field) over all its tiles.
 * Writes only the level's ghost store and second stage buffer; call between
 * sc_advance calls.  Synchronises. */
sc_status sc_time_ghost_kernels(sc_ctx* ctx, int level, int nrep, double* ms, long* counts);

/* Measurement (no counterpart in the paper; every kernel of this library is
 * bound by the FP64 pipe, whose rate depends on the operands).  Measures, on
 * the current device with CUDA events on cuda_stream, the issue rates of a
 * general FP64 fused multiply-add and of an FP64 addition (G instructions per
 * second, 8 independent chains per thread, 8 blocks of 256 threads per SM,
 * the best of three timed launches after an untimed one),
 * and reports the SM count and the maximum SM clock.  Allocates and frees a
 * small output buffer; synchronises.  Errors: SC_EINVAL, SC_ENOMEM, SC_ECUDA. */
sc_status sc_measure_fp64_peak(void* cuda_stream, double* dfma_g_per_s, double* dadd_g_per_s, int* sms,
                               double* sm_clock_mhz);

const char* sc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
