// sc_persist.cu -- the persistent coarse-step kernel of the scalar-wave
// system: one cooperative launch runs a whole coarse step (Sec. II steps 1-7
// on every level: all stages of every substep, the dense-output ghost fills,
// the prolongation of the parent's vectors and the restriction), phase after
// phase, with a grid-wide barrier between dependent phases, for one context
// or for a batch of contexts whose schedules have the same shape (the served
// form merges the active requests of a tick into one launch this way).
//
// Each phase runs the same device-function bodies as the stand-alone kernels
// (sc_device.cuh), so every value is computed by the same arithmetic as in
// the graph form.  The barrier waits are bounded: a block that has waited
// kBarrierTimeoutNs for the others sets kStatusTimeout in every context's
// status word and returns, so a launch can end early but never hangs.
#include "sc_device.cuh"
#include "sc_persist.h"

namespace sc {
namespace {

constexpr int kPThreads = 256;
constexpr unsigned long long kBarrierTimeoutNs = 5ull * 1000 * 1000 * 1000;
// dynamic shared memory: the larger of the prolongation and the restriction
// workspaces (2 groups each)
constexpr int kPSmemDoubles =
    2 * kProlongSmemPerGroup > 2 * kRestrictSmemPerGroup ? 2 * kProlongSmemPerGroup : 2 * kRestrictSmemPerGroup;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  The
// last block to arrive resets the count and advances the generation; the
// others wait for the generation to change, at most kBarrierTimeoutNs.
// Thread 0's fences order the whole block's writes (made visible to it by
// the preceding __syncthreads) before the arrival and the other blocks'
// writes before the block continues.  Returns false on timeout.
__device__ bool grid_barrier(GridBarrier* bar, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &bar->gen;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (unsigned spin = 1; *gen == g; ++spin) {
        if ((spin & 63) == 0 && globaltimer_ns() - t0 > kBarrierTimeoutNs) {
          good = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ void run_phase(const POp& op, const Weights& w, double* sm, int bid, int nb) {
  const FmaK K{1.0, -1.0, -0.0};
  switch (op.kind) {
    case kPhaseStage:
      if (op.ntiles) {
        if (op.order == 8) wave_stage_body<8>(op.a, op.tiles, op.ntiles, K, bid, nb);
        else wave_stage_body<4>(op.a, op.tiles, op.ntiles, K, bid, nb);
      }
      if (op.nphys) radiative_stage_body(op.a, op.phys, op.nphys, op.F, op.g, op.system, bid, nb);
      // the refinement-boundary ghosts of the next stage input, when the
      // phase table folded that fill in (its cells are ghosts of a buffer the
      // stage neither reads nor writes there)
      if (op.namr && op.nk >= 0)
        amr_apply_body(op.vec, op.fs, op.F, op.amr, op.namr, op.store, op.c[0], op.c[1], op.c[2], op.c[3], op.nk, bid,
                       nb);
      break;
    case kPhaseFill:
      if (op.namr && op.nk >= 0)
        amr_apply_body(op.vec, op.fs, op.F, op.amr, op.namr, op.store, op.c[0], op.c[1], op.c[2], op.c[3], op.nk, bid,
                       nb);
      if (op.nperiodic) periodic_copy_body(op.vec, op.fs, op.F, op.periodic, op.nperiodic, bid, nb);
      break;
    case kPhaseProlong:
      if (op.natiles)
        amr_prolong_tiles_body(op.pv[0], op.pv[1], op.pv[2], op.pv[3], op.pv[4], op.pfs, op.psy, op.psz, op.atiles,
                               op.natiles, op.aslots, op.namr, const_cast<double*>(op.store), op.F, w, op.nvec, bid, nb,
                               sm, 2);
      if (op.namr > op.namr_blocked)
        amr_prolong_cells_body(op.pv[0], op.pv[1], op.pv[2], op.pv[3], op.pv[4], op.pfs, op.psy, op.psz, op.amr,
                               op.namr_blocked, op.namr, const_cast<double*>(op.store), op.F, w, op.nvec, bid, nb);
      break;
    case kPhaseRestrict:
      if (op.nrblocks)
        restrict_blocks_body(op.parent, op.ppfs, op.ppsy, op.ppsz, op.fine, op.ffs, op.fsy, op.fsz, op.rblocks,
                             op.nrblocks, op.F, w, bid, nb, sm, 2);
      if (op.nrcells)
        restrict_cells_body(op.parent, op.ppfs, op.fine, op.ffs, op.fsy, op.fsz, op.rcells, op.nrcells, op.F, w, bid,
                            nb);
      break;
    case kPhaseCheck:
      if (op.ntiles) nonfinite_body(op.vec, op.fs, op.F, op.tiles, op.ntiles, op.a.sy, op.a.sz, op.status, bid, nb);
      break;
  }
}

// Three blocks per SM (at most 80 registers): more warps to hide the
// latency of the memory-bound phases than the two an unconstrained build
// allows.
__global__ void __launch_bounds__(kPThreads, 3) persistent_step_kernel(PBatch B) {
  extern __shared__ double sm[];
  // the phase record, staged in shared memory: one coalesced read per block
  // instead of one dependent global load per field
  __shared__ POp op;
  constexpr int kWords = (int)(sizeof(POp) / sizeof(int));
  static_assert(sizeof(POp) % sizeof(int) == 0, "POp is copied as ints");
  for (int i = 0; i < B.nops; ++i) {
    for (int r = 0; r < B.n; ++r) {
      if (i >= B.nops_r[r]) continue;
      const int* src = reinterpret_cast<const int*>(B.ops[r] + i);
      int* dst = reinterpret_cast<int*>(&op);
      for (int q = threadIdx.x; q < kWords; q += blockDim.x) dst[q] = src[q];
      __syncthreads();
      run_phase(op, B.w, sm, blockIdx.x, gridDim.x);
      __syncthreads();
    }
    if (i + 1 < B.nops && !grid_barrier(B.bar, gridDim.x)) {
      if (threadIdx.x == 0)
        for (int r = 0; r < B.n; ++r) atomicOr(B.status[r], kStatusTimeout);
      return;
    }
  }
}

int g_coop_blocks[64];  // co-resident blocks of the kernel per device (0 = not queried yet)

}  // namespace

cudaError_t persistent_max_blocks(int* nblocks) {
  int dev = 0, nsm = 0, occ = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (g_coop_blocks[dev & 63] == 0) {
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_step_kernel, kPThreads,
                                                           kPSmemDoubles * sizeof(double))) != cudaSuccess)
      return e;
    if (occ < 1) return cudaErrorNotSupported;
    g_coop_blocks[dev & 63] = nsm * occ;
  }
  *nblocks = g_coop_blocks[dev & 63];
  return cudaSuccess;
}

long phase_work_blocks(const POp& op) {
  auto cdiv = [](long a, long b) { return (a + b - 1) / b; };
  switch (op.kind) {
    case kPhaseStage:
      return op.ntiles + cdiv((long)op.nphys * op.F, kPThreads) +
             (op.nk >= 0 ? cdiv((long)op.namr * op.F, kPThreads) : 0);
    case kPhaseFill:
      return cdiv(((op.nk >= 0 ? (long)op.namr : 0) + op.nperiodic) * op.F, kPThreads);
    case kPhaseProlong:
      return (long)op.natiles * cdiv((long)op.nvec * op.F, 2) + cdiv((long)(op.namr - op.namr_blocked) * op.F, kPThreads);
    case kPhaseRestrict:
      return cdiv((long)op.nrblocks * op.F, 2) + cdiv((long)op.nrcells * op.F, kPThreads);
    case kPhaseCheck:
      return op.ntiles;
  }
  return 1;
}

cudaError_t launch_persistent_step(const PBatch& batch, int nblocks, cudaStream_t s) {
  if (batch.n < 1 || batch.nops < 1) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(&batch.bar->count, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  PBatch b = batch;
  void* args[] = {&b};
  return cudaLaunchCooperativeKernel((const void*)persistent_step_kernel, dim3(nblocks), dim3(kPThreads), args,
                                     kPSmemDoubles * sizeof(double), s);
}

}  // namespace sc
