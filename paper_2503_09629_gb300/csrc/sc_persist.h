// sc_persist.h -- phase table of the persistent coarse-step kernel (scalar
// wave).  Not part of the public ABI.
#pragma once

#include "sc_internal.h"

namespace sc {

enum { kPhaseStage = 0, kPhaseFill = 1, kPhaseProlong = 2, kPhaseRestrict = 3, kPhaseCheck = 4 };

// One phase of a coarse step: everything it does is independent within the
// phase; phases are separated by grid barriers.  Only the fields of the
// phase's kind are used.
struct POp {
  int kind;
  int F;
  // kPhaseStage: fused stage over the interior tiles (and the radiative
  // shell cells of a radiative level 0)
  StageArgs a;
  const Tile* tiles;
  int ntiles;
  int order;
  const int32_t* phys;
  int nphys;
  int system;
  Geom g;
  // kPhaseFill: refinement-boundary ghosts (nk >= 0: dense-output apply with
  // coefficients c; nk < 0: none) and periodic images; kPhaseCheck: vec
  double* vec;
  long fs;
  const AmrCell* amr;
  int namr;
  int namr_blocked;
  const double* store;
  double c[4];
  int nk;
  const int2* periodic;
  int nperiodic;
  // kPhaseProlong: parent vectors (y_n, then the stage vectors) into the store
  const double* pv[5];
  long pfs;
  int psy, psz;
  const AmrTile* atiles;
  int natiles;
  const int32_t* aslots;
  int nvec;
  // kPhaseRestrict
  double* parent;
  long ppfs;
  int ppsy, ppsz;
  const double* fine;
  long ffs;
  int fsy, fsz;
  const RestrictBlock* rblocks;
  int nrblocks;
  const RestrictCell* rcells;
  int nrcells;
  // kPhaseCheck: status word to flag
  int* status;
};

// Arrival count and generation of the grid barrier, on separate 128-byte
// lines so that the waiting blocks' polls of the generation do not queue
// behind the arrivals' atomics on the same line.
struct GridBarrier {
  unsigned count;
  unsigned pad0[31];
  unsigned gen;
  unsigned pad1[31];
};

constexpr int kMaxBatch = 128;

// Kernel parameter block: the phase tables (one per context), each
// context's phase count and status word, the barrier and the transfer
// weights (the same for every context).  Phase i of every context runs
// between the same two barriers: a context's phases depend only on its own
// earlier phases, so contexts of any shapes can share a launch.
struct PBatch {
  int n;
  int nops;  // the largest of nops_r: context r runs its phases 0..nops_r[r]-1
  GridBarrier* bar;
  Weights w;
  const POp* ops[kMaxBatch];
  int* status[kMaxBatch];
  int nops_r[kMaxBatch];
};

// Co-resident blocks of the persistent kernel on the current device (its
// cooperative-launch limit); cudaErrorNotSupported without cooperative launch.
cudaError_t persistent_max_blocks(int* nblocks);
// Thread blocks a phase can keep busy (the grid of a launch is the largest
// over its phases, capped by persistent_max_blocks).
long phase_work_blocks(const POp& op);
// One coarse step of every context of the batch: resets the barrier count,
// then one cooperative launch of nblocks blocks on stream s.
cudaError_t launch_persistent_step(const PBatch& batch, int nblocks, cudaStream_t s);

// What the server needs to merge persistent-form contexts into one launch:
// the device phase table of the current level-0 parity, its host copy and
// the context's status word (sc_host.cu).  SC_EINVAL for other forms.
struct PersistView {
  const POp* ops;
  const std::vector<POp>* host;
  int* status;
  Weights w;
};
sc_status persistent_view(sc_ctx* c, PersistView* v);
// The host-side bookkeeping of one coarse step launched outside sc_advance
// (level-0 parity, time, zone-update counts).
void persistent_step_done(sc_ctx* c);

}  // namespace sc
