// Launchers of the C-GBR interface sweep, one translation unit per
// (arithmetic form, dimension) so that the many instantiations (direction x
// grid kind x gradient kind x lines per tile) compile in parallel.  Forms:
// FP64 without FMA contraction (the oracle's operation order, bitwise
// reproducible), FP64 with contraction, FP32 (the mixed form, contracted).
#pragma once
#include "cg_kernels.cuh"

namespace cgk {

// Lines per tile an autotuner may choose for a sweep along dir.
constexpr int kSweepLwCands0[] = {4, 8};       // dir 0 (lines along x, contiguous)
constexpr int kSweepLwCands1[] = {4, 8, 16};   // dir 1, 2 (tile rows contiguous along x)

// Each returns a cudaError_t value (0 on success); cudaErrorInvalidValue for a
// combination that is not instantiated.
#define CGK_SWEEP_DECL(name)                                                                              \
  int name(int dir, int lw, bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A, \
           cudaStream_t st);
CGK_SWEEP_DECL(launch_sweep_f64_1)
CGK_SWEEP_DECL(launch_sweep_f64_2)
CGK_SWEEP_DECL(launch_sweep_f64_3)
CGK_SWEEP_DECL(launch_sweep_f64c_1)
CGK_SWEEP_DECL(launch_sweep_f64c_2)
CGK_SWEEP_DECL(launch_sweep_f64c_3)
CGK_SWEEP_DECL(launch_sweep_f32_1)
CGK_SWEEP_DECL(launch_sweep_f32_2)
CGK_SWEEP_DECL(launch_sweep_f32_3)
#undef CGK_SWEEP_DECL

constexpr int kSweepExact = 0, kSweepContracted = 1, kSweepFP32 = 2;

// Tile grid of a sweep along dir with lw lines per tile: along dir, tiles of
// SWEEP_TL interfaces overlapping by one node; across, groups of lw lines.
inline dim3 sweep_grid_dims(int dir, int lw, const DevGrid& g) {
  const int* n = g.n;
  if (dir == 0) {
    long long lines = (long long)n[1] * n[2];
    return dim3((n[0] + SWEEP_TL - 2) / (SWEEP_TL - 1), (unsigned)((lines + lw - 1) / lw), 1);
  }
  int other = dir == 1 ? n[2] : n[1];
  return dim3((n[0] + lw - 1) / lw, (n[dir] + SWEEP_TL - 2) / (SWEEP_TL - 1), other);
}

// ---------------------------------------------------------------- batched sweeps
// One grid of a batched sweep (2D, Cartesian): its arguments and its tile
// grid, which takes blocks [off_m, off_m + gx gy gz) of the one launch.
struct SweepJob {
  DevGrid g;
  GbrCfg q;
  StageArgs A;
  unsigned gx, gy, gz;
};

// Sweep along dir of every grid of a batch in one launch: jobs[nm], off[nm + 1]
// (off[nm] = total blocks) and mem[total] (the grid of every block) in device
// memory.  Returns a cudaError_t value; cudaErrorInvalidValue for a form or
// shape that is not instantiated (2D Cartesian, exact FP64 or FP32,
// non-compact gradients).
int launch_sweep_batched_f64_2(int dir, int lw, const SweepJob* jobs, const long long* off, const int* mem,
                               long long total, cudaStream_t st);
int launch_sweep_batched_f32_2(int dir, int lw, const SweepJob* jobs, const long long* off, const int* mem,
                               long long total, cudaStream_t st);

// ---------------------------------------------------------------- persistent stage
// One RK stage of a work table in a single cooperative launch: every phase
// (the jobs of one table launch) runs over its virtual blocks with a grid
// barrier after it.  A phase: its job array, block offsets, block -> member
// array and total blocks (device memory).
struct PhaseRef {
  const void* jobs = nullptr;
  const long long* off = nullptr;
  const int* mem = nullptr;
  long long total = 0;
};
struct PersistentStage {
  PhaseRef zero, cfl, fin, prim, omega, field, troubled, grad, coef, gauss[2], nodeflux[2], hflux[2], sweep[2];
  int with_cfl;        // first stage: the members' CFL time steps
  unsigned* bar;       // barrier: arrivals, generation (device, zero at rest)
  int* err;            // set to 1 when a barrier wait gave up (bounded wait)
  unsigned expect;     // arrivals a barrier waits for: the launch's blocks
};
// Blocks the persistent stage runs with (all co-resident: a cooperative
// launch); 0 if the shape is not instantiated.
int persistent_blocks_f64_2(int lw0, int lw1);
int persistent_blocks_f32_2(int lw0, int lw1);
// Enqueues one persistent stage with `blocks` blocks (cudaError_t value).
int launch_persistent_f64_2(int lw0, int lw1, const PersistentStage& P, int blocks, cudaStream_t st);
int launch_persistent_f32_2(int lw0, int lw1, const PersistentStage& P, int blocks, cudaStream_t st);

inline int launch_sweep_any(int form, int nd, int dir, int lw, bool cart, bool compact, const DevGrid& g,
                            const GbrCfg& q, const StageArgs& A, cudaStream_t st) {
  if (form == kSweepContracted) {
    if (nd == 1) return launch_sweep_f64c_1(dir, lw, cart, compact, g, q, A, st);
    if (nd == 2) return launch_sweep_f64c_2(dir, lw, cart, compact, g, q, A, st);
    return launch_sweep_f64c_3(dir, lw, cart, compact, g, q, A, st);
  }
  if (form == kSweepFP32) {
    if (nd == 1) return launch_sweep_f32_1(dir, lw, cart, compact, g, q, A, st);
    if (nd == 2) return launch_sweep_f32_2(dir, lw, cart, compact, g, q, A, st);
    return launch_sweep_f32_3(dir, lw, cart, compact, g, q, A, st);
  }
  if (nd == 1) return launch_sweep_f64_1(dir, lw, cart, compact, g, q, A, st);
  if (nd == 2) return launch_sweep_f64_2(dir, lw, cart, compact, g, q, A, st);
  return launch_sweep_f64_3(dir, lw, cart, compact, g, q, A, st);
}

}  // namespace cgk
