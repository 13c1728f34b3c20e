// Instantiations and launchers of the C-GBR interface sweep for one arithmetic
// form and dimension, selected at compile time by CGK_SWEEP_UNIT (0: FP64
// without contraction, 1: FP64 with fused multiply-add, 2: FP32 mixed form;
// the build passes the matching -fmad flag) and CGK_SWEEP_ND (1, 2 or 3).
#include "cg_sweep.h"
#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT != 1
#include "cg_batch_jobs.cuh"
#endif

#if !defined(CGK_SWEEP_ND) || !defined(CGK_SWEEP_UNIT)
#error "compile with -DCGK_SWEEP_ND=<1|2|3> -DCGK_SWEEP_UNIT=<0|1|2>"
#endif
#define CGK_SWEEP_FP32 (CGK_SWEEP_UNIT == 2)

namespace cgk {

namespace {

#if CGK_SWEEP_FP32
using ST = float;
#else
using ST = double;
#endif
constexpr int SND = CGK_SWEEP_ND;

// grid of tiles: along DIR, tiles of SWEEP_TL interfaces overlapping by one
// node; across, groups of LW lines
template <int DIR, int LW>
dim3 sweep_grid(const DevGrid& g) {
  return sweep_grid_dims(DIR, LW, g);
}

template <int DIR, bool CART, bool COMPACT, int LW>
int launch_one(const DevGrid& g, const GbrCfg& q, const StageArgs& A, cudaStream_t st) {
  size_t smem = sizeof(ST) * sweep_smem_doubles<SND, LW>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gbr_sweep<SND, DIR, CART, COMPACT, ST, LW, CGK_SWEEP_UNIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  k_gbr_sweep<SND, DIR, CART, COMPACT, ST, LW, CGK_SWEEP_UNIT><<<sweep_grid<DIR, LW>(g), 256, smem, st>>>(g, q, A);
  return (int)cudaGetLastError();
}

template <int DIR, int LW>
int launch_kind(bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A, cudaStream_t st) {
  if (cart) return compact ? launch_one<DIR, true, true, LW>(g, q, A, st) : launch_one<DIR, true, false, LW>(g, q, A, st);
  return compact ? launch_one<DIR, false, true, LW>(g, q, A, st) : launch_one<DIR, false, false, LW>(g, q, A, st);
}

template <int DIR>
int launch_dir(int lw, bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A,
               cudaStream_t st) {
  if (lw == 4) return launch_kind<DIR, 4>(cart, compact, g, q, A, st);
  if (lw == 8) return launch_kind<DIR, 8>(cart, compact, g, q, A, st);
  if (DIR > 0 && lw == 16) return launch_kind<DIR, 16>(cart, compact, g, q, A, st);
  return (int)cudaErrorInvalidValue;
}

#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT != 1
// Batched sweep: block b of the launch belongs to the grid m = mem[b]
// (off[m] <= b < off[m + 1]) and is that grid's tile (b - off[m]).
template <int DIR, int LW>
__global__ void __launch_bounds__(256, sweep_min_blocks<SND, true, ST>())
    k_gbr_sweep_batched(const SweepJob* __restrict__ jobs, const long long* __restrict__ off,
                        const int* __restrict__ mem) {
  const long long b = blockIdx.x;
  const int m = mem[b];
  const SweepJob& J = jobs[m];
  const long long r = b - off[m];
  const VBlock vb{(unsigned)(r % J.gx), (unsigned)((r / J.gx) % J.gy), (unsigned)(r / ((long long)J.gx * J.gy)),
                  J.gx, J.gy, J.gz};
  k_gbr_sweep_body<SND, DIR, true, false, ST, LW, CGK_SWEEP_UNIT>(vb, J.g, J.q, J.A);
}

template <int DIR, int LW>
int launch_batched_one(const SweepJob* jobs, const long long* off, const int* mem, long long total, cudaStream_t st) {
  size_t smem = sizeof(ST) * sweep_smem_doubles<SND, LW>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gbr_sweep_batched<DIR, LW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  if (total < 1 || total > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  k_gbr_sweep_batched<DIR, LW><<<(unsigned)total, 256, smem, st>>>(jobs, off, mem);
  return (int)cudaGetLastError();
}

int launch_batched(int dir, int lw, const SweepJob* jobs, const long long* off, const int* mem, long long total,
                   cudaStream_t st) {
  if (dir == 0 && lw == 4) return launch_batched_one<0, 4>(jobs, off, mem, total, st);
  if (dir == 0 && lw == 8) return launch_batched_one<0, 8>(jobs, off, mem, total, st);
  if (dir == 1 && lw == 4) return launch_batched_one<1, 4>(jobs, off, mem, total, st);
  if (dir == 1 && lw == 8) return launch_batched_one<1, 8>(jobs, off, mem, total, st);
  if (dir == 1 && lw == 16) return launch_batched_one<1, 16>(jobs, off, mem, total, st);
  return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- persistent stage
// Grid barrier with a bounded wait: thread 0 of every block arrives
// (atomic), the last one resets the count and advances the generation, the
// others wait for it with a spin of at most ~2^22 sleeps of 256 ns (about a
// second); a wait that runs out sets *err and returns false, and the kernel
// then returns (every block's wait runs out in turn).  The fences order each
// block's writes before its arrival and its later reads after the release.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned expect) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(bar, 1u) + 1u == expect) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      for (long long spin = 0; *gen == g0; ++spin) {
        if (spin > (1LL << 22)) {
          atomicExch(err, 1);
          good = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    ok = good && *(volatile int*)err == 0;
  }
  __syncthreads();
  return ok != 0;
}

// every virtual block of a phase, the block's threads together
template <class Job>
__device__ __forceinline__ void run_phase(const PhaseRef& K) {
  const Job* jobs = static_cast<const Job*>(K.jobs);
  for (long long b = blockIdx.x; b < K.total; b += gridDim.x) {
    const int m = K.mem[b];
    jobs[m].run((unsigned)(b - K.off[m]));
    __syncthreads();
  }
}

template <int DIR, int LW>
__device__ __forceinline__ void run_sweep_phase(const PhaseRef& K) {
  const SweepJob* jobs = static_cast<const SweepJob*>(K.jobs);
  for (long long b = blockIdx.x; b < K.total; b += gridDim.x) {
    const int m = K.mem[b];
    const SweepJob& J = jobs[m];
    const long long r = b - K.off[m];
    const VBlock vb{(unsigned)(r % J.gx), (unsigned)((r / J.gx) % J.gy), (unsigned)(r / ((long long)J.gx * J.gy)),
                    J.gx, J.gy, J.gz};
    k_gbr_sweep_body<SND, DIR, true, false, ST, LW, CGK_SWEEP_UNIT>(vb, J.g, J.q, J.A);
    __syncthreads();
  }
}

// One RK stage of the per-interface hybrid for every member of a work table:
// the phases of the table's launches, in their order, a grid barrier after
// each (independent phases share one).  No buffer a phase reads is written
// later in the same stage (the table gives the Gaussian's second pass and the
// second direction's node fluxes buffers of their own), so no SM can hold a
// stale line of it.
template <int LW0, int LW1>
__global__ void __launch_bounds__(256, sweep_min_blocks<SND, true, ST>()) k_stage_persistent(PersistentStage P) {
  using T = ST;
#define CGK_BARRIER() \
  if (!grid_barrier(P.bar, P.err, P.expect)) return
  run_phase<JobZero>(P.zero);
  if (P.with_cfl) {
    CGK_BARRIER();
    run_phase<JobCfl<T>>(P.cfl);
    CGK_BARRIER();
    run_phase<JobFinish>(P.fin);
  }
  run_phase<JobPrim<T>>(P.prim);
  CGK_BARRIER();
  run_phase<JobOmega<T>>(P.omega);
  run_phase<JobField<T>>(P.field);
  CGK_BARRIER();
  run_phase<JobTroubled<T>>(P.troubled);
  run_phase<JobGrad<T>>(P.grad);
  CGK_BARRIER();
  run_phase<JobCoef<T>>(P.coef);
  CGK_BARRIER();
  run_phase<JobGauss<T>>(P.gauss[0]);
  CGK_BARRIER();
  run_phase<JobGauss<T>>(P.gauss[1]);
  CGK_BARRIER();
  run_phase<JobNodeflux<T>>(P.nodeflux[0]);
  run_phase<JobNodeflux<T>>(P.nodeflux[1]);
  CGK_BARRIER();
  run_phase<JobHflux<T>>(P.hflux[0]);
  run_phase<JobHflux<T>>(P.hflux[1]);
  CGK_BARRIER();
  run_sweep_phase<0, LW0>(P.sweep[0]);
  CGK_BARRIER();
  run_sweep_phase<1, LW1>(P.sweep[1]);
#undef CGK_BARRIER
}

template <int LW0, int LW1>
constexpr size_t persistent_smem() {
  return sizeof(ST) * (sweep_smem_doubles<SND, LW0>() > sweep_smem_doubles<SND, LW1>() ? sweep_smem_doubles<SND, LW0>()
                                                                                         : sweep_smem_doubles<SND, LW1>());
}

template <int LW0, int LW1>
int persistent_blocks_one() {
  static int blocks = -1;
  if (blocks >= 0) return blocks;
  int dev = 0, nsm = 0, per = 0;
  const size_t smem = persistent_smem<LW0, LW1>();
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(k_stage_persistent<LW0, LW1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage_persistent<LW0, LW1>, 256, smem) != cudaSuccess)
    return 0;
  blocks = nsm * per;
  return blocks;
}

template <int LW0, int LW1>
int launch_persistent_one(const PersistentStage& P, int blocks, cudaStream_t st) {
  if (blocks < 1 || blocks > persistent_blocks_one<LW0, LW1>()) return (int)cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = persistent_smem<LW0, LW1>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_stage_persistent<LW0, LW1>, P);
}

int persistent_blocks(int lw0, int lw1) {
  if (lw0 == 4 && lw1 == 4) return persistent_blocks_one<4, 4>();
  if (lw0 == 4 && lw1 == 8) return persistent_blocks_one<4, 8>();
  if (lw0 == 8 && lw1 == 4) return persistent_blocks_one<8, 4>();
  if (lw0 == 8 && lw1 == 8) return persistent_blocks_one<8, 8>();
  return 0;
}

int launch_persistent(int lw0, int lw1, const PersistentStage& P, int blocks, cudaStream_t st) {
  if (lw0 == 4 && lw1 == 4) return launch_persistent_one<4, 4>(P, blocks, st);
  if (lw0 == 4 && lw1 == 8) return launch_persistent_one<4, 8>(P, blocks, st);
  if (lw0 == 8 && lw1 == 4) return launch_persistent_one<8, 4>(P, blocks, st);
  if (lw0 == 8 && lw1 == 8) return launch_persistent_one<8, 8>(P, blocks, st);
  return (int)cudaErrorInvalidValue;
}
#endif

}  // namespace

#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT == 0
int persistent_blocks_f64_2(int lw0, int lw1) { return persistent_blocks(lw0, lw1); }
int launch_persistent_f64_2(int lw0, int lw1, const PersistentStage& P, int blocks, cudaStream_t st) {
  return launch_persistent(lw0, lw1, P, blocks, st);
}
#endif
#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT == 2
int persistent_blocks_f32_2(int lw0, int lw1) { return persistent_blocks(lw0, lw1); }
int launch_persistent_f32_2(int lw0, int lw1, const PersistentStage& P, int blocks, cudaStream_t st) {
  return launch_persistent(lw0, lw1, P, blocks, st);
}
#endif

#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT == 0
int launch_sweep_batched_f64_2(int dir, int lw, const SweepJob* jobs, const long long* off, const int* mem,
                               long long total, cudaStream_t st) {
  return launch_batched(dir, lw, jobs, off, mem, total, st);
}
#endif
#if CGK_SWEEP_ND == 2 && CGK_SWEEP_UNIT == 2
int launch_sweep_batched_f32_2(int dir, int lw, const SweepJob* jobs, const long long* off, const int* mem,
                               long long total, cudaStream_t st) {
  return launch_batched(dir, lw, jobs, off, mem, total, st);
}
#endif

#define CGK_CAT3_(a, b, c) a##b##c
#define CGK_CAT3(a, b, c) CGK_CAT3_(a, b, c)
#if CGK_SWEEP_UNIT == 2
#define CGK_SWEEP_NAME CGK_CAT3(launch_sweep_f32_, CGK_SWEEP_ND, )
#elif CGK_SWEEP_UNIT == 1
#define CGK_SWEEP_NAME CGK_CAT3(launch_sweep_f64c_, CGK_SWEEP_ND, )
#else
#define CGK_SWEEP_NAME CGK_CAT3(launch_sweep_f64_, CGK_SWEEP_ND, )
#endif

int CGK_SWEEP_NAME(int dir, int lw, bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A,
                   cudaStream_t st) {
  if (dir == 0) return launch_dir<0>(lw, cart, compact, g, q, A, st);
#if CGK_SWEEP_ND >= 2
  if (dir == 1) return launch_dir<1>(lw, cart, compact, g, q, A, st);
#endif
#if CGK_SWEEP_ND >= 3
  if (dir == 2) return launch_dir<2>(lw, cart, compact, g, q, A, st);
#endif
  return (int)cudaErrorInvalidValue;
}

}  // namespace cgk
