// Instantiations and launchers of the C-GBR interface sweep for one arithmetic
// form and dimension, selected at compile time by CGK_SWEEP_UNIT (0: FP64
// without contraction, 1: FP64 with fused multiply-add, 2: FP32 mixed form;
// the build passes the matching -fmad flag) and CGK_SWEEP_ND (1, 2 or 3).
#include "cg_sweep.h"

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
#endif

}  // namespace

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
