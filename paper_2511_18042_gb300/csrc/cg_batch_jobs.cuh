// Work-table launches of a batch of 2D Cartesian grids: one launch runs one
// phase of an RK stage for every grid of the batch.  Block b of the launch
// belongs to the grid m = mem[b] (off[m] <= b < off[m + 1], off[nm] = the
// total) and runs that grid's block (b - off[m]) of the phase's kernel body,
// with the grid's own arguments (a job).  The bodies are those of the
// per-grid kernels, so a batched phase computes what the per-grid launches
// compute.
#pragma once
#include "cg_lad.cuh"

namespace cgk {

constexpr int BATCH_THREADS = 256;

// grid-stride bodies: nb virtual blocks along x
__device__ __forceinline__ VBlock vblock_1d(unsigned b, unsigned nb) { return VBlock{b, 0u, 0u, nb, 1u, 1u}; }

template <class Job>
__global__ void __launch_bounds__(BATCH_THREADS) k_batched(const Job* __restrict__ jobs,
                                                          const long long* __restrict__ off,
                                                          const int* __restrict__ mem) {
  const long long b = blockIdx.x;
  const int m = mem[b];
  jobs[m].run((unsigned)(b - off[m]));
}

// two independent phases in one launch: blocks [0, t1) run J1, the rest J2
template <class J1, class J2>
__global__ void __launch_bounds__(BATCH_THREADS) k_batched2(const J1* __restrict__ j1, const long long* __restrict__ o1,
                                                           const int* __restrict__ m1, long long t1,
                                                           const J2* __restrict__ j2, const long long* __restrict__ o2,
                                                           const int* __restrict__ m2) {
  const long long b = blockIdx.x;
  if (b < t1) {
    const int m = m1[b];
    j1[m].run((unsigned)(b - o1[m]));
  } else {
    const long long r = b - t1;
    const int m = m2[r];
    j2[m].run((unsigned)(r - o2[m]));
  }
}

// per-grid scalars set at the start of a stage (one block per grid)
struct JobZero {
  unsigned long long* cflmax;  // null: keep
  int* hyb_flag;
  unsigned long long* hyb_count;
  __device__ void run(unsigned) const {
    if (threadIdx.x == 0) {
      if (cflmax) *cflmax = 0ull;
      *hyb_flag = 0;
      *hyb_count = 0ull;
    }
  }
};

template <typename T>
struct JobCfl {
  DevGrid g;
  const double* U;
  unsigned long long* mx;
  unsigned nb;
  __device__ void run(unsigned b) const { k_cfl_max_body<2, true, T>(vblock_1d(b, nb), g, U, mx); }
};

struct JobFinish {
  const unsigned long long* mx;
  double cfl;
  double* dt;
  __device__ void run(unsigned b) const {
    if (threadIdx.x == 0) {
      // the maximum read at L2 (an atomic): the same value, and no stale
      // line in a persistent launch that zeroed and raised it
      const unsigned long long v = atomicAdd(const_cast<unsigned long long*>(mx), 0ull);
      k_cfl_finish_body(vblock_1d(b, 1u), &v, cfl, dt, nullptr, 0.0);
    }
  }
};

template <typename T>
struct JobPrim {
  DevGrid g;
  const double* U;
  T* W;
  unsigned nb;
  __device__ void run(unsigned b) const { k_prim_body<2, T>(vblock_1d(b, nb), g, U, W); }
};

template <typename T>
struct JobOmega {
  DevGrid g;
  const T* W;
  const T* G[3];
  LineBuf gb[3];
  T* om;
  Box ob;
  unsigned nb;
  __device__ void run(unsigned b) const {
    k_omega_body<2, true, false, T>(vblock_1d(b, nb), g, W, G[0], G[1], G[2], gb[0], gb[1], gb[2], om, ob, nullptr,
                                    0);
  }
};

template <typename T>
struct JobField {
  DevGrid g;
  const T* W;
  T* f;
  Box fbx;
  unsigned nb;
  __device__ void run(unsigned b) const { k_lad_fieldbuf_body<2, T>(vblock_1d(b, nb), g, W, f, fbx); }
};

template <typename T>
struct JobTroubled {
  DevGrid g;
  const T* W;
  double hr, hp;
  const T* om;
  Box ob;
  double thr;
  unsigned char* tr;
  Box tb;
  int* flag;
  unsigned long long* count;
  unsigned nb;
  int buf;
  __device__ void run(unsigned b) const {
    k_troubled_body<2, T>(vblock_1d(b, nb), g, W, hr, hp, om, ob, thr, tr, tb, flag, count, buf);
  }
};

template <typename T>
struct JobGrad {
  DevGrid g;
  const T* fb;
  Box fbx;
  LineBuf lb[3];
  T* gr;
  T* dv;
  Box b3;
  unsigned nb;
  __device__ void run(unsigned b) const {
    k_lad_grad_body<2, true, false, T>(vblock_1d(b, nb), g, fb, fbx, nullptr, nullptr, nullptr, lb[0], lb[1], lb[2],
                                       gr, dv, b3, nullptr, 0);
  }
};

template <typename T>
struct JobCoef {
  DevGrid g;
  const T* W;
  const T* fb;
  Box fbx;
  const T* gr;
  const T* dv;
  Box b3;
  double cb, ck;
  T* bt;
  T* kp;
  unsigned nb;
  __device__ void run(unsigned b) const {
    k_lad_coef_body<2, true, T>(vblock_1d(b, nb), g, W, fb, fbx, gr, dv, b3, cb, ck, bt, kp, nullptr, 0);
  }
};

template <typename T>
struct JobGauss {
  DevGrid g;
  int l;
  const T* a;
  const T* b;
  T* ao;
  T* bo;
  unsigned nb;
  __device__ void run(unsigned blk) const { k_gauss_body<2, T>(vblock_1d(blk, nb), g, l, a, b, ao, bo, nullptr, 0); }
};

template <typename T>
struct JobNodeflux {
  DevGrid g;
  int l;
  const T* W;
  const T* bt;
  const T* kp;
  const T* gr;
  const T* dv;
  Box b3;
  T* Fn;
  Box fb;
  unsigned nb;
  __device__ void run(unsigned b) const {
    k_lad_nodeflux_body<2, true, NF_LAD, T>(vblock_1d(b, nb), g, l, W, bt, kp, gr, dv, b3, nullptr, Box{}, Fn, fb,
                                            nullptr, 0);
  }
};

template <typename T>
struct JobHflux {
  DevGrid g;
  int l;
  const T* Fn;
  Box fb;
  T* H;
  Box hb;
  unsigned nb;
  __device__ void run(unsigned b) const { k_lad_hflux_body<2, T>(vblock_1d(b, nb), g, l, Fn, fb, H, hb); }
};

}  // namespace cgk
