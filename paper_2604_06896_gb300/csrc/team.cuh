// Teams of threads that own one tissue inside a persistent kernel.
//
// BlockTeam:   one CTA; barriers are __syncthreads; reductions go through
//              per-warp slots in the CTA's shared memory.
// ClusterTeam: a thread-block cluster of NR CTAs; barriers are the hardware
//              cluster barrier (barrier.cluster.arrive.release /
//              wait.acquire, which orders global and shared memory for the
//              whole cluster); each CTA reduces into its own slots and every
//              thread then reads all ranks' slots through distributed
//              shared memory, in rank order, so all threads obtain identical
//              (deterministic) sums.
//
// Items (cells, vertices, edges) are dealt to threads round-robin:
// item = first() + k * stride().
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

namespace vx {
namespace cg = cooperative_groups;

template <int T>
struct BlockTeam {
  static constexpr int kThreads = T;
  static constexpr int kWarps = T / 32;
  __device__ __forceinline__ int rank() const { return 0; }
  __device__ __forceinline__ int nranks() const { return 1; }
  __device__ __forceinline__ int first() const { return threadIdx.x; }
  __device__ __forceinline__ int stride() const { return T; }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool sync_or(bool p, double*) const { return __syncthreads_or(p); }
  // Sum (and max in slot MAXK if want_max) of NV values over the team.
  // `slots` holds kWarps * NV doubles; the caller must separate two uses of
  // the same slots by a team barrier.
  template <int NV>
  __device__ __forceinline__ void reduce(double (&v)[NV], double* slots, int nmax) const {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = (k >= NV - nmax) ? fmax(x, y) : x + y;
      }
      if (lane == 0) slots[w * NV + k] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = (k >= NV - nmax) ? 0.0 : 0.0;
      for (int q = 0; q < kWarps; ++q) {
        const double y = slots[q * NV + k];
        s = (k >= NV - nmax) ? fmax(s, y) : s + y;
      }
      v[k] = s;
    }
  }
};

template <int T, int NR>
struct ClusterTeam {
  static constexpr int kThreads = T;
  static constexpr int kWarps = T / 32;
  __device__ __forceinline__ int rank() const { return (int)cg::this_cluster().block_rank(); }
  __device__ __forceinline__ int nranks() const { return NR; }
  __device__ __forceinline__ int first() const { return rank() * T + (int)threadIdx.x; }
  __device__ __forceinline__ int stride() const { return T * NR; }
  __device__ __forceinline__ bool leader() const { return rank() == 0 && threadIdx.x == 0; }
  __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
  // Team-wide OR; uses `slots` like reduce().
  __device__ __forceinline__ bool sync_or(bool p, double* slots) const {
    double v[1] = {p ? 1.0 : 0.0};
    reduce<1>(v, slots, 1);
    return v[0] > 0.0;
  }
  // `slots` holds (kWarps + 2) * NV doubles.
  template <int NV>
  __device__ __forceinline__ void reduce(double (&v)[NV], double* slots, int nmax) const {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = (k >= NV - nmax) ? fmax(x, y) : x + y;
      }
      if (lane == 0) slots[w * NV + k] = x;
    }
    __syncthreads();
    // CTA total into row kWarps.
    if (threadIdx.x < NV) {
      const int k = threadIdx.x;
      double s = 0.0;
      for (int q = 0; q < kWarps; ++q) {
        const double y = slots[q * NV + k];
        s = (k >= NV - nmax) ? fmax(s, y) : s + y;
      }
      slots[kWarps * NV + k] = s;
    }
    cg::this_cluster().sync();
    // Warp 0 gathers the NR totals through distributed shared memory (lane q
    // reads rank q) and reduces them with a fixed shuffle tree into row
    // kWarps + 1; the other warps read that row after the CTA barrier.
    if (w == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const bool mx = k >= NV - nmax;
        double x = (lane < NR) ? *cg::this_cluster().map_shared_rank(&slots[kWarps * NV + k], lane)
                               : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, x, o);
          x = mx ? fmax(x, y) : x + y;
        }
        if (lane == 0) slots[(kWarps + 1) * NV + k] = x;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = slots[(kWarps + 1) * NV + k];
  }
};

}  // namespace vx
