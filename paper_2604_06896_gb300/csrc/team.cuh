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
// GridTeam:    m co-resident CTAs of a cooperative launch (any subset of
//              the GPU's SMs); barriers are a counter / generation pair in
//              global memory (atom.add.acq_rel + ld.acquire at GPU scope);
//              each CTA writes its partial sums to a global table and every
//              CTA then reads all m partials in rank order, so all threads
//              obtain identical sums.  Every wait is bounded: a CTA that
//              waits longer than kGridWaitNs raises the team's abort word,
//              all CTAs of the team then stop waiting and failed() is true.
//
// Items (cells, vertices, edges) are dealt to threads round-robin:
// item = first() + k * stride().
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

namespace vx {
namespace cg = cooperative_groups;

// Warp totals of NV FP32 values (sum, or max for the last nmax), fixed
// shuffle tree, converted to FP64.
template <int NV>
__device__ __forceinline__ void warp_tree_f(const float (&v)[NV], double (&out)[NV], int nmax) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k >= NV - nmax) ? fmaxf(x, y) : x + y;
    }
    out[k] = (double)x;
  }
}

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
  __device__ __forceinline__ bool failed() const { return false; }
  // Sum (and max in slot MAXK if want_max) of NV values over the team.
  // `slots` holds kWarps * NV doubles; the caller must separate two uses of
  // the same slots by a team barrier.
  // FP32 values: the warp stage in FP32 (FP64 issues slowly on this GPU),
  // the team stage in FP64 as in reduce().
  template <int NV>
  __device__ __forceinline__ void reduce_f(const float (&v)[NV], double (&out)[NV], double* slots,
                                           int nmax) const {
    warp_tree_f<NV>(v, out, nmax);
    reduce<NV, true>(out, slots, nmax);
  }
  // kTreeDone: v already holds warp totals (in every lane).
  template <int NV, bool kTreeDone = false>
  __device__ __forceinline__ void reduce(double (&v)[NV], double* slots, int nmax) const {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = v[k];
      if (!kTreeDone)
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
  __device__ __forceinline__ bool failed() const { return false; }
  // Team-wide OR; uses `slots` like reduce().
  __device__ __forceinline__ bool sync_or(bool p, double* slots) const {
    const float f[1] = {p ? 1.0f : 0.0f};
    double v[1];
    reduce_f<1>(f, v, slots, 1);
    return v[0] > 0.0;
  }
  // `slots` holds (kWarps + 2) * NV doubles.
  // FP32 values: the warp stage in FP32 (FP64 issues slowly on this GPU),
  // the team stage in FP64 as in reduce().
  template <int NV>
  __device__ __forceinline__ void reduce_f(const float (&v)[NV], double (&out)[NV], double* slots,
                                           int nmax) const {
    warp_tree_f<NV>(v, out, nmax);
    reduce<NV, true>(out, slots, nmax);
  }
  // kTreeDone: v already holds warp totals (in every lane).
  template <int NV, bool kTreeDone = false>
  __device__ __forceinline__ void reduce(double (&v)[NV], double* slots, int nmax) const {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = v[k];
      if (!kTreeDone)
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

// Barrier words of one grid team (zeroed before the launch).
struct GridBar {
  unsigned count;  // arrivals at the current barrier
  unsigned gen;    // completed barriers
  unsigned abort;  // set by a CTA whose wait timed out
  unsigned pad;
};

constexpr unsigned long long kGridWaitNs = 4000000000ull;  // 4 s

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// acq_rel: the last arriver must see what the others released before it
// publishes the new generation.
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned x) {
  unsigned v;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "r"(x) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned x) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned* p, unsigned x) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Called by one thread per CTA; false when the team aborted (this CTA or
// another waited longer than wait_ns).
__device__ __forceinline__ bool grid_arrive_wait(GridBar* b, unsigned m,
                                                 unsigned long long wait_ns = kGridWaitNs) {
  const unsigned g = ld_relaxed_gpu(&b->gen);
  if (atom_add_acq_rel_gpu(&b->count, 1u) == m - 1) {
    st_relaxed_gpu(&b->count, 0u);
    st_release_gpu(&b->gen, g + 1u);
    return true;
  }
  const unsigned long long t0 = global_ns();
  for (unsigned k = 0;; ++k) {
    if (ld_acquire_gpu(&b->gen) != g) return true;
    if (ld_relaxed_gpu(&b->abort)) return false;
    if ((k & 63u) == 63u && global_ns() - t0 > wait_ns) {
      st_relaxed_gpu(&b->abort, 1u);
      return false;
    }
  }
}

// State of a grid team, in the CTA's shared memory (so that the team costs
// no registers in the solver loops).
struct GridState {
  GridBar* bar;
  double* part;  // [2][total][4] partial sums, double-buffered
  int base;      // first CTA of the team
  int m;         // CTAs in the team
  int total;     // CTAs in the launch (row length of `part`)
  int phase;     // reductions so far
  int fail;      // this CTA saw the team abort
};

template <int T>
struct GridTeam {
  static constexpr int kThreads = T;
  static constexpr int kWarps = T / 32;
  GridState* s;
  __device__ __forceinline__ int rank() const { return (int)blockIdx.x - s->base; }
  __device__ __forceinline__ int nranks() const { return s->m; }
  __device__ __forceinline__ int first() const { return rank() * T + (int)threadIdx.x; }
  __device__ __forceinline__ int stride() const { return T * s->m; }
  __device__ __forceinline__ bool leader() const { return rank() == 0 && threadIdx.x == 0; }
  __device__ __forceinline__ bool failed() const { return *(volatile int*)&s->fail != 0; }
  __device__ __forceinline__ void sync() const {
    __syncthreads();
    if (threadIdx.x == 0 && !s->fail && !grid_arrive_wait(s->bar, (unsigned)s->m)) s->fail = 1;
    __syncthreads();
  }
  __device__ __forceinline__ bool sync_or(bool p, double* slots) const {
    const float f[1] = {p ? 1.0f : 0.0f};
    double v[1];
    reduce_f<1>(f, v, slots, 1);
    return v[0] > 0.0;
  }
  // `slots` holds (kWarps + 2) * NV doubles, NV <= 4.  Two consecutive
  // reduces use the two halves of `part`; a third may reuse the first half
  // because every CTA has passed the second one's barrier, after its reads
  // of the first.
  // FP32 values: the warp stage in FP32 (FP64 issues slowly on this GPU),
  // the team stage in FP64 as in reduce().
  template <int NV>
  __device__ __forceinline__ void reduce_f(const float (&v)[NV], double (&out)[NV], double* slots,
                                           int nmax) const {
    warp_tree_f<NV>(v, out, nmax);
    reduce<NV, true>(out, slots, nmax);
  }
  // kTreeDone: v already holds warp totals (in every lane).
  template <int NV, bool kTreeDone = false>
  __device__ __forceinline__ void reduce(double (&v)[NV], double* slots, int nmax) const {
    static_assert(NV <= 4, "at most 4 values per reduction");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = v[k];
      if (!kTreeDone)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, x, o);
          x = (k >= NV - nmax) ? fmax(x, y) : x + y;
        }
      if (lane == 0) slots[w * NV + k] = x;
    }
    __syncthreads();
    double* row = s->part + (size_t)(s->phase & 1) * s->total * 4;
    if (threadIdx.x < NV) {
      const int k = threadIdx.x;
      double a = 0.0;
      for (int q = 0; q < kWarps; ++q) {
        const double y = slots[q * NV + k];
        a = (k >= NV - nmax) ? fmax(a, y) : a + y;
      }
      __stcg(&row[(size_t)blockIdx.x * 4 + k], a);
    }
    sync();
    // Warp 0: lane q combines ranks q, q + 32, ... in order, then a fixed
    // shuffle tree; the result goes to row kWarps + 1 for the other warps.
    if (w == 0) {
      const int base = s->base, m = s->m;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const bool mx = k >= NV - nmax;
        double x = 0.0;
        for (int q = lane; q < m; q += 32) {
          const double y = __ldcg(&row[(size_t)(base + q) * 4 + k]);
          x = mx ? fmax(x, y) : x + y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double y = __shfl_xor_sync(0xffffffffu, x, o);
          x = mx ? fmax(x, y) : x + y;
        }
        if (lane == 0) slots[(kWarps + 1) * NV + k] = x;
      }
      if (lane == 0) ++s->phase;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = slots[(kWarps + 1) * NV + k];
  }
};

}  // namespace vx
