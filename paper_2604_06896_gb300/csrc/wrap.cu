// Exit-time wrap (Methods, "Periodic mode"): every vertex is put back into
// the primary box [0, Lx) x [0, Ly) and the offsets of the half-edges are
// changed so that each unwrapped edge vector keeps its value.  Solves keep
// positions unwrapped (offsets stay fixed inside a solve, which gives the
// same geometry); the wrap runs once when a solve returns.
//
// Per coordinate: k = floor(x / L), x' = x - k L; one period is added or
// taken away when rounding left x' outside [0, L); a result that rounds to
// L is taken as 0.  A half-edge s -> t then gets the offset off + k_t - k_s.
// The arithmetic is spelled out with explicitly rounded operations so that
// no contraction into fused multiply-adds changes a result.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

__global__ void k_wrap_pos(double* X, int V, double Lx, double Ly, int2* kv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    int kx, ky;
    const double x = wrap_coord(X[2 * i], Lx, kx);
    const double y = wrap_coord(X[2 * i + 1], Ly, ky);
    X[2 * i] = x;
    X[2 * i + 1] = y;
    kv[i] = make_int2(kx, ky);
  }
}

// Both half-edges of edge e (internal numbering: 2e and 2e + 1).  An offset
// that would leave {-1, 0, 1} (an edge longer than half the box) is left
// unchanged and reported as VX_ERR_TOPOLOGY in *status (when given).
__global__ void k_wrap_tgt(uint32_t* tgt, int E, const int2* kv, int* status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const uint32_t t0 = tgt[2 * e], t1 = tgt[2 * e + 1];
    const int a = tgt_v(t1), b = tgt_v(t0);  // 2e runs a -> b
    const int2 ka = kv[a], kb = kv[b];
    const int ox = tgt_ox(t0) + kb.x - ka.x, oy = tgt_oy(t0) + kb.y - ka.y;
    if (ox < -1 || ox > 1 || oy < -1 || oy > 1) {
      if (status) *status = VX_ERR_TOPOLOGY;
      continue;
    }
    tgt[2 * e] = pack_tgt(b, ox, oy);
    tgt[2 * e + 1] = pack_tgt(a, -ox, -oy);
  }
}

vx_status wrap_tissue(vx_tissue_s* t, double* X, int* status_dev, cudaStream_t s) {
  const int th = 256;
  if (status_dev && cudaMemsetAsync(status_dev, 0, sizeof(int), s) != cudaSuccess) {
    set_error("wrap: status reset failed");
    return VX_ERR_CUDA;
  }
  k_wrap_pos<<<(t->V + th - 1) / th, th, 0, s>>>(X, t->V, t->Lx, t->Ly, t->wrapk);
  k_wrap_tgt<<<(t->E + th - 1) / th, th, 0, s>>>(t->tgt, t->E, t->wrapk, status_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = rebuild_flat(t, s);
  if (e != cudaSuccess) {
    set_error(std::string("wrap: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

}  // namespace vx
