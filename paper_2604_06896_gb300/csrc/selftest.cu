// vx_grid_barrier_selftest: the bounded wait of the GRID path's barrier,
// exercised without a fault.  One cooperative launch of m co-resident CTAs
// passes `rounds` barriers through grid_arrive_wait (the function GridTeam
// uses); the CTA of rank `absent` (if any) returns before the first one, so
// the others' waits run out after wait_ns, the team's abort word is raised
// and every waiting CTA reports VX_ERR_TIMEOUT.  Nothing hangs: every wait
// is bounded and the absent CTA has exited.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "team.cuh"
#include "vx_internal.h"

namespace vx {

__global__ void k_grid_bar_selftest(GridBar* bar, int m, int absent, int rounds,
                                    unsigned long long wait_ns, int* result) {
  __shared__ int fail;
  const int r = (int)blockIdx.x;
  if (r == absent) {
    if (threadIdx.x == 0) result[r] = -1;
    return;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < rounds; ++k) {
    if (threadIdx.x == 0 && !fail && !grid_arrive_wait(bar, (unsigned)m, wait_ns)) fail = 1;
    __syncthreads();
    if (fail) break;
  }
  if (threadIdx.x == 0) result[r] = fail ? (int)VX_ERR_TIMEOUT : (int)VX_OK;
}

}  // namespace vx

extern "C" vx_status vx_grid_barrier_selftest(int32_t ctas, int32_t absent_rank, int32_t rounds,
                                              double wait_s, int32_t* status, void* stream) {
  if (!status || ctas < 1 || rounds < 1 || absent_rank >= ctas || !(wait_s > 0) || wait_s > 10) {
    vx::set_error("vx_grid_barrier_selftest: invalid arguments");
    return VX_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vx::k_grid_bar_selftest, 64, 0) !=
          cudaSuccess ||
      ctas > per_sm * sms) {
    vx::set_error("vx_grid_barrier_selftest: the CTAs cannot all be resident");
    return VX_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  vx::GridBar* bar = nullptr;
  int* res = nullptr;
  cudaError_t e = cudaMalloc(&bar, sizeof(vx::GridBar));
  if (e == cudaSuccess) e = cudaMalloc(&res, sizeof(int) * ctas);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(vx::GridBar), s);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas, 1, 1);
    cfg.blockDim = dim3(64, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned long long ns = (unsigned long long)(wait_s * 1e9);
    e = cudaLaunchKernelEx(&cfg, vx::k_grid_bar_selftest, bar, (int)ctas, (int)absent_rank,
                           (int)rounds, ns, res);
  }
  std::vector<int> h(ctas, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), res, sizeof(int) * ctas, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (bar) cudaFree(bar);
  if (res) cudaFree(res);
  if (e != cudaSuccess) {
    vx::set_error(std::string("vx_grid_barrier_selftest: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  vx_status worst = VX_OK;
  for (int r = 0; r < ctas; ++r) {
    status[r] = h[r];
    if (h[r] == VX_ERR_TIMEOUT) worst = VX_ERR_TIMEOUT;
  }
  return worst;
}
