// The vx_tissue handle: one tissue's device topology and workspace.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "device_math.cuh"
#include "kernels.cuh"
#include "../../include/vx.h"

struct vx_tissue_s {
  int device;
  int n, V, E, HE;
  double Lx, Ly;
  int dtype;
  // topology (internal half-edge numbering: edge e owns 2e and 2e + 1)
  uint32_t* tgt;
  int32_t *nxt, *face, *vout, *ffirst;
  // host maps between the caller's half-edge indices and the internal ones
  std::vector<int32_t> ext2int, int2ext;
  // workspace
  void* Xw;      // positions, internal representation [V]
  void* vel;     // FIRE velocities [V][2] (compute precision)
  void* F;       // forces [V][2] (compute precision)
  void* cellc;   // per-cell (cA, cP) [n][2]
  uint32_t* shortbits;
  uint32_t* touched;
  double* partE;  // per-block energy partials
  double* partF;  // per-block FIRE partials
  vx::FireCtrl* ctrl;
  vx::MinOut* dout;
  // flat tables (see View): per vertex [3][V], per cell [n][16]
  uint32_t* vnb;
  int32_t *vfc, *ccnt;
  uint32_t* ccor;
  int32_t* cedge;
  // topology at creation (for vx_tissue_restore)
  uint32_t* tgt0;
  int32_t *nxt0, *face0, *vout0, *ffirst0;
  // adjoint workspace (float64 vectors [V][2] and per-cell sums)
  double* work;
  size_t work_doubles;
};

namespace vx {
vx_status energy_forces(vx_tissue_s* t, const double* X, const ParamsD& prm, double* F, double* E,
                        cudaStream_t s);
vx_status minimize(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp, int path,
                   int check_every, MinOut* out, int* path_used, cudaStream_t s);
size_t resident_smem_bytes(vx_tissue_s* t);
vx_status minimize_many(vx_tissue_s* const* ts, int count, double* const* Xs, const ParamsD* prms,
                        const MinParams& mp, int path, MinOut* outs, int* paths, cudaStream_t s);
// Recompute the flat tables from the half-edge tables (after a resident
// solve rewrote the latter).
cudaError_t rebuild_flat(vx_tissue_s* t, cudaStream_t s);
vx_status hessian_vector(vx_tissue_s* t, const double* X, const ParamsD& prm, const double* vec,
                         double* Hv, cudaStream_t s);
vx_status equilibrium_grad(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                           const double* dCdX, const vx_grad_opts* o, double* g_lambda, double* g_A0,
                           double* g_P0, vx_grad_result* r, cudaStream_t s);
size_t aniso_scratch_doubles(int n);
vx_status aniso_cost_view(const View<PolF64>& v, const double* q_target, double* gradX,
                          double* scratch, double* C, cudaStream_t s);
}  // namespace vx
