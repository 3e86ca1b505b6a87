// The vx_tissue handle: one tissue's device topology and workspace.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
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
  // image shifts of the exit-time wrap [V]
  int2* wrapk;
};

namespace vx {
// The internal tables of one tissue, built on the host from the caller's
// half-edge tables: the internal numbering (edge e owns half-edges 2e and
// 2e + 1, the caller's smaller index first) both ways, packed targets,
// next, face, the counter-clockwise out-lists [3][V] and each face's first
// half-edge.
struct HostTables {
  std::vector<int32_t> ext2int, int2ext;
  std::vector<uint32_t> tgt;
  std::vector<int32_t> nxt, face, vout, ff;
};
// Validates the caller's tables and builds the internal ones (host only, no
// device call); returns "" or the reason the tables are refused.
std::string build_host_tables(const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                              int n, int HE, HostTables* ht);

// The float64 workspace `work`, allocated once by vx_tissue_create, in three
// regions that calls use at the same time without overlap:
//   solver: CG vectors of the plain adjoint (x, r, p, h, 2x2 blocks), the
//           per-cell 4-vectors of the persistent adjoint and of the
//           Hessian-vector product, partial sums and control words;
//   ep:     the two nudged equilibria of equilibrium propagation, the cost
//           and the two phases' results;
//   aniso:  grad_X C of the anisotropy cost and its per-cell scratch.
// Each region is a multiple of 32 doubles (256 bytes), so that every region
// (and every [V][2] vector at an even offset inside it) is aligned for
// double2 / double4 access.
inline size_t work_r32(size_t x) { return (x + 31) & ~size_t(31); }
inline size_t work_solver_doubles(int n, int V) {
  return work_r32(12 * (size_t)V + 4 * (size_t)n + 3 * (size_t)((V + 255) / 256) + 128);
}
inline size_t work_ep_doubles(int V) { return work_r32(4 * (size_t)V + 64); }
inline size_t work_aniso_doubles(int n, int V) {
  return work_r32(2 * (size_t)V + 3 * (size_t)n + 3 * (size_t)((n + 255) / 256) + 64);
}
inline size_t work_total_doubles(int n, int V) {
  return work_solver_doubles(n, V) + work_ep_doubles(V) + work_aniso_doubles(n, V);
}
inline double* work_ep(vx_tissue_s* t) { return t->work + work_solver_doubles(t->n, t->V); }
inline double* work_aniso(vx_tissue_s* t) { return work_ep(t) + work_ep_doubles(t->V); }

vx_status energy_forces(vx_tissue_s* t, const double* X, const ParamsD& prm, double* F, double* E,
                        cudaStream_t s);
vx_status minimize(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp, int path,
                   int check_every, MinOut* out, int* path_used, cudaStream_t s);
// Exit-time wrap of X (device [V][2]) and of the tissue's offsets; an
// offset that would leave {-1, 0, 1} sets *status_dev to VX_ERR_TOPOLOGY
// (the slot is cleared first).  Rebuilds the flat tables.
vx_status wrap_tissue(vx_tissue_s* t, double* X, int* status_dev, cudaStream_t s);
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
// r_host: synchronous (result to the host); r_dev: asynchronous (the GPU
// writes the result), exactly one of them non-NULL.
vx_status equilibrium_grad_impl(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                                const double* dCdX, const vx_grad_opts* o, double* g_lambda,
                                double* g_A0, double* g_P0, vx_grad_result* r_host,
                                vx_grad_result* r_dev, cudaStream_t s);
vx_status minimize_launch(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                          int path, MinOut* out_dev, int* path_used, cudaStream_t s);
vx_status sensitivity(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const double* dCdX,
                      int count, const int32_t* kind, const int32_t* index, bool minres,
                      double rtol, int max_iter, int check_every, double* out, int32_t* status,
                      cudaStream_t s);
// Newton steps X += H^-1 F towards force balance from a near-equilibrium:
// F in FP64 arithmetic, H^-1 F by the plain-path CG on the tissue's
// Hessian-vector product.  Stops at max|F| < tol, after max_steps, at a
// step that does not lower max|F| (undone), or when CG meets negative
// curvature.  *steps: accepted steps; *fmax: max|F| at the returned X.
vx_status newton_refine(vx_tissue_s* t, double* X, const ParamsD& prm, double tol,
                        int max_steps, int* steps, double* fmax, cudaStream_t s);
size_t aniso_scratch_doubles(int n);
vx_status aniso_cost_view(const View<PolF64>& v, const double* q_target, double* gradX,
                          double* scratch, double* C, cudaStream_t s);
}  // namespace vx
