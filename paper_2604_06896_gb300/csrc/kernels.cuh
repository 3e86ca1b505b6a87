// Kernel entry points and their host-side launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_math.cuh"
#include "../../include/vx.h"

namespace vx {

// Inner-minimiser parameters as the kernels see them.
struct MinParams {
  int method;  // 0 FIRE, 1 GD
  double tol;
  int patience, max_iter;
  double gd_lr, dt0, dt_max;
  int n_min;
  double f_inc, f_dec, alpha0, f_alpha;
  double l_min;
  // Nudged phase of equilibrium propagation: force += -s Pi grad_X C.
  int cost;              // 0 none, 1 v2v, 2 anisotropy
  double nudge_s;
  const double* cost_data;  // X_target [V][2] (v2v) or q_target [2] (anisotropy)
  // anisotropy nudging: per-cell centroids double2 [n] followed by corner
  // counts int [n], and the per-vertex nudge double2 [V] (global memory,
  // any residency)
  double* aniso_ws;
  double* aniso_nudge;
  // Exit-time wrap of positions and offsets (applied by the host launcher
  // after the solve).
  int wrap;
  // Optional per-edge decision counters [E][2] (stretches, T1s).
  int* edge_events;
};

// Control block of the global-memory minimiser (one per tissue).
struct FireCtrl {
  double dt, alpha;
  int npos, below, it, done, status;
  double P, FF, VV, fmax2;
  double mixA, mixB, dt_step;
  int zero_v;
  unsigned int counter;
  int any_short;
  int n_t1, n_stretch;
};

// Result block written by the minimisers (device side).
struct MinOut {
  int status, iters, n_t1, n_stretch, n_short, n_inverted, force_evals;
  int wrap_err;  // set by the exit-time wrap when an offset would leave {-1, 0, 1}
  double fmax, energy;
};

template <class P>
struct Workspace {
  using R = typename P::R;
  using R2 = typename std::conditional<std::is_same<R, double>::value, double2, float2>::type;
};

}  // namespace vx
