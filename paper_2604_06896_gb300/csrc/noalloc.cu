// vx_energy_forces_noalloc: energy and forces for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a stream capture
// whose memory pool is frozen, plugins handed a fixed memory budget by their
// host application, or real-time loops that must not touch the allocator.
// This entry point needs no vx_tissue handle (whose creation allocates): the
// caller passes the topology tables, positions and outputs in its own device
// memory, and the scratch the kernels need (per-cell coefficients, per-vertex
// out-half-edge slots, per-block energy partials) lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded and
// held by every GPU that loads it until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device_math.cuh"
#include "vx_internal.h"

namespace vx {

// Largest tissue the static scratch holds.
constexpr int kNoAllocMaxCells = 32768;
constexpr int kNoAllocMaxVertices = 2 * kNoAllocMaxCells;
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = (kNoAllocMaxVertices + kNoAllocThreads - 1) / kNoAllocThreads;

// Layout (doubles): cell coefficients [2 n] | block partials [kNoAllocMaxBlocks]
// | then int32: out-slot counters [V] | out half-edges [3 V].
constexpr size_t kScratchDoubles =
    2 * (size_t)kNoAllocMaxCells + kNoAllocMaxBlocks +
    ((size_t)kNoAllocMaxVertices * 4 * sizeof(int32_t) + sizeof(double) - 1) / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Status bits written by the kernels (see vx.h).
constexpr int kBadValence = 1;
constexpr int kBadIndex = 2;

// Per cell: cA = 2 K_A (A - A0), cP = 2 K_P (P - P0) and its energy; one
// partial energy per block (cell terms plus 1/2 Lambda l per half-edge).
// Every table index is checked before it is used: an index out of range
// sets kBadIndex and ends the cell's walk.
__global__ void k_na_cells(const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                           int n, double Lx, double Ly, const double* X, ParamsD prm,
                           double* scratch, int* bad) {
  __shared__ double red[kNoAllocThreads / 32];
  double* cc = scratch;
  double* part = scratch + 2 * (size_t)kNoAllocMaxCells;
  const int V = 2 * n, HE = 6 * n, E = 3 * n;
  double e = 0.0;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) {
    const int h0 = face_he[c];
    bool ok = h0 >= 0 && h0 < HE;
    const int v0 = ok ? he[8 * h0 + 3] : 0;
    ok = ok && v0 >= 0 && v0 < V;
    double qx = 0, qy = 0, A2 = 0, P = 0, el = 0;
    if (ok) {
      const double x0 = X[2 * v0], y0 = X[2 * v0 + 1];
      int ox = 0, oy = 0, h = h0, guard = 0;
      do {
        const int32_t* r = he + 8 * h;
        const int t = r[4], eid = edge_id[h], hn = r[1];
        if (t < 0 || t >= V || eid < 0 || eid >= E || hn < 0 || hn >= HE) {
          ok = false;
          break;
        }
        ox += r[6];
        oy += r[7];
        const double nx = (X[2 * t] + ox * Lx) - x0, ny = (X[2 * t + 1] + oy * Ly) - y0;
        A2 += qx * ny - nx * qy;
        const double l = sqrt((nx - qx) * (nx - qx) + (ny - qy) * (ny - qy));
        P += l;
        el += 0.5 * prm.la(eid) * l;
        qx = nx;
        qy = ny;
        h = hn;
      } while (h != h0 && ++guard < 4096);
    }
    if (!ok) atomicOr(bad, kBadIndex);
    const double dA = 0.5 * A2 - prm.a0(c), dP = P - prm.p0(c);
    cc[2 * c] = 2.0 * prm.ka(c) * dA;
    cc[2 * c + 1] = 2.0 * prm.kp(c) * dP;
    e = prm.ka(c) * dA * dA + prm.kp(c) * dP * dP + el;
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// Out-half-edge slots per vertex; the counters start at zero (cleared by the
// caller of this kernel on the same stream).  A source index out of range
// sets kBadIndex and is not counted.
__global__ void k_na_slots(const int32_t* he, int HE, int V, int32_t* cnt, int32_t* slots,
                           int* bad) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= HE) return;
  const int s = he[8 * h + 3];
  if (s < 0 || s >= V) {
    atomicOr(bad, kBadIndex);
    return;
  }
  const int k = atomicAdd(&cnt[s], 1);
  if (k < 3) slots[3 * s + k] = h;
}

// kBadValence when a vertex is not the source of exactly three half-edges
// (run on every call, whether or not forces are asked for).
__global__ void k_na_valence(const int32_t* cnt, int V, int* bad) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < V && cnt[s] != 3) atomicOr(bad, kBadValence);
}

__device__ __forceinline__ void edge_d(const int32_t* he, int h, const double* X, double Lx,
                                       double Ly, double& dx, double& dy) {
  const int32_t* r = he + 8 * h;
  dx = (X[2 * r[4]] + r[6] * Lx) - X[2 * r[3]];
  dy = (X[2 * r[4] + 1] + r[7] * Ly) - X[2 * r[3] + 1];
}

// F_s = sum over the out-half-edges h of s (taken in increasing index, so
// the sum is deterministic) of (Lambda_e + cP_f + cP_f') u_h
// - 1/2 cA_f rot(d_h + d_prev(h)), f = face(h), f' = face(twin(h)).
// A vertex that is not 3-valent, or whose tables hold an index out of
// range, gets no force (its status bit is set by k_na_valence, or here).
__global__ void k_na_vertices(const int32_t* he, const int32_t* edge_id, int n, double Lx,
                              double Ly, const double* X, ParamsD prm, const double* cc,
                              const int32_t* cnt, const int32_t* slots, double* F, int* bad) {
  const int V = 2 * n, HE = 6 * n, E = 3 * n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  if (cnt[s] != 3) return;
  int hs[3] = {slots[3 * s], slots[3 * s + 1], slots[3 * s + 2]};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (hs[j] > hs[j + 1]) {
        const int t = hs[j];
        hs[j] = hs[j + 1];
        hs[j + 1] = t;
      }
  auto in = [](int x, int m) { return x >= 0 && x < m; };
  double fx = 0, fy = 0;
  for (int k = 0; k < 3; ++k) {
    const int h = hs[k];
    const int32_t* r = he + 8 * h;
    const int hp = r[0], tw = r[2], eid = edge_id[h];
    bool ok = in(hp, HE) && in(tw, HE) && in(eid, E) && in(r[4], V) && in(r[5], n);
    if (ok) {
      const int32_t* rp = he + 8 * hp;
      ok = in(rp[3], V) && in(rp[4], V) && in(he[8 * tw + 5], n);
    }
    if (!ok) {
      atomicOr(bad, kBadIndex);
      return;
    }
    double dx, dy, px, py;
    edge_d(he, h, X, Lx, Ly, dx, dy);
    edge_d(he, hp, X, Lx, Ly, px, py);
    const double l = sqrt(dx * dx + dy * dy);
    const int f = r[5], f2 = he[8 * tw + 5];
    const double T = prm.la(eid) + cc[2 * f + 1] + cc[2 * f2 + 1];
    fx += T * dx / l;
    fy += T * dy / l;
    const double wx = dx + px, wy = dy + py;  // r_next - r_prev
    fx -= 0.5 * cc[2 * f] * wy;
    fy += 0.5 * cc[2 * f] * wx;
  }
  F[2 * s] = fx;
  F[2 * s + 1] = fy;
}

__global__ void k_na_energy(const double* part, int nb, double* E) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0;
  for (int b = 0; b < nb; ++b) s += part[b];
  *E = s;
}

}  // namespace

// Device address of the static scratch on the current device; looked up
// once per device (with that device current) and cached.
static double* noalloc_scratch(std::string* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = "no current CUDA device";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return (double*)g_addr[dev];
}

}  // namespace vx

extern "C" vx_status vx_energy_forces_noalloc(const int32_t* he, const int32_t* face_he,
                                              const int32_t* edge_id, int32_t n_cells, double Lx,
                                              double Ly, const double* X, const vx_params* p,
                                              double* F, double* E, int32_t* status,
                                              void* stream) {
  if (!he || !face_he || !edge_id || !X || !p || !status) {
    vx::set_error("vx_energy_forces_noalloc: NULL argument");
    return VX_ERR_INVALID_ARG;
  }
  if (n_cells < 1 || n_cells > vx::kNoAllocMaxCells) {
    vx::set_error("vx_energy_forces_noalloc: n_cells must be in [1, " +
                  std::to_string(vx::kNoAllocMaxCells) + "] (the size of the static scratch)");
    return VX_ERR_INVALID_ARG;
  }
  if (!(Lx > 0) || !(Ly > 0)) {
    vx::set_error("vx_energy_forces_noalloc: box sides must be positive");
    return VX_ERR_INVALID_ARG;
  }
  std::string err;
  double* scratch = vx::noalloc_scratch(&err);
  if (!scratch) {
    vx::set_error(err);
    return VX_ERR_CUDA;
  }
  vx::ParamsD prm;
  prm.KA = p->KA;
  prm.KP = p->KP;
  prm.A0 = p->A0;
  prm.P0 = p->P0;
  prm.lam = p->lambda;
  prm.KA_s = p->KA_s;
  prm.KP_s = p->KP_s;
  prm.A0_s = p->A0_s;
  prm.P0_s = p->P0_s;
  prm.lam_s = p->lambda_s;
  const int n = n_cells, V = 2 * n, HE = 6 * n, T = vx::kNoAllocThreads;
  cudaStream_t s = (cudaStream_t)stream;
  double* cc = scratch;
  double* part = scratch + 2 * (size_t)vx::kNoAllocMaxCells;
  int32_t* cnt = (int32_t*)(part + vx::kNoAllocMaxBlocks);
  int32_t* slots = cnt + vx::kNoAllocMaxVertices;
  const int nbc = (n + T - 1) / T;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * V, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    vx::k_na_slots<<<(HE + T - 1) / T, T, 0, s>>>(he, HE, V, cnt, slots, status);
    vx::k_na_valence<<<(V + T - 1) / T, T, 0, s>>>(cnt, V, status);
    vx::k_na_cells<<<nbc, T, 0, s>>>(he, face_he, edge_id, n, Lx, Ly, X, prm, scratch, status);
    if (F)
      vx::k_na_vertices<<<(V + T - 1) / T, T, 0, s>>>(he, edge_id, n, Lx, Ly, X, prm, cc, cnt,
                                                       slots, F, status);
    if (E) vx::k_na_energy<<<1, 32, 0, s>>>(part, nbc, E);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    vx::set_error(std::string("vx_energy_forces_noalloc: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}
