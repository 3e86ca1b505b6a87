// Launchers of the persistent per-tissue kernels: one CTA with the tissue in
// shared memory ("resident"), or a 16-CTA thread-block cluster with the
// tissue in L2-resident global memory ("cluster"), for the minimiser and the
// adjoint; plus the path choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "persistent.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

template <class P>
vx_status minimize_plain_t(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                           int check_every, MinOut* out_h, cudaStream_t s);

// dynamic shared memory of a resident tissue: 227 KiB per CTA less room for
// the kernels' static shared memory (the T1 pass keeps its candidates there)
constexpr int kSmemMax = 224 * 1024;
constexpr int kClusterT = 256;  // 255 registers per thread: no spills
constexpr int kClusterNR = 16;
// Cells one T1 pass may change before the team falls back to a full cell
// pass (four per candidate).
constexpr int kDirtyCap = 1024;

__host__ __device__ inline size_t a16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared memory of a resident tissue: positions, topology, per-cell
// coefficients (nc4 = 2 for the minimiser, 4 for the adjoint), tensions,
// the CG direction (adjoint), bit masks and reduction slots.
template <class P>
size_t res_bytes(int n, int V, int E, int HE, int T, bool adjoint) {
  using R = typename P::R;
  size_t b = a16(sizeof(typename P::Pos) * V) + 3 * a16(4 * (size_t)HE) + a16(12 * (size_t)V) +
             a16(4 * (size_t)n) + a16((adjoint ? 4 : 2) * sizeof(R) * n) + a16(sizeof(R) * E) +
             a16(4 * (size_t)((E + 31) / 32)) + a16(4 * (size_t)((V + 31) / 32)) +
             3 * a16(8 * 4 * (size_t)(T / 32 + 1));
  if (adjoint) b += a16(2 * sizeof(R) * V);
  return b;
}

struct PersistArgs {
  const double* Xin;
  double* Xout;
  int n, V, E, HE;
  double Lx, Ly;
  uint32_t* tgt;
  int32_t *nxt, *face, *vout, *ffirst;
  ParamsD prm;
  MinParams mp;
  AdjParams ap;
  MinOut* out;
  AdjOut* aout;
  // global workspace (cluster variant)
  void* Xw;
  void* cell;
  void* pvec;
  uint32_t* shortbits;
  uint32_t* touched;
  uint32_t* vnb;
  int32_t *vfc, *ccnt;
  uint32_t* ccor;
  int32_t* cedge;
  // grid variant: CTAs grid_base .. grid_base + grid_m - 1 own the tissue
  int grid_base, grid_m;
};

template <class P>
__device__ __forceinline__ View<P> global_view(const PersistArgs& g) {
  View<P> v;
  v.X = (typename P::Pos*)g.Xw;
  v.tgt = g.tgt;
  v.nxt = g.nxt;
  v.face = g.face;
  v.vout = g.vout;
  v.ffirst = g.ffirst;
  v.n = g.n;
  v.V = g.V;
  v.E = g.E;
  v.box = P::make_box(g.Lx, g.Ly);
  v.Lx = g.Lx;
  v.Ly = g.Ly;
  v.vnb = g.vnb;
  v.vfc = g.vfc;
  v.ccnt = g.ccnt;
  v.ccor = g.ccor;
  v.cedge = g.cedge;
  return v;
}

// Copies the tissue into shared memory; returns the view and carves the
// remaining buffers.
template <class P, int T>
__device__ __forceinline__ View<P> load_resident(const PersistArgs& g, unsigned char* smem,
                                                 bool adjoint, void** cell, void** lamR,
                                                 void** pvec, uint32_t** sh, uint32_t** tc,
                                                 Slots* sl) {
  using R = typename P::R;
  using Pos = typename P::Pos;
  const int n = g.n, V = g.V, E = g.E, HE = g.HE, tid = threadIdx.x;
  unsigned char* p = smem;
  Pos* sX = (Pos*)p;             p += a16(sizeof(Pos) * V);
  uint32_t* sTgt = (uint32_t*)p; p += a16(4 * (size_t)HE);
  int32_t* sNxt = (int32_t*)p;   p += a16(4 * (size_t)HE);
  int32_t* sFace = (int32_t*)p;  p += a16(4 * (size_t)HE);
  int32_t* sVout = (int32_t*)p;  p += a16(12 * (size_t)V);
  int32_t* sFf = (int32_t*)p;    p += a16(4 * (size_t)n);
  *cell = p;                     p += a16((adjoint ? 4 : 2) * sizeof(R) * n);
  R* sLam = (R*)p;               p += a16(sizeof(R) * E);
  *sh = (uint32_t*)p;            p += a16(4 * (size_t)((E + 31) / 32));
  *tc = (uint32_t*)p;            p += a16(4 * (size_t)((V + 31) / 32));
  const size_t sb = a16(8 * 4 * (size_t)(T / 32 + 1));
  sl->a = (double*)p;            p += sb;
  sl->b = (double*)p;            p += sb;
  sl->c = (double*)p;            p += sb;
  if (adjoint) *pvec = p;
  for (int h = tid; h < HE; h += T) {
    sTgt[h] = g.tgt[h];
    sNxt[h] = g.nxt[h];
    sFace[h] = g.face[h];
  }
  for (int k = tid; k < 3 * V; k += T) sVout[k] = g.vout[k];
  for (int c = tid; c < n; c += T) sFf[c] = g.ffirst[c];
  for (int e = tid; e < E; e += T) sLam[e] = (R)g.prm.la(e);
  for (int w = tid; w < (E + 31) / 32; w += T) (*sh)[w] = 0;
  for (int w = tid; w < (V + 31) / 32; w += T) (*tc)[w] = 0;
  *lamR = sLam;
  View<P> v;
  v.X = sX;
  v.tgt = sTgt;
  v.nxt = sNxt;
  v.face = sFace;
  v.vout = sVout;
  v.ffirst = sFf;
  v.n = n;
  v.V = V;
  v.E = E;
  v.box = P::make_box(g.Lx, g.Ly);
  v.Lx = g.Lx;
  v.Ly = g.Ly;
  v.vnb = nullptr;
  v.vfc = nullptr;
  v.ccnt = nullptr;
  v.ccor = nullptr;
  v.cedge = nullptr;
  return v;
}

template <class P, int T>
__device__ __forceinline__ void store_topology(const PersistArgs& g, const View<P>& v) {
  const int tid = threadIdx.x;
  for (int h = tid; h < g.HE; h += T) {
    g.tgt[h] = v.tgt[h];
    g.nxt[h] = v.nxt[h];
    g.face[h] = v.face[h];
  }
  for (int k = tid; k < 3 * g.V; k += T) g.vout[k] = v.vout[k];
  for (int c = tid; c < g.n; c += T) g.ffirst[c] = v.ffirst[c];
}

template <class P, int T, int MAXC>
__global__ void __launch_bounds__(T) k_min_res(PersistArgs g) {
  using R2 = typename Vec2Of<typename P::R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  void *cell, *lam, *pvec;
  uint32_t *sh, *tc;
  Slots sl;
  View<P> v = load_resident<P, T>(g, smem, false, &cell, &lam, &pvec, &sh, &tc, &sl);
  __syncthreads();
  BlockTeam<T> tm;
  min_body<P, BlockTeam<T>, MAXC>(tm, v, (R2*)cell, (const typename P::R*)lam, sh, tc, sl, g.prm,
                                  g.mp, g.Xin, g.Xout, g.out);
  __syncthreads();
  store_topology<P, T>(g, v);
}

template <class P, int T, int MAXC>
__global__ void __launch_bounds__(T) k_adj_res(PersistArgs g) {
  using R2 = typename Vec2Of<typename P::R>::T;
  using R4 = typename Vec2Of<typename P::R>::T4;
  extern __shared__ __align__(16) unsigned char smem[];
  void *cell, *lam, *pvec;
  uint32_t *sh, *tc;
  Slots sl;
  View<P> v = load_resident<P, T>(g, smem, true, &cell, &lam, &pvec, &sh, &tc, &sl);
  __syncthreads();
  BlockTeam<T> tm;
  adj_body<P, BlockTeam<T>, MAXC>(tm, v, (R4*)cell, (const typename P::R*)lam, (R2*)pvec, sl,
                                  g.prm, g.ap, g.Xin, g.aout);
}

template <class P, int T, int NR, int MAXC>
__global__ void __launch_bounds__(T) k_min_cluster(PersistArgs g) {
  using R2 = typename Vec2Of<typename P::R>::T;
  __shared__ double slots[3][4 * (T / 32 + 2)];
  __shared__ int dirty[kDirtyCap];
  ClusterTeam<T, NR> tm;
  for (int w = tm.first(); w < (g.E + 31) / 32; w += tm.stride()) g.shortbits[w] = 0;
  for (int w = tm.first(); w < (g.V + 31) / 32; w += tm.stride()) g.touched[w] = 0;
  Slots sl = {slots[0], slots[1], slots[2]};
  sl.dirty = dirty;
  sl.dirty_cap = kDirtyCap;
  min_body<P, ClusterTeam<T, NR>, MAXC>(tm, global_view<P>(g), (R2*)g.cell, g.prm.lam, g.shortbits,
                                        g.touched, sl, g.prm, g.mp, g.Xin, g.Xout, g.out);
  tm.sync();
}

// Several tissues in one launch: cluster k (blocks k*NR .. k*NR+NR-1) solves
// tissue k with the same body as k_min_cluster.
template <class P, int T, int NR, int MAXC>
__global__ void __launch_bounds__(T) k_min_cluster_many(const PersistArgs* args) {
  using R2 = typename Vec2Of<typename P::R>::T;
  __shared__ double slots[3][4 * (T / 32 + 2)];
  __shared__ int dirty[kDirtyCap];
  const PersistArgs& g = args[blockIdx.x / NR];
  ClusterTeam<T, NR> tm;
  for (int w = tm.first(); w < (g.E + 31) / 32; w += tm.stride()) g.shortbits[w] = 0;
  for (int w = tm.first(); w < (g.V + 31) / 32; w += tm.stride()) g.touched[w] = 0;
  Slots sl = {slots[0], slots[1], slots[2]};
  sl.dirty = dirty;
  sl.dirty_cap = kDirtyCap;
  min_body<P, ClusterTeam<T, NR>, MAXC>(tm, global_view<P>(g), (R2*)g.cell, g.prm.lam, g.shortbits,
                                        g.touched, sl, g.prm, g.mp, g.Xin, g.Xout, g.out);
  tm.sync();
}

// Several resident tissues in one launch: CTA k solves tissue k.
template <class P, int T, int MAXC>
__global__ void __launch_bounds__(T) k_min_res_many(const PersistArgs* args) {
  using R2 = typename Vec2Of<typename P::R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const PersistArgs& g = args[blockIdx.x];
  void *cell, *lam, *pvec;
  uint32_t *sh, *tc;
  Slots sl;
  View<P> v = load_resident<P, T>(g, smem, false, &cell, &lam, &pvec, &sh, &tc, &sl);
  __syncthreads();
  BlockTeam<T> tm;
  min_body<P, BlockTeam<T>, MAXC>(tm, v, (R2*)cell, (const typename P::R*)lam, sh, tc, sl, g.prm,
                                  g.mp, g.Xin, g.Xout, g.out);
  __syncthreads();
  store_topology<P, T>(g, v);
}

// Several tissues in one cooperative launch: tissue k owns the CTAs
// args[k].grid_base .. + grid_m - 1 (bases ascending), which synchronise
// through bars[k]; part is the [2][gridDim.x][4] table of partial sums.
template <class P, int T, int MAXC>
__global__ void __launch_bounds__(T) k_min_grid(const PersistArgs* args, int count, GridBar* bars,
                                                double* part) {
  using R2 = typename Vec2Of<typename P::R>::T;
  __shared__ double slots[3][4 * (T / 32 + 2)];
  __shared__ int dirty[kDirtyCap];
  __shared__ GridState gs;
  int k = 0;
  while (k + 1 < count && args[k + 1].grid_base <= (int)blockIdx.x) ++k;
  const PersistArgs& g = args[k];
  if (threadIdx.x == 0) gs = GridState{bars + k, part, g.grid_base, g.grid_m, (int)gridDim.x, 0, 0};
  __syncthreads();
  GridTeam<T> tm{&gs};
  for (int w = tm.first(); w < (g.E + 31) / 32; w += tm.stride()) g.shortbits[w] = 0;
  for (int w = tm.first(); w < (g.V + 31) / 32; w += tm.stride()) g.touched[w] = 0;
  Slots sl = {slots[0], slots[1], slots[2]};
  sl.dirty = dirty;
  sl.dirty_cap = kDirtyCap;
  min_body<P, GridTeam<T>, MAXC>(tm, global_view<P>(g), (R2*)g.cell, g.prm.lam, g.shortbits,
                                 g.touched, sl, g.prm, g.mp, g.Xin, g.Xout, g.out);
  tm.sync();
}

template <class P, int T, int NR, int MAXC>
__global__ void __launch_bounds__(T) k_adj_cluster(PersistArgs g) {
  using R2 = typename Vec2Of<typename P::R>::T;
  using R4 = typename Vec2Of<typename P::R>::T4;
  __shared__ double slots[3][4 * (T / 32 + 2)];
  ClusterTeam<T, NR> tm;
  Slots sl = {slots[0], slots[1], slots[2]};
  adj_body<P, ClusterTeam<T, NR>, MAXC>(tm, global_view<P>(g), (R4*)g.cell, g.prm.lam,
                                        (R2*)g.pvec, sl, g.prm, g.ap, g.Xin, g.aout);
  tm.sync();
}

// ------------------------------------------------------------------ host

static PersistArgs make_args(vx_tissue_s* t, const double* Xin, double* Xout, const ParamsD& prm) {
  PersistArgs a = {};
  a.Xin = Xin;
  a.Xout = Xout;
  a.n = t->n;
  a.V = t->V;
  a.E = t->E;
  a.HE = t->HE;
  a.Lx = t->Lx;
  a.Ly = t->Ly;
  a.tgt = t->tgt;
  a.nxt = t->nxt;
  a.face = t->face;
  a.vout = t->vout;
  a.ffirst = t->ffirst;
  a.prm = prm;
  a.out = t->dout;
  a.aout = (AdjOut*)t->dout;
  a.Xw = t->Xw;
  a.cell = t->cellc;
  a.pvec = t->vel;
  a.shortbits = t->shortbits;
  a.touched = t->touched;
  a.vnb = t->vnb;
  a.vfc = t->vfc;
  a.ccnt = t->ccnt;
  a.ccor = t->ccor;
  a.cedge = t->cedge;
  return a;
}

// Kernels whose attributes were set (and, for clusters, whose occupancy was
// checked) on a device: done once, so that a later call recorded in a CUDA
// graph enqueues launches only.
static std::mutex g_cfg_mu;
static std::vector<std::pair<const void*, int>> g_cfg_done;
static bool configured(const void* k) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  for (const auto& x : g_cfg_done)
    if (x.first == k && x.second == dev) return true;
  return false;
}
static void mark_configured(const void* k) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg_done.emplace_back(k, dev);
}

template <class K>
static cudaError_t launch_res(K kernel, int T, size_t smem, const PersistArgs& a, cudaStream_t s) {
  if (!configured((const void*)kernel)) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e != cudaSuccess) return e;
    mark_configured((const void*)kernel);
  }
  kernel<<<1, T, smem, s>>>(a);
  return cudaGetLastError();
}

// One 256-thread CTA (the largest size whose 255-register budget holds the
// loop without spilling); each thread owns up to MAXC cells and 2 MAXC
// vertices.
constexpr int kResT = 256;

template <class P, bool ADJ>
static cudaError_t dispatch_res(vx_tissue_s* t, const PersistArgs& a, cudaStream_t s) {
  const int n = t->n;
  const size_t smem = res_bytes<P>(t->n, t->V, t->E, t->HE, kResT, ADJ);
  const int mc = (n + kResT - 1) / kResT;
  if (ADJ) {
    if (mc <= 1) return launch_res(k_adj_res<P, kResT, 1>, kResT, smem, a, s);
    if (mc <= 2) return launch_res(k_adj_res<P, kResT, 2>, kResT, smem, a, s);
    if (mc <= 3) return launch_res(k_adj_res<P, kResT, 3>, kResT, smem, a, s);
    if (mc <= 4) return launch_res(k_adj_res<P, kResT, 4>, kResT, smem, a, s);
    return launch_res(k_adj_res<P, kResT, 6>, kResT, smem, a, s);
  }
  if (mc <= 1) return launch_res(k_min_res<P, kResT, 1>, kResT, smem, a, s);
  if (mc <= 2) return launch_res(k_min_res<P, kResT, 2>, kResT, smem, a, s);
  if (mc <= 3) return launch_res(k_min_res<P, kResT, 3>, kResT, smem, a, s);
  if (mc <= 4) return launch_res(k_min_res<P, kResT, 4>, kResT, smem, a, s);
  return launch_res(k_min_res<P, kResT, 6>, kResT, smem, a, s);
}

template <class K>
static cudaError_t launch_cluster(K kernel, const PersistArgs& a, cudaStream_t s) {
  const bool ready = configured((const void*)kernel);
  cudaError_t e = cudaSuccess;
  if (!ready) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterNR, 1, 1);
  cfg.blockDim = dim3(kClusterT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterNR;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!ready) {
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    mark_configured((const void*)kernel);
  }
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <class P, bool ADJ>
static cudaError_t dispatch_cluster(vx_tissue_s* t, const PersistArgs& a, cudaStream_t s) {
  const int per = kClusterT * kClusterNR;
  const int mc = (t->n + per - 1) / per;
  if (ADJ) {
    if (mc <= 1) return launch_cluster(k_adj_cluster<P, kClusterT, kClusterNR, 1>, a, s);
    if (mc <= 2) return launch_cluster(k_adj_cluster<P, kClusterT, kClusterNR, 2>, a, s);
    if (mc <= 3) return launch_cluster(k_adj_cluster<P, kClusterT, kClusterNR, 3>, a, s);
    return launch_cluster(k_adj_cluster<P, kClusterT, kClusterNR, 4>, a, s);
  }
  if (mc <= 1) return launch_cluster(k_min_cluster<P, kClusterT, kClusterNR, 1>, a, s);
  if (mc <= 2) return launch_cluster(k_min_cluster<P, kClusterT, kClusterNR, 2>, a, s);
  if (mc <= 3) return launch_cluster(k_min_cluster<P, kClusterT, kClusterNR, 3>, a, s);
  return launch_cluster(k_min_cluster<P, kClusterT, kClusterNR, 4>, a, s);
}

bool resident_fits(vx_tissue_s* t, bool adjoint) {
  const size_t b = t->dtype == VX_F64 ? res_bytes<PolF64>(t->n, t->V, t->E, t->HE, kResT, adjoint)
                                      : res_bytes<PolF32>(t->n, t->V, t->E, t->HE, kResT, adjoint);
  return b <= (size_t)kSmemMax && t->n <= 6 * kResT;
}

bool cluster_fits(vx_tissue_s* t) { return t->n <= 4 * kClusterT * kClusterNR; }

size_t resident_smem_bytes(vx_tissue_s* t) {
  return t->dtype == VX_F64 ? res_bytes<PolF64>(t->n, t->V, t->E, t->HE, kResT, false)
                            : res_bytes<PolF32>(t->n, t->V, t->E, t->HE, kResT, false);
}

bool grid_fits(vx_tissue_s* t);

// A single tissue larger than this runs faster on a cluster (16 SMs) than
// in one SM's shared memory, although it may fit there (measured: 1,000
// FP32 cells take 38.6 us per FIRE iteration resident, 15.7 on a cluster).
constexpr int kResidentAutoMaxCells = 512;

static int choose_path(vx_tissue_s* t, int path, bool adjoint) {
  if (path == VX_PATH_AUTO) {
    if (t->n <= kResidentAutoMaxCells && resident_fits(t, adjoint)) return VX_PATH_RESIDENT;
    if (cluster_fits(t)) return VX_PATH_CLUSTER;
    return adjoint ? -1 : VX_PATH_PLAIN;
  }
  if (path == VX_PATH_RESIDENT && !resident_fits(t, adjoint)) return -1;
  if (path == VX_PATH_CLUSTER && !cluster_fits(t)) return -1;
  if (path == VX_PATH_GRID && adjoint) return cluster_fits(t) ? VX_PATH_CLUSTER : -1;
  if (path == VX_PATH_GRID && !grid_fits(t)) return -1;
  if (path == VX_PATH_PLAIN && adjoint) return cluster_fits(t) ? VX_PATH_CLUSTER : -1;
  return path;
}

vx_status minimize_launch(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                          int path, MinOut* out_dev, int* path_used, cudaStream_t s) {
  const int p = choose_path(t, path, false);
  if (p != VX_PATH_RESIDENT && p != VX_PATH_CLUSTER) {
    set_error("without a host synchronisation only the resident and cluster paths can run "
              "this tissue");
    return VX_ERR_INVALID_ARG;
  }
  *path_used = p;
  const bool f64 = t->dtype == VX_F64;
  PersistArgs a = make_args(t, X, X, prm);
  a.mp = mp;
  a.out = out_dev;
  cudaError_t e;
  if (p == VX_PATH_RESIDENT) {
    e = f64 ? dispatch_res<PolF64, false>(t, a, s) : dispatch_res<PolF32, false>(t, a, s);
    if (e == cudaSuccess && mp.l_min > 0 && !mp.wrap) e = rebuild_flat(t, s);
  } else {
    e = f64 ? dispatch_cluster<PolF64, false>(t, a, s) : dispatch_cluster<PolF32, false>(t, a, s);
  }
  if (e != cudaSuccess) {
    set_error(std::string("persistent minimiser launch: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  if (mp.wrap && wrap_tissue(t, X, &out_dev->wrap_err, s) != VX_OK) return VX_ERR_CUDA;
  return VX_OK;
}

vx_status minimize(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp, int path,
                   int check_every, MinOut* out, int* path_used, cudaStream_t s) {
  const int p = choose_path(t, path, false);
  if (p < 0) {
    set_error("the requested path cannot hold this tissue");
    return VX_ERR_INVALID_ARG;
  }
  *path_used = p;
  if (p == VX_PATH_GRID) {
    vx_tissue_s* ts[1] = {t};
    double* Xs[1] = {X};
    int used = 0;
    return minimize_many(ts, 1, Xs, &prm, mp, VX_PATH_GRID, out, &used, s);
  }
  const bool f64 = t->dtype == VX_F64;
  if (p == VX_PATH_PLAIN)
    return f64 ? minimize_plain_t<PolF64>(t, X, prm, mp, check_every, out, s)
               : minimize_plain_t<PolF32>(t, X, prm, mp, check_every, out, s);
  PersistArgs a = make_args(t, X, X, prm);
  a.mp = mp;
  cudaError_t e;
  if (p == VX_PATH_RESIDENT) {
    e = f64 ? dispatch_res<PolF64, false>(t, a, s) : dispatch_res<PolF32, false>(t, a, s);
    if (e == cudaSuccess && mp.l_min > 0 && !mp.wrap) e = rebuild_flat(t, s);
  } else {
    e = f64 ? dispatch_cluster<PolF64, false>(t, a, s) : dispatch_cluster<PolF32, false>(t, a, s);
  }
  if (e != cudaSuccess) {
    set_error(std::string("persistent minimiser launch: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  if (mp.wrap && wrap_tissue(t, X, &t->dout->wrap_err, s) != VX_OK) return VX_ERR_CUDA;
  if (cudaMemcpyAsync(out, t->dout, sizeof(MinOut), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("vx_minimize: ") + cudaGetErrorString(cudaGetLastError()));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

// ------------------------------------------------------- many tissues

namespace {
std::mutex g_many_mu;
std::mutex g_many_call_mu;
void* g_many_buf[64] = {};
size_t g_many_bytes[64] = {};

// A device buffer for the argument and result arrays of vx_minimize_many,
// grown on demand and kept per device.
void* many_buffer(size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_many_mu);
  if (g_many_bytes[dev] < bytes) {
    if (g_many_buf[dev]) cudaFree(g_many_buf[dev]);
    g_many_buf[dev] = nullptr;
    g_many_bytes[dev] = 0;
    if (cudaMalloc(&g_many_buf[dev], bytes) != cudaSuccess) return nullptr;
    g_many_bytes[dev] = bytes;
  }
  return g_many_buf[dev];
}

template <class P>
cudaError_t launch_res_many(const std::vector<vx_tissue_s*>& ts, const PersistArgs* d_args,
                            cudaStream_t s) {
  int nmax = 0;
  size_t smem = 0;
  for (vx_tissue_s* t : ts) {
    nmax = std::max(nmax, t->n);
    smem = std::max(smem, res_bytes<P>(t->n, t->V, t->E, t->HE, kResT, false));
  }
  const int mc = (nmax + kResT - 1) / kResT;
  auto go = [&](auto kernel) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e != cudaSuccess) return e;
    kernel<<<(int)ts.size(), kResT, smem, s>>>(d_args);
    return cudaGetLastError();
  };
  if (mc <= 1) return go(k_min_res_many<P, kResT, 1>);
  if (mc <= 2) return go(k_min_res_many<P, kResT, 2>);
  if (mc <= 3) return go(k_min_res_many<P, kResT, 3>);
  if (mc <= 4) return go(k_min_res_many<P, kResT, 4>);
  return go(k_min_res_many<P, kResT, 6>);
}

template <class P>
cudaError_t launch_cluster_many(const std::vector<vx_tissue_s*>& ts, const PersistArgs* d_args,
                                cudaStream_t s) {
  int nmax = 0;
  for (vx_tissue_s* t : ts) nmax = std::max(nmax, t->n);
  const int mc = (nmax + kClusterT * kClusterNR - 1) / (kClusterT * kClusterNR);
  auto go = [&](auto kernel) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterNR * (unsigned)ts.size(), 1, 1);
    cfg.blockDim = dim3(kClusterT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterNR;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, d_args);
  };
  if (mc <= 1) return go(k_min_cluster_many<P, kClusterT, kClusterNR, 1>);
  if (mc <= 2) return go(k_min_cluster_many<P, kClusterT, kClusterNR, 2>);
  if (mc <= 3) return go(k_min_cluster_many<P, kClusterT, kClusterNR, 3>);
  return go(k_min_cluster_many<P, kClusterT, kClusterNR, 4>);
}

constexpr int kGridT = 256;
constexpr int kGridMaxC = 4;

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// CTAs per tissue on the grid path: one per kGridT cells when the SMs
// suffice, else shares proportional to those demands (at least one each),
// at most one CTA per SM in total.  Returns the cells-per-thread bound, or
// 0 if the tissues do not fit.
int grid_plan(const std::vector<vx_tissue_s*>& ts, int sms, std::vector<int>* m) {
  long long demand = 0;
  m->assign(ts.size(), 1);
  for (size_t k = 0; k < ts.size(); ++k) {
    (*m)[k] = (ts[k]->n + kGridT - 1) / kGridT;
    demand += (*m)[k];
  }
  if ((long long)ts.size() > sms) return 0;
  if (demand > sms) {
    long long used = 0;
    for (size_t k = 0; k < ts.size(); ++k) {
      (*m)[k] = std::max(1, (int)((*m)[k] * (long long)sms / demand));
      used += (*m)[k];
    }
    if (used > sms) return 0;
  }
  int mc = 1;
  for (size_t k = 0; k < ts.size(); ++k)
    mc = std::max(mc, (ts[k]->n + (*m)[k] * kGridT - 1) / ((*m)[k] * kGridT));
  return mc <= kGridMaxC ? mc : 0;
}

template <class P>
cudaError_t launch_grid_many(int mc, int total, int count, const PersistArgs* d_args, GridBar* bars,
                             double* part, cudaStream_t s) {
  auto go = [&](auto kernel) -> cudaError_t {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGridT, 0);
    if (e != cudaSuccess) return e;
    if (per_sm * sm_count() < total) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total, 1, 1);
    cfg.blockDim = dim3(kGridT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, d_args, count, bars, part);
  };
  if (mc <= 1) return go(k_min_grid<P, kGridT, 1>);
  if (mc <= 2) return go(k_min_grid<P, kGridT, 2>);
  if (mc <= 3) return go(k_min_grid<P, kGridT, 3>);
  return go(k_min_grid<P, kGridT, 4>);
}
}  // namespace

bool grid_fits(vx_tissue_s* t) {
  std::vector<int> m;
  return grid_plan({t}, sm_count(), &m) > 0;
}

vx_status minimize_many(vx_tissue_s* const* ts, int count, double* const* Xs, const ParamsD* prms,
                        const MinParams& mp, int path, MinOut* outs, int* paths, cudaStream_t s) {
  const int dtype = ts[0]->dtype;
  if (path == VX_PATH_PLAIN) {
    set_error("vx_minimize_many: the plain path takes one tissue at a time (vx_minimize)");
    return VX_ERR_INVALID_ARG;
  }
  std::vector<vx_tissue_s*> res, clu, grd;
  std::vector<PersistArgs> ares, aclu, agrd;
  std::vector<int> ires, iclu, igrd;
  for (int k = 0; k < count; ++k) {
    vx_tissue_s* t = ts[k];
    if (t->dtype != dtype) {
      set_error("vx_minimize_many: all tissues must have the same dtype");
      return VX_ERR_INVALID_ARG;
    }
    PersistArgs a = make_args(t, Xs[k], Xs[k], prms[k]);
    a.mp = mp;
    if (path == VX_PATH_GRID) {
      grd.push_back(t);
      agrd.push_back(a);
      igrd.push_back(k);
      paths[k] = VX_PATH_GRID;
    } else if (path != VX_PATH_CLUSTER && resident_fits(t, false)) {
      res.push_back(t);
      ares.push_back(a);
      ires.push_back(k);
      paths[k] = VX_PATH_RESIDENT;
    } else if (path != VX_PATH_RESIDENT && cluster_fits(t)) {
      clu.push_back(t);
      aclu.push_back(a);
      iclu.push_back(k);
      paths[k] = VX_PATH_CLUSTER;
    } else {
      set_error("vx_minimize_many: tissue " + std::to_string(k) + " does not fit the requested path");
      return VX_ERR_INVALID_ARG;
    }
  }
  std::vector<int> gm;
  int gmc = 0, total = 0;
  if (!grd.empty()) {
    gmc = grid_plan(grd, sm_count(), &gm);
    if (gmc == 0) {
      set_error("vx_minimize_many: the tissues do not fit the grid path (at most one CTA per SM, "
                "4 x 256 cells per CTA)");
      return VX_ERR_INVALID_ARG;
    }
    for (size_t q = 0; q < agrd.size(); ++q) {
      agrd[q].grid_base = total;
      agrd[q].grid_m = gm[q];
      total += gm[q];
    }
  }
  // One buffer per device holds the argument, result, barrier and partial
  // sum arrays; calls are serialised so that they never share it.
  std::lock_guard<std::mutex> call_lock(g_many_call_mu);
  const size_t nargs = (size_t)count;
  const size_t o_out = a16(nargs * sizeof(PersistArgs));
  const size_t o_bar = o_out + a16(nargs * sizeof(MinOut));
  const size_t o_part = o_bar + a16(grd.size() * sizeof(GridBar));
  const size_t bytes = o_part + (size_t)2 * total * 4 * sizeof(double) + 256;
  unsigned char* buf = (unsigned char*)many_buffer(bytes);
  if (!buf) {
    set_error("vx_minimize_many: out of device memory for the argument arrays");
    return VX_ERR_OOM;
  }
  PersistArgs* d_args = (PersistArgs*)buf;
  MinOut* d_out = (MinOut*)(buf + o_out);
  GridBar* d_bar = (GridBar*)(buf + o_bar);
  double* d_part = (double*)(buf + o_part);
  // results of tissue k go to d_out[k]
  for (size_t q = 0; q < ares.size(); ++q) ares[q].out = d_out + ires[q];
  for (size_t q = 0; q < aclu.size(); ++q) aclu[q].out = d_out + iclu[q];
  for (size_t q = 0; q < agrd.size(); ++q) agrd[q].out = d_out + igrd[q];
  std::vector<PersistArgs> all(ares);
  all.insert(all.end(), aclu.begin(), aclu.end());
  all.insert(all.end(), agrd.begin(), agrd.end());
  cudaError_t e = cudaMemcpyAsync(d_args, all.data(), all.size() * sizeof(PersistArgs),
                                  cudaMemcpyHostToDevice, s);
  const bool f64 = dtype == VX_F64;
  if (e == cudaSuccess && !grd.empty()) {
    e = cudaMemsetAsync(d_bar, 0, grd.size() * sizeof(GridBar), s);
    const PersistArgs* da = d_args + ares.size() + aclu.size();
    if (e == cudaSuccess)
      e = f64 ? launch_grid_many<PolF64>(gmc, total, (int)grd.size(), da, d_bar, d_part, s)
              : launch_grid_many<PolF32>(gmc, total, (int)grd.size(), da, d_bar, d_part, s);
  }
  if (e == cudaSuccess && !clu.empty())
    e = f64 ? launch_cluster_many<PolF64>(clu, d_args + ares.size(), s)
            : launch_cluster_many<PolF32>(clu, d_args + ares.size(), s);
  if (e == cudaSuccess && !res.empty())
    e = f64 ? launch_res_many<PolF64>(res, d_args, s) : launch_res_many<PolF32>(res, d_args, s);
  if (e == cudaSuccess && mp.l_min > 0 && !mp.wrap)
    for (vx_tissue_s* t : res)
      if (e == cudaSuccess) e = rebuild_flat(t, s);
  if (e == cudaSuccess && mp.wrap)
    for (int k = 0; k < count; ++k)
      if (wrap_tissue(ts[k], Xs[k], &d_out[k].wrap_err, s) != VX_OK) return VX_ERR_CUDA;
  if (e == cudaSuccess) e = cudaMemcpyAsync(outs, d_out, nargs * sizeof(MinOut), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("vx_minimize_many: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

// The persistent adjoint.  The kernel writes its result to out_dev (the
// tissue's result block when NULL); with out_host it is then copied there
// and the stream synchronised, without it the call returns at once.
vx_status adjoint_solve(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int path, AdjOut* out_host, AdjOut* out_dev, cudaStream_t s) {
  const int p = choose_path(t, path, true);
  if (p < 0) {
    set_error("the tissue is too large for the adjoint kernels");
    return VX_ERR_INVALID_ARG;
  }
  if (!out_dev) out_dev = (AdjOut*)t->dout;
  PersistArgs a = make_args(t, Xstar, nullptr, prm);
  a.ap = ap;
  a.aout = out_dev;
  // per-cell 4-vectors of the cluster path in the solver region of the
  // workspace (4 n doubles)
  if (p == VX_PATH_CLUSTER) a.cell = t->work;
  const bool f64 = t->dtype == VX_F64;
  cudaError_t e;
  if (p == VX_PATH_RESIDENT)
    e = f64 ? dispatch_res<PolF64, true>(t, a, s) : dispatch_res<PolF32, true>(t, a, s);
  else
    e = f64 ? dispatch_cluster<PolF64, true>(t, a, s) : dispatch_cluster<PolF32, true>(t, a, s);
  if (e != cudaSuccess) {
    set_error(std::string("adjoint launch: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  if (!out_host) return VX_OK;
  if (cudaMemcpyAsync(out_host, out_dev, sizeof(AdjOut), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("adjoint: ") + cudaGetErrorString(cudaGetLastError()));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

}  // namespace vx
