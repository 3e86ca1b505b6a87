// The extern "C" entry points of vx.h: argument validation, the tissue
// handle, and dispatch to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tissue.h"
#include "vx_internal.h"

namespace vx {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace vx

using vx::set_error;

#define VX_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA;         \
    }                                                                            \
  } while (0)

namespace {

vx_status invalid(const std::string& m) {
  set_error(m);
  return VX_ERR_INVALID_ARG;
}

// Checks that (he, face_he, edge_id) is a 3-valent periodic half-edge mesh
// with n faces; returns "" when valid.
std::string check_tables(const int32_t* he, const int32_t* face_he, const int32_t* edge_id, int n,
                         int HE) {
  if (n < 1) return "n_cells must be positive";
  if (HE != 6 * n) return "a 3-valent tessellation of the torus has 6 n half-edges";
  const int V = HE / 3, E = HE / 2;
  std::vector<int> outdeg(V, 0), ecount(E, 0);
  for (int h = 0; h < HE; ++h) {
    const int32_t* r = he + 8 * h;
    for (int k = 0; k < 5; ++k) {
      const int lim = (k < 3) ? HE : V;
      if (r[k] < 0 || r[k] >= lim) return "he[" + std::to_string(h) + "] index out of range";
    }
    if (r[5] < 0 || r[5] >= n) return "he[" + std::to_string(h) + "] face out of range";
    if (r[6] < -1 || r[6] > 1 || r[7] < -1 || r[7] > 1) return "offsets must be in {-1, 0, 1}";
    if (edge_id[h] < 0 || edge_id[h] >= E) return "edge_id out of range";
    ecount[edge_id[h]]++;
    outdeg[r[3]]++;
  }
  for (int h = 0; h < HE; ++h) {
    const int32_t* r = he + 8 * h;
    const int32_t* tw = he + 8 * r[2];
    if (r[2] == h || tw[2] != h) return "twin is not an involution at " + std::to_string(h);
    if (tw[3] != r[4] || tw[4] != r[3]) return "twin endpoints do not match";
    if (tw[6] != -r[6] || tw[7] != -r[7]) return "twin offsets must be negated";
    if (he[8 * r[1] + 0] != h) return "prev(next(h)) != h";
    if (he[8 * r[1] + 3] != r[4]) return "next(h) does not start at target(h)";
    if (he[8 * r[1] + 5] != r[5]) return "next(h) lies in another face";
    if (edge_id[r[2]] != edge_id[h]) return "twins must share an edge id";
  }
  for (int e = 0; e < E; ++e)
    if (ecount[e] != 2) return "every edge id must own exactly two half-edges";
  for (int v = 0; v < V; ++v)
    if (outdeg[v] != 3) return "vertex " + std::to_string(v) + " is not 3-valent";
  std::vector<char> seen(HE, 0);
  for (int c = 0; c < n; ++c) {
    const int h0 = face_he[c];
    if (h0 < 0 || h0 >= HE || he[8 * h0 + 5] != c) return "face_he[" + std::to_string(c) + "]";
    int h = h0, k = 0;
    do {
      if (seen[h]) return "a half-edge lies on two face cycles";
      seen[h] = 1;
      h = he[8 * h + 1];
    } while (h != h0 && ++k < HE);
    int ox = 0, oy = 0;
    h = h0;
    do {
      ox += he[8 * h + 6];
      oy += he[8 * h + 7];
      h = he[8 * h + 1];
    } while (h != h0);
    if (ox || oy) return "offsets around face " + std::to_string(c) + " do not cancel";
  }
  for (int h = 0; h < HE; ++h)
    if (!seen[h]) return "half-edge " + std::to_string(h) + " lies on no face cycle";
  return "";
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

bool params_ok(const vx_params* p, std::string* m) {
  if (!p) {
    *m = "params is NULL";
    return false;
  }
  const double sc[5] = {p->KA_s, p->KP_s, p->A0_s, p->P0_s, p->lambda_s};
  for (double x : sc)
    if (!std::isfinite(x)) {
      *m = "scalar parameters must be finite";
      return false;
    }
  return true;
}

vx::ParamsD to_params(const vx_params* p) {
  vx::ParamsD d;
  d.KA = p->KA;
  d.KP = p->KP;
  d.A0 = p->A0;
  d.P0 = p->P0;
  d.lam = p->lambda;
  d.KA_s = p->KA_s;
  d.KP_s = p->KP_s;
  d.A0_s = p->A0_s;
  d.P0_s = p->P0_s;
  d.lam_s = p->lambda_s;
  return d;
}

}  // namespace

namespace vx {

std::string build_host_tables(const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                              int n, int HE, HostTables* ht) {
  const std::string m = check_tables(he, face_he, edge_id, n, HE);
  if (!m.empty()) return m;
  const int V = HE / 3;
  std::vector<int32_t>& ext2int = ht->ext2int;
  std::vector<int32_t>& int2ext = ht->int2ext;
  ext2int.assign(HE, 0);
  int2ext.assign(HE, 0);
  for (int h = 0; h < HE; ++h) {
    const int tw = he[8 * h + 2];
    const int hi = 2 * edge_id[h] + (h > tw ? 1 : 0);
    ext2int[h] = hi;
    int2ext[hi] = h;
  }
  std::vector<uint32_t>& tgt = ht->tgt;
  std::vector<int32_t>&nxt = ht->nxt, &face = ht->face, &vout = ht->vout, &ff = ht->ff;
  tgt.assign(HE, 0u);
  nxt.assign(HE, 0);
  face.assign(HE, 0);
  vout.assign(3 * (size_t)V, -1);
  ff.assign(n, 0);
  std::vector<int> firstout(V, -1);
  for (int hc = 0; hc < HE; ++hc) {
    const int32_t* r = he + 8 * hc;
    const int hi = ext2int[hc];
    tgt[hi] = pack_tgt(r[4], r[6], r[7]);
    nxt[hi] = ext2int[r[1]];
    face[hi] = r[5];
    const int s = r[3];
    if (firstout[s] < 0 || hi < firstout[s]) firstout[s] = hi;
  }
  // Out-lists in counter-clockwise order: h, twin(prev(h)), twin(prev(.)).
  for (int v = 0; v < V; ++v) {
    int h = firstout[v];
    for (int a = 0; a < 3; ++a) {
      vout[a * V + v] = h;
      const int hp = ext2int[he[8 * int2ext[h] + 0]];
      h = hp ^ 1;
    }
    if (h != firstout[v]) return "vertex " + std::to_string(v) + ": out-half-edges do not close";
  }
  for (int c = 0; c < n; ++c) ff[c] = ext2int[face_he[c]];
  for (int c = 0; c < n; ++c) {
    int h = ff[c], k = 0;
    do {
      ++k;
      h = nxt[h];
    } while (h != ff[c] && k <= kMaxCorners);
    if (k > kMaxCorners - 1)
      return "cell " + std::to_string(c) + " has more than " + std::to_string(kMaxCorners - 1) +
             " edges";
  }
  return "";
}

}  // namespace vx

extern "C" {

const char* vx_last_error(void) { return vx::g_err.c_str(); }

const char* vx_version(void) { return "vx 0.1 sm_103a"; }

vx_status vx_build_mesh(const double* seeds_xy, int32_t n_cells, double Lx, double Ly,
                        double* vert_xy, int32_t* he, int32_t* face_he, int32_t* edge_id) {
  if (!seeds_xy || !vert_xy || !he || !face_he || !edge_id) return invalid("NULL pointer");
  if (n_cells < 3) return invalid("n_cells must be >= 3");
  if (n_cells > (1 << 24)) return invalid("n_cells too large");
  if (!(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly))
    return invalid("box sides must be positive and finite");
  for (int i = 0; i < n_cells; ++i) {
    const double x = seeds_xy[2 * i], y = seeds_xy[2 * i + 1];
    if (!(x >= 0 && x < Lx && y >= 0 && y < Ly)) return invalid("seeds must lie in [0,Lx) x [0,Ly)");
  }
  std::string err;
  const vx_status s = vx::build_mesh(seeds_xy, n_cells, Lx, Ly, vert_xy, he, face_he, edge_id, &err);
  if (s != VX_OK) set_error(err);
  return s;
}

vx_status vx_seed_order(const double* seeds_xy, int32_t n_cells, double Lx, double Ly,
                        int32_t* order) {
  if (!seeds_xy || !order) return invalid("NULL pointer");
  if (n_cells < 1) return invalid("n_cells must be positive");
  if (!(Lx > 0) || !(Ly > 0)) return invalid("box sides must be positive");
  vx::seed_order(seeds_xy, n_cells, Lx, Ly, order);
  return VX_OK;
}

vx_status vx_tissue_create(const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                           int32_t n_cells, int32_t n_half_edges, double Lx, double Ly,
                           int32_t dtype, void* stream, vx_tissue* out) {
  if (!he || !face_he || !edge_id || !out) return invalid("NULL pointer");
  if (dtype != VX_F64 && dtype != VX_F32) return invalid("dtype must be VX_F64 or VX_F32");
  if (!(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly))
    return invalid("box sides must be positive and finite");
  if (n_cells > (1 << 24)) return invalid("n_cells too large");
  vx::HostTables ht;
  const std::string m = vx::build_host_tables(he, face_he, edge_id, n_cells, n_half_edges, &ht);
  if (!m.empty()) return invalid(m);
  const int n = n_cells, HE = n_half_edges, V = HE / 3, E = HE / 2;
  vx_tissue_s* t = new vx_tissue_s();
  cudaGetDevice(&t->device);
  t->n = n;
  t->V = V;
  t->E = E;
  t->HE = HE;
  t->Lx = Lx;
  t->Ly = Ly;
  t->dtype = dtype;
  t->ext2int = std::move(ht.ext2int);
  t->int2ext = std::move(ht.int2ext);
  const std::vector<uint32_t>& tgt = ht.tgt;
  const std::vector<int32_t>&nxt = ht.nxt, &face = ht.face, &vout = ht.vout, &ff = ht.ff;
  auto bytes = [](size_t b) { return b < 16 ? (size_t)16 : b; };
  const int nbc = (n + 255) / 256 + 1, nbv = (V + 255) / 256 + 1;
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&t->tgt, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->nxt, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->face, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->vout, bytes(12 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->ffirst, bytes(4 * (size_t)n));
  if (e == cudaSuccess) e = cudaMalloc(&t->Xw, bytes(16 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->vel, bytes(16 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->F, bytes(16 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->cellc, bytes(16 * (size_t)n));
  if (e == cudaSuccess) e = cudaMalloc(&t->shortbits, bytes(4 * (size_t)(E / 32 + 1)));
  if (e == cudaSuccess) e = cudaMalloc(&t->touched, bytes(4 * (size_t)(V / 32 + 1)));
  if (e == cudaSuccess) e = cudaMalloc(&t->partE, bytes(3 * 8 * (size_t)nbc));
  if (e == cudaSuccess) e = cudaMalloc(&t->partF, bytes(4 * 8 * (size_t)nbv));
  if (e == cudaSuccess) e = cudaMalloc(&t->vnb, bytes(12 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->vfc, bytes(12 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->ccnt, bytes(4 * (size_t)n));
  if (e == cudaSuccess) e = cudaMalloc(&t->ccor, bytes(4 * (size_t)vx::kMaxCorners * n));
  if (e == cudaSuccess) e = cudaMalloc(&t->cedge, bytes(4 * (size_t)vx::kMaxCorners * n));
  if (e == cudaSuccess) e = cudaMalloc(&t->tgt0, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->nxt0, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->face0, bytes(4 * (size_t)HE));
  if (e == cudaSuccess) e = cudaMalloc(&t->vout0, bytes(12 * (size_t)V));
  if (e == cudaSuccess) e = cudaMalloc(&t->ffirst0, bytes(4 * (size_t)n));
  if (e == cudaSuccess) e = cudaMalloc(&t->ctrl, sizeof(vx::FireCtrl));
  if (e == cudaSuccess) e = cudaMalloc(&t->dout, sizeof(vx::MinOut));
  if (e == cudaSuccess) e = cudaMalloc(&t->wrapk, bytes(sizeof(int2) * (size_t)V));
  t->work = nullptr;
  t->work_doubles = vx::work_total_doubles(n, V);
  if (e == cudaSuccess) e = cudaMalloc(&t->work, 8 * t->work_doubles);
  if (e != cudaSuccess) {
    vx_tissue_destroy(t);
    set_error(std::string("vx_tissue_create: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA;
  }
  cudaStream_t s = as_stream(stream);
  auto upload = [&]() -> cudaError_t {
    cudaError_t r = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t b) {
      if (r == cudaSuccess) r = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s);
    };
    up(t->tgt, tgt.data(), 4 * (size_t)HE);
    up(t->nxt, nxt.data(), 4 * (size_t)HE);
    up(t->face, face.data(), 4 * (size_t)HE);
    up(t->vout, vout.data(), 12 * (size_t)V);
    up(t->ffirst, ff.data(), 4 * (size_t)n);
    up(t->tgt0, tgt.data(), 4 * (size_t)HE);
    up(t->nxt0, nxt.data(), 4 * (size_t)HE);
    up(t->face0, face.data(), 4 * (size_t)HE);
    up(t->vout0, vout.data(), 12 * (size_t)V);
    up(t->ffirst0, ff.data(), 4 * (size_t)n);
    if (r == cudaSuccess) r = cudaMemsetAsync(t->shortbits, 0, 4 * (size_t)(E / 32 + 1), s);
    if (r == cudaSuccess) r = cudaMemsetAsync(t->touched, 0, 4 * (size_t)(V / 32 + 1), s);
    if (r == cudaSuccess) r = vx::rebuild_flat(t, s);
    // the host tables are locals: wait for the copies before returning
    const cudaError_t w = cudaStreamSynchronize(s);
    return r == cudaSuccess ? w : r;
  };
  e = upload();
  if (e != cudaSuccess) {
    vx_tissue_destroy(t);
    set_error(std::string("vx_tissue_create: upload: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA;
  }
  *out = t;
  return VX_OK;
}

vx_status vx_tissue_destroy(vx_tissue t) {
  if (!t) return VX_OK;
  void* ptrs[] = {t->tgt,  t->nxt,   t->face,      t->vout,    t->ffirst, t->Xw,
                  t->vel,  t->F,     t->cellc,     t->shortbits, t->touched, t->partE,
                  t->partF, t->ctrl, t->dout,      t->work,    t->tgt0,   t->nxt0,
                  t->face0, t->vout0, t->ffirst0, t->vnb,   t->vfc,    t->ccnt,
                  t->ccor,  t->cedge, t->wrapk};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete t;
  return VX_OK;
}

vx_status vx_tissue_restore(vx_tissue t, void* stream) {
  if (!t) return invalid("NULL tissue");
  cudaStream_t s = as_stream(stream);
  const size_t HE = t->HE, V = t->V, n = t->n;
  VX_CUDA_TRY(cudaMemcpyAsync(t->tgt, t->tgt0, 4 * HE, cudaMemcpyDeviceToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(t->nxt, t->nxt0, 4 * HE, cudaMemcpyDeviceToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(t->face, t->face0, 4 * HE, cudaMemcpyDeviceToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(t->vout, t->vout0, 12 * V, cudaMemcpyDeviceToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(t->ffirst, t->ffirst0, 4 * n, cudaMemcpyDeviceToDevice, s));
  VX_CUDA_TRY(vx::rebuild_flat(t, s));
  return VX_OK;
}

vx_status vx_hessian_vector(vx_tissue t, const double* X, const vx_params* p, const double* v,
                            double* Hv, void* stream) {
  if (!t || !X || !v || !Hv) return invalid("NULL tissue, X, v or Hv");
  std::string m;
  if (!params_ok(p, &m)) return invalid(m);
  const vx_status s = vx::hessian_vector(t, X, to_params(p), v, Hv, as_stream(stream));
  if (s != VX_OK) set_error(std::string("vx_hessian_vector: ") + cudaGetErrorString(cudaGetLastError()));
  return s;
}

vx_status vx_tissue_sizes(vx_tissue t, int32_t* n_cells, int32_t* n_vertices, int32_t* n_edges,
                          int32_t* n_half_edges) {
  if (!t) return invalid("NULL tissue");
  if (n_cells) *n_cells = t->n;
  if (n_vertices) *n_vertices = t->V;
  if (n_edges) *n_edges = t->E;
  if (n_half_edges) *n_half_edges = t->HE;
  return VX_OK;
}

vx_status vx_tissue_topology(vx_tissue t, int32_t* he, int32_t* face_he, int32_t* edge_id) {
  if (!t || !he || !face_he || !edge_id) return invalid("NULL pointer");
  const int HE = t->HE, V = t->V, n = t->n;
  std::vector<uint32_t> tgt(HE);
  std::vector<int32_t> nxt(HE), face(HE), vout(3 * V), ff(n);
  VX_CUDA_TRY(cudaMemcpy(tgt.data(), t->tgt, 4 * (size_t)HE, cudaMemcpyDeviceToHost));
  VX_CUDA_TRY(cudaMemcpy(nxt.data(), t->nxt, 4 * (size_t)HE, cudaMemcpyDeviceToHost));
  VX_CUDA_TRY(cudaMemcpy(face.data(), t->face, 4 * (size_t)HE, cudaMemcpyDeviceToHost));
  VX_CUDA_TRY(cudaMemcpy(vout.data(), t->vout, 12 * (size_t)V, cudaMemcpyDeviceToHost));
  VX_CUDA_TRY(cudaMemcpy(ff.data(), t->ffirst, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  for (int hi = 0; hi < HE; ++hi) {
    const int s = vx::tgt_v(tgt[hi ^ 1]);
    int slot = 0;
    while (slot < 3 && vout[slot * V + s] != hi) ++slot;
    if (slot == 3) {
      set_error("device topology is inconsistent");
      return VX_ERR_TOPOLOGY;
    }
    const int prev = vout[((slot + 1) % 3) * V + s] ^ 1;
    int32_t* r = he + 8 * t->int2ext[hi];
    r[0] = t->int2ext[prev];
    r[1] = t->int2ext[nxt[hi]];
    r[2] = t->int2ext[hi ^ 1];
    r[3] = s;
    r[4] = vx::tgt_v(tgt[hi]);
    r[5] = face[hi];
    r[6] = vx::tgt_ox(tgt[hi]);
    r[7] = vx::tgt_oy(tgt[hi]);
    edge_id[t->int2ext[hi]] = hi >> 1;
  }
  for (int c = 0; c < n; ++c) face_he[c] = t->int2ext[ff[c]];
  return VX_OK;
}

vx_status vx_energy_forces(vx_tissue t, const double* X, const vx_params* p, double* F, double* E,
                           void* stream) {
  if (!t || !X) return invalid("NULL tissue or X");
  std::string m;
  if (!params_ok(p, &m)) return invalid(m);
  const vx_status s = vx::energy_forces(t, X, to_params(p), F, E, as_stream(stream));
  if (s != VX_OK) set_error(std::string("vx_energy_forces: ") + cudaGetErrorString(cudaGetLastError()));
  return s;
}

void vx_min_opts_default(vx_min_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = VX_FIRE;
  o->tol = 1e-8;
  o->patience = 1;
  o->max_iter = 100000;
  o->gd_lr = 1e-2;
  o->dt0 = 0.01;
  o->dt_max = 0.5;
  o->n_min = 5;
  o->f_inc = 1.1;
  o->f_dec = 0.5;
  o->alpha0 = 0.1;
  o->f_alpha = 0.99;
  o->l_min = 0.0;
  o->path = VX_PATH_AUTO;
  o->check_every = 50;
  o->wrap = 1;
  o->edge_events = nullptr;
  o->refine_tol = 0.0;
}

static bool min_opts_ok(const vx_min_opts* o, std::string* m) {
  if (!o) {
    *m = "opts is NULL";
    return false;
  }
  if (o->method != VX_FIRE && o->method != VX_GD) *m = "method must be VX_FIRE or VX_GD";
  else if (!(o->tol >= 0)) *m = "tol must be >= 0";
  else if (o->patience < 1) *m = "patience must be >= 1";
  else if (o->max_iter < 0) *m = "max_iter must be >= 0";
  else if (!(o->dt0 > 0) || !(o->dt_max > 0)) *m = "dt0 and dt_max must be positive";
  else if (!(o->gd_lr > 0)) *m = "gd_lr must be positive";
  else if (o->path < VX_PATH_AUTO || o->path > VX_PATH_GRID) *m = "unknown path";
  else return true;
  return false;
}

static vx::MinParams to_min_params(const vx_min_opts* o) {
  vx::MinParams mp = {};
  mp.method = o->method;
  mp.tol = o->tol;
  mp.patience = o->patience;
  mp.max_iter = o->max_iter;
  mp.gd_lr = o->gd_lr;
  mp.dt0 = o->dt0;
  mp.dt_max = o->dt_max;
  mp.n_min = o->n_min;
  mp.f_inc = o->f_inc;
  mp.f_dec = o->f_dec;
  mp.alpha0 = o->alpha0;
  mp.f_alpha = o->f_alpha;
  mp.l_min = o->l_min;
  mp.wrap = o->wrap ? 1 : 0;
  mp.edge_events = o->edge_events;
  return mp;
}

vx_status vx_minimize(vx_tissue t, double* X, const vx_params* p, const vx_min_opts* o,
                      vx_min_result* r, void* stream) {
  if (!t || !X || !r) return invalid("NULL tissue, X or result");
  std::string m;
  if (!params_ok(p, &m) || !min_opts_ok(o, &m)) return invalid(m);
  vx::MinOut out = {};
  int used = 0;
  const vx::ParamsD prm = to_params(p);
  vx::MinParams mp = to_min_params(o);
  const bool refine = t->dtype == VX_F32 && o->refine_tol > o->tol;
  if (refine) {
    mp.tol = o->refine_tol;
    mp.wrap = 0;
  }
  vx_status s = vx::minimize(t, X, prm, mp, o->path, o->check_every, &out, &used,
                             as_stream(stream));
  if (s != VX_OK) return s;
  if (refine && out.status == VX_OK && out.iters < o->max_iter) {
    // Newton steps (FP64 residuals, CG on the Hessian), then FP64 FIRE from
    // there to tol: the FIRE stage checks the T1 rule and the stop rule at
    // its first iteration and ends at once when the Newton steps reached
    // tol (X is FP64 in and out; the tissue's buffers hold either precision)
    int nsteps = 0;
    double fm = 0.0;
    s = vx::newton_refine(t, X, prm, o->tol, 8, &nsteps, &fm, as_stream(stream));
    if (s != VX_OK) return s;
    out.force_evals += 2 * nsteps + 1;
    const vx::MinOut first = out;
    vx::MinParams mp2 = to_min_params(o);
    mp2.max_iter = o->max_iter - first.iters;
    const int saved = t->dtype;
    t->dtype = VX_F64;
    out = vx::MinOut{};
    s = vx::minimize(t, X, prm, mp2, o->path, o->check_every, &out, &used, as_stream(stream));
    t->dtype = saved;
    if (s != VX_OK) return s;
    out.iters += first.iters;
    out.n_t1 += first.n_t1;
    out.n_stretch += first.n_stretch;
    out.force_evals += first.force_evals;
  } else if (refine && o->wrap) {
    vx::MinParams mw = to_min_params(o);
    mw.max_iter = 0;    // no step and no T1 check: the exit-time wrap only
    mw.l_min = 0.0;
    const vx::MinOut first = out;
    s = vx::minimize(t, X, prm, mw, o->path, o->check_every, &out, &used, as_stream(stream));
    if (s != VX_OK) return s;
    const int wrap_err = out.wrap_err;
    out = first;
    out.wrap_err = wrap_err;
  }
  r->status = out.status;
  r->iters = out.iters;
  r->n_t1 = out.n_t1;
  r->n_stretch = out.n_stretch;
  r->n_short_edges = out.n_short;
  r->n_inverted = out.n_inverted;
  r->fmax = out.fmax;
  r->energy = out.energy;
  r->path_used = used;
  r->force_evals = out.force_evals;
  if (out.wrap_err) r->status = VX_ERR_TOPOLOGY;
  const vx_status st = (vx_status)r->status;
  return st == VX_ERR_NONFINITE || st == VX_ERR_TIMEOUT || st == VX_ERR_TOPOLOGY ? st : VX_OK;
}

vx_status vx_minimize_many(vx_tissue* tissues, int32_t count, double* const* X,
                           const vx_params* params, const vx_min_opts* o, vx_min_result* r,
                           void* stream) {
  if (!tissues || !X || !params || !r || count < 1) return invalid("NULL argument or count < 1");
  std::string m;
  if (!min_opts_ok(o, &m)) return invalid(m);
  std::vector<vx::ParamsD> prms(count);
  for (int k = 0; k < count; ++k) {
    if (!tissues[k] || !X[k]) return invalid("NULL tissue or X at " + std::to_string(k));
    if (!params_ok(&params[k], &m)) return invalid(m);
    prms[k] = to_params(&params[k]);
    for (int q = 0; q < k; ++q)
      if (tissues[q] == tissues[k]) return invalid("a tissue appears twice");
  }
  std::vector<vx::MinOut> out(count);
  std::vector<int> paths(count);
  const vx_status s = vx::minimize_many(tissues, count, X, prms.data(), to_min_params(o), o->path,
                                        out.data(), paths.data(), as_stream(stream));
  if (s != VX_OK) return s;
  vx_status worst = VX_OK;
  for (int k = 0; k < count; ++k) {
    r[k].status = out[k].status;
    r[k].iters = out[k].iters;
    r[k].n_t1 = out[k].n_t1;
    r[k].n_stretch = out[k].n_stretch;
    r[k].n_short_edges = out[k].n_short;
    r[k].n_inverted = out[k].n_inverted;
    r[k].fmax = out[k].fmax;
    r[k].energy = out[k].energy;
    r[k].path_used = paths[k];
    r[k].force_evals = out[k].force_evals;
    if (out[k].wrap_err) r[k].status = VX_ERR_TOPOLOGY;
    if (r[k].status == VX_ERR_NONFINITE || r[k].status == VX_ERR_TIMEOUT ||
        r[k].status == VX_ERR_TOPOLOGY)
      worst = (vx_status)r[k].status;
  }
  return worst;
}

void vx_grad_opts_default(vx_grad_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = VX_ADJOINT_CG;
  o->beta = 1e-3;
  o->cg_rtol = 1e-10;
  o->cg_max_iter = 20000;
  o->cost = VX_COST_NONE;
  o->cost_data = nullptr;
  vx_min_opts_default(&o->inner);
  o->inner.tol = 1e-10;
  o->ep_f64 = 1;
}

}  // extern "C"

namespace {

// The minimiser's device result block as the caller's vx_min_result (in
// device or pinned host memory).
__global__ void k_min_result(const vx::MinOut* o, int path, vx_min_result* r) {
  if (threadIdx.x || blockIdx.x) return;
  vx_min_result x;
  x.status = o->wrap_err ? (int)VX_ERR_TOPOLOGY : o->status;
  x.iters = o->iters;
  x.n_t1 = o->n_t1;
  x.n_stretch = o->n_stretch;
  x.n_short_edges = o->n_short;
  x.n_inverted = o->n_inverted;
  x.fmax = o->fmax;
  x.energy = o->energy;
  x.path_used = path;
  x.force_evals = o->force_evals;
  *r = x;
}

std::string grad_opts_error(const double* dCdX, const vx_grad_opts* o) {
  std::string m;
  if (o->mode != VX_ADJOINT_CG && o->mode != VX_EP_CENTERED && o->mode != VX_EP_FORWARD &&
      o->mode != VX_ADJOINT_MINRES)
    return "unknown gradient mode";
  const bool ep = o->mode == VX_EP_CENTERED || o->mode == VX_EP_FORWARD;
  if (!ep && !dCdX && o->cost == VX_COST_NONE) return "adjoint needs dCdX or a built-in cost";
  if (ep && o->cost == VX_COST_NONE) return "equilibrium propagation needs a built-in cost";
  if (o->cost != VX_COST_NONE && o->cost != VX_COST_V2V && o->cost != VX_COST_ANISO)
    return "unknown cost";
  if (o->cost != VX_COST_NONE && !o->cost_data) return "cost_data is NULL";
  if (ep && !(o->beta > 0)) return "beta must be positive";
  if (!min_opts_ok(&o->inner, &m)) return m;
  return "";
}

}  // namespace

extern "C" {

vx_status vx_minimize_async(vx_tissue t, double* X, const vx_params* p, const vx_min_opts* o,
                            vx_min_result* r, void* stream) {
  if (!t || !X || !r) return invalid("NULL tissue, X or result");
  std::string m;
  if (!params_ok(p, &m) || !min_opts_ok(o, &m)) return invalid(m);
  if (o->path == VX_PATH_PLAIN || o->path == VX_PATH_GRID)
    return invalid("vx_minimize_async runs the resident or cluster path only");
  cudaStream_t s = as_stream(stream);
  int used = 0;
  const vx_status st = vx::minimize_launch(t, X, to_params(p), to_min_params(o), o->path, t->dout,
                                           &used, s);
  if (st != VX_OK) return st;
  k_min_result<<<1, 1, 0, s>>>(t->dout, used, r);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("vx_minimize_async: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

vx_status vx_sensitivity_grad(vx_tissue t, const double* Xstar, const vx_params* p,
                              const double* dCdX, int32_t count, const int32_t* kind,
                              const int32_t* index, int32_t solver, double rtol, int32_t max_iter,
                              double* out, int32_t* status, void* stream) {
  if (!t || !Xstar || !dCdX || !kind || !index || !out) return invalid("NULL argument");
  if (count < 0) return invalid("count must be >= 0");
  std::string m;
  if (!params_ok(p, &m)) return invalid(m);
  if (solver != VX_ADJOINT_CG && solver != VX_ADJOINT_MINRES)
    return invalid("solver must be VX_ADJOINT_CG or VX_ADJOINT_MINRES");
  if (!(rtol >= 0) || max_iter < 0) return invalid("invalid solver options");
  for (int k = 0; k < count; ++k) {
    const int lim = kind[k] == VX_PARAM_LAMBDA ? t->E : t->n;
    if (kind[k] < VX_PARAM_LAMBDA || kind[k] > VX_PARAM_P0) return invalid("unknown parameter kind");
    if (index[k] < 0 || index[k] >= lim) return invalid("parameter index out of range");
  }
  return vx::sensitivity(t, Xstar, to_params(p), dCdX, count, kind, index,
                         solver == VX_ADJOINT_MINRES, rtol, max_iter, 50, out, status,
                         as_stream(stream));
}

vx_status vx_equilibrium_grad_async(vx_tissue t, const double* Xstar, const vx_params* p,
                                    const double* dCdX, const vx_grad_opts* o, double* g_lambda,
                                    double* g_A0, double* g_P0, vx_grad_result* r, void* stream) {
  if (!t || !Xstar || !o || !r) return invalid("NULL tissue, X*, opts or result");
  std::string m;
  if (!params_ok(p, &m)) return invalid(m);
  m = grad_opts_error(dCdX, o);
  if (!m.empty()) return invalid(m);
  if (o->inner.path == VX_PATH_PLAIN || o->inner.path == VX_PATH_GRID)
    return invalid("vx_equilibrium_grad_async runs the persistent paths only");
  return vx::equilibrium_grad_impl(t, Xstar, to_params(p), dCdX, o, g_lambda, g_A0, g_P0, nullptr, r,
                                   as_stream(stream));
}

vx_status vx_equilibrium_grad(vx_tissue t, const double* Xstar, const vx_params* p,
                              const double* dCdX, const vx_grad_opts* o, double* g_lambda,
                              double* g_A0, double* g_P0, vx_grad_result* r, void* stream) {
  if (!t || !Xstar || !o || !r) return invalid("NULL tissue, X*, opts or result");
  std::string m;
  if (!params_ok(p, &m)) return invalid(m);
  m = grad_opts_error(dCdX, o);
  if (!m.empty()) return invalid(m);
  return vx::equilibrium_grad(t, Xstar, to_params(p), dCdX, o, g_lambda, g_A0, g_P0, r,
                              as_stream(stream));
}

}  // extern "C"
