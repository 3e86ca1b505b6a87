/*
 * vx.h — C ABI of the GB300-native periodic vertex model.
 *
 * The library computes, on one GPU, the hot path of a confluent periodic 2D
 * vertex model (VertAX, arXiv 2604.06896): cell areas and perimeters, edge
 * lengths, the energy
 *
 *     E(X) = sum_cells K_A (A - A0)^2 + K_P (P - P0)^2 + sum_edges Lambda l
 *
 * (Methods, "Vertex model formulation": the E1 form with per-cell moduli plus
 * the line-tension term of E2), its analytic gradient on the 3-valent
 * vertices, relaxation to force balance by FIRE or gradient descent with T1
 * transitions (Methods, "Simulation engine", "T1 transitions"), and the
 * gradient of an outer cost taken at the equilibrium, by the implicit adjoint
 * (Methods, "Implicit differentiation") or by equilibrium propagation
 * (Methods, "Equilibrium propagation").
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns a vx_status and never throws across the ABI.  On
 *   an error, vx_last_error() returns a message for the calling thread.
 * - Arguments are validated before anything is launched; an invalid argument
 *   leaves every output untouched.
 * - "dev" pointers are CUDA device pointers on the current device, "host"
 *   pointers are ordinary (pageable or pinned) host memory.  The caller owns
 *   every buffer it passes; the library never frees them.  A vx_tissue owns
 *   its device topology and workspace, allocated in vx_tissue_create and
 *   released by vx_tissue_destroy.
 * - Positions X are float64 [V][2] (x, y interleaved).  Forces and gradients
 *   are float64.  The compute precision is chosen per tissue (VX_F64 or
 *   VX_F32: FP32 arithmetic on hi/lo FP32 position pairs, FP64 reductions).
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls that return results to the host synchronise it.
 *
 * Topology format (Methods, "System state and data structure")
 * ------------------------------------------------------------
 *   he      int32 [HE][8]: prev, next, twin, source, target, face, offx, offy
 *           (offx, offy in {-1, 0, 1}: the target vertex sits at
 *           X[target] + (offx Lx, offy Ly) as seen from the source)
 *   face_he int32 [n]: one half-edge of each face
 *   edge_id int32 [HE]: the undirected edge of each half-edge, 0 .. E-1
 * A periodic Voronoi tessellation of n generic seeds has V = 2n vertices,
 * E = 3n edges and HE = 6n half-edges.
 */
#ifndef VX_H
#define VX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VX_OK = 0,
  VX_NOT_CONVERGED = 1,      /* non-fatal: outputs hold the last iterate   */
  VX_ERR_INVALID_ARG = 2,
  VX_ERR_DEGENERATE_SEEDS = 3,
  VX_ERR_CUDA = 4,
  VX_ERR_OOM = 5,
  VX_ERR_INDEFINITE = 6,     /* CG met p^T H p <= 0 (non-convex energy)    */
  VX_ERR_TIMEOUT = 7,
  VX_ERR_NONFINITE = 8,      /* NaN or Inf met in positions or forces      */
  VX_ERR_TOPOLOGY = 9        /* T1 bookkeeping found an inconsistency      */
} vx_status;

enum { VX_F64 = 0, VX_F32 = 1 };
enum { VX_FIRE = 0, VX_GD = 1 };
enum { VX_ADJOINT_CG = 0, VX_EP_CENTERED = 1, VX_EP_FORWARD = 2, VX_ADJOINT_MINRES = 3 };
/* Parameter kinds of vx_sensitivity_grad. */
enum { VX_PARAM_LAMBDA = 0, VX_PARAM_A0 = 1, VX_PARAM_P0 = 2 };
enum { VX_COST_NONE = 0, VX_COST_V2V = 1, VX_COST_ANISO = 2 };
/* Execution paths of the persistent solvers:
 *   RESIDENT: one CTA holds the whole tissue in shared memory for the whole
 *             solve (tissues up to ~1,500 cells in FP32);
 *   CLUSTER:  a 16-CTA thread-block cluster holds it in L2-resident global
 *             memory, synchronised by the hardware cluster barrier (up to
 *             16,384 cells);
 *   PLAIN:    one kernel launch per sub-step, convergence polled by the
 *             host every check_every steps (the reference GPU path);
 *   GRID:     m co-resident CTAs of a cooperative launch (one per 256
 *             cells, at most one per SM) hold it in L2-resident global
 *             memory, synchronised by a bounded-wait barrier in global
 *             memory (up to 4 x 256 cells per SM).  A barrier wait longer
 *             than 4 s ends the solve with status VX_ERR_TIMEOUT.
 *   AUTO picks RESIDENT for tissues of up to 512 cells that fit, then
 *   CLUSTER, then PLAIN (vx_minimize_many: RESIDENT whenever it fits). */
enum { VX_PATH_AUTO = 0, VX_PATH_RESIDENT = 1, VX_PATH_PLAIN = 2, VX_PATH_CLUSTER = 3,
       VX_PATH_GRID = 4 };

/* Message of the last error on the calling thread ("" if none). */
const char* vx_last_error(void);

/* Library version, e.g. "vx 0.1 sm_103a". */
const char* vx_version(void);

/*
 * vx_build_mesh — periodic Voronoi tessellation of n seeds (host only).
 *
 * Methods, "Mesh initialization" and "Periodic mode": the tessellation of the
 * seeds on the torus [0,Lx) x [0,Ly); every polygon of a primary seed is
 * kept, and half-edges crossing the box get the offset of their target.
 * Indexing is canonical (identical for identical seeds on any machine):
 *   face alpha = seed alpha; a vertex is a Delaunay triangle of the torus,
 *   keyed by its three (seed, image shift) corners in CCW order, translated
 *   so that the first corner has shift 0, smallest rotation first; vertices
 *   are numbered by increasing key; a vertex sits at the circumcentre of its
 *   key triangle wrapped into the box; the half-edges of each face are
 *   contiguous (faces in order), counter-clockwise from the face's smallest
 *   vertex index; an edge's id is the rank of its smaller half-edge index.
 *
 * seeds_xy  host float64 [n][2], each in [0,Lx) x [0,Ly)
 * n_cells   n >= 3
 * vert_xy   host float64 [2n][2]   (out)
 * he        host int32 [6n][8]     (out)
 * face_he   host int32 [n]         (out; the first half-edge of each face)
 * edge_id   host int32 [6n]        (out)
 * Returns VX_ERR_DEGENERATE_SEEDS when four seeds are (nearly) cocircular
 * (a Voronoi edge shorter than 1e-9 sqrt(Lx Ly / n)), when a cell touches
 * its own periodic image, or when a cell spans more than one box copy.
 */
vx_status vx_build_mesh(const double* seeds_xy, int32_t n_cells, double Lx, double Ly,
                        double* vert_xy, int32_t* he, int32_t* face_he, int32_t* edge_id);

/*
 * vx_seed_order — an ordering of the seeds along a Hilbert curve through the
 * box (order[k] = index of the k-th seed).  The canonical numbering of
 * vx_build_mesh follows the seed order, so building from the reordered
 * seeds gives the same tissue with cells, vertices and edges numbered in
 * spatial order: neighbouring threads then touch neighbouring memory, which
 * is what the global-memory kernels need to coalesce their gathers.
 * seeds_xy host float64 [n][2]; order host int32 [n] (out).
 */
vx_status vx_seed_order(const double* seeds_xy, int32_t n_cells, double Lx, double Ly,
                        int32_t* order);

/* Opaque handle: one tissue (topology on the device + workspace). */
typedef struct vx_tissue_s* vx_tissue;

/*
 * vx_tissue_create — upload a topology and allocate the workspace.
 * he, face_he, edge_id: host tables in the format above (any valid
 * 3-valent periodic half-edge mesh, not only canonical ones).
 * dtype: VX_F64 or VX_F32.  The handle is bound to the current device.
 */
vx_status vx_tissue_create(const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                           int32_t n_cells, int32_t n_half_edges, double Lx, double Ly,
                           int32_t dtype, void* stream, vx_tissue* out);
vx_status vx_tissue_destroy(vx_tissue t);

/*
 * vx_tissue_restore — put back the topology the tissue had at creation
 * (undoes the T1 transitions of earlier vx_minimize calls).  Asynchronous.
 */
vx_status vx_tissue_restore(vx_tissue t, void* stream);

/* Sizes of a tissue: cells, vertices, edges, half-edges. */
vx_status vx_tissue_sizes(vx_tissue t, int32_t* n_cells, int32_t* n_vertices,
                          int32_t* n_edges, int32_t* n_half_edges);

/*
 * vx_tissue_topology — copy the tissue's current topology (T1 transitions
 * made by vx_minimize change it) back to host tables of the input format.
 * Half-edge and edge identities are kept through T1 transitions.
 */
vx_status vx_tissue_topology(vx_tissue t, int32_t* he, int32_t* face_he, int32_t* edge_id);

/*
 * Model parameters.  Each pointer is a device float64 array (K_A, K_P, A0,
 * P0 per cell [n]; lambda per edge [E]) or NULL, in which case the scalar
 * beside it is used for every cell / edge.
 */
typedef struct {
  const double* KA;  const double* KP;  const double* A0;  const double* P0;
  const double* lambda;
  double KA_s, KP_s, A0_s, P0_s, lambda_s;
} vx_params;

/*
 * vx_energy_forces — energy and forces at X.
 * Energy: Methods, "Vertex model formulation"; forces F = -grad_X E
 * (Results, "Energy functions").
 * X  dev float64 [V][2]; F dev float64 [V][2] or NULL; E dev float64 [1] or
 * NULL.  Asynchronous on `stream`; deterministic (no atomics).
 */
vx_status vx_energy_forces(vx_tissue t, const double* X, const vx_params* p,
                           double* F, double* E, void* stream);

/*
 * vx_hessian_vector — Hv = (grad^2_X E) v at X (the operator the adjoint
 * solves with; Methods, "Implicit differentiation").  X, v, Hv dev float64
 * [V][2].  Asynchronous on `stream`.
 */
vx_status vx_hessian_vector(vx_tissue t, const double* X, const vx_params* p, const double* v,
                            double* Hv, void* stream);

/* Inner minimiser options (defaults from vx_min_opts_default). */
typedef struct {
  int32_t method;      /* VX_FIRE or VX_GD                                  */
  double  tol;         /* stop when max_i |F_i| < tol ...                   */
  int32_t patience;    /* ... for this many consecutive iterations         */
  int32_t max_iter;
  double  gd_lr;       /* gradient-descent step eta                         */
  double  dt0, dt_max; /* FIRE time steps                                   */
  int32_t n_min;       /* FIRE N_min                                        */
  double  f_inc, f_dec, alpha0, f_alpha;
  double  l_min;       /* T1 threshold; <= 0 disables T1 checks             */
  int32_t path;        /* VX_PATH_AUTO / RESIDENT / CLUSTER / PLAIN / GRID  */
  int32_t check_every; /* PLAIN path: host polls convergence every k steps  */
  int32_t wrap;        /* 1 (default): on return every vertex is wrapped into
                          the box and the offsets fixed (Methods, "Periodic
                          mode"); 0: positions are left unwrapped          */
  int32_t* edge_events;/* dev int32 [E][2] or NULL: per edge, the number of
                          stretches ([e][0]) and T1s ([e][1]) the T1 passes
                          made are added (a diagnostic of repeated events) */
  double  refine_tol;  /* FP32 tissues, vx_minimize only: when > tol, the
                          solve runs in FP32 arithmetic until max|F| <
                          refine_tol, then takes up to 8 Newton steps
                          X += H^-1 F (F in FP64 arithmetic, H^-1 F by CG on
                          the Hessian-vector product; a step that does not
                          lower max|F| is undone) and finishes with FP64
                          FIRE to tol (FP32 forces carry ~3e-7 relative
                          rounding, below which FP32 FIRE stalls); the FIRE
                          budget is shared; 0 (default): one precision
                          throughout                                       */
} vx_min_opts;

typedef struct {
  int32_t status;      /* VX_OK or VX_NOT_CONVERGED (or an error)           */
  int32_t iters;       /* position updates made                             */
  int32_t n_t1, n_stretch;
  int32_t n_short_edges; /* edges shorter than l_min at the end             */
  int32_t n_inverted;  /* cells with A <= 0 at the end                      */
  double  fmax;        /* max_i |F_i| at the returned X                     */
  double  energy;
  int32_t path_used;   /* VX_PATH_RESIDENT, _CLUSTER, _PLAIN or _GRID       */
  int32_t force_evals;
} vx_min_result;

void vx_min_opts_default(vx_min_opts* o);

/*
 * vx_minimize — relax X to force balance (Methods, "Simulation engine"):
 * FIRE (Bitzek et al., PRL 97, 170201, 2006; unit masses, semi-implicit
 * Euler step) or gradient descent X <- X - eta grad E; stop rule
 * max_i |F_i| < tol for `patience` consecutive iterations, or max_iter.
 * Each iteration first checks the edges for T1 transitions (Methods, "T1
 * transitions"; both candidates at length 1.5 l_min, lower energy kept).
 * X dev float64 [V][2], in/out.  Inside the solve positions are unwrapped
 * and the offsets fixed; with o->wrap (the default) every vertex is then
 * put back into [0, Lx) x [0, Ly) and the tissue's offsets are changed so
 * that every unwrapped edge vector keeps its value (an offset that would
 * leave {-1, 0, 1} gives VX_ERR_TOPOLOGY).  r host (out).  Synchronises
 * `stream`.
 */
vx_status vx_minimize(vx_tissue t, double* X, const vx_params* p, const vx_min_opts* o,
                      vx_min_result* r, void* stream);

/*
 * vx_minimize_many — vx_minimize for several tissues at once: one persistent
 * launch holds every tissue that fits a CTA's shared memory (one CTA each)
 * and one holds the others (one 16-CTA cluster each), or, with o->path =
 * VX_PATH_GRID, one cooperative launch holds them all, each on a share of
 * the SMs proportional to its cell count.  Independent relaxations (a
 * parameter sweep, the members of an ensemble) so share the GPU instead of
 * running one after another.  Each tissue gets the same result as from
 * vx_minimize on the path it was given (r[k].path_used).  o->path AUTO
 * puts small tissues on CTAs and large ones on clusters, CLUSTER puts all
 * on clusters, RESIDENT requires every tissue to fit a CTA; PLAIN is
 * rejected.  tissues [count], X [count] (dev float64 [V_k][2], in/out),
 * params [count], r host [count] (out).  Tissues must be distinct and of
 * one dtype.  Calls are serialised.  Synchronises `stream`.
 */
vx_status vx_minimize_many(vx_tissue* tissues, int32_t count, double* const* X,
                           const vx_params* params, const vx_min_opts* o, vx_min_result* r,
                           void* stream);

/* Outer-gradient options. */
typedef struct {
  int32_t mode;        /* VX_ADJOINT_CG, VX_EP_CENTERED, VX_EP_FORWARD      */
  double  beta;        /* EP nudging strength                               */
  double  cg_rtol;     /* CG stops at |r| <= cg_rtol |b|                    */
  int32_t cg_max_iter;
  int32_t cost;        /* built-in cost for EP (and for adjoint if dCdX NULL) */
  const double* cost_data; /* dev: X_target [V][2] (v2v) or q_target [2]     */
  vx_min_opts inner;   /* nudged phases (T1 is not applied in them, nor the
                          exit-time wrap)                                   */
  int32_t ep_f64;      /* EP on an FP32 tissue: 1 (default) runs the nudged
                          phases in FP64 arithmetic (the estimate divides a
                          difference of two equilibria by beta, so their
                          force balance must be finer than FP32 forces
                          allow); 0 keeps them in FP32 (about 4e-2 relative
                          error against the FP64 estimate at beta = 1e-2) */
} vx_grad_opts;

typedef struct {
  int32_t status;
  int32_t cg_iters;
  double  cg_rel_residual;
  double  cost;        /* C at X* (built-in costs)                          */
  int32_t nudged_iters[2];
} vx_grad_result;

void vx_grad_opts_default(vx_grad_opts* o);

/*
 * vx_equilibrium_grad — gradient of an outer cost C(X*) with respect to the
 * line tensions Lambda_e and the targets A0, P0 at an equilibrium X*.
 * VX_ADJOINT_CG (Methods, "Implicit differentiation", adjoint form):
 *   solve H lam = Pi grad_X C by conjugate gradients on a Hessian-vector
 *   product (Pi removes the two rigid translations, the null space of H),
 *   then g_theta = -(d^2 E / dX dtheta)^T lam.  The CG runs in one
 *   persistent launch (o->inner.path AUTO, RESIDENT, CLUSTER; GRID runs it
 *   on a cluster), or, with o->inner.path = VX_PATH_PLAIN, as one launch per
 *   sub-step with FP64 vectors and the status polled every
 *   o->inner.check_every iterations (the reference GPU path).
 * VX_ADJOINT_MINRES (Methods, "Implicit differentiation": Krylov solves for
 *   Hessians that are not positive definite): the same adjoint with the
 *   linear system solved by MINRES (Paige and Saunders 1975; no
 *   preconditioner) on the plain path, for the indefinite Hessians on which
 *   CG stops with VX_ERR_INDEFINITE.
 * VX_EP_CENTERED / VX_EP_FORWARD (Methods, "Equilibrium propagation"):
 *   re-minimise E +/- (beta/2) C (or E + beta C and the free X*) from X*,
 *   nudging with the translation-free part of grad_X C, and difference
 *   d_theta E over beta.  The built-in cost is VX_COST_V2V or
 *   VX_COST_ANISO (its gradient is recomputed from the cells' shapes at
 *   every iteration of the nudged phases).
 * Xstar dev float64 [V][2]; dCdX dev float64 [V][2] (adjoint; NULL uses the
 * built-in cost).  g_lambda dev [E], g_A0 dev [n], g_P0 dev [n], each may be
 * NULL.  r host (out).  Synchronises `stream`.
 */
vx_status vx_equilibrium_grad(vx_tissue t, const double* Xstar, const vx_params* p,
                              const double* dCdX, const vx_grad_opts* o,
                              double* g_lambda, double* g_A0, double* g_P0,
                              vx_grad_result* r, void* stream);

/*
 * vx_sensitivity_grad — the forward form of implicit differentiation
 * (Methods, "Implicit differentiation", sensitivity form): for each listed
 * parameter theta_k (kind[k] VX_PARAM_LAMBDA with index[k] an edge id,
 * VX_PARAM_A0 / VX_PARAM_P0 with a cell), solve H s_k = d(grad_X E)/d theta_k
 * (solver VX_ADJOINT_CG or VX_ADJOINT_MINRES, to rtol, on the plain path)
 * and return dC/d theta_k = -grad_X C . s_k: one linear solve per
 * parameter, the same numbers as the adjoint (which needs one solve for
 * all).  Xstar, dCdX dev float64 [V][2]; kind, index host int32 [count];
 * out host float64 [count]; status host int32 [count] or NULL (per solve
 * VX_OK / VX_NOT_CONVERGED / VX_ERR_INDEFINITE).  Synchronises `stream`.
 */
vx_status vx_sensitivity_grad(vx_tissue t, const double* Xstar, const vx_params* p,
                              const double* dCdX, int32_t count, const int32_t* kind,
                              const int32_t* index, int32_t solver, double rtol, int32_t max_iter,
                              double* out, int32_t* status, void* stream);

/*
 * Asynchronous forms, for CUDA graphs.  Every call above that takes a
 * vx_tissue allocates nothing (the workspace is sized by vx_tissue_create);
 * these two also never synchronise: everything is enqueued on `stream` and
 * the GPU writes the result struct into r, which is device memory or pinned
 * (page-locked) host memory, when the work is done.  So they can be
 * recorded in a CUDA graph and replayed; arguments are checked when the
 * call is made, the statuses in r describe the run.
 *
 * vx_minimize_async — vx_minimize on the persistent paths (o->path AUTO,
 *   RESIDENT or CLUSTER; AUTO must resolve to one of them); PLAIN and GRID
 *   are rejected (they poll the host or stage arguments through it).
 *   r->status is VX_OK, VX_NOT_CONVERGED, VX_ERR_NONFINITE or
 *   VX_ERR_TOPOLOGY.
 * vx_equilibrium_grad_async — vx_equilibrium_grad with the persistent
 *   adjoint or the persistent nudged phases (o->inner.path not PLAIN or
 *   GRID); r->status as in the synchronous form (VX_ERR_INDEFINITE when CG
 *   met non-positive curvature).
 */
vx_status vx_minimize_async(vx_tissue t, double* X, const vx_params* p, const vx_min_opts* o,
                            vx_min_result* r, void* stream);
vx_status vx_equilibrium_grad_async(vx_tissue t, const double* Xstar, const vx_params* p,
                                    const double* dCdX, const vx_grad_opts* o,
                                    double* g_lambda, double* g_A0, double* g_P0,
                                    vx_grad_result* r, void* stream);

/*
 * vx_energy_forces_noalloc — vx_energy_forces for callers that cannot
 * allocate device memory (a stream capture whose memory pool is frozen, a
 * plugin with a fixed memory budget, a real-time loop that must not touch
 * the allocator).  The paper has no counterpart: this is an interface of the
 * library, not a step of the method.
 *
 * It needs no vx_tissue (creating one allocates).  The caller passes, in its
 * own device memory, the topology tables in the format of this header
 * (he int32 [6n][8], face_he int32 [n], edge_id int32 [6n]), X float64
 * [2n][2], and the outputs F float64 [2n][2] (or NULL) and E float64 [1] (or
 * NULL), plus status int32 [1], which every call clears and then sets to
 * the OR of: 1 when a vertex is not the source of exactly three half-edges
 * (that vertex gets no force), 2 when a table holds an index out of range
 * (the access is skipped; F and E are then not meaningful).  Both checks run
 * whether or not F is asked for.  Arithmetic is FP64.  Nothing is allocated
 * and no allocating library routine is called: the kernels' scratch lives in
 * one static device array sized for at most 32,768 cells (196,864 doubles =
 * 1,574,912 bytes, about 1.5 MiB, held by every GPU that loads the library
 * until the process exits); larger tissues are rejected with
 * VX_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (with that device current) and caches it: make that first
 * call before any stream capture.  All calls share the one array: calls
 * that overlap on the GPU (on different streams) race and must be ordered
 * by the caller.  Asynchronous on `stream`.
 */
vx_status vx_energy_forces_noalloc(const int32_t* he, const int32_t* face_he,
                                   const int32_t* edge_id, int32_t n_cells, double Lx, double Ly,
                                   const double* X, const vx_params* p, double* F, double* E,
                                   int32_t* status, void* stream);

/*
 * vx_grid_barrier_selftest — exercises the bounded wait of the GRID path's
 * barrier without a fault (the paper has no counterpart: this checks the
 * library's failure detection).  One cooperative launch of `ctas`
 * co-resident CTAs passes `rounds` barriers with the same barrier code the
 * GRID minimiser uses, each wait limited to wait_s seconds (0 < wait_s
 * <= 10).  The CTA of rank absent_rank (or none, when it is negative)
 * leaves before the first barrier, so the others' waits run out.
 * status host int32 [ctas] (out): VX_OK for a CTA that passed every
 * barrier, VX_ERR_TIMEOUT for one whose wait ran out (or that saw another
 * CTA's time-out), -1 for the absent CTA.  Returns VX_ERR_TIMEOUT if any
 * CTA timed out, VX_ERR_INVALID_ARG if the CTAs cannot all be resident.
 * Allocates a few bytes of device memory for the barrier; synchronises
 * `stream`.
 */
vx_status vx_grid_barrier_selftest(int32_t ctas, int32_t absent_rank, int32_t rounds,
                                   double wait_s, int32_t* status, void* stream);

/* ------------------------------------------------------------ batches */

/*
 * A batch: many independent tissues of uneven size solved in one persistent
 * launch (the workload's batched forward path; the paper runs tissues one at
 * a time).  Tissue k's tables use indices local to the tissue; they are
 * concatenated in order: he [sum 6 n_k][8], face_he [sum n_k],
 * edge_id [sum 6 n_k]; box [count][2] = (Lx, Ly).  Positions are the
 * concatenation of the tissues' [2 n_k][2] arrays.
 */
typedef struct vx_batch_s* vx_batch;

typedef struct {
  const double *KA, *KP, *A0, *P0;  /* dev, per cell [sum n_k] or NULL       */
  const double* lambda;             /* dev, per edge [sum 3 n_k] or NULL     */
  const double *KA_t, *KP_t, *A0_t, *P0_t, *lambda_t; /* host, per tissue or NULL */
  double KA_s, KP_s, A0_s, P0_s, lambda_s;             /* used when both NULL */
} vx_batch_params;

vx_status vx_batch_create(int32_t count, const int32_t* n_cells, const double* box,
                          const int32_t* he, const int32_t* face_he, const int32_t* edge_id,
                          int32_t dtype, void* stream, vx_batch* out);
vx_status vx_batch_destroy(vx_batch b);
/* Put back every tissue's topology at creation (asynchronous). */
vx_status vx_batch_restore(vx_batch b, void* stream);
vx_status vx_batch_sizes(vx_batch b, int32_t* count, int32_t* n_total, int32_t* v_total,
                         int32_t* e_total);
/* The batch's current topologies, concatenated in the input format. */
vx_status vx_batch_topology(vx_batch b, int32_t* he, int32_t* face_he, int32_t* edge_id);

/*
 * vx_minimize_batched — vx_minimize for every tissue of the batch in one
 * persistent launch (replayed from a CUDA graph captured at the first call
 * with these arguments).  Tissues whose working set fits a CTA's
 * shared-memory allocation are solved there, one CTA each, taken largest
 * first; larger ones (up to 6,144 cells) by 8-CTA thread-block clusters from
 * L2-resident global memory, on a share of the SMs proportional to their
 * cells, in a second launch that runs beside the first; the CTA launch
 * takes tissues from the clusters' queue once its own is empty (a tissue
 * above 6,144 cells is solved by one CTA from L2).  X dev float64
 * [sum V][2] in/out; r host [count] (out).  opts->path and check_every are
 * ignored.  Synchronises `stream`.
 */
vx_status vx_minimize_batched(vx_batch b, double* X, const vx_batch_params* p,
                              const vx_min_opts* o, vx_min_result* r, void* stream);

/*
 * vx_batch_autotune — time `probe_iters`-iteration runs of the batch for
 * every (threads per CTA, shared memory per CTA) pair in {128, 256} x
 * {220, 108, 70, 52} KiB and keep the fastest for later calls (the shared-memory
 * size is the residency cutoff and sets how many CTAs share an SM).  X is
 * not modified.  Outputs may be NULL.
 */
vx_status vx_batch_autotune(vx_batch b, double* X, const vx_batch_params* p,
                            const vx_min_opts* o, int32_t probe_iters, int32_t* threads_out,
                            int32_t* smem_out, void* stream);

/*
 * vx_equilibrium_grad_batched — the adjoint gradient (Methods, "Implicit
 * differentiation", adjoint form; as vx_equilibrium_grad with
 * VX_ADJOINT_CG) for every tissue of the batch in one persistent launch:
 * CTAs take tissues largest first and run the block-Jacobi preconditioned CG
 * on each, tissue and CG vectors in L2-resident global memory.  The
 * topology is the batch's current one (after vx_minimize_batched).
 * Xstar dev float64 [sum V][2]; dCdX dev float64 [sum V][2] (the outer
 * cost's gradient, e.g. from vx_batch_aniso_cost); CG stops at
 * |r| <= cg_rtol |b| or after cg_max_iter iterations; g_lambda dev
 * [sum E], g_A0, g_P0 dev [sum n], each may be NULL; r host [count] (out).
 * Returns VX_ERR_INDEFINITE if CG met non-positive curvature in a tissue
 * (see r[k].status).  Synchronises `stream`.
 */
vx_status vx_equilibrium_grad_batched(vx_batch b, const double* Xstar, const vx_batch_params* p,
                                      const double* dCdX, double cg_rtol, int32_t cg_max_iter,
                                      double* g_lambda, double* g_A0, double* g_P0,
                                      vx_grad_result* r, void* stream);

/*
 * vx_batch_grad — the batched gradient workload in one persistent launch
 * (replayed from a CUDA graph captured at the first call with these
 * arguments): for every tissue of the batch, taken largest first by the
 * CTAs of the launch, (1) the free relaxation from X to X* under
 * free_opts (Methods, "Simulation engine", "T1 transitions"); (2) the
 * built-in outer cost go->cost (VX_COST_V2V with go->cost_data = X_target
 * dev [sum V][2], or VX_COST_ANISO with q_target dev [2]) and its gradient
 * at X*; (3) with what & VX_GRAD_ADJOINT, the adjoint gradient (Methods,
 * "Implicit differentiation": preconditioned CG to go->cg_rtol, FP64
 * reductions); (4) with what & VX_GRAD_EP, equilibrium propagation
 * (Methods, "Equilibrium propagation"): the nudged phases E +/- (beta/2) C
 * (go->mode VX_EP_CENTERED) or E + beta C (VX_EP_FORWARD) from X* under
 * go->inner without T1, in FP64 arithmetic when go->ep_f64, then the
 * difference of d_theta E over beta.  Each tissue is run by one CTA, or
 * by one cluster (8 CTAs up to 10,240 cells, 16 up to 12,288) when every
 * tissue has at least 4,096 cells and at most 12,288 (free_opts->path
 * VX_PATH_RESIDENT forces one CTA, VX_PATH_CLUSTER 16-CTA clusters;
 * CLUSTER with a tissue above 12,288 cells is VX_ERR_INVALID_ARG).
 * X dev float64 [sum V][2] in/out
 * (X*, wrapped per free_opts->wrap).  Gradients (each may be NULL): ga_*
 * adjoint, ge_* EP; lambda dev [sum E], A0 and P0 dev [sum n].  r host
 * [count] (out).  Nothing is allocated (the workspace is sized by
 * vx_batch_create).  Synchronises `stream`.
 */
enum { VX_GRAD_ADJOINT = 1, VX_GRAD_EP = 2 };
typedef struct {
  vx_min_result free;      /* the free relaxation to X*                      */
  vx_grad_result adjoint;  /* status, CG iterations, residual; cost at X*    */
  vx_grad_result ep;       /* status, nudged iterations; cost at X*          */
} vx_batch_grad_result;
vx_status vx_batch_grad(vx_batch b, double* X, const vx_batch_params* p,
                        const vx_min_opts* free_opts, const vx_grad_opts* go, int32_t what,
                        double* ga_lambda, double* ga_A0, double* ga_P0, double* ge_lambda,
                        double* ge_A0, double* ge_P0, vx_batch_grad_result* r, void* stream);

/*
 * vx_batch_aniso_cost — the anisotropy cost of every tissue (the batched
 * inverse-design workload's outer cost; the mean cell-shape tensor Q,
 * q = ((Qxx - Qyy) / tr Q, 2 Qxy / tr Q), C = |q - q_target|^2) and its
 * gradient.  X dev float64 [sum V][2]; q_target dev float64 [2]; C host
 * [count] (out); dCdX dev float64 [sum V][2] (out).  Synchronises `stream`.
 */
vx_status vx_batch_aniso_cost(vx_batch b, const double* X, const double* q_target, double* C,
                              double* dCdX, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VX_H */
