/*
 * irk.h - C ABI of libirk: one stage-parallel Radau IIA step of the heat
 * equation on a GB300 GPU (sm_103a).
 *
 * The problem (arXiv 2209.06700, Sec. 2 and Sec. 5): the semi-discrete heat
 * equation M u'(t) + K u(t) = g(t) on the unit square/cube [0,1]^d, with
 * continuous tensor-product Lagrange elements of degree k on a uniform mesh
 * of N cells per direction, Gauss-Legendre (k+1)^d quadrature and homogeneous
 * Dirichlet conditions, advanced by the Q-stage Radau IIA method with step
 * tau.  Each step solves the transformed stage system of Eq. (irk:A),
 *     (A_Q^{-1} (x) M + tau I_Q (x) K) k = (A_Q^{-1} (x) I)(gbar - 1_Q (x) K y_n),
 * with FP64 flexible GMRES preconditioned by Eq. (irk:P),
 *     P^{-1} = (S~ (x) I) (Lambda~ (x) M + tau I (x) K)^{-1} (S~^{-1} (x) I),
 * (A_Q^{-1} = L U, L = S~ Lambda~ S~^{-1}), each block (lambda_i M + tau K)
 * approximated by one geometric-multigrid V-cycle with a Chebyshev/point-
 * Jacobi smoother; then y_{n+1} = y_n + tau sum_i b_i k_i (Sec. 1).  The
 * directly diagonalised variant (Eq. (irk:Ainv) in real 2x2-block form,
 * Sec. 6, PRESB preconditioner Eq. (presb:p)) is selected by
 * irk_options.variant = IRK_VARIANT_DIAG.
 *
 * Conventions for every call:
 *  - Vectors are FP64 (or FP32 where stated) arrays over the (kN+1)^d node
 *    grid, lexicographic with x fastest.  Entries at boundary nodes are zero on
 *    input and are left zero on output.  Stage-blocked vectors hold Q such
 *    vectors back to back with stride irk_stage_stride(h) elements.
 *  - Unless stated otherwise, pointers are DEVICE pointers owned by the
 *    caller, on the device current when the handle was created, and all work
 *    is enqueued on the handle's CUDA stream (irk_create's `cuda_stream`,
 *    NULL = legacy default stream).  A call on a handle makes the handle's
 *    GPU current while it runs and restores the caller's current device, so
 *    one process may drive handles on several GPUs.  The library owns every internal buffer
 *    (Krylov bases, multigrid hierarchy) and frees it in irk_destroy.
 *  - Errors are returned as irk_status codes; no C++ exception crosses the
 *    ABI.  irk_last_error(h) gives a one-line message for the last failure.
 *    Every call that takes a handle returns IRK_EINVAL for a NULL handle and
 *    for the NULL or out-of-range arguments named at the call, IRK_ENOMEM when
 *    an allocation fails and IRK_ECUDA when a CUDA call fails; the size queries
 *    return -1 instead of a status.
 *  - A handle is not thread-safe; distinct handles may be used from distinct
 *    threads.
 */
#ifndef IRK_H_
#define IRK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IRK_OK = 0,
  IRK_EINVAL = -1,    /* bad argument (sizes, degree, stage count, NULL) */
  IRK_ENOMEM = -2,    /* device allocation failed */
  IRK_ENOTCONV = -3,  /* FGMRES did not reach rtol within max_it; y unchanged */
  IRK_ENUMERIC = -4,  /* NaN/Inf met in a residual norm; y unchanged */
  IRK_ETIMEOUT = -5,  /* a bounded device wait gave up */
  IRK_ECUDA = -6,     /* a CUDA runtime call failed */
  IRK_EBUSY = -7      /* admission refused: memory budget exhausted */
} irk_status;

enum { IRK_VARIANT_LU = 0, IRK_VARIANT_DIAG = 1 };

typedef struct {
  int dim;            /* 2 or 3 */
  int cells_per_axis; /* N >= 1; the domain is [0,1]^dim */
} irk_mesh;

typedef struct {
  double rtol;        /* outer FGMRES: stop when ||r|| <= rtol ||rhs|| (default 1e-10; > 0) */
  int max_it;         /* maximum FGMRES iterations per step, all restarts (default 200; >= 1) */
  int restart;        /* Krylov basis size before restart (default 30; 1..60) */
  int cheb_degree;    /* Chebyshev smoother degree per half V-cycle (default 3; 1..16) */
  int variant;        /* IRK_VARIANT_LU (Eq. irk:P) or IRK_VARIANT_DIAG (Eq. irk:Ainv + PRESB) */
  int mg_precision;   /* 0 (default): chosen at create from the preconditioner's basis change:
                         FP32 while cond_F(S~) (DIAG: cond_F(T)) <= 2e5, i.e. Q <= 5, FP64 above,
                         where the basis change would magnify FP32 rounding beyond the V-cycle's
                         own error; 32: FP32 V-cycle; 64: FP64 V-cycle */
  int batched;        /* 1: all stage blocks in one launch per kernel (default); 0: per-stage launches */
  int use_graph;      /* 1: replay the preconditioner as a CUDA graph (default 1) */
  int eig_steps;      /* Lanczos steps for the Chebyshev interval (default 20; >= 2) */
  double smoothing_range; /* Chebyshev interval [hi/range, hi] (default 10; > 1) */
  double eig_safety;  /* hi = safety * Lanczos estimate (default 1.2; >= 1) */
  int shared_cheb;    /* 1: one Chebyshev interval for all blocks (batched mode of Sec. 5.4) */
  int op_ff;          /* arithmetic of the outer solver (stage operator, Krylov vectors, stage
                         combinations): 0 native FP64 (default); 1 float-float on the FP32 pipe
                         (about 48 significant bits, |values| within 1e-30..1e30; faster on GPUs
                         with a narrow FP64 pipe, not FP64) */
  int autotune;       /* 1: time the 3D operator kernels' launch shapes (tile width, z chunk,
                         cluster) at create on the handle's own buffers and keep the fastest,
                         process-wide per kernel and size (default 1); 0: cost model only */
  int pair_precond;   /* DIAG variant, 2x2 pair blocks: 0 PRESB (Eq. presb:p, two V-cycles on
                         (alpha+beta) M + tau K, default); 1 one V-cycle on the coupled 2x2 system
                         itself (Sec. 6, GMG applied directly to Eq. complex:twobytwo) */
  double deform;      /* 0 (default): the uniform Cartesian mesh.  eps > 0: the curved mesh
                         Phi(xi) = xi + eps prod_a sin(pi xi_a) (1, .., 1) of the same cube
                         (boundary fixed, non-affine cells; needs eps < 1 / (dim pi)).  The
                         stage operator, K y_n, the load and the initial interpolant then use
                         the mapping data w det J and w det J J^-1 J^-T at every Gauss point
                         (Sec. 3.4: read once per cell for all stages of a launch), with FP64
                         stage vectors; op_ff then picks the operator's arithmetic (1 float-float,
                         0 native FP64).  The preconditioner keeps the Cartesian blocks of
                         Eq. (irk:P) (flexible GMRES absorbs the difference) */
  int gs_reorth;      /* second classical Gram-Schmidt pass of the outer FGMRES: 0 (default) where
                         one pass would leave the Krylov basis orthogonal to worse than 2^-16
                         (estimated loss; the residuals and stopping test are then those of an
                         orthogonal basis to within 0.1 %); 1 at every step */
} irk_options;

typedef struct {
  int iterations;       /* FGMRES iterations of the last step (sum over DIAG blocks) */
  int vcycles;          /* V-cycles applied (per block, sequential count as in Sec. 5 tables) */
  double rel_residual;  /* final ||r|| / ||rhs|| (max over DIAG blocks) */
  double ms_total;      /* host wall time of the step, ms */
  int reorth_passes;    /* Gram-Schmidt second passes taken (see gs_reorth) */
} irk_stats;

typedef struct irk_problem* irk_handle;

/* Fill `opt` with the defaults listed above. */
void irk_default_options(irk_options* opt);

/* Create a solver for the heat problem on `mesh` with degree k (1..4), Q stages
 * (1..9; DIAG variant 2..9) and step tau > 0.  Builds the tableau factors, the
 * multigrid hierarchy (levels N, N/2, ... to the first odd N or the coarsest
 * mesh with an interior node; the coarsest level is solved exactly, by a dense
 * FP64 inverse up to 9^3 unknowns and by fast diagonalisation above), the Chebyshev
 * intervals (Lanczos on D^{-1}A per level and block) and the dense coarse
 * inverses, and allocates all work memory on the current device.
 * `cuda_stream` is a cudaStream_t (NULL: default stream).  On success *out
 * holds the handle; on failure *out is NULL and nothing is leaked.  The setup
 * follows Sec. 5 (solver setup) with the readings of the multigrid stated above.
 * IRK_EINVAL: NULL mesh or out, dim not 2 or 3, cells_per_axis outside 1..4096,
 * degree outside 1..4, Q outside 1..9 (DIAG: 2..9), tau not positive and finite,
 * no interior node, or invalid options; IRK_ENOMEM / IRK_ECUDA as above. */
irk_status irk_create(const irk_mesh* mesh, int degree, int Q, double tau,
                      const irk_options* opt, void* cuda_stream, irk_handle* out);

/* One Radau IIA step from t_n (Sec. 2: the stage system of Eq. (irk:A) solved by
 * flexible GMRES preconditioned by Eq. (irk:P), then the update of Sec. 1).
 * y (device, irk_ndofs(h) doubles): in y_n,
 * out y_{n+1}.  stage_load: NULL = the built-in manufactured source
 * g(t) = (d pi^2 cos t - sin t) G with G_j = int prod sin(pi x_a) phi_j;
 * otherwise a device array [Q][stride] with g(t_n + c_i tau) per stage.
 * stats may be NULL.  Returns after the step is complete on the stream
 * (the FGMRES convergence test reads residual norms on the host).
 * IRK_EINVAL for a NULL y.  On IRK_ENOTCONV / IRK_ENUMERIC y is unchanged. */
irk_status irk_step(irk_handle h, double* y, double t_n, const double* stage_load,
                    irk_stats* stats);
/* (irk_step refuses a group handle with IRK_EINVAL: groups step with irk_step_group.) */

/* Advance `count` independent problems by one step each.  hs[i], ys[i],
 * t_ns[i] as in irk_step (built-in source).  Distinct handles run concurrently
 * on host threads, each enqueueing on its own handle's stream, so their FGMRES
 * iterations interleave and their kernels overlap on the device (batching
 * across requests; give each handle its own stream for overlap).  Items that
 * repeat a handle run in array order.  per_item (host, count entries, may be
 * NULL) receives each item's status.  Returns IRK_OK if every item
 * succeeded, else the status of the lowest failing index; failed items leave
 * their y unchanged as in irk_step. */
irk_status irk_solve_batch(irk_handle* hs, double** ys, const double* t_ns, int count,
                           irk_status* per_item);

/* ---- groups of requests: shared launches across requests ----
 * Not in the paper: the paper batches the Q stages of one problem into the same operator and
 * multigrid sweeps (Sec. 3.4, Sec. 5.4); a group extends that batch across requests.  R independent
 * heat problems of the same shape (dim, cells, degree, Q), each with its own step tau_r, live in one
 * handle: their stage vectors are [R][Q][stride], every stage-operator launch, K y_n launch and
 * V-cycle launch covers all R Q stage vectors or blocks, and each request keeps its own FGMRES
 * (Krylov basis, Hessenberg matrix, convergence test) in lockstep with the others, one device->host
 * read-back per iteration for all of them.  Every launch takes the launch shape of a single
 * request's stage count and every per-stage or per-block result is computed as for that request
 * alone, so each request's y_{n+1} equals the result of a one-request handle (to rounding, 1e-12
 * relative).  Groups use the LU variant on the Cartesian mesh; R Q <= 16. */

/* Create a group handle for R requests (taus: host, R steps > 0) of the shape given as in
 * irk_create.  The multigrid hierarchy holds R Q blocks (lambda~_i M + tau_r K), the Krylov space
 * R interleaved bases.  IRK_EINVAL as irk_create, and for NULL taus, R < 1, R Q > 16, a
 * non-positive tau, the DIAG variant or a curved mesh. */
irk_status irk_create_group(const irk_mesh* mesh, int degree, int Q, int R, const double* taus,
                            const irk_options* opt, void* cuda_stream, irk_handle* out);

/* One Radau IIA step of every request of a group (or one-request) handle from t_ns[r] (host, R
 * values): ys (host array of R device pointers, irk_ndofs doubles each) y_n in, y_{n+1} out.  The
 * built-in source.  stats (host, R entries) and per_item (host, R statuses) may be NULL.  Returns
 * IRK_OK when every request succeeded, else the first failing status; a failed request (IRK_ENOTCONV,
 * IRK_ENUMERIC) leaves its y unchanged while the others complete.  IRK_EINVAL for NULL ys or t_ns,
 * a NULL entry of ys, or a handle of the DIAG variant or curved mesh. */
irk_status irk_step_group(irk_handle h, double* const* ys, const double* t_ns, irk_stats* stats,
                          irk_status* per_item);

/* New steps for the requests of a handle (taus: host, irk_group_size(h) values > 0), so that a
 * handle can serve a later request of the same shape: only what depends on tau is rebuilt, on the
 * handle's memory (Chebyshev intervals by Lanczos, coarse inverses, fused-cycle parameters; the
 * captured V-cycle graph is recaptured at the next step).  IRK_EINVAL for NULL taus, a
 * non-positive tau or the DIAG variant. */
irk_status irk_set_tau(irk_handle h, const double* taus);

/* Requests in the handle (1 for irk_create), -1 for NULL. */
int irk_group_size(irk_handle h);

/* ---- serving: continuous batching of single-step requests ---- */
typedef struct {
  int dim, cells, degree, Q;  /* problem of the request (as irk_create) */
  double tau;                 /* step */
  double t0;                  /* the step goes from t0 to t0 + tau, y(t0) = interpolant */
  double arrival_s;           /* arrival time, seconds after irk_serve starts */
} irk_request;

typedef struct {
  irk_status status;
  int iterations;             /* FGMRES iterations */
  double latency_ms;          /* arrival -> y_{n+1} ready (on the host if requested) */
  double queue_ms;            /* arrival -> admission */
  double setup_ms;            /* handle creation (hierarchy, Chebyshev intervals) and y_0 */
  double solve_ms;            /* irk_step */
  long long ndofs, ninterior;
  double mem_bytes;           /* device memory reserved for the request at admission */
  int group_size;             /* requests that shared this request's launches (irk_create_group) */
  int handle_reused;          /* 1: the group's handle came from the cache (irk_set_tau), 0: created */
} irk_result;

typedef struct {
  int max_active;             /* concurrent requests (slots, one stream and one host worker each) */
  double mem_budget_bytes;    /* device memory for resident requests; <= 0: 80% of the free memory */
  int realtime;               /* 1: honour arrival_s; 0: every request arrives at time 0 */
  irk_options solver;         /* solver options of every request */
  int max_group;              /* requests of one shape that share launches (1 = none; 0 = up to 16/Q) */
  int reuse_handles;          /* 1: keep idle handles per shape and group size and reuse them for later
                                 requests (irk_set_tau), evicted least recently used when memory is
                                 needed; 0: create and destroy a handle per group */
  int smallest_first;         /* 1 (default): a free slot takes the waiting request with the fewest
                                 stage-DoFs (oldest among equals); 0: the oldest waiting request */
} irk_serve_options;

/* Default serving options: 16 slots, automatic budget, real time, groups up to 16/Q requests,
 * handle reuse on, smallest request first, solver defaults with restart 16 and autotune 0 (concurrent requests would time
 * each other's kernels; the cost model's launch shapes, or shapes tuned earlier in the process,
 * are used). */
void irk_default_serve_options(irk_serve_options* opt);

/* Serve `count` requests with continuous batching (not in the paper: the serving form of this
 * library).  Arrived requests wait; a free slot (a host worker) takes the smallest waiting request
 * (fewest stage-DoFs, the oldest among equals; the oldest with smallest_first = 0) together with the
 * other waiting requests of the same shape (dim, cells, degree, Q), up to
 * max_group, as one group whose operator and V-cycle launches they share (irk_create_group), on a
 * handle taken from the cache of idle handles of that shape and size (irk_set_tau) or created when
 * the memory budget allows (evicting idle handles if needed), each handle on its own CUDA stream.
 * Each request takes one step from the interpolant of u(., t0); groups run concurrently, so
 * requests arriving while others are on the GPU start as soon as a slot and memory are free.
 * Every request's result is independent of the mix (a group member's result equals its result
 * alone; same launch shapes, deterministic reductions).  results (host, count entries) receive
 * per-request timing, status and group size; out_host (optional, count pointers, each NULL or a
 * host array of irk_ndofs doubles) receives y_{n+1}.  A request larger than the whole budget fails
 * with IRK_EBUSY.  Every cached handle is destroyed before the call returns.  Returns IRK_OK if
 * every request succeeded, else the first failing status. */
irk_status irk_serve(const irk_request* reqs, int count, const irk_serve_options* opt, irk_result* results,
                     double** out_host);

/* Release every resource of the handle (NULL is accepted).  Returns IRK_OK. */
irk_status irk_destroy(irk_handle h);

/* ---- sizes and helpers (the size queries return -1 for a NULL handle) ---- */
long long irk_ndofs(irk_handle h);            /* (kN+1)^d */
long long irk_ninterior(irk_handle h);        /* (kN-1)^d unknowns per stage */
long long irk_stage_stride(irk_handle h);     /* elements between stage vectors in [Q][stride] arrays */
int irk_num_levels(irk_handle h);             /* multigrid levels, finest first */
/* Static text of a status code (never NULL). */
const char* irk_strerror(irk_status s);
/* Message of the handle's last failure ("" before any; "NULL handle" for NULL); the string is
 * owned by the handle and valid until its next failing call or irk_destroy. */
const char* irk_last_error(irk_handle h);

/* Text report of the launch shapes chosen by the autotuner so far in this process, one line
 * per kernel and size ("<kernel> k=.. <epilogue> N=.. stages=..: cxs=.. zc=.. cluster=.. <us>
 * (model ...)").  Writes at most len-1 bytes and a terminating NUL into buf (buf may be NULL);
 * returns the full length of the report.  No paper counterpart (implementation detail of the
 * batched launches of Sec. 5.4). */
int irk_autotune_report(char* buf, int len);

/* Launch-shape control of the 3D operator kernels (no paper counterpart: it lets tests reach every
 * launch shape of the streaming kernel, Sec. 3's matrix-free evaluation tiled for the GPU).
 * irk_op_shape_force makes every later 3D streaming operator launch of one element size use the
 * given shape, process-wide, until cleared with cxs = 0: elem_bytes 4 for the FP32 multigrid
 * kernels (level operator, Chebyshev step, residual), 8 for the FP64-accurate stage operator and
 * K y_n; cxs the cells per warp segment (8, 16 or 32; below 32 only for elem_bytes 4), zc the
 * cells per z chunk (>= 1), cluster 1 to run the chunks of a tile as one thread-block cluster
 * (2..16 chunks that the device can hold).  Levels of at most 8 cells per axis keep the cell
 * kernel.  A forced shape the kernel cannot run makes the launching call fail (IRK_ECUDA); CUDA
 * graphs captured before the call keep their shapes.  Returns IRK_EINVAL for an unknown element
 * size or a shape outside these ranges.
 * irk_op_shape_last writes (cxs, zc, cluster, number of z chunks) of the last such launch of that
 * element size into out4 (host, 4 ints; -1 each before any launch); IRK_EINVAL for a NULL out4 or
 * an unknown element size. */
irk_status irk_op_shape_force(int elem_bytes, int cxs, int zc, int cluster);
irk_status irk_op_shape_last(int elem_bytes, int* out4);

/* y (device, irk_ndofs doubles) <- nodal interpolant of the manufactured solution
 * u = prod sin(pi x_a) cos t (the initial value of the step; on the curved mesh at the mapped
 * nodes).  IRK_EINVAL for a NULL y. */
irk_status irk_interpolate_initial(irk_handle h, double* y, double t);

/* Host copies of the tableau factors (row-major Q x Q or length Q), FP64:
 * which = 0 A, 1 b, 2 c, 3 A^{-1}, 4 L, 5 U, 6 S~, 7 S~^{-1}, 8 lambda~ (diag L),
 * 9 T (real Jordan basis of A^{-1}), 10 T^{-1}, 11 J (real block form)
 * (Sec. 2; Eq. (irk:P); Eq. (irk:Ainv)).  out_host is owned by the caller.  IRK_EINVAL for a
 * NULL out_host or an unknown which. */
irk_status irk_get_tableau(irk_handle h, int which, double* out_host);

/* The same factors without a handle or a device: Radau IIA with Q stages (1..9; Sec. 2, the
 * collocation tableau), the Crout factors of A^{-1} with its eigen-decomposition (Eq. irk:P) and
 * the real block form (Eq. irk:Ainv), built by the host routine irk_create uses.  which as in
 * irk_get_tableau; out_host holds Q x Q (row-major) or Q doubles, owned by the caller.  Returns
 * IRK_EINVAL for a NULL out_host, Q outside 1..9 or an unknown which, IRK_ENUMERIC if the
 * construction fails.  Runs on the host only (no CUDA call). */
irk_status irk_tableau_factors(int Q, int which, double* out_host);

/* One-dimensional Q_k element data on the reference cell [0, 1] as the operators use it, built
 * on the host without a handle or a device (Sec. 5: tensor-product Lagrange elements with the
 * consistent (k+1)-point Gauss rule; nodes at the Gauss-Lobatto-Legendre points; the
 * prolongation is the Q_k embedding of a cell split in two).  k in 1..4, p = k + 1; which:
 * 0 nodes (p), 1 mass matrix (p x p), 2 stiffness matrix (p x p), 3 prolongation block
 * ((2k+1) x p: coarse basis i at fine node m, row-major [m][i]), 4 Gauss points (p), 5 Gauss
 * weights (p), 6 basis values and 7 basis derivatives at the Gauss points (p x p, [q][i]).
 * out_host is owned by the caller.  Returns IRK_EINVAL for a NULL out_host, k outside 1..4 or an
 * unknown which, IRK_ENUMERIC if the construction fails.  Host only (no CUDA call). */
irk_status irk_element_factors(int k, int which, double* out_host);

/* Chebyshev interval of the smoother (Sec. 5) on level l (0 = finest) and block i of the
 * hierarchy chosen by irk_mg_select: out_host[0] = lo, [1] = hi (host, caller-owned).
 * IRK_EINVAL for a NULL out_host, a level without a smoother (the coarsest is solved exactly)
 * or a block the hierarchy does not have. */
irk_status irk_get_cheb_interval(irk_handle h, int level, int block, double* out_host);

/* ---- the steps of the hot path, exposed one by one (all device pointers) ---- */

/* v = (Cm (x) M + Ck (x) K) u on the finest mesh, FP64, with ns stage vectors
 * of stride irk_stage_stride(h); Cm, Ck are host row-major ns x ns matrices
 * (ns <= 9).  With Cm = A^{-1}, Ck = tau I this is the operator of Eq. (irk:A);
 * Sec. 2's "generalized vector scaling" (I (x) C) u is Cm = diag, Ck = diag. */
irk_status irk_apply_op(irk_handle h, const double* u, double* v, int ns,
                        const double* Cm_host, const double* Ck_host);

/* v = calA u with calA = A^{-1} (x) M + tau I (x) K (Eq. irk:A), [Q][stride] FP64; on a group
 * handle every request's [Q][stride] block with its own tau, u and v [R][Q][stride].
 * IRK_EINVAL for NULL u or v. */
irk_status irk_apply(irk_handle h, const double* u, double* v);

/* rhs = (A^{-1} (x) I)(gbar - 1 (x) K y_n) (Eq. irk:A right-hand side) with the
 * built-in source; rhs is [Q][stride] FP64.  IRK_EINVAL for NULL y or rhs and for a group handle. */
irk_status irk_stage_rhs(irk_handle h, const double* y, double t_n, double* rhs);

/* z = P^{-1} r (Eq. irk:P): basis change S~^{-1}, one V-cycle per block in the
 * configured MG precision, basis change S~.  [Q][stride] FP64 in and out ([R][Q][stride] on a
 * group handle, one V-cycle launch sequence over all R Q blocks).
 * IRK_EINVAL for NULL r or z. */
irk_status irk_precondition(irk_handle h, const double* r, double* z);

/* The two basis changes of Eq. (irk:P) around the block V-cycles, on their own (LU variant; the
 * kernels irk_precondition runs, on the caller's buffers):
 *   to_mg:   b = S~^{-1} r in FP64, rounded to the multigrid's element type (float for the FP32
 *            hierarchy, round to nearest with ties to even; double for the FP64 one);
 *            r [Q][stride] FP64, b [Q][stride] of that type;
 *   from_mg: z = S~ x, x [Q][stride] in the multigrid's element type (widened exactly), z
 *            [Q][stride] FP64.
 * stride = irk_level_stride(h, 0).  Asynchronous on the handle's stream.
 * IRK_EINVAL for NULL vectors, a DIAG-variant handle or a group handle. */
irk_status irk_basis_to_mg(irk_handle h, const double* r, void* b);
irk_status irk_basis_from_mg(irk_handle h, const void* x, double* z);

/* Multigrid pieces on level `level` (0 = finest) for all Q LU blocks at once,
 * in the MG precision's element type (float for 32, double for 64):
 *   smooth:    x <- degree-m Chebyshev iteration on (lambda_i M + tau K) x = b
 *              from x (x_is_zero = 1 means start from 0); m = cheb_degree.
 *   residual:  r = b - (lambda_i M + tau K) x
 *   restrict:  b_c = P^T r (level -> level+1, Q_k embedding transposed)
 *   prolongate:x += P e_c (level+1 -> level)
 *   coarse:    x = (lambda_i M_c + tau K_c)^{-1} b on the coarsest level (dense FP64)
 *   vcycle:    x = V-cycle(b) starting from level `level`.
 * Vectors are [Q][level stride] of the level's (k N_l + 1)^d nodes; strides from
 * irk_level_stride.  The V-cycle of Sec. 5 (geometric multigrid, Chebyshev smoother around
 * point-Jacobi) taken apart.  On a group handle the hierarchy holds R Q blocks (block r Q + i is
 * block i of request r, with that request's tau).  IRK_EINVAL for NULL vectors or a level out of range: smooth,
 * restrict and prolongate need level < levels - 1, residual and vcycle level < levels;
 * irk_level_ndofs / irk_level_stride return -1 for a NULL handle or a bad level. */
long long irk_level_ndofs(irk_handle h, int level);
long long irk_level_stride(irk_handle h, int level);
irk_status irk_mg_smooth(irk_handle h, int level, const void* b, void* x, int x_is_zero);
irk_status irk_mg_residual(irk_handle h, int level, const void* b, const void* x, void* r);
irk_status irk_mg_restrict(irk_handle h, int level, const void* r_fine, void* b_coarse);

/* Allocation-free variant of irk_mg_restrict (the paper has no counterpart: this
 * serves callers that cannot allocate device memory at this point, such as a
 * serving process whose whole device budget is already held by request state,
 * or a latency-critical loop where a cudaMalloc/cudaFree, which may synchronise
 * the device, is not acceptable).  Same arguments and result as
 * irk_mg_restrict; the intermediate grids of the axis passes live in one
 * library-owned device array of 24 MiB per device (held by every GPU that loads
 * the library until the process exits) instead of the handle's buffers, and no
 * allocating routine is called.  Like the other irk_mg_* calls it works
 * whatever device is current: the array used is the one on the GPU the handle
 * was created on.  The first call that uses a GPU resolves the array's device
 * address there (making that GPU current for the lookup and restoring the
 * caller's device) and should come before any stream capture; if the lookup
 * fails it returns IRK_ECUDA and irk_last_error says why.  The address is
 * cached for the process: after a cudaDeviceReset of that GPU (which also
 * invalidates every handle created there) the entry point must not be used.
 * Levels needing more than 24 MiB of intermediate grids are rejected with
 * IRK_EINVAL (irk_last_error names the sizes).  Every call shares the array
 * and clears the part it uses; calls that overlap on the GPU race on it and
 * must be serialised by the caller. */
irk_status irk_mg_restrict_noalloc(irk_handle h, int level, const void* r_fine, void* b_coarse);
irk_status irk_mg_prolongate(irk_handle h, int level, const void* e_coarse, void* x_fine);
irk_status irk_mg_coarse_solve(irk_handle h, const void* b, void* x);
irk_status irk_mg_vcycle(irk_handle h, int level, const void* b, void* x);

/* Hierarchy the irk_mg_* calls and irk_get_cheb_interval act on: 0 the LU blocks (default);
 * 1 + i the DIAG variant's block i in irk_get_tableau(J) order: a real block gamma M + tau K
 * (one vector); a 2x2 pair with pair_precond = 0 the PRESB block (alpha + beta) M + tau K (one
 * vector); a 2x2 pair with pair_precond = 1 the coupled system of Sec. 6 (two vectors
 * [2][stride]).  IRK_EINVAL for a block the handle does not have. */
irk_status irk_mg_select(irk_handle h, int which);

/* The generalized mat-vec of Sec. 2, v = (D (x) I) u, D host row-major
 * nout x nin, u [nin][stride], v [nout][stride], FP64.  IRK_EINVAL for NULL
 * pointers or nin / nout outside 1..9. */
irk_status irk_stage_combine(irk_handle h, const double* u, int nin, double* v, int nout,
                             const double* D_host);

/* Wait for the handle's stream; IRK_ECUDA if the stream reports an error. */
irk_status irk_synchronize(irk_handle h);

/* ---- launch accounting (no counterpart in the paper: measurement support) ----
 * Every kernel launch of the handle is counted per category; launches of the
 * categories whose bit is set in `mask` are also bracketed by CUDA events on the
 * handle's stream.  irk_profile resets the counters (after synchronising the
 * stream); irk_profile_read returns, for one category, the summed device time
 * of the timed launches in ms, the number of launches, and the number timed
 * (host pointers; IRK_EINVAL for an unknown category). */
enum {
  IRK_PROF_APPLY64 = 0,   /* FP64-accurate stage-operator kernel of Eq. (irk:A) */
  IRK_PROF_MG_OP = 1,     /* level-operator kernels (Chebyshev steps, residuals), coarser levels */
  IRK_PROF_MG_POINT = 2,  /* first Chebyshev step from zero */
  IRK_PROF_TRANSFER = 3,  /* restriction / prolongation passes */
  IRK_PROF_COARSE = 4,    /* dense coarse-grid solve */
  IRK_PROF_COMBINE = 5,   /* stage combinations and precision casts */
  IRK_PROF_KRYLOV = 6,    /* FGMRES vector kernels */
  IRK_PROF_RHS = 7,       /* K y_n, stage right-hand side, solution update, interpolation */
  IRK_PROF_MG_OP_FINE = 8,  /* level-operator kernels on the finest level */
  IRK_PROF_NCAT = 9
};
irk_status irk_profile(irk_handle h, unsigned mask);
irk_status irk_profile_read(irk_handle h, int category, double* ms, long long* launches, long long* timed);

#ifdef __cplusplus
}
#endif
#endif /* IRK_H_ */
