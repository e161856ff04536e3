/*
 * glls.h - C ABI of the GB300 (sm_103a) GLL spectral-element Poisson solver:
 * outer Krylov (flexible CG) preconditioned by a p-multigrid gamma-cycle with
 * line smoothers solved by cyclic reduction.
 *
 * Paper passages (arXiv 2504.10710):
 *   Sec. 2.2, eq. (discreteBilinear)   stiffness A_p, diagonal mass M_p
 *   Sec. 2.3                            Dirichlet lifting f0 = M f - A v, u = w + v
 *   Def. 3.1, Def. 3.2, Fig. 4          line systems R A_p P, line preconditioners
 *   Algorithm 1, Prop. 3.7, Thm. 3.8,
 *   Cor. 3.9                            cyclic reduction as a direct multigrid
 *   Sec. 3.3, Def. 3.12, Algorithm 2    p-transfers, gamma-cycle, M_0^-1 = A_0^-1
 *   Def. 3.5, Prop. 3.7, Thm. 3.8
 *   (blocks m > 1), Cor. 3.9            block cyclic reduction of the coarsest level
 *
 * Conventions for every entry point:
 *   - Return value: GLLS_OK (0) or a negative glls_status.  The message of the
 *     last error on the calling thread is returned by glls_last_error().  No
 *     call aborts the process or throws across the ABI.
 *   - Nodal vectors use the global lexicographic grid of their level, x
 *     fastest ("left-right, bottom-top", Fig. 4): index = (k*Ny + j)*Nx + i,
 *     with N_a = nelem[a]*p_level + 1 nodes along axis a, boundary included.
 *     Vectors handed to level operations must be zero on the boundary nodes
 *     (the unknowns are the interior nodes; boundary values are Dirichlet).
 *   - "Device" pointers are CUDA global-memory pointers on the problem's device
 *     (e.g. torch tensor data_ptr()); "host" pointers are ordinary memory.  The
 *     caller owns every buffer it passes; the library copies what it keeps.
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Device-pointer
 *     operations are asynchronous on that stream unless stated otherwise.
 *   - Levels are numbered 0 (coarsest: p = 1 when every axis has at least two
 *     elements, else p = 2) to L (finest), with p_{l-1} = floor(p_l / 2).
 */
#ifndef GLLS_H
#define GLLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GLLS_NOT_READY = 1,           /* glls_poll: the request has not finished yet */
    GLLS_OK = 0,
    GLLS_ERR_INVALID = -1,        /* bad argument, size, level or axis */
    GLLS_ERR_OOM = -2,            /* device or host allocation failed */
    GLLS_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    GLLS_ERR_NOT_CONVERGED = -4,  /* max_iter reached; last iterate returned */
    GLLS_ERR_BREAKDOWN = -5,      /* p.Ap <= 0, NaN/Inf, zero pivot, bad Jacobian; a solve that
                                     breaks down clears the problem's work vectors before it
                                     returns, so the next solve starts clean */
    GLLS_ERR_TIMEOUT = -6,
    GLLS_ERR_BUDGET = -7
} glls_status;

/* Precision of a solve:
 *   FP64   everything in FP64;
 *   MIXED  the gamma-cycle in FP32 and, for tol >= 1e-12, the outer apply in
 *          float-float arithmetic (glls_apply_partials_ff); the outer Krylov
 *          vectors, dots and updates stay FP64.  The residuals and directions
 *          must stay inside the FP32 exponent range (about 1e-38 .. 3e38 in
 *          magnitude): data far outside it overflows or underflows in the
 *          cycle and the solve reports GLLS_ERR_BREAKDOWN; scale it, or use
 *          FP64. */
enum { GLLS_PREC_FP64 = 0, GLLS_PREC_MIXED = 1 };
/* Line systems of the line smoother (Def. 3.2):
 *   GLL        the line blocks R A_p P, i.e. every coupling of A_p between two
 *              nodes of the grid line (half-bandwidth p; solved exactly by
 *              condensing each element segment's interior and cyclic reduction
 *              on the element-boundary vertices, Thm. 3.8 / Prop. 3.7 /
 *              Cor. 3.9).  Lines of at most 256 elements and 2047 interior
 *              nodes; on p = 1 levels the block is tridiagonal.
 *   FEM        R A~_p P of the bilinear FEM matrix on the GLL nodes (tridiagonal).
 *   GLL_BAND1  the band-1 part (Def. 3.1, half-bandwidth 1) of the GLL line
 *              blocks: diagonal and neighbour couplings along the line. */
enum { GLLS_SMOOTHER_GLL = 0, GLLS_SMOOTHER_FEM = 1, GLLS_SMOOTHER_GLL_BAND1 = 2 };
enum { GLLS_RESTRICT_TRANSPOSE = 0, GLLS_RESTRICT_INTERP = 1 };
enum { GLLS_KRYLOV_FCG = 0, GLLS_KRYLOV_PCG = 1, GLLS_KRYLOV_GMRES = 2 };
/* Exact solver of the coarsest level (A_0^-1 of Algorithm 2):
 *   AUTO     block cyclic reduction over the blocks of the slowest grid axis
 *            (lines in 2-D, planes in 3-D) to the depth a launch-and-bytes
 *            cost model prefers, then the dense inverse of what is left
 *            (depth 0 = the dense inverse of A_0);
 *   DENSE    the dense inverse of A_0 (one matrix-vector product; at most
 *            16384 interior unknowns, larger systems are refused);
 *   BLOCK_CR coarse_cr_levels levels of block CR (0 = the model's depth, at
 *            least one), clamped to floor(log2(blocks)).
 * Every choice gives A_0^-1 r up to rounding.  AUTO takes at least one level
 * of block CR above 16384 unknowns; block CR stores dense blocks of the
 * slowest axis (lines in 2-D, planes in 3-D) and refuses blocks of more than
 * 2048 unknowns. */
enum { GLLS_COARSE_AUTO = 0, GLLS_COARSE_DENSE = 1, GLLS_COARSE_BLOCK_CR = 2 };
/* Direct stiffness summation of the operator applies (the sum over elements of
 * A = sum_e Q_e^T A_e Q_e, Sec. 2):
 *   ATOMIC   one launch; nodes shared by elements are accumulated with atomic
 *            adds, so their summation order, and with it the last bits of an
 *            FP32 or FP64 result, follows the GPU's scheduling.
 *   COLORED  one launch per element colour (the 2^dim parity classes of the
 *            element coordinates, no two elements of a class share a node)
 *            in a fixed order: every shared node sums its contributions in the
 *            same order on every run.  A solve is then the same bits alone, in
 *            a graph-branch batch and in the serving loop, at the cost of the
 *            node-per-thread apply kernel (not the specialised ones) and 2^dim
 *            launches per apply.  A multi-right-hand-side solve gives each
 *            right-hand side the bits of its single solve (every kernel does
 *            the same arithmetic per right-hand side), so grouped requests in
 *            the serving loop keep them too.  Work-list batches refuse such
 *            problems. */
enum { GLLS_SUM_ATOMIC = 0, GLLS_SUM_COLORED = 1 };

typedef struct glls_problem glls_problem;   /* opaque, library-owned */

/* Mesh of a structured grid of dim-dimensional GLL elements of order `order`.
 * coords: HOST array [dim][N] of physical node coordinates on the fine grid
 * (x-coordinates of all nodes, then y, then z), i.e. the isoparametric map
 * sampled at the GLL nodes (glls_gll gives the reference nodes). */
typedef struct {
    int dim;              /* 2 or 3 */
    int nelem[3];         /* elements along x, y, z (z ignored in 2-D) */
    int order;            /* p >= 1 (p >= 2 for a single element) */
    const double* coords; /* host, [dim][N] */
    int smoother;         /* GLLS_SMOOTHER_* */
    int restriction;      /* GLLS_RESTRICT_* */
    int device;           /* CUDA device ordinal */
    int coarse_solver;    /* GLLS_COARSE_* (0 = AUTO) */
    int coarse_cr_levels; /* block-CR levels for GLLS_COARSE_BLOCK_CR (0 = automatic) */
    int summation;        /* GLLS_SUM_* (0 = ATOMIC) */
} glls_mesh_desc;

typedef struct {
    double tol;      /* stop when ||r_k||_2 <= tol ||r_0||_2 (interior nodes, x0 = 0) */
    int max_iter;    /* outer iterations */
    int gamma;       /* coarse visits per level visit, >= 1 (Algorithm 2) */
    int m;           /* smoothing steps per direction, >= 1 */
    double alpha;    /* damping of the line smoothing step */
    int precision;   /* GLLS_PREC_FP64 or GLLS_PREC_MIXED */
    int krylov;      /* GLLS_KRYLOV_FCG (Polak-Ribiere beta), _PCG (Fletcher-Reeves), or _GMRES:
                        right-preconditioned flexible GMRES without restart, the paper's outer
                        solver (Sec. 3), at most min(max_iter, 400) steps, host-driven loop;
                        its residual test is the Arnoldi least-squares estimate */
    int use_graph;   /* 0: host loop, kernels launched per iteration;
                        1: host loop, each outer iteration replayed as a captured CUDA graph;
                        2: the whole solve as one captured graph whose outer loop is a
                           device-side conditional WHILE node (one host synchronisation) */
    int check_every; /* host loops (use_graph 0/1): read the residual back every k iterations */
} glls_solve_opts;

typedef struct {
    int iterations;
    double rel_residual;
    double setup_ms;
    double solve_ms;
    int status;
    long long kernels;   /* kernels this solve launched (graph kernel nodes x loop trips) */
    double queue_ms;     /* served requests: submission to the start of their work (else 0) */
    int setup_kind;      /* served requests: 0 resident instance, 1 mesh set up for it, 2 clone made for it */
    int group;           /* served requests: requests solved together with it, itself included (else 0) */
} glls_stats;

typedef struct {
    int dim, levels;            /* number of levels L + 1 */
    int order[8];               /* p per level, index 0 = coarsest */
    int nodes[8][3];            /* nodes per axis per level */
    long long ndof[8];          /* total nodes per level */
    long long coarse_unknowns;  /* interior unknowns of level 0 */
    size_t device_bytes;        /* device memory held by the problem */
    int coarse_cr_levels;       /* block-CR levels of the coarsest solve (0 = dense inverse) */
    long long coarse_dense_unknowns;   /* size of the densely inverted system */
    size_t instance_bytes;      /* device memory this instance owns alone: what a clone adds */
    int nrhs;                   /* right-hand sides solved together (glls_problem_create_nrhs) */
    double setup_phase_ms[6];   /* set-up wall time by phase: coarse-level coordinates, geometry
                                   factors, line data (bands, line blocks), transfers, coarsest-level
                                   factorisation (all host), device upload and allocation */
} glls_info;

/* Reference GLL(p) nodes and weights (Def. 2.1); xi, rho: host arrays of p+1. */
glls_status glls_gll(int p, double* xi, double* rho);

/* Build every level: geometry factors, line bands, CR-ready data, transfers and
 * the coarsest-level factor, and upload them to the device.  Synchronous. */
glls_status glls_problem_create(const glls_mesh_desc* desc, glls_problem** out);
/* As glls_problem_create, with nrhs >= 1 right-hand sides solved together:
 * glls_set_rhs takes nrhs x N values ([nrhs][N], right-hand side j at j N),
 * glls_set_dirichlet one N-vector shared by all, and glls_solve writes nrhs x
 * N values into u and fills stats[0 .. nrhs-1].  Every kernel of the solve
 * processes all right-hand sides in one launch with the right-hand side
 * fastest in its CTA order, so the mesh data (geometry factors, line blocks,
 * coarsest-level operators) is read from HBM about once per launch for all
 * of them.  Each right-hand side has its own flexible-CG scalars and stops
 * on its own (converged or broken down) while the others continue; the
 * call returns the worst status.  Solves with nrhs > 1 run as one graph with
 * a device-side loop (use_graph = 2) with FCG or PCG; level operations act
 * on a single vector as for nrhs = 1.  (Multi-RHS block CR: Thm. 3.8 with
 * the block products applied to all right-hand sides of a launch.) */
glls_status glls_problem_create_nrhs(const glls_mesh_desc* desc, int nrhs, glls_problem** out);
/* A second problem on the same mesh: it shares every read-only device array of
 * prob (geometry factors, line bands, transfers, coarsest inverse, mass; held
 * until the last of them is destroyed) and owns its own right-hand side,
 * Dirichlet data and Krylov state.  Several right-hand sides of one mesh are
 * solved together as clones in one glls_solve_batch.  Autotuned tiles are
 * copied.  Synchronous. */
glls_status glls_problem_clone(const glls_problem* prob, glls_problem** out);
/* As glls_problem_clone, with nrhs right-hand sides solved together (as
 * glls_problem_create_nrhs) whatever the count of prob. */
glls_status glls_problem_clone_nrhs(const glls_problem* prob, int nrhs, glls_problem** out);
void glls_problem_destroy(glls_problem* prob);
/* Failure injection for tests (no counterpart in the paper): after n more
 * device allocations by the library, further ones fail as if the device were
 * out of memory (the calls report GLLS_ERR_OOM and free what they had
 * allocated); n < 0 turns it off.  Process-wide. */
void glls_debug_fail_alloc_after(long long n);
glls_status glls_problem_info(const glls_problem* prob, glls_info* out);

/* Dirichlet data g (N fine-grid values; only boundary entries are read) and
 * right-hand side f (N nodal values; M f is formed inside).  on_device selects
 * how the pointer is read; with on_device = 0 the copy is synchronous. */
glls_status glls_set_dirichlet(glls_problem* prob, const double* g, int on_device, void* stream);
glls_status glls_set_rhs(glls_problem* prob, const double* f, int on_device, void* stream);

/* Solve A u = M f with u = g on the boundary (Sec. 2.3): lifting, outer Krylov
 * to opts->tol, u = w + v.  u: N values (device or host per on_device).  Host
 * output makes the call synchronous.  Returns GLLS_ERR_NOT_CONVERGED (u holds
 * the last iterate) or GLLS_ERR_BREAKDOWN; stats may be NULL. */
glls_status glls_solve(glls_problem* prob, const glls_solve_opts* opts, double* u, int on_device,
                       void* stream, glls_stats* stats);

/* Solve several independent problems (any sizes, orders, dimensions, on one
 * device) together: one graph launch whose parallel branches are the
 * problems' whole solves, each with its own device-side loop; their kernels
 * overlap on the GPU.  u[i]: N_i values per problem (device or host per
 * on_device); stats: n entries or NULL.  The graph is cached per (problem
 * list, options).  Returns GLLS_OK if every problem converged, else the
 * first failure status (per-problem status in stats[i].status). */
glls_status glls_solve_batch(glls_problem* const* probs, int n, const glls_solve_opts* opts, double* const* u,
                             int on_device, void* stream, glls_stats* stats);
/* The same batched solve with work-list kernels (the batched form of the
 * solve loop): the problems are grouped by their chain of orders, and inside
 * a group every step of the outer iteration (each apply, line solve,
 * transfer, coarsest-solve step and outer-Krylov kernel) is one launch over
 * a work list whose items are (problem, level, tile range): item j carries
 * problem j's level data and vectors and owns a contiguous range of the
 * launch's CTAs.  Each group is one branch of one graph with its own
 * device-side loop that runs while any of its problems is active; a
 * problem that has stopped keeps its iterate.  The launch covers every
 * problem whatever its element count, so a step costs one launch per group
 * instead of one per problem.  Requirements: 2-D, one right-hand side per
 * problem, the GLL line-block smoother, orders up to 16, FCG or PCG
 * (GLLS_ERR_INVALID otherwise).  The plan (item arrays and graph) is cached
 * per problem list and options and released with its problems.  stats[0].kernels
 * holds the kernels of the whole launch. */
glls_status glls_solve_batch_worklist(glls_problem* const* probs, int n, const glls_solve_opts* opts,
                                      double* const* u, int on_device, void* stream, glls_stats* stats);

/* Autotuner: for every level >= 1, precision and direction, time the line
 * solve on the problem's own data with each candidate number of lines per
 * CTA and keep the fastest: for the Def. 3.2 line blocks (GLL smoother)
 * 1, 2, 4, 8, 16 (at most 256 element segments per CTA) or 0, the launch
 * heuristic; for the band-1 and FEM line kernels 2, 4, 8 and (FP32 only) 16.
 * chosen / best_us (optional): levels x 2 (FP32, FP64) x 3 entries,
 * index (level * 2 + precision) * 3 + axis, the chosen value and its time in
 * microseconds per launch.  Cached graphs are rebuilt on the next solve.
 * Synchronous. */
glls_status glls_autotune(glls_problem* prob, int* chosen, float* best_us);

/* Device bytes glls_problem_create would allocate for desc (estimate used for
 * admission by an HBM budget; no allocation, no device work). */
glls_status glls_estimate_bytes(const glls_mesh_desc* desc, size_t* bytes);

/* ---- serving: a request loop with admission by HBM budget ----------------
 * A server owns `slots` worker threads, each with its own CUDA stream, and a
 * cache of resident problems (meshes with their geometry factors, line data
 * and Krylov state) keyed by the mesh.  Requests are admitted in arrival
 * order as soon as a slot is free and the resident bytes plus the request's
 * estimate fit the budget (idle cached meshes are evicted, least recently
 * used first).  A request for a resident mesh runs on an idle instance of it;
 * when every instance is busy it runs on a new clone (glls_problem_clone:
 * the mesh data is shared, the clone adds its instance_bytes) if those bytes
 * fit, else it waits for an instance while later requests go ahead.  Admitted
 * requests run concurrently on the device.  A request whose estimate exceeds
 * the whole budget fails with GLLS_ERR_BUDGET. */
typedef struct glls_server glls_server;
typedef struct {
    unsigned long long submitted, completed, failed, queued, running;
    size_t resident_bytes, budget_bytes;
    int cached_problems;         /* resident meshes */
    int cached_instances;        /* their instances (set-up problems and clones) */
    unsigned long long clones;   /* clones created so far */
    unsigned long long grouped;  /* requests served by multi-right-hand-side solves */
} glls_server_info;

glls_status glls_server_create(int device, size_t hbm_budget_bytes, int slots, glls_server** out);
/* Waits for running requests, then frees every cached problem. */
void glls_server_destroy(glls_server* server);
/* Queue one solve.  mesh (with its coords), f and g (N host values each; g may
 * be NULL for homogeneous data) are copied; u (N host values) is written when
 * the request completes and must stay valid until then.  Returns a ticket. */
glls_status glls_submit(glls_server* server, const glls_mesh_desc* mesh, const double* f, const double* g,
                        const glls_solve_opts* opts, double* u, unsigned long long* ticket);
/* Registers a mesh with the server (its coordinates are copied and keyed
 * once) and returns an id for glls_submit_mesh; nothing is set up until the
 * first request on it runs.  Registered meshes stay known until the server
 * is destroyed (their device data is still subject to eviction). */
glls_status glls_server_register(glls_server* server, const glls_mesh_desc* mesh, unsigned long long* mesh_id);
/* As glls_submit, on a registered mesh, without copying: f and g (N host
 * values each; g may be NULL) are read when the request runs, so they stay
 * valid and unchanged, like u, until its ticket is polled to completion or
 * cancelled. */
glls_status glls_submit_mesh(glls_server* server, unsigned long long mesh_id, const double* f, const double* g,
                             const glls_solve_opts* opts, double* u, unsigned long long* ticket);
/* GLLS_NOT_READY while queued or running (wait = 0), else the request's
 * status with stats filled: stats->solve_ms is the request's latency
 * (submission to result in u: queue, any set-up and the solve),
 * stats->queue_ms the part before a worker took it, stats->setup_ms and
 * stats->setup_kind the set-up or clone done for it; wait = 1 blocks until done.  A
 * finished ticket is released by the first poll that returns its result. */
glls_status glls_poll(glls_server* server, unsigned long long ticket, int wait, glls_stats* stats);
glls_status glls_server_info_get(glls_server* server, glls_server_info* out);
/* Grouping (default 1: off).  With max_group > 1 a worker that takes a
 * request for a resident mesh also takes the queued requests of that mesh
 * with the same Dirichlet data pointer and options, up to the largest power
 * of two <= max_group available, and solves them together on an instance
 * with that many right-hand sides (glls_problem_clone_nrhs), so the mesh
 * data is read once per kernel launch for all of them.  Only requests with
 * use_graph = 2 and FCG or PCG are grouped.  Each request still gets its own
 * solution, status and stats (stats->group = the group size). */
glls_status glls_server_set_max_group(glls_server* server, int max_group);
/* Removes a request that is still queued: GLLS_OK (its ticket is released and
 * u is never written), GLLS_NOT_READY if it is already running, or
 * GLLS_ERR_INVALID for an unknown or released ticket. */
glls_status glls_cancel(glls_server* server, unsigned long long ticket);

/* ---- level operations on device vectors (parity tests, custom drivers) ----
 * Each exists as _f64 and _f32; the FP32 variant uses the FP32 copies of the
 * level data (the mixed-precision gamma-cycle). */

/* y = A_l x on interior rows (boundary rows of y set to 0), eq. (discreteBilinear). */
/* The FP64 apply as the outer iteration launches it (Sec. 2.2; the p.Ap of
 * flexible CG fused): y += A_l x on interior rows, and `partials` (device,
 * `capacity` doubles) receives the per-CTA partial sums of x.(A x), whose sum
 * is x.(A x) for x zero on the boundary.  y must be zero on entry (element-
 * boundary rows are accumulated); *count (host) is set to the number of
 * partials, and GLLS_ERR_INVALID is returned without device work when
 * capacity is smaller. */
glls_status glls_apply_partials_f64(glls_problem* prob, int level, const double* x, double* y, double* partials,
                                    int capacity, int* count, void* stream);
/* The same product and partials computed in float-float arithmetic (each
 * value a pair of FP32 numbers, about 48 significant bits: Knuth's two-sum and
 * the FMA exact product), as the mixed-precision solve's outer iteration runs
 * it for solves with tol >= 1e-12 (GB300 runs FP32 at 64 times its FP64
 * rate).  x and y are FP64 as above; the relative rounding is near 2^-44 per
 * contraction instead of 2^-53.  Only the finest level of a problem with
 * 2 <= p <= 16 (2-D) or 2 <= p <= 8 (3-D, even-odd line sweeps) and
 * GLLS_SUM_ATOMIC (else GLLS_ERR_INVALID without device work); *count is this
 * kernel's partial count (in 2-D the same as glls_apply_partials_f64's). */
glls_status glls_apply_partials_ff(glls_problem* prob, int level, const double* x, double* y, double* partials,
                                   int capacity, int* count, void* stream);
glls_status glls_apply_f64(glls_problem* prob, int level, const double* x, double* y, void* stream);
glls_status glls_apply_f32(glls_problem* prob, int level, const float* x, float* y, void* stream);
/* y = A_l x for nrhs vectors at once (x, y: nrhs x N_l values, vector j at
 * j N_l), in one launch with the vector fastest in the CTA order, so the
 * geometry factors of each element are read from HBM once for all nrhs
 * (the multi-right-hand-side apply of the solve). */
glls_status glls_apply_multi_f64(glls_problem* prob, int level, const double* x, double* y, int nrhs, void* stream);
glls_status glls_apply_multi_f32(glls_problem* prob, int level, const float* x, float* y, int nrhs, void* stream);

/* x = B_s^-1 g: every interior grid line along axis s solved by cyclic
 * reduction (Def. 3.2, Cor. 3.9); x is written on interior nodes only.  The
 * FP32 variant takes each pivot's reciprocal from the hardware approximation
 * (at most 1 ulp from the rounded quotient). */
glls_status glls_line_solve_f64(glls_problem* prob, int level, int axis, const double* g, double* x, void* stream);
glls_status glls_line_solve_f32(glls_problem* prob, int level, int axis, const float* g, float* x, void* stream);

/* The line update of a smoothing step alone (Def. 3.2, Algorithm 2), as the
 * gamma-cycle launches it after y = A_l x: x += alpha B_s^-1 (r - y) on
 * interior nodes.  y is consumed: its element-boundary entries are reset to
 * 0 (the accumulating apply needs them zero), its other entries are left. */
glls_status glls_line_update_f64(glls_problem* prob, int level, int axis, double alpha, const double* r, double* y,
                                 double* x, void* stream);
glls_status glls_line_update_f32(glls_problem* prob, int level, int axis, float alpha, const float* r, float* y,
                                 float* x, void* stream);
/* One damped line-smoothing step x <- x + alpha B_s^-1 (r - A_l x) (Algorithm 2). */
glls_status glls_smooth_f64(glls_problem* prob, int level, int axis, double alpha, const double* r, double* x, void* stream);
glls_status glls_smooth_f32(glls_problem* prob, int level, int axis, float alpha, const float* r, float* x, void* stream);

/* rc = R_l (r - A_l x) on level l-1 (coarse boundary rows 0), Sec. 3.3. level >= 1. */
glls_status glls_restrict_f64(glls_problem* prob, int level, const double* r, const double* x, double* rc, void* stream);
glls_status glls_restrict_f32(glls_problem* prob, int level, const float* r, const float* x, float* rc, void* stream);

/* x += P_l e, e on level l-1, x on level l (Sec. 3.3). level >= 1. */
glls_status glls_prolong_add_f64(glls_problem* prob, int level, const double* e, double* x, void* stream);
glls_status glls_prolong_add_f32(glls_problem* prob, int level, const float* e, float* x, void* stream);

/* e = A_0^-1 r on the coarsest level (M_0^-1 of Algorithm 2). */
glls_status glls_coarse_solve_f64(glls_problem* prob, const double* r, double* e, void* stream);
glls_status glls_coarse_solve_f32(glls_problem* prob, const float* r, float* e, void* stream);

/* z = M_L^-1 r: one gamma-cycle on the finest level (Algorithm 2, x0 = 0),
 * using opts->gamma, opts->m, opts->alpha. */
glls_status glls_precondition_f64(glls_problem* prob, const glls_solve_opts* opts, const double* r, double* z, void* stream);
glls_status glls_precondition_f32(glls_problem* prob, const glls_solve_opts* opts, const float* r, float* z, void* stream);

/* f0 = M f - A v on interior nodes (0 on the boundary), v = g on the boundary
 * and 0 inside (Sec. 2.3); f, g, f0: fine-grid device vectors. */
glls_status glls_lift_f64(glls_problem* prob, const double* f, const double* g, double* f0, void* stream);

/* rc = R_l (r - A_l x), like glls_restrict_f32, for callers that cannot
 * call cudaMalloc: code running under an external allocator that owns all
 * device memory (a framework's caching pool sized to the whole GPU), or on a
 * path that must not pay cudaMalloc's cost and implicit synchronisation
 * between steps.  This entry point allocates nothing and does not
 * use the problem's own scratch: the apply result and the transfer
 * temporaries live in one fixed library-wide device array of 3 x 262,144
 * floats (3 MiB), which every GPU that loads the library holds until the
 * process exits.  It has no counterpart in the paper.
 *   - Level l must have at most 262,144 nodes; larger levels return
 *     GLLS_ERR_INVALID with the limit in the message.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - Every call shares the array and leaves its contents behind; each call
 *     clears what must start at zero.  Calls that overlap on the GPU (other
 *     streams, concurrent graphs) race on the array and must be serialised.
 * Arguments as glls_restrict_f32 (device vectors, asynchronous on stream). */
glls_status glls_restrict_noalloc_f32(glls_problem* prob, int level, const float* r, const float* x, float* rc,
                                      void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* glls_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GLLS_H */
