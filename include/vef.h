/*
 * vef.h -- C ABI of the GB300 DG S_N transport sweep and VEF closure library (libvef.so).
 *
 * The library computes, on one CUDA GPU, the data-parallel hot path of the Variable
 * Eddington Factor (VEF) fixed-point iteration of Olivier & Haut, "High-Order Mixed
 * Finite Element Variable Eddington Factor Methods":
 *   - the inversion of the streaming-plus-collision operator of the discrete-ordinates
 *     transport equation (paper Eq. transport with boundary condition Eq. trans_bc)
 *     discretised with the DG space Y_p on curved Q_m quadrilaterals (paper Sec.
 *     "Transport Discretizations", "Discontinuous Galerkin", "Description of the Mesh");
 *   - the angular moments and VEF closures, scalar flux phi, current J, Eddington
 *     tensor E and boundary factor E_b (paper Eq. vef_disc) and the inflow partial
 *     current J_in (paper, the definitions following Eq. mlbc);
 *   - source iteration (paper Sec. "VEF Algorithm", the fixed-point loop) and an
 *     adjoint sweep giving cross-section gradients (not in the paper).
 *
 * Discretisation (the paper defers the sweep's weak form to its transport solver; this
 * library fixes it as follows).  Per direction Omega_d and element K, find psi in Q_p(K):
 *     - int_K psi (Omega.grad v) + int_dK (Omega.n) psi_hat v + int_K sigma_t psi v
 *         = int_K (sigma_s phi_in / (4 pi) + q_d) v        for all v in Q_p(K),
 * psi_hat = interior trace where Omega.n >= 0, else the upwind neighbour's trace or
 * the inflow data psi_bar, decided pointwise at every face quadrature point.
 * Basis: tensor Lagrange at the (p+1)^2 Gauss-Lobatto points of the reference square,
 * local dof a + (p+1) b.  Quadrature: tensor Gauss-Legendre with nq = p+2 points per
 * direction; faces use the same nq-point rule.  Mesh: nx x ny structured elements of
 * [0,1]^2, element e = j*nx + i, Q_m map through (m+1)^2 Gauss-Lobatto control points.
 * Faces: 0 bottom, 1 right, 2 top, 3 left; face points in increasing reference
 * coordinate.  Boundary faces (N_bf = 2 nx + 2 ny): bottom row (i = 0..nx-1), right
 * column (j = 0..ny-1), top row (i), left column (j).
 *
 * A sweep returns psi_d = L_d^{-1} b_d for every direction, independent of any
 * ordering: the library orders elements per direction along the upwind dependency
 * graph (one thread-block cluster per direction walks its levels) and solves the rare
 * strongly coupled element groups (curved faces that are partly inflow and partly
 * outflow) as units: directly, through the dense system for the face traces the
 * group's elements exchange (its inverse is formed with the element factorisations;
 * groups of up to 32 elements for p <= 2, 16 for p >= 3, and up to 128 trace values),
 * else by an inner block Gauss-Seidel iteration to a relative change below
 * `vef_opts.tol`.
 *
 * Conventions
 *   - Array arguments marked [device] are caller-owned device memory: contiguous FP64,
 *     on the current device, in the layouts stated.  Arguments marked [host] are
 *     caller-owned host memory read during the call.
 *   - Calls are stream-ordered on `stream` (NULL = legacy default stream) and
 *     asynchronous, except where a call states that it synchronises.
 *   - A mesh handle owns device memory (geometry, schedules, scratch).  Calls that use
 *     the same handle must not overlap on the GPU: issue them on one stream or
 *     serialise them.
 *   - The status returned covers argument validation and launch.  Failures detected
 *     on the device (an inner iteration that did not converge, a singular local
 *     system, a non-positive closure denominator) are recorded in the handle and are
 *     returned by the next call that synchronises: vef_mesh_sync(), or any call given
 *     a non-NULL vef_info.
 *   - No exceptions cross the ABI.  There is no CPU fallback: without a usable CUDA
 *     device every compute call returns VEF_ERR_CUDA.
 */
#ifndef VEF_H
#define VEF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VEF_OK = 0,
  VEF_ERR_INVALID_ARG = 1,
  VEF_ERR_CUDA = 2,
  VEF_ERR_OOM = 3,
  VEF_ERR_TIMEOUT = 4,            /* a bounded device-side wait (staging copy) gave up */
  VEF_ERR_NOT_CONVERGED = 5,      /* an inner or defect-correction iteration hit its cap */
  VEF_ERR_NONPOSITIVE_DENOM = 6,  /* sum_d w_d psi_d <= 1e-300 at a closure point (NaN written) */
  VEF_ERR_NOT_IMPLEMENTED = 7,
  VEF_ERR_BOUNDS = 8              /* bounds-checked build only: a kernel met an index outside its
                                     array (the access was skipped; results are undefined) */
} vef_status;

enum { VEF_FP64 = 0, VEF_MIXED = 1 };

/* vef_opts.flags */
enum {
  VEF_GROUPS_ITERATIVE = 1, /* solve every coupled group by the inner iteration */
  VEF_SWEEP_CLUSTER = 2,    /* sweep each direction (forward or adjoint) with a
                               thread-block cluster, as the batched sweep does, instead of
                               one CTA */
  VEF_APPLY_SEPARATE = 4,   /* compute y = A^{-1} b by a launch of its own before the
                               single-CTA sweep (always so for p >= 3, whose A^{-1} reads
                               the free SMs alone cannot stream fast enough); by default,
                               for p <= 2, the SMs the directions leave free do it inside
                               the sweep launch, which is then a
                               cooperative launch sized from the device's SM count (a
                               context limited to fewer SMs, e.g. under MPS, should set
                               this flag: the CUDA driver refuses a cooperative grid that
                               does not fit, and the call returns VEF_ERR_CUDA) */
  VEF_PIVOT_ALWAYS = 8,     /* refactorise every (element, direction) system with partial
                               pivoting, as the library does by itself only for the systems
                               whose unpivoted elimination meets a small pivot (see
                               VEF_PIVOT_FLOOR_LOG2_FP64); slow, meant for testing */
  VEF_REUSE_FACTORS = 16,   /* keep the local factorisation of the previous call with this
                               mesh and direction set in this precision instead of forming it
                               again (vef_sweep, vef_source_iterate, vef_batch_sweep): the
                               caller guarantees sigma_t is unchanged, as in the outer
                               iterations of the VEF method, where only the scattering
                               source changes.  Without a previous factorisation the call
                               factorises as usual. */
  VEF_CKPT_FP32 = 32        /* vef_adjoint_sweep: psi_ckpt points to an FP32 copy of the
                               forward psi (float [D][E][n], half the memory of the FP64
                               checkpoint); the gradients then carry its rounding, about
                               1e-7 relative */
};

typedef struct vef_mesh_s* vef_mesh;

/* Pivot guard of the element solves.  Each (element, direction) system is inverted by
 * Gauss-Jordan elimination without pivoting; a system whose pivot at some step is zero, not
 * finite, or below 2^VEF_PIVOT_FLOOR_LOG2_FP64 (FP64 solves) / 2^VEF_PIVOT_FLOOR_LOG2_FP32
 * (FP32 solves) times the largest entry of that row of the assembled matrix is inverted
 * again with partial pivoting.  vef_info.pivoted_tasks reports how many were.  (Over the
 * level-symmetric sets S4..S16, p = 1..4, void to optically thick elements and sine-curved
 * meshes up to alpha = 0.1 the smallest such ratio is about 0.1.) */
#define VEF_PIVOT_FLOOR_LOG2_FP64 (-33)
#define VEF_PIVOT_FLOOR_LOG2_FP32 (-13)

/* Environment: VEF_TRACE_SLOTS=<k>, read when a schedule is built (the first sweep of a
 * mesh with a given direction set), caps the shared-memory trace slots of the single-CTA
 * sweeps at k; the couplings left over are read from global memory.  Meant for testing
 * that path; results do not depend on it. */

/* Sweep options.  NULL means the defaults listed. */
typedef struct {
  int precision;     /* VEF_FP64 (default): FP64 assembly and solves.
                        VEF_MIXED: FP32 assembly and solves inside an FP64
                        defect-correction loop r = b - L psi (FP64), psi += L32^{-1} r.
                        vef_sweep forms r matrix-free from the element's M, Gx, Gy and
                        its face terms; vef_source_iterate stores the FP64 element
                        systems once and reuses them for the residuals of its K
                        inversions. */
  double tol;        /* relative tolerance: inner coupled-group iteration (FP64: 1e-15) and
                        defect correction ||r||_2 / ||b||_2 (mixed: 1e-13).
                        tol < 0 with VEF_MIXED: a fixed number of passes instead, exactly
                        max_passes sweeps (default 2) with an FP64 residual between
                        consecutive ones and none after the last, and no host
                        synchronisation inside the call; vef_info.rel_residual then
                        reports the residual the last correction started from */
  int max_passes;    /* cap on defect-correction passes (default 8) and, x4, on inner
                        coupled-group iterations */
  int tile_override; /* 0 = library choice; else 100 * (CTAs per direction cluster, 1..16)
                        + (warps per CTA, 1..16) of the cluster sweep kernel (implies
                        VEF_SWEEP_CLUSTER) */
  int flags;         /* bit set of VEF_GROUPS_ITERATIVE, VEF_SWEEP_CLUSTER,
                        VEF_APPLY_SEPARATE, VEF_PIVOT_ALWAYS (default 0: direct group
                        solves, one CTA per direction, fused apply, pivoting only where
                        the guard asks for it) */
} vef_opts;

/* Filled by calls given a non-NULL pointer (those calls synchronise `stream`). */
typedef struct {
  int passes;                 /* sweeps executed (1 for FP64; 1 + corrections for mixed) */
  double rel_residual;        /* mixed: final ||b - L psi||_2 / ||b||_2 (FP64 path: -1) */
  long long coupled_groups;   /* (element group, direction) tasks with more than one element */
  long long lagged_face_points; /* inflow face points between elements of one coupled group */
  int max_inner_iterations;   /* largest inner Gauss-Seidel count used by a coupled group
                                 (0 when every group was solved directly) */
  int timed_out;              /* 1 if a bounded device-side wait gave up */
  int levels;                 /* dependency levels of the schedule (critical path length) */
  long long pivoted_tasks;    /* element systems of the last factorisation inverted with
                                 partial pivoting (see VEF_PIVOT_FLOOR_LOG2_FP64) */
} vef_info;

/* Mesh description returned by vef_mesh_query. */
typedef struct {
  int nx, ny, mesh_order, p;
  int n;          /* (p+1)^2 dofs per element */
  int nq;         /* p+2 quadrature points per direction */
  long long E;    /* nx*ny */
  long long nbf;  /* 2 nx + 2 ny boundary faces */
} vef_mesh_desc;

/* Create a mesh of [0,1]^2 with nx x ny elements, map order mesh_order (1..4), DG
 * order p (1..4) and sine distortion amplitude alpha (paper Sec. "Solver Performance on
 * Curved Meshes": x -> x + alpha sin(2 pi x) sin(2 pi y) (1,1)) applied to the
 * Gauss-Lobatto control points (paper Sec. "Description of the Mesh").
 * ctrl_pts: [host] optional [E][(m+1)^2][2] control points (replaces the generated
 * ones; alpha is then ignored).  Computes the geometric factors on the device.
 * Synchronises the current device's legacy stream.  *out receives the handle. */
vef_status vef_mesh_create(int nx, int ny, int mesh_order, int p, double alpha,
                           const double* ctrl_pts, vef_mesh* out);
vef_status vef_mesh_destroy(vef_mesh mesh);
vef_status vef_mesh_query(vef_mesh mesh, vef_mesh_desc* out);
/* Waits for the handle's work on `stream` and returns (then clears) the first
 * device-side failure recorded since the last check. */
vef_status vef_mesh_sync(vef_mesh mesh, void* stream);

/* One transport inversion for every direction (paper Eq. transport, trans_bc):
 *   sigma_t, sigma_s [device] [E] per-element cross sections (sigma_t > 0);
 *   phi_in  [device] [E][n] scattering scalar flux (DG nodal values) or NULL (= 0);
 *   source  [device] [E][n] isotropic q per steradian, or [D][E][n] when
 *           source_aniso != 0; NULL = 0;
 *   inflow  [device] [D][N_bf][nq] psi_bar at the boundary face points; only values
 *           at inflow points (Omega.n < 0) are read; NULL = vacuum;
 *   omega   [host] [D][2] direction cosines (mu, eta); weights [host] [D] (not used
 *           by the sweep itself; validated and kept for the moment calls);
 *   psi     [device] [D][E][n] output.
 * The first call with a given direction set builds its schedule on the host (this
 * synchronises `stream`; do it before any stream capture). */
vef_status vef_sweep(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                     const double* phi_in, const double* source, int source_aniso,
                     const double* inflow, const double* omega, const double* weights, int D,
                     const vef_opts* opts, double* psi, vef_info* info, void* stream);

/* Moments and closures (paper Eq. vef_disc and the definitions of E, E_b, J_in):
 *   psi [device] [D][E][n]; omega, weights [host] as for vef_sweep;
 *   inflow [device] [D][N_bf][nq] or NULL (then Jin is set to 0);
 * outputs, each [device] and optional (NULL = skip):
 *   phi [E][n], J [2][E][n] (x, y), P [3][E][n] (xx, xy, yy) as DG nodal values;
 *   Eten [3][E][nq*nq] = P/phi at the volume quadrature points (point k1 + nq k2);
 *   Eb [N_bf][nq] = sum w |Omega.n_hat| psi / sum w psi with the interior trace;
 *   Jin [N_bf][nq] = sum_{Omega.n<0} w (Omega.n_hat) psi_bar.
 * All sums are accumulated in FP64.  A denominator <= 1e-300 writes NaN and records
 * VEF_ERR_NONPOSITIVE_DENOM. */
vef_status vef_moments(vef_mesh mesh, const double* psi, const double* omega,
                       const double* weights, int D, const double* inflow, double* phi,
                       double* J, double* P, double* Eten, double* Eb, double* Jin,
                       void* stream);

/* Source iteration (paper Sec. "VEF Algorithm", fixed-point loop): phi^0 = phi0
 * ([device] [E][n], NULL = 0), then K times psi = sweep(phi^k), phi^{k+1} = sum_d w_d psi_d.
 * phi_out [device] [E][n] receives phi^K; psi [device] [D][E][n] the last sweep
 * (required); dphi_inf [device] [K] receives max |phi^{k+1} - phi^k| (optional). */
vef_status vef_source_iterate(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                              const double* phi0, const double* source, int source_aniso,
                              const double* inflow, const double* omega, const double* weights,
                              int D, int K, const vef_opts* opts, double* phi_out, double* psi,
                              double* dphi_inf, vef_info* info, void* stream);

/* g [device] [E][n] such that sum_{e,j} g[e][j] phi[e][j] = int over the box
 * [x0,x1] x [y0,y1] of phi dx, for phi given by its DG nodal values; the box indicator
 * is evaluated at the volume Gauss points (its integral is exact for elements inside or
 * outside the box).  The right-hand side of vef_adjoint_sweep for a region functional. */
vef_status vef_region_weights(vef_mesh mesh, double x0, double y0, double x1, double y1, double* g,
                              void* stream);

/* Adjoint sweep for R = sum_{e,j} g[e][j] phi[e][j] of one transport inversion with fixed
 * phi_in: solves L_d^T lambda_d = w_d g (directions reversed: downwind order), then
 *   dR_dsigma_t[e] = - sum_d lambda_{d,e}^T M_e psi_{d,e},
 *   dR_dsigma_s[e] =   sum_d lambda_{d,e}^T M_e phi_in,e / (4 pi)
 * with M_e the element mass matrix.  psi_ckpt [device] [D][E][n] is the forward sweep's
 * psi (checkpoint; FP64, or FP32 with VEF_CKPT_FP32 in opts->flags, read as const float*);
 * g [device] [E][n]; lambda [device] [D][E][n] output or NULL (then a
 * library buffer is used); dR_dsigma_t, dR_dsigma_s [device] [E] outputs.  opts: tol and
 * max_passes bound the inner iteration of coupled groups beyond the direct limits;
 * VEF_SWEEP_CLUSTER or a tile_override selects the cluster form of the backward sweep
 * (default: one CTA per direction with the forward sweep's shared-memory slots). */
vef_status vef_adjoint_sweep(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                             const double* phi_in, const double* omega, const double* weights,
                             int D, const double* psi_ckpt, const double* g, double* lambda,
                             double* dR_dsigma_t, double* dR_dsigma_s, const vef_opts* opts,
                             vef_info* info, void* stream);

/* Batches of independent problems (uneven mesh sizes, DG orders and direction sets).
 * Each problem has its own mesh handle (distinct handles); the batch fixes each problem's direction set
 * (omega[k] [host] [D[k]][2], weights[k] [host] [D[k]]) and builds its schedule.  One
 * vef_batch_sweep call runs, per problem, the dependency-free kernels (right-hand side,
 * local factorisation unless VEF_REUSE_FACTORS, apply), then one launch per DG order sweeps
 * every (problem, direction) of that order: one CTA per (problem, direction) with the
 * single-CTA sweep, largest problems first, or one cluster per (problem, direction) when
 * the tuner or opts->tile_override chose a cluster shape.  FP64 only.  No device
 * synchronisation unless info is given, so a call can be captured in a CUDA graph after a
 * first (allocating) call. */
typedef struct vef_batch_s* vef_batch;
vef_status vef_batch_create(const vef_mesh* meshes, int nprob, const double* const* omega,
                            const double* const* weights, const int* D, vef_batch* out);
vef_status vef_batch_destroy(vef_batch batch);
/* Per-problem arrays of [device] pointers, layouts as in vef_sweep (isotropic source,
 * entries of phi_in / source / inflow may be NULL, and so may these arrays).  The
 * per-problem kernel arguments live in a pinned host table that each call rewrites and
 * copies to the device asynchronously; a call first waits (host side) for the previous
 * call's copy.  A captured call copies the table when the graph is replayed, so new
 * calls on the same batch must not overlap replays still in flight. */
vef_status vef_batch_sweep(vef_batch batch, const double* const* sigma_t, const double* const* sigma_s,
                           const double* const* phi_in, const double* const* source,
                           const double* const* inflow, double* const* psi, const vef_opts* opts,
                           vef_info* info, void* stream);
/* Autotuner: times the batched sweep of each DG order in its single-CTA form (one CTA per
 * (problem, direction), the default) and in a set of cluster shapes (CTAs per direction x
 * warps per CTA) on the data of the last vef_batch_sweep call and keeps the fastest for later
 * calls; tiles_out (optional, [4]) receives the choice per order p = 1..4 as 100 x CTAs +
 * warps for a cluster shape, 1 for the single-CTA form, 0 when no problem has that order.
 * When the environment variable VEF_TUNE_CACHE names a file, the choices are appended to it
 * keyed by the device and the problems of each order, and vef_batch_create reads them back
 * for a batch with the same key (a missing or unreadable file is ignored; the last line
 * for a key wins); an order whose choice came from the file is not timed again.
 * Synchronises `stream`. */
vef_status vef_batch_tune(vef_batch batch, void* stream, int* tiles_out);

/* Hybridized Raviart-Thomas VEF solve (paper Sec. "Hybridization": "Extension to VEF" and
 * "Implementation Details"), the VEF step of the outer iteration that follows a transport
 * sweep and its closures.  On the mesh's elements it discretises
 *     div J + sigma_a phi = Q0,   div(E phi) + sigma_t J = Q1,   J.n = E_b phi + 2 J_in on the boundary
 * (paper Eqs. zeroth, first, mlbc) with a broken RT_p current (x component in Q_{p+1} x Q_p,
 * y component in Q_p x Q_{p+1}, nodal at the p+2 Gauss-Lobatto points across and the p+1
 * Gauss-Legendre points along, contravariant Piola transform), the transport's DG scalar
 * flux and degree-p Lagrange multipliers on the interior faces (nodal at the p+1
 * Gauss-Legendre points; {E n} averaged from the two sides).  Each element's local mixed
 * system is assembled and inverted on the GPU (block inverse [[W, X], [Y, Z]]); its share
 * of the reduced system H = C1 W C2 for the multiplier is solved by BiCGStab with a
 * two-level additive Schwarz preconditioner standing in for the paper's algebraic
 * multigrid: per element, H restricted to its interior faces' multipliers, inverted; plus
 * a coarse correction on bilinear functions over a grid of at most 11 x 11 cells of whole
 * elements (its operator R0 H R0^T inverted once per call, in FP32: it steers the FP64
 * iteration, not its answer).  The matrix is applied face by face from the elements' H_e;
 * the current and scalar flux then follow element by element.
 *   sigma_t, sigma_s [device] [E];  phi_tr [device] [E][n], P_tr [device] [3][E][n]: the
 *   transport's nodal scalar flux and second moment (vef_moments' phi and P), giving
 *   E = P / phi at the quadrature points and on each side of each face;  Eb, Jin [device]
 *   [N_bf][nq] (vef_moments' Eb and Jin);  Q0 [device] [E][n] nodal zeroth source moment,
 *   Q1 [device] [2][E][n] nodal first moment or NULL (zero);
 *   tol: relative residual of the multiplier solve; max_iter: its iteration cap;
 *   outputs phi [device] [E][n] (DG nodal), J [device] [E][2 (p+2)(p+1)] (RT dofs: x part
 *   a + (p+2) b, then y part a + (p+1) b), lambda [device] [faces][p+1] or NULL (interior
 *   faces: vertical ones first, j (nx-1) + i, then horizontal, (nx-1) ny + j nx + i).
 * Synchronises `stream` (the Krylov scalars stay on the device; the host reads the
 * convergence state back every 16 iterations).  Uses the handle's
 * scratch.  Errors: VEF_ERR_INVALID_ARG, VEF_ERR_NOT_CONVERGED (tolerance not reached in
 * max_iter iterations, or a singular local system). */
typedef struct {
  int iterations;          /* BiCGStab iterations of the multiplier system */
  double rel_residual;     /* final ||r - H lambda||_2 / ||r||_2 */
  long long multipliers;   /* unknowns of the reduced system: interior faces x (p+1) */
} vef_hrt_info;

vef_status vef_hrt_solve(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                         const double* phi_tr, const double* P_tr, const double* Eb,
                         const double* Jin, const double* Q0, const double* Q1, double tol,
                         int max_iter, double* phi, double* J, double* lambda,
                         vef_hrt_info* info, void* stream);

/* VEF fixed-point iteration (paper Sec. "VEF Algorithm"): from phi^0 ([device] [E][n],
 * NULL = 0), repeat
 *   1) invert the transport equation with the scattering source sigma_s phi^k / (4 pi) + q
 *      (vef_sweep; the factorisation is formed on the first iteration and kept after it,
 *      sigma_t being fixed; opts selects the precision and sweep forms as for vef_sweep);
 *   2) form the Eddington tensor, boundary factor and inflow partial current from its
 *      angular flux (vef_moments);
 *   3) solve the VEF equations by the hybridized RT method (vef_hrt_solve) with
 *      Q0 = 4 pi q and Q1 = 0, and take their scalar flux as phi^{k+1};
 * until max |phi^{k+1} - phi^k| <= tol (the max norm of the difference of successive
 * iterates, the paper's stopping rule) or max_outer iterations.
 *   source [device] [E][n] isotropic q per steradian (NULL = 0); inflow [device]
 *   [D][N_bf][nq] or NULL (vacuum); omega, weights [host] as for vef_sweep;
 *   hrt_tol, hrt_max_iter: the multiplier solve of each VEF step;
 *   phi_out [device] [E][n] the last VEF scalar flux; J_out [device] [E][2 (p+2)(p+1)] its
 *   current (RT dofs) or NULL; psi [device] [D][E][n] the last transport solution
 *   (required); dphi [device] [max_outer] the max-norm changes, or NULL.
 * Synchronises `stream`.  Returns VEF_ERR_NOT_CONVERGED if max_outer iterations did not
 * reach tol (the outputs then hold the last iterate). */
typedef struct {
  int iterations;        /* fixed-point iterations performed */
  int converged;         /* 1 if the last change was <= tol */
  double last_change;    /* max |phi^{k+1} - phi^k| of the last iteration */
  int hrt_iterations;    /* BiCGStab iterations summed over the VEF solves */
} vef_vef_info;

vef_status vef_vef_iterate(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                           const double* source, const double* inflow, const double* omega,
                           const double* weights, int D, const double* phi0, int max_outer,
                           double tol, double hrt_tol, int hrt_max_iter, const vef_opts* opts,
                           double* phi_out, double* J_out, double* psi, double* dphi,
                           vef_vef_info* info, void* stream);

/* Kernel classes for the per-kernel timing counters. */
enum {
  VEF_K_GEOMETRY = 0, /* mesh geometric factors */
  VEF_K_FACTOR = 1,   /* local assembly + inversion of every (element, direction) system */
  VEF_K_SWEEP = 2,    /* dependency-driven wavefront solve */
  VEF_K_RESIDUAL = 3, /* FP64 residual of the mixed-precision defect correction */
  VEF_K_SOURCE = 4,   /* direction-independent right-hand side and scalar-flux updates */
  VEF_K_MOMENTS = 5,  /* moments, Eddington tensor, boundary factor */
  VEF_K_ADJOINT = 6,  /* adjoint sweep */
  VEF_K_GROUP = 7,    /* trace systems of the coupled element groups (after VEF_K_FACTOR) */
  VEF_K_HRT = 8,      /* hybridized RT VEF solve: element-local elimination and recovery */
  VEF_K_COUNT = 9
};
typedef struct {
  long long launches;  /* kernel launches since the counters were last reset */
  double ms;           /* summed CUDA-event time of those launches (when timing is on) */
} vef_kernel_stat;

/* Turns per-kernel CUDA-event timing on (enable != 0) or off for calls using `mesh`, and
 * resets the counters.  Events are recorded on the stream each kernel is launched on. */
vef_status vef_profile(vef_mesh mesh, int enable);
/* Synchronises the recorded events and writes VEF_K_COUNT entries to out. */
vef_status vef_profile_read(vef_mesh mesh, vef_kernel_stat* out);

/* Measures this device's FMA throughput for FP64 (precision = VEF_FP64) or FP32
 * (VEF_MIXED) with independent FMA chains in every warp slot; *flops_per_s receives
 * the rate.  Diagnostic for roofline denominators; synchronises the device. */
vef_status vef_measure_fma_peak(int precision, double* flops_per_s);

/* Dependency schedule of the sweep, computed on the host from the face normals alone (the
 * scheduler behind vef_sweep; no CUDA call, for tests and tooling).  The paper sweeps in a
 * topological order of the elements and lags the couplings that re-entrant faces make
 * cyclic (Sec. "Thick Diffusion Limit", citing its graph-sweep reference); here the
 * upwind graph, decided pointwise at the face Gauss points, is condensed by its strongly
 * connected components, which the sweep solves as coupled groups, and the components are
 * levelled (Kahn) so that every donor lies at an earlier level.
 *   nds    [E][4][p+2][2] outward n ds at the face Gauss points, E = nx*ny, element
 *          e = j*nx + i, faces 0..3 towards (i, j-1), (i+1, j), (i, j+1), (i-1, j);
 *          a face point with Omega . n ds < 0 is inflow, = 0 neither (host array)
 *   omega  [D][2] directions (host); D in 1..1023
 *   levels [D] out: dependency levels of each direction
 *   groups [D] out: coupled groups of two or more elements
 *   level, comp_size  [D][E] out, each may be NULL: the level of each element's component
 *          and that component's size (1 for an element swept on its own).
 * Errors: VEF_ERR_INVALID_ARG (sizes, NULL required pointers), VEF_ERR_OOM (host memory). */
vef_status vef_schedule_host(int nx, int ny, int p, const double* nds, const double* omega, int D,
                             int* levels, long long* groups, int* level, int* comp_size);

/* Failure-detection self-test (the paper has no counterpart: its CPU sweeps do not wait on
 * other processors' flags).  Every wait in the library's kernels is a bounded poll that, when
 * it runs out, sets a timeout bit in a device status word and lets the kernel finish, so the
 * call returns VEF_ERR_TIMEOUT and the CUDA context stays usable.  This call runs one such
 * wait in a one-thread kernel on `stream` and synchronises it:
 *   kind 0  acquire loads of a global flag (the form of the fused apply's band waits),
 *   kind 1  try-waits on a shared-memory mbarrier phase (the form of the staging waits);
 *   satisfied != 0: the flag is set / the phase completed before the wait -> VEF_OK;
 *   satisfied == 0: nothing completes it -> VEF_ERR_TIMEOUT after `polls` polls.
 * polls in 1..2^24, else VEF_ERR_INVALID_ARG (checked before any CUDA call).  Allocates and
 * frees 8 bytes of device memory. */
vef_status vef_wait_selftest(int kind, int satisfied, long long polls, void* stream);

/* The elimination pivots' reciprocal (an approximate reciprocal refined by two
 * Newton-Raphson steps; FP32: the correctly rounded reciprocal) against the correctly
 * rounded 1/x, on n device-generated inputs across the normal range (exponents -500..500,
 * hashed mantissas, both signs; FP32 inputs within 2^+-99): *max_rel_err and
 * *max_rel_err_f32 receive the largest relative differences.  n in 1..2^30, else
 * VEF_ERR_INVALID_ARG.  Synchronous (default stream); allocates 16 bytes of device memory. */
vef_status vef_rcp_selftest(long long n, double* max_rel_err, double* max_rel_err_f32);

/* Device status bits: what a kernel records when a bounded wait runs out, an iteration
 * hits its cap, a closure denominator is not positive, an element system is singular, or
 * (bounds-checked build) an index falls outside its array; the next synchronising call
 * maps them to VEF_ERR_TIMEOUT, VEF_ERR_NOT_CONVERGED, VEF_ERR_NONPOSITIVE_DENOM,
 * VEF_ERR_NOT_CONVERGED and VEF_ERR_BOUNDS. */
enum {
  VEF_STATUS_TIMEOUT = 1,
  VEF_STATUS_NOT_CONVERGED = 2,
  VEF_STATUS_NONPOSITIVE = 4,
  VEF_STATUS_SINGULAR = 8,
  VEF_STATUS_BOUNDS = 16
};

/* Failure-detection test hook (the paper has no counterpart): ORs `bits` (VEF_STATUS_*)
 * into the handle's device status word on `stream`, as a device-side failure would.  Kernels
 * launched after it see the bits: a staging wait of the sweeps finding VEF_STATUS_TIMEOUT
 * set stops polling at once, and its warp stops reading staged data (the call's results are
 * then undefined), so a call made while a timeout is recorded and not yet collected returns
 * quickly; the next synchronising call returns the error and clears the word.
 * Errors: VEF_ERR_INVALID_ARG (NULL mesh, bits empty or outside the five values, another
 * device). */
vef_status vef_mesh_inject_status(vef_mesh mesh, unsigned int bits, void* stream);

/* 1 when this library is the bounds-checked build (libvef_checked.so: compiled with
 * VEF_CHECKED, see the package's build(checked=True)), 0 for the normal build.  The checked
 * build tests the indices the sweep, adjoint, group and factorisation kernels take from the
 * schedule (record and member indices, element indices, shared-memory trace-slot ids)
 * before each access; an index outside its array sets VEF_STATUS_BOUNDS and the access is
 * skipped, so the next synchronising call returns VEF_ERR_BOUNDS instead of the kernel
 * touching memory it does not own.  It stands in for a memory checker; the arithmetic is
 * the normal build's. */
int vef_build_checked(void);

/* Eddington tensor without device allocation (the paper has no counterpart: this is a
 * library interface).  Same result as vef_moments with only Eten requested:
 *   Eten [device] [3][E][(p+2)^2] = P / phi at the volume Gauss points, from
 *   psi [device] [D][E][(p+1)^2]; omega [host] [D][2] and weights [host] [D].
 * For callers that cannot allocate device memory: applications that hand all device
 * memory to their own pool at start-up, or loops that must avoid the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  Such callers cannot create a mesh
 * handle either, so the mesh enters only through E and p.  The call allocates nothing:
 * the nodal moments go through one fixed 16 MiB device array that every GPU loading
 * the library holds until the process exits.  Limits: D <= 256 and
 * E * (p+1)^2 <= 524288; larger inputs return VEF_ERR_INVALID_ARG.
 * The first call on a device looks up that array's device address (with the device
 * current) and keeps it; make that first call before any stream capture.  A
 * cudaDeviceReset of that device invalidates the kept address: do not call this entry
 * point on a device after resetting it in the same process.  All calls share the
 * array: calls that overlap on the GPU (different streams or devices' work racing on
 * one device) corrupt each other's result, so serialise them.  Each call writes every
 * scratch entry it reads, so nothing carries over between calls.  A non-positive
 * denominator writes NaN at that point.  Stream-ordered on `stream`. */
vef_status vef_eddington_noalloc(const double* psi, const double* omega, const double* weights,
                                 int D, long long E, int p, double* Eten, void* stream);

/* Human-readable name of a status code (static string). */
const char* vef_status_string(vef_status s);
/* Last error message of the calling thread (static buffer, "" if none). */
const char* vef_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VEF_H */
