/*
 * hfv.h -- C ABI of libhfv: the hybrid Linear / CWENOZ / MUSCL finite-volume
 * residual of Tong & Tsoutsanis (arXiv 2510.25906) for the compressible Euler
 * equations on unstructured mixed-element meshes, on one NVIDIA GB300 GPU.
 *
 * The calls follow the paper's statement of the problem:
 *   build the mesh and its stencils ............ Sec. 2.1 (stencil selection)
 *   precompute the reconstruction operators .... Sec. 2.1 (pseudo-inverse,
 *                                                computed once), Sec. 2.3 (OI)
 *   compute the residual ....................... Sec. 2 (eq. EulerEquationsDetails)
 *                                                with the pipeline of Sec. 2.5
 *   advance a step ............................. Sec. 2.4 (explicit SSP
 *                                                Runge-Kutta; three-stage here)
 *
 * Conventions
 *   - Every function returns an int status: HFV_OK (0) or a negative HFV_ERR_*
 *     code.  No C++ exception crosses this interface.  hfv_last_error()
 *     returns a message for the calling thread's last failure.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the current device.  Streams are cudaStream_t passed
 *     as void* (NULL = legacy default stream).  Calls marked "async" only
 *     enqueue work on that stream; calls marked "sync" wait for it.
 *   - Cell states are conserved variables, structure of arrays:
 *     U[v * n_cells + c], v = 0..nv-1, nv = dim + 2, order
 *     (rho, rho u, rho v[, rho w], E).
 *   - Handles are opaque and owned by the library until *_destroy.
 *   - Not thread-safe per handle: one host thread drives a given scheme.
 */
#ifndef HFV_H
#define HFV_H

#include <stdint.h>

#if defined(__GNUC__)
#define HFV_API __attribute__((visibility("default")))
#else
#define HFV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HFV_OK 0
#define HFV_ERR_ARG (-1)          /* invalid argument (NULL, size, enum) */
#define HFV_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define HFV_ERR_OOM (-3)          /* device or host allocation failed */
#define HFV_ERR_MESH (-4)         /* degenerate cell, unmatched or over-shared face */
#define HFV_ERR_STENCIL (-5)      /* too few cells reachable, or a rank-deficient least-squares system */
#define HFV_ERR_NONPHYSICAL (-6)  /* a state with rho <= 0, p <= 0 or a non-finite value was seen */
#define HFV_ERR_TIMEOUT (-7)      /* a bounded device wait gave up */
#define HFV_ERR_STATE (-8)        /* call not valid for this handle (e.g. wrong precision) */

/* cell types; local vertex order: TRI, QUAD counter-clockwise; HEX v0..v3
 * bottom face counter-clockwise seen from +z, v4..v7 above them.  3D meshes
 * may mix TET, PRISM, PYRAMID and HEX; a mesh holding any cell but HEX is
 * built for orders 2 and 3. */
#define HFV_TRI 1
#define HFV_QUAD 2
#define HFV_TET 3     /* positive volume v0 v1 v2 v3 */
#define HFV_HEX 4
#define HFV_PRISM 5   /* triangle v0 v1 v2 counter-clockwise seen from v3 v4 v5; v3, v4, v5 joined to v0, v1, v2 */
#define HFV_PYRAMID 6 /* base v0 v1 v2 v3 counter-clockwise seen from the apex v4 */

/* Riemann solvers at the face quadrature points (Sec. 2.4) */
#define HFV_RUSANOV 0
#define HFV_HLLC 1
#define HFV_HLL 2

/* reconstruction schemes */
#define HFV_HYBRID 0       /* the paper's detector-driven hybrid (Sec. 2.5) */
#define HFV_PURE_LINEAR 1  /* every cell linear (still Harten-bounded) */
#define HFV_PURE_CWENOZ 2  /* every cell CWENOZ (still Harten-bounded) */
#define HFV_PURE_MUSCL 3   /* every cell MUSCL (still Harten-bounded) */

/* arithmetic of the residual path */
#define HFV_FP64 0 /* operators, gathers, reconstruction and fluxes in FP64 */
#define HFV_FP32 1 /* the same in FP32; setup and the Runge-Kutta accumulation stay FP64 */

/* time integration and MUSCL limiter (hfv_scheme_params) */
#define HFV_SSPRK3 0
#define HFV_SSPRK54 1
#define HFV_BARTH_JESPERSEN 0
#define HFV_VENKATAKRISHNAN 1
#define HFV_CONSERVED 0
#define HFV_CHARACTERISTIC 1

/* cell classes written by the pipeline (Sec. 2.5; the paper's figures call
 * them Scheme 0 / 1 / 3 / -1) */
#define HFV_CLASS_LINEAR 0
#define HFV_CLASS_CWENOZ 1
#define HFV_CLASS_MUSCL 2
#define HFV_CLASS_FIRST 3  /* Harten bound violated: first-order (cell mean) */

typedef struct hfv_mesh hfv_mesh;
typedef struct hfv_scheme hfv_scheme;

/* Mesh description.  All arrays are host memory owned by the caller and
 * copied by hfv_mesh_create. */
typedef struct {
    int dim;                       /* 2 or 3 */
    int64_t n_nodes, n_cells;
    const double* node_xyz;        /* [n_nodes][dim] */
    const uint8_t* cell_type;      /* [n_cells] HFV_TRI / HFV_QUAD (2D); HFV_TET / PRISM / PYRAMID / HEX (3D) */
    const int64_t* cell_node_ptr;  /* [n_cells + 1] CSR offsets, from cell_node_ptr[0] >= 0 */
    const int32_t* cell_node_idx;  /* [cell_node_ptr[n_cells]] vertex ids in local order: cell c's are
                                      cell_node_idx[cell_node_ptr[c] .. cell_node_ptr[c+1] - 1] */
    const double* period;          /* [dim] periodic length per axis, 0 = open (transmissive) */
} hfv_mesh_desc;

/* Scheme parameters.  hfv_default_params fills the defaults given here. */
typedef struct {
    int order;          /* r + 1 (default 3), "order" as in Sec. 2.1: 2..7 in 2D, 2..6 on
                           hexahedra, 2..3 on meshes with tetrahedra, prisms or pyramids;
                           hfv_residual_vjp: 2..5 in 2D, 2..4 on hexahedra */
    int flux;           /* HFV_RUSANOV / HFV_HLLC / HFV_HLL (default HLLC) */
    int scheme;         /* HFV_HYBRID (default) or a pure scheme */
    int nad_vars;       /* detector variables: bit0 density, bit1 pressure,
                           bit2 the remaining conserved variables (default 3) */
    int precision;      /* HFV_FP64 (default) or HFV_FP32 */
    int time_scheme;    /* hfv_step: HFV_SSPRK3 (default, three-stage SSP) or HFV_SSPRK54
                           (the five-stage, fourth-order SSP method of Spiteri and Ruuth the
                           paper integrates with, Sec. 2) */
    double gamma;       /* 1.4 (Sec. 2) */
    double alpha_m, beta_m, alpha_w, beta_w;  /* detector margins, eqs. marginm and marginw;
                                                 default 5e-3, 0.5, 0, 0 (Fig. NADMargin (a)) */
    double kappa, n_exp;   /* deactivation threshold (kappa dx)^n, eq. NADDeactivatedCriteria; default 1, 1 */
    double lambda1_prime;  /* CWENOZ central weight lambda_1' (Sec. 2.3); default 1e3 */
    double cweno_eps, cweno_b;          /* 1e-3 and 4 (Sec. 2.3) */
    double harten_theta, harten_eps;    /* 0.9 and 1e-14 (eq. harten_jump_fix) */
    double stencil_factor;              /* M = stencil_factor * K(r, d); default 2 (Sec. 2.1) */
    int limiter;        /* MUSCL limiter: HFV_BARTH_JESPERSEN (default, Sec. 2.2) or
                           HFV_VENKATAKRISHNAN (the smooth limiter the paper runs with K = 5) */
    int cweno_vars;     /* CWENOZ variables (Sec. 2.3 leaves the choice open): HFV_CONSERVED
                           (default, component-wise) or HFV_CHARACTERISTIC (per face, projected
                           with the eigenvectors of the flux Jacobian along its normal at the
                           cell mean) */
    double venkat_k;    /* Venkatakrishnan threshold eps^2 = (K dx)^3, dx = |V|^(1/d); default 5 */
    /* viscous terms (Sec. 2, eq. EulerEquationsDetails; Navier-Stokes when mu0 > 0):
     *   mu = mu0 (T / t0)^(3/2) (t0 + sutherland_s) / (T + sutherland_s)  (eq. sutherlandlaw),
     *   T = p / rho, heat flux mu / prandtl gamma / (gamma - 1) grad T   (eq. HeatConduct),
     *   face gradient = mean of the two sides' gradients + (visc_alpha / L_int)(W_R - W_L) n
     *   (eq. viscous_jump; L_int between the cells' vertex means).  The gradients
     *   are those of each side's unlimited least-squares polynomial (Sec. 2).
     *   Defaults: mu0 = 0 (Euler), t0 = 1, sutherland_s = 110.4 / 288.15,
     *   prandtl = 0.72, visc_alpha = 4/3 */
    double mu0, t0, sutherland_s, prandtl, visc_alpha;
    /* chained steps (hfv_step with HFV_SSPRK3; default 0 = off).  1: the last
     * stage of every step also writes the next step's FP32/FP64 stage copy of
     * the state and, in CFL mode, reduces the next step's time step, so that a
     * following hfv_step on the same U pointer, in the same mode (CFL or fixed
     * dt) and with the same cfl, skips its stage-in copy and time-step
     * reduction.  The caller promises that U is not written between such calls;
     * calls that overwrite the scheme's stage copy (hfv_residual,
     * hfv_compute_dt, hfv_autotune, hfv_residual_vjp, hfv_advance_host's
     * upload) end the chain and the next step starts afresh.  The chain knows
     * the state by its address only: new contents at the same address (U
     * written by the caller, or a buffer freed and allocated again at that
     * address) must be preceded by one of those calls, e.g. hfv_compute_dt,
     * or they are stepped from the stale copy.  Results are the same bits as
     * with 0. */
    int step_chain;
} hfv_scheme_params;

/* Fill *p with the defaults listed above (the paper's values of Sec. 2.3-2.5
 * and Fig. NADMargin (a) where it gives them).  Errors: HFV_ERR_ARG (p NULL). */
HFV_API int hfv_default_params(hfv_scheme_params* p);

/* Build faces, face neighbours, periodic pairing and cell geometry.
 * Sec. 2 (mixed-element meshes).  The offsets, vertex ids and coordinates are
 * checked before anything is read through the offsets.  sync.  Errors:
 * HFV_ERR_ARG (NULL array, dim not 2 or 3, no cells or nodes, 2^31 cells or
 * more, a period negative or not finite), HFV_ERR_MESH (a type not of the
 * dimension, offsets that are negative or do not step by each cell's vertex
 * count, a vertex id outside 0..n_nodes-1, a non-finite coordinate, zero or
 * negative volume, a face shared by more than two cells, a cell that is its
 * own neighbour), HFV_ERR_OOM. */
HFV_API int hfv_mesh_create(const hfv_mesh_desc* desc, hfv_mesh** out);

/* A batch of independent problems as one mesh (the batched workload of many
 * 2D problems of uneven size): the meshes are concatenated, node and cell ids
 * offset per mesh, and problem k becomes the cells
 * cell_offsets[k] .. cell_offsets[k+1] - 1 (hfv_mesh_segments), in the given
 * order.  No face is shared between problems, so stencils (Sec. 2.1),
 * detector bounds (Sec. 2.5) and fluxes never couple them, and a residual of
 * the batch equals, cell by cell, the residuals of the problems alone.
 * hfv_step and hfv_compute_dt take one time step per problem.  The paper
 * solves one problem at a time; batching is a property of this library.
 * All meshes must have the same dim and be open (period 0).  Errors:
 * HFV_ERR_ARG (bad descriptor, periodic mesh), HFV_ERR_MESH, HFV_ERR_OOM. */
HFV_API int hfv_mesh_create_batch(const hfv_mesh_desc* descs, int n_meshes, hfv_mesh** out);

/* Problems of a mesh (1 for hfv_mesh_create): *n_segments, and when
 * cell_offsets (host, n_segments + 1 int64) is non-NULL their first cells
 * and the total.  A property of this library's batching (the paper solves one
 * problem at a time).  sync.  Errors: HFV_ERR_ARG (mesh or n_segments NULL). */
HFV_API int hfv_mesh_segments(const hfv_mesh* mesh, int* n_segments, int64_t* cell_offsets);

/* Cell measures |V_c| (host output, caller-owned, n_cells doubles): areas
 * in 2D, volumes in 3D, as the scheme uses them (Sec. 2).  sync.  Errors:
 * HFV_ERR_ARG (NULL argument). */
HFV_API int hfv_mesh_volumes(const hfv_mesh* mesh, double* vol);

/* Sizes of a mesh (Sec. 2): cells, faces, dimension.  Any output pointer may
 * be NULL.  sync.  Errors: HFV_ERR_ARG (mesh NULL). */
HFV_API int hfv_mesh_info(const hfv_mesh* mesh, int64_t* n_cells, int64_t* n_faces, int* dim);

/* Face neighbours in canonical per-cell form (host outputs, caller-owned):
 * nbr[c * 6 + f] = cell across local face f of c or -1 on an open boundary,
 * nbrf[c * 6 + f] = that face's local index inside the neighbour (or -1).
 * Unused slots (f >= faces of c) are -1.  The face adjacency the stencils of
 * Sec. 2.1 grow along.  sync.  Errors: HFV_ERR_ARG (NULL argument). */
HFV_API int hfv_mesh_connectivity(const hfv_mesh* mesh, int32_t* nbr, int8_t* nbrf);

/* Build the central and directional stencils (Sec. 2.1, 2.3), then, on the
 * GPU in FP64, the reference maps, the least-squares matrices, their
 * Householder-QR pseudo-inverses (computed once, Sec. 2.1), the
 * oscillation-indicator matrices (Sec. 2.3) and the folded per-cell
 * operators; allocate the device scratch of the residual.  The mesh must
 * outlive the scheme.  sync (the setup runs on `stream` and is waited for).
 * Errors: HFV_ERR_ARG, HFV_ERR_STENCIL (fewer than M cells within 16 face
 * layers, or a rank-deficient system; hfv_last_error names the cell),
 * HFV_ERR_CUDA, HFV_ERR_OOM. */
HFV_API int hfv_scheme_create(hfv_mesh* mesh, const hfv_scheme_params* params, void* stream, hfv_scheme** out);

/* Sizes: info[0..7] = N (unknown coefficients, K(r,d)-1), M (central stencil
 * size, 2 K(r,d); Sec. 2.1), Md (directional / MUSCL stencil size), nq (Gauss
 * points per face direction), nfp (points per face), nv, Q_total (sum over
 * cells of face points), precision.  Host output, 8 int64.  sync.  Errors:
 * HFV_ERR_ARG (NULL argument). */
HFV_API int hfv_scheme_info(const hfv_scheme* s, int64_t* info);

/* Stencils, for bit-exact checks (host outputs, caller-owned):
 * central[c * M + m] = m-th cell of c's central stencil, in the order
 * (face layer, quantised distance, id); dir[(c * 6 + f) * Md + k] = local
 * index (0..M-1) of the k-th cell of the directional stencil of face f, or
 * -1 past its size; dir may be NULL.  The central stencil of Sec. 2.1 and
 * the directional stencils of Sec. 2.3.  sync.  Errors: HFV_ERR_ARG (s or
 * central NULL). */
HFV_API int hfv_get_stencils(const hfv_scheme* s, int32_t* central, int32_t* dir);

/* The same stencils without a scheme or a GPU: the host builder that
 * hfv_scheme_create runs (central stencil of Sec. 2.1, directional stencils
 * of Sec. 2.3), for a mesh at an order, so the lists equal hfv_get_stencils'
 * of a scheme of that order.  sizes[0..1] (required) receive M and Md; central
 * (NULL: sizes only) and dir (may be NULL) have the layouts of
 * hfv_get_stencils: [n_cells][M] and [n_cells][6][Md].  Host outputs,
 * caller-owned.  Errors: HFV_ERR_ARG (NULL mesh or sizes, order outside
 * 2..7), HFV_ERR_STENCIL (a cell reaches fewer than M cells within 16 face
 * layers), HFV_ERR_OOM.  sync; touches no GPU. */
HFV_API int hfv_stencils_host(const hfv_mesh* mesh, int order, int32_t* sizes, int32_t* central, int32_t* dir);

/* One residual evaluation R(U) = dU/dt (eq. EulerEquationsDetails, inviscid)
 * with the hybrid pipeline of Sec. 2.5: linear candidate, detector
 * (eqs. DMP, NADMUSCL, NADCWENOZ, marginm, marginw, NADDeactivatedCriteria),
 * tagging of the flagged cells' face neighbourhoods, CWENOZ and MUSCL
 * recomputation, Harten bound (eq. harten_jump_fix), Riemann fluxes.
 *   U            device, [nv][n_cells], double (HFV_FP64) or float (HFV_FP32)
 *   R            device, same layout and type; written for every cell
 *   forced_class device uint8 [n_cells] or NULL.  Non-NULL: skip the
 *                detector and tagging and use these classes (0..3); the
 *                Harten bound still applies to classes 0..2.  Other values
 *                are not checked (the array is device memory): the kernels
 *                use their low two bits, bit 7 reads as a failed Harten
 *                test, and no memory access depends on them.
 *   class_out    device uint8 [n_cells] or NULL: the final class per cell.
 * async; allocates nothing; capturable in a CUDA graph.  Errors: HFV_ERR_ARG.
 * A non-physical state is recorded for hfv_status, not returned here. */
HFV_API int hfv_residual(hfv_scheme* s, const void* U, void* R, const uint8_t* forced_class, uint8_t* class_out, void* stream);

/* Stable time step dt = cfl * min_c |V_c| / sum_f (|u_c . n_f| + a_c) |S_f|
 * from the cell averages of U (device, FP64 [nv][n_cells]), the minimum taken
 * over each problem's cells; result written to dt_dev (device, one double per
 * problem of the mesh, hfv_mesh_segments).  The time discretisation of
 * Sec. 2.4 gives only the CFL number; this convective bound (with the
 * diffusion limit 4 nu sum_f |S_f|^2 / |V| added when mu0 > 0) is the reading
 * taken.  async.  Errors: HFV_ERR_ARG (NULL argument, cfl <= 0),
 * HFV_ERR_CUDA. */
HFV_API int hfv_compute_dt(hfv_scheme* s, const double* U, double cfl, double* dt_dev, void* stream);

/* One SSP Runge-Kutta step of U in place, Shu-Osher form (the temporal
 * discretisation of Sec. 2.4; the paper's own runs use the SSP scheme of
 * Spiteri and Ruuth).  time_scheme
 * HFV_SSPRK3 (three stages):
 *   U1 = U + dt R(U);  U2 = 3/4 U + 1/4 (U1 + dt R(U1));
 *   U  = 1/3 U + 2/3 (U2 + dt R(U2));
 * HFV_SSPRK54: the five-stage, fourth-order method of Spiteri and Ruuth
 *   u_i = sum_j alpha_ij u_j + beta_ij dt R(u_j), u_0 = U, U = u_5.
 *   U   device FP64 [nv][n_cells] (the accumulation is FP64 in both precisions;
 *       in HFV_FP32 each stage's residual is evaluated on an FP32 copy)
 *   dt  > 0: that step for every problem; <= 0: each problem's own step
 *       computed from U with `cfl` (hfv_compute_dt)
 *   dt_used  host double* (one per problem of the mesh) or NULL; non-NULL
 *       makes the call sync.
 * async otherwise; allocates nothing.  Errors: HFV_ERR_ARG (s or U NULL,
 * neither dt nor cfl positive), HFV_ERR_CUDA. */
HFV_API int hfv_step(hfv_scheme* s, double* U, double cfl, double dt, double* dt_used, void* stream);

/* Vector-Jacobian product of the residual: g = lam^T dR/dU at U, with the
 * cell classes frozen (the detector, tagging and Harten decisions of
 * Sec. 2.5) and every branch inside the reconstructions and the Riemann
 * solver (limiter bounds and minimum, |x|, HLLC wave pattern) taken as in
 * the evaluation at U; the derivative of that branch.
 *   U    device FP64 [nv][n_cells]
 *   cls  device uint8 [n_cells], classes as hfv_residual's class_out (a
 *        forced LINEAR or CWENOZ cell that breaks the Harten bound at U falls
 *        back to FIRST as in hfv_residual)
 *   lam  device FP64 [nv][n_cells], the adjoint of R
 *   g    device FP64 [nv][n_cells], output
 * FP64 schemes of the Euler residual (mu0 = 0) only.  The first call allocates the adjoint's scratch
 * (face-point adjoints, per-stencil-entry contributions and the inverse
 * stencil map, about (Q_max + M + 1) nv 8 + 12 M bytes per cell), kept until
 * hfv_scheme_destroy.  The paper states no adjoint; this is the
 * differentiation of its residual.  async.  Errors: HFV_ERR_ARG,
 * HFV_ERR_OOM, HFV_ERR_CUDA. */
HFV_API int hfv_residual_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, const double* lam, double* g,
                             void* stream);

/* One SSP-RK3 step (Sec. 2.4) that records (forced = 0) or imposes
 * (forced != 0) the classes (Sec. 2.5) of its three stages: U (device FP64 [nv][n_cells], the step's
 * start) -> U_out (device, another buffer), with U1 = U + dt R(U),
 * U2 = 3/4 U + 1/4 (U1 + dt R(U1)), U_out = 1/3 U + 2/3 (U2 + dt R(U2));
 * cls device uint8 [3][n_cells], stage k's final classes (as hfv_residual's
 * class_out).  The forward sweep of a checkpointed adjoint: the state and
 * cls of every step are its checkpoint.  Same schemes as hfv_residual_vjp;
 * uses the adjoint's scratch.  async.  Errors: HFV_ERR_ARG, HFV_ERR_OOM. */
HFV_API int hfv_step_classes(hfv_scheme* s, const double* U, double dt, uint8_t* cls, int forced, double* U_out,
                             void* stream);

/* The adjoint of one SSP-RK3 step with its stages' classes frozen (the
 * differentiation of hfv_step_classes; the paper states no adjoint): lam
 * (device FP64 [nv][n_cells]) holds dJ/dU_{n+1} on entry and dJ/dU_n on
 * return, for the step from U with step size dt and stage classes cls
 * ([3][n_cells], as recorded by hfv_step_classes).  The stage states are
 * recomputed from U; with J_k = dR/dU at stage k (its classes frozen):
 *   l2 = 2/3 lam + dt J_2^T (2/3 lam),   l1 = 1/4 l2 + dt J_1^T (1/4 l2),
 *   lam <- 1/3 lam + 3/4 l2 + l1 + dt J_0^T l1.
 * async.  Errors: HFV_ERR_ARG, HFV_ERR_OOM, HFV_ERR_CUDA. */
HFV_API int hfv_step_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, double dt, double* lam, void* stream);

/* Autotuner of the residual's launch shape for this scheme and state (a
 * property of this library; the paper has no counterpart): the
 * persistent candidate kernel's tile shape (2D FP32 orders 2-3: 0 = tiles of
 * 48 cells, three CTAs per SM; 1 = tiles of 64 cells, two CTAs per SM; one
 * shape elsewhere) and resident CTAs per SM, and the CWENOZ / MUSCL
 * kernel's blocks per SM and the share of them given to the CWENOZ queue.
 * Coordinate descent over candidate values, each timed twice with CUDA
 * events over `reps` residuals of U (device, the scheme's precision,
 * [nv][n_cells]) on `stream` (the better time counts); a candidate replaces
 * the current value only when 2 % faster, and the shape found is kept for
 * every later call on the scheme.
 * shape (host, 4 ints, may be NULL) receives it: {candidate CTAs per SM
 * (0: as many as fit), nonlinear blocks per SM, CWENOZ share in %, tile
 * shape}.  The results of the residual do not depend on the shape.  sync.
 * Errors: HFV_ERR_ARG, HFV_ERR_CUDA. */
HFV_API int hfv_autotune(hfv_scheme* s, const void* U, int reps, void* stream, int* shape);

/* Set the launch shape hfv_autotune reports (host, 4 ints, same order and
 * meaning), e.g. one tuned earlier for the same mesh and order; a tile shape
 * that the configuration lacks falls back to its only one.  The paper has no
 * counterpart.  Errors: HFV_ERR_ARG (NULL, a value out of range: CTAs per SM
 * 0..64, blocks per SM 1..64, share 1..99 %, tile 0 or 1). */
HFV_API int hfv_scheme_set_shape(hfv_scheme* s, const int* shape);

/* hfv_step (Sec. 2.4) on several schemes at once, each on its own stream forked from
 * `stream` and joined back into it (so their kernels may run concurrently,
 * and a stream capture records one graph with one branch per scheme): the
 * form a batch of problems of different orders takes, one batched mesh per
 * order.  U[k] is scheme k's state; cfl and dt as for hfv_step.  Schemes
 * must be distinct.  async; allocates nothing.  Errors: HFV_ERR_ARG (NULL
 * entry, a scheme listed twice), HFV_ERR_CUDA and those of hfv_step; a
 * failure still joins the branches forked before it into `stream`. */
HFV_API int hfv_step_many(hfv_scheme* const* schemes, double* const* U, int n, double cfl, double dt, void* stream);

/* End-to-end helper: copy U (host, FP64 [nv][n_cells], caller-owned) to the
 * scheme's own device state, take n_steps steps as hfv_step (Sec. 2.4), copy
 * the result back into U.  Allocates nothing; ends a step chain.  sync.
 * Errors: HFV_ERR_ARG (s or U NULL, n_steps < 0), HFV_ERR_CUDA and those of
 * hfv_step. */
HFV_API int hfv_advance_host(hfv_scheme* s, double* U_host, int n_steps, double cfl, double dt, void* stream);

/* Class queues of the last residual (the tagged classes of Sec. 2.5; host
 * outputs, caller-owned): counts[0] = CWENOZ cells, counts[1] = MUSCL cells; queues may be NULL or hold
 * [2][n_cells] int32, each queue in ascending cell order.  sync.  Errors:
 * HFV_ERR_ARG (NULL scheme or counts), HFV_ERR_CUDA (a copy failed, or the
 * device holds a queue length outside 0..n_cells; queues is then left
 * unwritten). */
HFV_API int hfv_get_queues(const hfv_scheme* s, int32_t* counts, int32_t* queues);

/* Sticky status bits (host output): bit0 = a state with rho <= 0, p <= 0 or
 * a non-finite value reached hfv_residual (the positivity the bound of
 * Sec. 2.4 protects); bit2 = a bounded wait on a bulk
 * copy inside the candidate kernel gave up (the kernel skipped the rest of
 * its cells and returned; the residual of that launch is incomplete).
 * reset != 0 clears them.  sync.  Returns HFV_ERR_TIMEOUT when bit2 is set,
 * else HFV_ERR_NONPHYSICAL when bit0 is set, else HFV_OK; HFV_ERR_ARG (s or
 * flags NULL), HFV_ERR_CUDA. */
HFV_API int hfv_status(hfv_scheme* s, int* flags, int reset);

/* Testing aid for the bounded waits of the candidate kernel (the paper has no
 * counterpart).  consumer_wait_ns in 1..2e9 replaces the 2 s limit of its
 * consumer warps' waits for the bulk copies (0: back to 2 s);
 * withhold_copies != 0 makes its producer warp issue no copy at all, so that
 * the consumers' first wait runs out: every later residual on the scheme then
 * skips its candidates, records bit 2 for hfv_status (HFV_ERR_TIMEOUT) and
 * returns -- its R is meaningless -- with no copy in flight and the context
 * intact.  (0, 0) restores normal operation.  Errors: HFV_ERR_ARG. */
HFV_API int hfv_debug_wait(hfv_scheme* s, int64_t consumer_wait_ns, int withhold_copies);

/* Wall time of hfv_scheme_create's two phases (host output, 2 doubles, ms):
 * ms[0] the stencils (host threads), ms[1] the operators (device, FP64).
 * Instrumentation; sync.  Errors: HFV_ERR_ARG (NULL argument). */
HFV_API int hfv_scheme_setup_ms(const hfv_scheme* s, double* ms);

/* Switch an existing scheme between the detector-driven hybrid and the pure
 * schemes (HFV_HYBRID, HFV_PURE_LINEAR, HFV_PURE_CWENOZ, HFV_PURE_MUSCL): the
 * stencils and operators do not depend on this choice (Sec. 2.5 selects among
 * reconstructions built on the same stencils), so a comparison of hybrid and
 * pure CWENOZ needs one setup.  Takes effect at the next residual; ends a
 * step chain.  Errors: HFV_ERR_ARG. */
HFV_API int hfv_scheme_set_kind(hfv_scheme* s, int scheme);

/* Device bytes held by the scheme (operators + scratch; host output).
 * Instrumentation; sync.  Errors: HFV_ERR_ARG (NULL argument). */
HFV_API int hfv_scheme_device_bytes(const hfv_scheme* s, int64_t* bytes);

/* Per-kernel timer of the hot path (instrumentation for benchmarks).
 * enable != 0: every kernel the scheme launches afterwards is bracketed by a
 * pair of CUDA events recorded on its launch stream (at most 512 pending
 * launches between reads).  enable == 0 switches it off.  Instrumentation
 * (the paper has no counterpart).  sync.  Errors: HFV_ERR_ARG (s NULL),
 * HFV_ERR_CUDA (event creation; the timer is then off). */
HFV_API int hfv_kernel_timer(hfv_scheme* s, int enable);

/* Fold the pending event pairs into per-kernel totals and read them (host
 * outputs, 16 entries each): ms[k] total milliseconds and launches[k] count
 * of kernel k: 0 linear candidate + detector, 1 tagging and queue
 * compaction, 5 CWENOZ, 6 MUSCL, 7 fluxes, 8 Runge-Kutta stage, 9 time
 * step, 10 FP32 conversion, 11 viscous gradients, 12 flux VJP, 13
 * reconstruction VJPs (linear and first-order cells, CWENOZ and MUSCL
 * queues), 14 stencil gather of the VJP (2, 3, 4: no kernel).  reset != 0
 * zeroes the totals after reading.  sync.  Errors: HFV_ERR_ARG (NULL
 * argument), HFV_ERR_CUDA. */
HFV_API int hfv_kernel_times(hfv_scheme* s, double* ms, int64_t* launches, int reset);

/* Number of kernels launched by this library in this process so far (host
 * output).  Instrumentation.  Errors: HFV_ERR_ARG (count NULL). */
HFV_API int hfv_launch_count(int64_t* count);

/* Fused multiply-add throughput of the current device's CUDA cores, the ALU
 * ceiling of the residual paths (instrumentation; the paper has no
 * counterpart).  kind 0 = FP64 (DFMA), 1 = FP32 (FFMA), 2 = packed FP32
 * (FFMA2, two FMAs per instruction).  Every SM runs 2,048 threads of eight
 * independent dependent-FMA chains; the loop count is calibrated so that a
 * launch takes about target_ms (0 < target_ms <= 2000), and the best of three
 * timed launches (CUDA events on `stream`) is written to *flops_per_s as
 * 2 x FMAs / second.  sync.  Errors: HFV_ERR_ARG, HFV_ERR_CUDA. */
HFV_API int hfv_fma_rate(int kind, double target_ms, double* flops_per_s, void* stream);

/* The FP32 kernels' conversions between FP32 and FP64 (the Runge-Kutta
 * update's increment and new state, the stage copy of the FP64 state, the
 * time step's FP64 bits) applied to an array, for checking them against the
 * hardware conversion (instrumentation; the paper has no counterpart).  They
 * use integer instructions on the IEEE 754 bit layouts, because the
 * conversion instruction occupies this GPU's FP64 pipe.  to_f32 = 1: in is
 * device double [n], out device float [n], rounded to nearest, ties to even;
 * to_f32 = 0: in device float [n], out device double [n], exact.  Every
 * result equals the conversion instruction's, NaN payloads included.  async
 * on `stream`.  Errors: HFV_ERR_ARG (bad to_f32, n < 0 or above
 * (2^31 - 1) * 255, null buffer with n > 0), HFV_ERR_CUDA. */
HFV_API int hfv_convert(int to_f32, int64_t n, const void* in, void* out, void* stream);

/* The FP64 kernels' reciprocal (the Riemann solvers, the pressure) applied
 * to an array: out[i] ~ 1 / in[i] from the hardware's approximate reciprocal
 * refined by two Newton-Raphson steps, within about an ulp for normal inputs
 * with normal reciprocals (instrumentation; the paper has no counterpart).
 * in, out: device double [n].  async on `stream`.  Errors: HFV_ERR_ARG
 * (n < 0 or above (2^31 - 1) * 255, null buffer with n > 0), HFV_ERR_CUDA. */
HFV_API int hfv_rcp64(int64_t n, const double* in, double* out, void* stream);

/* Class-queue compaction that allocates nothing (the paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory when they need the queues, e.g. code running inside a CUDA stream
 * capture, or a solver whose host framework's pool allocator owns all device
 * memory).  Given classes (device uint8 [n_cells], values 0..3), writes
 * counts[0] = number of CWENOZ cells (class 1), counts[1] = number of MUSCL
 * cells (class 2) (device int32 [2]) and the two queues in ascending cell
 * order to queues[0..counts[0]) and queues[n_cells..n_cells+counts[1])
 * (device int32 [2 * n_cells]) -- the same compaction the residual applies
 * to its tagged classes.  Scratch: a file-scope device array of 2 x 65,536
 * int32 block counts, held by every device that loads the library until the
 * process exits; n_cells above 16,777,216 is rejected with HFV_ERR_ARG.  The
 * first call on a device looks up that array's device address (set-up once
 * per device, under a host lock); make that first call before any stream
 * capture.  All calls share the one array: calls that overlap on the GPU
 * (different streams, concurrently) race.  No entry of the array needs to
 * start at zero: each call writes every entry it reads.  async. */
HFV_API int hfv_class_queues_static(const uint8_t* classes, int64_t n_cells, int32_t* counts, int32_t* queues,
                                    void* stream);

/* Message of the calling thread's last failure ("" if none); the string
 * belongs to the library and stays valid until the thread's next failing
 * call.  Never fails. */
HFV_API const char* hfv_last_error(void);

/* Release a scheme (its device arena, streams, events and the adjoint's
 * scratch) or a mesh; NULL is a no-op.  A mesh must outlive its schemes. */
HFV_API void hfv_scheme_destroy(hfv_scheme* s);
HFV_API void hfv_mesh_destroy(hfv_mesh* m);

#ifdef __cplusplus
}
#endif

#endif /* HFV_H */
