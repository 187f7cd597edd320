/*
 * gb.h -- C ABI of libgb, the B300 (sm_103a) solver for the arbitrary
 * Lagrangian-Eulerian (ALE) nodal discontinuous Galerkin form of the
 * Galerkin-Boltzmann equations (2D triangles, 6 fields; 3D tetrahedra, 10
 * fields) with semi-analytic Runge-Kutta (SARK) time stepping (arXiv
 * 2607.00199, Secs. 2-6).  Everything below describes the 2D solver; the
 * section "three dimensions" near the end lists what changes for dim = 3.
 *
 * Conventions (every entry point):
 *  - Returns GB_OK (0) or a negative GB_E* code; gb_last_error() gives a
 *    one-line message for the solver (or the last failed create, with NULL).
 *  - No call takes ownership of caller memory.  Host pointers are read or
 *    written during the call only.  The library allocates and owns all of
 *    the solver's device memory (cudaMalloc in gb_create, freed by
 *    gb_destroy).
 *  - All device work is enqueued on the CUDA stream given to gb_create
 *    (NULL = the legacy default stream).  Calls that return host data
 *    synchronise that stream; gb_step and gb_rhs only enqueue.
 *  - Field layout ("canonical"): q[k][f][i], k < n_elem elements, f < 6
 *    fields, i < Np nodes, row-major, FP64.  Node order: Warp & Blend nodes
 *    (Warburton 2006) on the reference triangle (-1,-1), (1,-1), (-1,1),
 *    by rows of constant barycentric coordinate of (-1,1) (bottom row
 *    first), left to right inside a row; Np = (N+1)(N+2)/2.
 *  - Fields (Sec. 2): q1 = rho, q2 = rho u / c, q3 = rho v / c, q4..q6 the
 *    second-order Hermite coefficients; c = sqrt(RT) = 1/Ma, tau = Ma^2/Re
 *    (lengths and the reference velocity scaled to 1, rho0 = 1).
 *  - There is no CPU fallback: every computation runs in the library's CUDA
 *    kernels; without a usable GPU the calls fail with GB_ECUDA.
 */
#ifndef GB_H
#define GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK       0
#define GB_EINVAL  (-1)  /* bad argument (NULL pointer, unsupported N, non-positive Ma/Re/dt ...) */
#define GB_ENOMEM  (-2)  /* device or host allocation failed */
#define GB_ECUDA   (-3)  /* a CUDA call failed (message in gb_last_error) */
#define GB_EMESH   (-4)  /* invalid mesh, or an element with J <= 0 at some stage */
#define GB_ENAN    (-5)  /* a NaN or Inf appeared in the fields */

#define GB_FP64   0      /* FP64 everywhere (the reference form) */
#define GB_MIXED  1      /* FP32 perturbation fields around the rest state; FP64 geometry and SARK coefficients */

#define GB_MOTION_STATIC 0
#define GB_MOTION_SINXY  1
#define GB_MOTION_PLUNGE 2   /* rigid plunge: every vertex moves by (0, A sin(2 pi t / T)) */
#define GB_MOTION_TGV3D  3   /* dim = 3: the deformation of the moving Taylor-Green vortex (below) */

#define GB_BC_INTERIOR 0     /* face shared with another element (or its periodic copy) */
#define GB_BC_WALL     1     /* wall moving with the mesh: bounce-back ghost state */
#define GB_BC_FARFIELD 2     /* far field: the free-stream equilibrium as the exterior state */

typedef struct gb_solver gb_solver;   /* opaque */

/* Straight-sided periodic simplex mesh (Sec. 3: affine simplices, fixed topology).
 * The 2D layout is given here; for dim = 3 see "three dimensions" below. */
typedef struct {
  int32_t dim;               /* 2 (triangles) or 3 (tetrahedra) */
  int64_t n_vert;            /* number of unique vertices (periodic images share one id) */
  const double *X;           /* n_vert x 2, Lagrangian (initial) vertex coordinates, host */
  int64_t n_elem;            /* K */
  const int32_t *EToV;       /* n_elem x 3 vertex ids, counter-clockwise, host */
  const double *elem_shift;  /* n_elem x 3 x 2 periodic unwrap offsets (element vertex j of element k
                                sits at X[EToV[k][j]] + elem_shift[k][j]); NULL = no offsets.  Every
                                offset must be an integer multiple (|m| <= 7) of one period per direction. */
} gb_mesh;

/* Prescribed grid motion (Sec. 5 and the free-stream test of Sec. 7.1):
 * GB_MOTION_SINXY displaces both coordinates of a vertex with Lagrangian
 * position X by A sin(2 pi t / T) sin(2 pi X / Lx) sin(2 pi Y / Ly);
 * GB_MOTION_PLUNGE moves every vertex by (0, A sin(2 pi t / T)) (the rigid plunge of
 * the airfoil case of Sec. 7; Lx, Ly unused);
 * GB_MOTION_TGV3D (dim = 3 only; Sec. 7.2, Eq. TGV_deformation) moves each coordinate of
 * the vertex at (X, Y, Z) by A sin(2 pi t / T) S(a) S(b) over the other two coordinates
 * a, b, with S(s) = sin(2 pi (s + L/2) / L), L = Lx (Ly unused); the paper's cube
 * [-pi, pi]^3 takes A = pi/6, T = 20, L = 2 pi. */
typedef struct {
  int32_t kind;              /* GB_MOTION_STATIC, GB_MOTION_SINXY, GB_MOTION_PLUNGE or GB_MOTION_TGV3D */
  double A, T, Lx, Ly;
} gb_motion;

/* gb_create: validate the mesh (GB_EMESH if a face is not shared by exactly two
 * elements or an element has J <= 0), build the order-N reference operators in
 * FP64 (Sec. 3), upload mesh and operators, allocate the state.  N in 1..6.
 * Ma > 0, Re > 0.  precision is GB_FP64 or GB_MIXED.  cuda_stream is a
 * cudaStream_t (NULL = default stream).  The fields start at zero, the vertices
 * at X, the time at 0, the motion static.  On success *out owns the solver. */
int gb_create(const gb_mesh *mesh, int N, double Ma, double Re, int precision,
              void *cuda_stream, gb_solver **out);

/* gb_create_bounded: gb_create for a 2D mesh with boundary faces (the plunging-airfoil
 * O-grid of Sec. 7).  face_bc (host, n_elem x 3, face f running from local vertex f to
 * f + 1) tags each face GB_BC_INTERIOR, GB_BC_WALL or GB_BC_FARFIELD; every interior face
 * must be shared by exactly two elements (periodic copies allowed) and no boundary face
 * may be.  far_state = (rho, u, v) of the free stream.  The paper gives neither condition;
 * the library reads them as: at a wall the particle velocities are reflected about the
 * wall velocity (the grid velocity at the face node), which maps the moments to
 * q1+ = q1, q2+ = 2 wx q1 - q2, q3+ = 2 wy q1 - q3, q4+ = q4 + 4 wx wy q1 - 2 wx q3 - 2 wy q2,
 * q5+ = q5 + 2 sqrt2 (wx^2 q1 - wx q2), q6+ = q6 + 2 sqrt2 (wy^2 q1 - wy q3) with
 * (wx, wy) = v_G / c; at the far field the exterior state is the free-stream equilibrium
 * (no perfectly matched layer).  Both enter the upwind flux as q+.  N in 1..4; groups
 * reject such solvers; everything else as gb_create (dim = 2 only). */
int gb_create_bounded(const gb_mesh *mesh, const int8_t *face_bc, const double *far_state, int N, double Ma,
                      double Re, int precision, void *cuda_stream, gb_solver **out);

/* Perfectly matched layer (dim = 2; the airfoil case's outer boundary, Sec. 7).  The paper
 * uses a PML with auxiliary fields but prints no equations.  Reading implemented here:
 * complex stretching of one direction e (planar approximation) with frequency shift alpha,
 *   dq/dt   = L(q) + Ntilde(q) - sigma Phi,
 *   dPhi/dt = R_e(q) - (alpha + sigma) Phi,
 * L = R_e + R_t the advective terms split into their part along e and the rest: in the
 * volume (A_e + v_G . e) e . grad q with A_e = -c (e_x Atilde_x + e_y Atilde_y); on the faces
 * 1/2 (n.e)(A_e + v_G . e) dq (the central part of the upwind flux along e) plus
 * (n.e)^2 times its dissipation 1/2 (c |Atilde_n| + |v_G . n|) dq, lifted.  Phi (6 fields
 * per node) lives on the layer's elements and advances by the RK4 stages; -sigma Phi joins
 * every field's SARK combinations.  sigma(r) = sigma_max ((r - r0)/d)^power for r > r0, else
 * 0, with r and e at each node's Lagrangian position X:
 *   GB_PML_RADIAL   r = |X - (cx, cy)|, e = (X - (cx, cy)) / r   (an outer ring);
 *   GB_PML_SLAB     r = |(X - (cx, cy)) . u|, e = sign((X - (cx, cy)) . u) u,
 *                   u = (ex, ey) normalised (two layers facing away from a centre line);
 *   GB_PML_UNIFORM  sigma = sigma_max and e = u everywhere (r0, d, power unused).
 * The layer = the elements with a node where sigma > 0. */
#define GB_PML_RADIAL  0
#define GB_PML_SLAB    1
#define GB_PML_UNIFORM 2
typedef struct {
  int32_t kind;              /* GB_PML_RADIAL, GB_PML_SLAB or GB_PML_UNIFORM */
  double cx, cy;             /* centre (radial) or a point on the centre line (slab) */
  double ex, ey;             /* direction u (slab, uniform) */
  double r0, d;              /* the layer starts at r = r0 and grades over depth d > 0 */
  double sigma_max, power;   /* sigma_max >= 0, power >= 0 */
  double alpha;              /* frequency shift >= 0 */
} gb_pml;

/* gb_set_pml: install the layer (copied; NULL removes it) and set Phi = 0.  N <= 4.
 * Synchronises the stream.  gb_set_fields also zeroes Phi.  gb_rhs and gb_rhs_noalloc
 * leave the layer out (they take no Phi); with a layer, gb_set_diagnostics records through
 * separate reduction launches after each step, and gb_step_timed's kernel_ms[i] includes
 * the layer's launch that follows stage kernel i.  Groups reject solvers with a layer.
 * GB_EINVAL for a 3D solver, non-finite or out-of-range parameters. */
int gb_set_pml(gb_solver *s, const gb_pml *p);

/* gb_pml_fields: *n_layer = the number of layer elements; if phi_out (host, n_layer x 6 x Np
 * doubles; FP32 values widened in GB_MIXED) and/or elem_out (host, n_layer) are non-NULL,
 * copy Phi_n and the canonical element ids (ascending, the order of phi_out).
 * Synchronises the stream. */
int gb_pml_fields(gb_solver *s, double *phi_out, int64_t *elem_out, int64_t *n_layer);

/* gb_set_motion: prescribe the vertex velocity d/dt of the displacement above,
 * evaluated at the Lagrangian X (Sec. 5).  Copied; takes effect at the next step. */
int gb_set_motion(gb_solver *s, const gb_motion *m);

/* gb_set_fields: upload q (host, canonical layout, K*6*Np doubles) and set the time t. */
int gb_set_fields(gb_solver *s, const double *q_host, double t);

/* gb_fields: synchronise, check the device status, copy q (canonical FP64) and t
 * to the host.  In GB_MIXED mode q is the FP32 perturbation plus the rest state,
 * widened to FP64.  Returns GB_ENAN / GB_EMESH if a step flagged one. */
int gb_fields(gb_solver *s, double *q_host_out, double *t_out);

/* gb_set_vertices / gb_vertices: current vertex positions x_n (n_vert x 2, host). */
int gb_set_vertices(gb_solver *s, const double *x_host);
int gb_vertices(gb_solver *s, double *x_host_out);

/* gb_nodes: physical node coordinates at the current vertex positions, host,
 * n_elem x Np x 2 (the P1 map of Sec. 3). */
int gb_nodes(gb_solver *s, double *xy_out);

/* gb_rhs: F = L(q) + Ntilde(q) (Sec. 4 splitting; the stiff -Lambda q part is not
 * included) for device arrays q_dev, F_dev in canonical layout (K*6*Np; FP64 in
 * GB_FP64 mode; in GB_MIXED mode FP32, q_dev holding perturbations q - (1,0,0,0,0,0)
 * and F_dev receiving F itself), at the current vertex positions with the grid
 * velocity of time t.  Both arrays are caller-owned device memory, used on the
 * solver's stream; enqueue only.  GB_MIXED uses the solver's stage buffers as
 * scratch, so the call must not overlap a gb_step on another stream. */
int gb_rhs(gb_solver *s, double t, const void *q_dev, void *F_dev);

/* gb_step: enqueue nsteps SARK steps of size dt (Sec. 4): per stage, the vertex
 * positions and velocities (Sec. 5), the geometric factors (GCL), the volume,
 * surface and cubature terms and the SARK combination.  Enqueue only; errors of
 * the device computation are reported by gb_sync / gb_fields.  On a non-default
 * stream and for nsteps >= 2 one step is captured as a CUDA graph (after one
 * direct step with the same dt) and replayed; the graph is rebuilt after a
 * change of dt, motion or stream.  gb_set_graph(s, 0) turns this off. */
int gb_step(gb_solver *s, double dt, int64_t nsteps);
int gb_set_graph(gb_solver *s, int enable);

/* gb_launch_config: the GB_MIXED launch shape (0 for GB_FP64):
 *   1, 2, 4  the mma.sync kernel: 16-element warp tiles, that many warps per CTA;
 *   8        the tcgen05 kernel: 128-element CTA tiles, accumulators in tensor
 *            memory (orders 1..4, meshes without boundary faces).
 * Both compute the same right-hand side and SARK step (they agree to rounding; the
 * three warp-tile shapes agree bit for bit).  With the fused diagnostics the last
 * stage of shape 8 runs on the 4-warp kernel.  The first gb_step / gb_step_timed of
 * a GB_MIXED solver tunes the shape: it times the right-hand-side kernel on the
 * solver's own data for each applicable shape (the state is not changed) and keeps
 * the fastest (a smaller shape must win by 3%); the choice is cached in the process
 * per device and per (N, size class of K), the size class being the bit length of
 * K - 1.
 * For dim = 3 solvers (GB_MIXED; 0 for GB_FP64):
 *   1..8     the tensor-core kernel: 16-element warp tiles on mma.sync TF32 split
 *            products, that many warps per CTA sharing the operator table in shared
 *            memory (orders 1..3; at most as many as fit, 7 at N = 3 and 8 at N <= 2);
 *   16       the FP32 one-thread-per-node kernel (every order; the only one at N = 4).
 * Before the first step of an untuned solver this reports the tensor-core kernel with
 * the most warps; that step then times stages 0..2 of it against shape 16 on the
 * solver's own data and keeps the faster (shape 16 must win by 3%), for that solver
 * (not cached: which one wins depends on the mesh and motion).  The two agree to
 * rounding; all warp counts agree bit for bit. */
int gb_launch_config(gb_solver *s, int *warps_per_cta);
/* gb_set_launch_config: fix the GB_MIXED launch shape (1, 2, 4 or 8; for dim = 3:
 * 1..8 as above or 16) and skip the tuner.  GB_EINVAL for other values, for a shape that
 * does not apply to the solver's order or mesh, and for GB_FP64 solvers. */
int gb_set_launch_config(gb_solver *s, int warps_per_cta);

/* gb_step_timed: gb_step that also records a CUDA event pair around every kernel
 * launch on the solver's stream (tracing), synchronises, and adds the device time
 * in milliseconds of each kernel kind to kernel_ms[0..4]: the fused stage kernels
 * of stages 0..3, then the vertex update.  kernel_ms is host memory of 5 doubles
 * (not cleared).  Returns the device status like gb_sync. */
int gb_step_timed(gb_solver *s, double dt, int64_t nsteps, double *kernel_ms);

/* gb_diagnostics: integrals of the current state over the moving mesh (the kinetic
 * energy diagnostic of Sec. 7.2 and conservation checks), each the exact integral
 * of the degree-N nodal interpolant (J sum_i w_i f_i per element, w = 1^T Mhat):
 * out[0] = int rho, out[1] = E_K = (1/|Omega|) int rho |u|^2 / 2 (rho_inf = 1),
 * out[2] = int rho u, out[3] = int rho v, out[4] = |Omega|.  Host array of 5
 * doubles; synchronises the stream.  Reductions in FP64 in both precisions. */
int gb_diagnostics(gb_solver *s, double *out);

/* gb_set_diagnostics: record the integrals of gb_diagnostics after every `every`-th
 * step of gb_step, gb_step_timed and gb_group_step, on the device and without host
 * synchronisation (the launches join the step, and its CUDA graph), into a ring of
 * `capacity` records of 6 doubles: t, int rho, E_K, int rho u, int rho v, |Omega|.
 * Counting starts at this call; every = 0 stops recording and frees the ring.
 * Synchronises the stream.  GB_EINVAL for every < 0 or capacity outside 1 .. 2^32. */
int gb_set_diagnostics(gb_solver *s, int every, int64_t capacity);

/* gb_diagnostics_history: copy the most recent records (at most max; host array of
 * max x 6 doubles), oldest first; *count = records copied, *total (may be NULL) =
 * records written since recording began (those beyond `capacity` are overwritten).
 * Synchronises the stream; *count = 0 when recording is off. */
int gb_diagnostics_history(gb_solver *s, double *out, int64_t max, int64_t *count, int64_t *total);

/* gb_sync: synchronise the stream, return and clear the device status
 * (GB_OK, GB_ENAN or GB_EMESH). */
int gb_sync(gb_solver *s);

/* gb_set_stream: finish the work enqueued on the solver's current stream, then use
 * cuda_stream for all later work (e.g. set a solver up on one stream and step it
 * in a group on another). */
int gb_set_stream(gb_solver *s, void *cuda_stream);

/* gb_info: sizes and derived constants.  Any output pointer may be NULL. */
int gb_info(gb_solver *s, int *Np, int *Nfp, int *Nc, int64_t *n_elem, int64_t *n_vert,
            double *c, double *tau, int64_t *device_bytes);

/* ---- groups (batched stepping of many simulations) --------------------------
 * A group steps several GB_MIXED solvers of the same order N with one launch
 * per SARK stage (a persistent kernel over the 16-element tiles of all of them,
 * the mma.sync kernel) plus one vertex-update launch per step.  Every solver
 * keeps its own fields, mesh, motion, time and step size; the result of each
 * solver is bitwise the same as stepping it alone with gb_step on a warp-tile
 * launch shape (1, 2 or 4).  The first gb_group_step of an order and size class
 * (the group's tile count, in powers of two) times the group kernel with 4, 2
 * and 1 warps per CTA on the group's own data (stage-0 launches, which only write
 * buffers the step rewrites) and keeps the fastest, cached for the process.
 * gb_group_create allocates the
 * descriptor buffers for up to `capacity` solvers (device and pinned host
 * memory) and uses `cuda_stream` for all its work; the solvers of a group must
 * have been created on that same stream.  gb_group_step enqueues nsteps steps
 * of solvers[0..n-1] with step sizes dt[0..n-1] (enqueue only; per-solver
 * device errors are reported by gb_sync / gb_fields of each solver). */
typedef struct gb_group gb_group;
int gb_group_create(int capacity, void *cuda_stream, gb_group **out);
int gb_group_step(gb_group *g, gb_solver *const *solvers, const double *dt, int n, int64_t nsteps);
int gb_group_destroy(gb_group *g);
const char *gb_group_last_error(gb_group *g);
/* gb_group_launch_config: the group kernel's warps per CTA last used for order N
 * (0 before the first gb_group_step of that order).  GB_EINVAL for NULL or N out of
 * 1..6. */
int gb_group_launch_config(gb_group *g, int N, int *warps_per_cta);
/* gb_group_set_launch_config: fix the group kernel's warps per CTA (1, 2 or 4) for
 * order N and skip its tuner (all shapes give bitwise-equal results).  GB_EINVAL for
 * other values or N out of 1..6. */
int gb_group_set_launch_config(gb_group *g, int N, int warps_per_cta);

/* gb_state_ptr: the device address of the current fields, owned by the solver and
 * valid until gb_destroy: the canonical FP64 layout in GB_FP64 mode; in GB_MIXED
 * mode an internal layout (FP32 perturbations, elements renumbered along a Morton
 * curve, padded element stride) that only gb_fields translates. */
int gb_state_ptr(gb_solver *s, void **q_dev);

/* gb_rhs_noalloc: the same F as gb_rhs, for GB_MIXED solvers, without the
 * library touching any device memory it allocated for scratch.  (The paper has
 * no counterpart; this is an interface for a particular kind of caller.)
 *
 * Who needs it: a process whose device memory is handed out by its own pool or
 * budget -- for instance a serving host that reserves its HBM at start-up --
 * must not have a library call cudaMalloc or cudaFree behind its back, and may
 * also want to evaluate a right-hand side without disturbing the solver's
 * stage buffers, which gb_rhs of a GB_MIXED solver uses as scratch.  This call
 * allocates and frees nothing: its scratch (the kernel-layout copies of q and
 * F) is a static device array of 16 MiB that every GPU loading libgb holds
 * until the process exits.
 *
 * Arguments and layout are those of gb_rhs in GB_MIXED mode (q_dev: canonical
 * FP32 perturbations, F_dev: canonical FP32 F, both caller-owned device
 * memory); work is enqueued on the solver's stream.  Limits and errors:
 *  - GB_EINVAL for a GB_FP64 solver (its gb_rhs needs no scratch) and for a
 *    mesh whose two internal copies exceed the array (at N = 4 about 22.8k
 *    elements, N = 3 35k, N = 2 58k), with the limit in gb_last_error.
 *  - GB_EINVAL for a non-finite t, and when the current device is not the
 *    solver's (the device current at gb_create): make it current first.
 *  - The first call for a solver of a given device looks up the array's
 *    device address on that device (cudaGetSymbolAddress, once per device,
 *    under a lock); make that first call before any stream capture.
 *  - Every call, on any solver and stream, shares the one array, which keeps
 *    the last call's contents (the call clears what it needs cleared): calls
 *    that overlap on the GPU race and must be ordered by the caller. */
int gb_rhs_noalloc(gb_solver *s, double t, const void *q_dev, void *F_dev);

int gb_destroy(gb_solver *s);
const char *gb_last_error(gb_solver *s);

/* ---- host-side queries (no GPU needed) ---------------------------------- */

/* gb_reference_operators: the library's order-N reference operators (Sec. 3),
 * row-major FP64: r, s [Np]; Dr, Ds [Np x Np]; LIFT [Np x 3 Nfp] (face nodes
 * counter-clockwise: face 0 from (-1,-1) to (1,-1), face 1 to (-1,1), face 2 back);
 * Icub [Nc x Np]; Pcub [Np x Nc]; cubature points/weights cr, cs, cw [Nc].  Any
 * output may be NULL; *Nc_out receives Nc (the degree-3N Stroud rule). */
int gb_reference_operators(int N, double *r, double *s, double *Dr, double *Ds, double *LIFT,
                           double *Icub, double *Pcub, double *cr, double *cs, double *cw,
                           int *Nc_out);

/* gb_sark_coefficients: SARK-4 coefficients of Sec. 4 for gamma = -dt/tau <= 0:
 * E[5] = exp(c_i gamma) (i = 0..3) and exp(gamma); A[16] row-major atilde (strictly
 * lower); B[4] btilde.  Evaluated through phi-functions (series for |gamma| < 1). */
int gb_sark_coefficients(double gamma, double *E, double *A, double *B);

/* ---- three dimensions (tetrahedra, 10 fields) --------------------------------
 * The paper runs the same scheme on tetrahedra (Sec. 3: simplices in two and
 * three dimensions; Sec. 2: n = 10 Hermite coefficients in 3D).  gb_create with
 * mesh->dim == 3 builds a 3D solver; then:
 *  - mesh: X is n_vert x 3, EToV n_elem x 4 with det[v1-v0, v2-v0, v3-v0] > 0,
 *    elem_shift n_elem x 4 x 3 (integer multiples |m| <= 7 of one period per
 *    direction); n_elem < 2^26; every face (vertex-id triple) shared by exactly
 *    two elements (periodic meshes).  N in 1..4.
 *  - reference tetrahedron (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1); canonical
 *    field layout q[k][f][i] with f < 10 fields and i < Np = (N+1)(N+2)(N+3)/6
 *    Warp & Blend nodes (Warburton 2006, tetrahedral alpha), ordered by the
 *    equidistant lattice indices (i, j, k) = N (l1, l2, l3) before warping,
 *    i fastest, k slowest (l1 = (1+r)/2, l2 = (1+s)/2, l3 = (1+t)/2).
 *  - fields: moments of multi-index (0,0,0); (1,0,0), (0,1,0), (0,0,1); (1,1,0),
 *    (1,0,1), (0,1,1); (2,0,0), (0,2,0), (0,0,2): q1 = rho, q2..q4 = rho u / c,
 *    q5..q10 the second-order coefficients (equilibrium q_{i+j} = q_i q_j / q1,
 *    q_{2i} = q_i^2 / (sqrt2 q1)); fields 1..4 step with RK4, 5..10 with the
 *    exponential SARK coefficients.
 *  - motion: gb_set_wave_motion (below), or gb_set_motion with GB_MOTION_STATIC or
 *    GB_MOTION_TGV3D (GB_EINVAL for non-finite A, T <= 0 or Lx = 0).
 *  - gb_nodes writes n_elem x Np x 3; gb_vertices / gb_set_vertices n_vert x 3.
 *  - GB_MIXED: FP32 perturbations around the rest state in the canonical layout
 *    (gb_rhs takes and returns that layout; gb_state_ptr points at it), FP64
 *    geometry, motion and SARK coefficients; no tensor-core contractions.
 *  - gb_step, gb_step_timed (kernel_ms[0..4] as in 2D), gb_rhs, gb_sync, gb_info,
 *    gb_set_graph, gb_set_stream, gb_state_ptr, gb_destroy and gb_last_error
 *    work as in 2D.
 *  - diagnostics: gb_diagnostics gives out[4] = the volume |Omega| (the rest as in 2D);
 *    gb_diagnostics3d (below) adds int rho w.  gb_set_diagnostics and
 *    gb_diagnostics_history work as in 2D with the same 6-double records (t, int rho,
 *    E_K, int rho u, int rho v, |Omega|), taken by separate reduction launches at the
 *    end of the recorded steps (inside the step's CUDA graph).
 *  - groups, gb_rhs_noalloc and launch configuration return GB_EINVAL. */

/* Travelling-wave lateral motion of a deforming channel (dim = 3): the vertex with
 * Lagrangian position (X, Y, Z) moves in y by
 *   A(X) sin(2 pi X / wavelength - omega t) exp(-r^2 / r0sq),
 *   A(X) = A0 + A1 X / Lx,  r^2 = (Y - yc)^2 + (Z - zc)^2,
 * with the velocity of that Lagrangian point (Sec. 5). */
typedef struct {
  double A0, A1, Lx, wavelength, omega, r0sq, yc, zc;
} gb_wave_motion;

/* gb_set_wave_motion: set the motion of a dim = 3 solver (copied; takes effect at
 * the next step).  A0 = A1 = 0 or omega = 0 is a static mesh.  GB_EINVAL for a
 * 2D solver, non-finite parameters, Lx = 0, wavelength = 0 or r0sq <= 0. */
int gb_set_wave_motion(gb_solver *s, const gb_wave_motion *m);

/* gb_diagnostics3d: integrals of the current state of a dim = 3 solver, each the exact
 * integral of the degree-N nodal interpolant (J sum_i w_i f_i per tetrahedron,
 * w = 1^T Mhat): out[0] = int rho, out[1] = E_K = (1/|Omega|) int rho |u|^2 / 2
 * (rho_inf = 1; the kinetic energy of Sec. 7.2), out[2..4] = int rho u, rho v, rho w,
 * out[5] = |Omega|.  Host array of 6 doubles; synchronises the stream; FP64 reductions
 * in a fixed order in both precisions.  GB_EINVAL for a 2D solver. */
int gb_diagnostics3d(gb_solver *s, double *out);

/* gb_reference_operators3d: the library's order-N tetrahedral operators (Sec. 3),
 * row-major FP64, host only: r, s, t [Np]; Dr, Ds, Dt [Np x Np]; LIFT [Np x 4 Nfp]
 * (faces (v0,v1,v2), (v0,v1,v3), (v1,v2,v3), (v0,v2,v3), face nodes in increasing
 * volume index, face measure of area 2 per face); Icub [Nc x Np]; Pcub [Np x Nc];
 * cr, cs, ct, cw [Nc] (conical-product rule exact for degree 3N, Nc = q^3,
 * q = ceil((3N+1)/2)).  Any output may be NULL.  N in 1..4. */
int gb_reference_operators3d(int N, double *r, double *s, double *t, double *Dr, double *Ds, double *Dt,
                             double *LIFT, double *Icub, double *Pcub, double *cr, double *cs, double *ct,
                             double *cw, int *Nc_out);

#ifdef __cplusplus
}
#endif
#endif /* GB_H */
