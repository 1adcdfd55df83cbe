/*
 * dgimex.h -- C ABI of the GB300 (sm_103a) hot path of a rotating IMEX-DG
 * solver for the compressible Euler equations on quad/hex meshes with 2:1
 * hanging faces (Bottani, Benacchio, Orlando, Bonaventura, Engsig-Karup:
 * "An IMEX-DG solver with non-conforming mesh refinement for atmospheric
 * dynamics with rotation").
 *
 * Discretisation (Section 3): nodal DG on (r+1)^d Gauss-Legendre points per
 * cell (collocated with the quadrature), Rusanov flux with
 * lambda = max(|u-.n|, |u+.n|) for advection, centred fluxes for pressure
 * and enthalpy, ARK2 IMEX stepping (TR-BDF2 implicit tableau,
 * chi = 2 - sqrt 2, a32 = 1/2), Picard iteration over the Schur complement
 * of the momentum/energy system (strategies R1 and R2), GMRES on the
 * pressure system, (A+R)^{-1} = (I + beta J)^{-1} A^{-1} with the closed-form
 * 3x3 inverse (Section 3.1).
 *
 * Conventions for every call:
 *  - All functions return a dg_status; nothing throws across the ABI.
 *  - Device arrays are caller-owned, contiguous, FP64, on the context's
 *    device.  Field-major SoA: array[field][cell][node]; nodes of a cell in
 *    tensor order with x fastest.  N = n_elem * (r+1)^d nodes.
 *    State q has 5 fields (rho, rho u, rho v, rho w, rho E) -- in 2D (x-z
 *    vertical slice, eq. vertical_slice) v is carried but has no derivative.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    apply_* calls are asynchronous on it; calls that fill an info struct
 *    synchronise the stream before returning.
 *  - Library-owned workspace (traces, face fluxes, Krylov basis) is
 *    allocated lazily per mesh and released by dg_mesh_destroy.  A context
 *    and its meshes are not thread-safe.
 */
#ifndef DGIMEX_H
#define DGIMEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,           /* invalid argument or inconsistent mesh lists */
  DG_ERR_UNSUPPORTED = -2,   /* valid but not implemented (e.g. GLL nodes) */
  DG_ERR_CUDA = -3,          /* CUDA runtime error (message: dg_last_error) */
  DG_ERR_NOT_CONVERGED = -4, /* iteration limit hit; best iterate returned */
  DG_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  DG_ERR_NONFINITE = -6,     /* NaN/Inf met in a norm or reduction */
  DG_ERR_OOM = -7            /* device allocation failed */
} dg_status;

enum { DG_NODES_GL = 0, DG_NODES_GLL = 1 };
enum { DG_BC_WALL = 1, DG_BC_FARFIELD = 2 };
enum { DG_R1 = 1, DG_R2 = 2 };
enum { DG_FP64 = 0, DG_MIXED = 1, DG_MIXED_EXPLICIT = 2, DG_PAIRS = 3 };

typedef struct dg_ctx dg_ctx;
typedef struct dg_mesh dg_mesh;

/* Human-readable name of a status code; message of the last failure. */
const char* dg_status_string(int status);
const char* dg_last_error(void);

/* Create a context on CUDA device `device` (makes it current). */
int dg_ctx_create(int device, dg_ctx** out);
void dg_ctx_destroy(dg_ctx* ctx);

/*
 * Mesh description (host arrays, copied by dg_mesh_create).
 *  dim        2 (x-z slice) or 3.
 *  degree     r in 1..4; nodes per cell (r+1)^dim.
 *  node_set   DG_NODES_GL (Section 3: Gauss-Legendre nodes) or DG_NODES_GLL
 *             (Gauss-Lobatto nodes, always with (r+1)-point Gauss-Legendre
 *             quadrature: the mass matrix S^T W S and its inverse
 *             S^{-1} W^{-1} S^{-T} of Section 3.1).  With GLL every nodal
 *             array of every call is in the GLL basis (nodes at the GLL
 *             points, dg_mesh_node_coords gives them); the library runs the
 *             operators in the GL basis of the same polynomials and changes
 *             basis per cell on the way in and out.  GLL meshes support the
 *             explicit and implicit operators, the Schur right-hand side,
 *             the velocity recovery, unpreconditioned GMRES and the
 *             host-driven step in DG_FP64 and DG_MIXED; the rest
 *             (preconditioners, graph mode, DG_MIXED_EXPLICIT, damping
 *             layers, E_geo, ensembles, the no-alloc call) answers
 *             DG_ERR_UNSUPPORTED.
 *  vertices   n_elem x 2^dim x dim doubles: corner v of a cell sits at
 *             reference corner (v&1, (v>>1)&1[, (v>>2)&1]); the cell map is
 *             multilinear (curved terrain-following cells included).
 *  int_faces  n_int x 4: [eL, fL, eR, fR], face f = 2a+s is xi_a = s;
 *             requires fL = 2a+1, fR = 2a (eL on the low side; periodic
 *             pairs listed the same way); tangential axes aligned.
 *  hang_faces n_hang x 5: [e_coarse, f_coarse, e_fine, f_fine, subface];
 *             2:1 only; f_fine = f_coarse ^ 1; bit t of subface selects the
 *             half along the t-th tangential axis.
 *  bdry_faces n_bdry x 3: [e, f, bc]: DG_BC_WALL (slip wall, mirror state)
 *             or DG_BC_FARFIELD (the non-reflecting top of Section 4.3, read
 *             as a far-field face whose outer state is a given background
 *             state: dg_mesh_set_far_state).
 * Every face of every cell must be covered exactly once (interior side,
 * fine hanging side, one of the 2^(dim-1) coarse subfaces, or boundary);
 * otherwise DG_ERR_ARG.
 */
typedef struct {
  int dim, degree, node_set;
  int64_t n_elem;
  const double* vertices;
  int64_t n_int;
  const int64_t* int_faces;
  int64_t n_hang;
  const int64_t* hang_faces;
  int64_t n_bdry;
  const int64_t* bdry_faces;
} dg_mesh_desc;

int dg_mesh_create(dg_ctx* ctx, const dg_mesh_desc* desc, dg_mesh** out);
void dg_mesh_destroy(dg_mesh* mesh);

/* Host-only check of a mesh description: every rule dg_mesh_create applies
 * before it touches the GPU (dim, degree, node set, list ranges, face
 * coverage, finite vertices), with the same status and message, and no
 * context or device needed.  Not checked here: det(J) > 0 at the nodes,
 * which dg_mesh_create tests with its geometry kernels. */
int dg_mesh_validate(const dg_mesh_desc* desc);

typedef struct {
  int dim, degree, n1d, nodes_per_elem;
  int64_t n_elem, n_nodes, n_face_points, n_hang_points;
  int64_t workspace_bytes;   /* library-owned device memory held now */
  int tile_fp64[3];          /* cells-per-block multipliers (1, 2, 4) of the */
  int tile_fp32[3];          /* explicit, gradient and divergence cell kernels
                                (entries 1 and 2: the schedule-2 vmult passes;
                                the other fused schedules run one tile size) */
  int terrain_following;     /* 1: every cell has x = x(xi_1) (and y = y(xi_2)),
                                so the cell kernels skip the metric terms that
                                vanish exactly (not in the paper) */
  int fused_stage[3];        /* FP64, FP32, FP32-pair Schur vmult: 1 =
                                plus-side face values from the neighbour
                                cells' node lines, 0 = from a trace array
                                written by a separate pass, 2 = one thread
                                per x-line (see dg_mesh_set_fused_stage) */
} dg_mesh_stats;
int dg_mesh_info(const dg_mesh* mesh, dg_mesh_stats* out);

/* Schedule autotuner (not in the paper): times the explicit operator's
 * cell kernel with 1, 2 and 4 times the base number of cells per thread
 * block, and whole Schur vmults with every fused-kernel schedule (see
 * dg_mesh_set_fused_stage; schedule 2, on three-dimensional degree-3
 * terrain-following meshes, with 1, 2 and 4 times its base cells per
 * block), on this mesh (synthetic coefficients, CUDA
 * events), and keeps the fastest, for FP64 and, when precision is DG_MIXED
 * or DG_MIXED_EXPLICIT, for the FP32 vmult too, when it is DG_PAIRS for the
 * FP32-pair vmult.  Allocates temporary device memory; synchronises
 * `stream`.  Results in dg_mesh_stats. */
int dg_mesh_autotune(dg_ctx* ctx, dg_mesh* mesh, int precision, void* stream);

/* Schedule of the fused face + cell kernels of the Schur vmult, right-hand
 * side and velocity recovery (not in the paper): per precision (FP64, FP32,
 * FP32 pairs of DG_PAIRS), 1 reads the neighbour cell's node line through
 * each face point and contracts it to the face in the kernel (no trace
 * pass, more arithmetic), 0 reads the neighbour's face values from a trace
 * array that a separate pass writes (less arithmetic, more memory
 * traffic), 2 runs the two vmult passes with one thread per x-line of a
 * cell (three dimensions, degree 3, vectors 16-byte aligned: 128-bit loads,
 * the x-direction work in registers; elsewhere, and for the right-hand
 * side and the recovery, 2 acts as 1).  All give the same results up to
 * rounding.  Defaults: FP64 0, FP32 1, pairs 0; dg_mesh_autotune times them
 * and keeps the fastest.  DG_ERR_ARG for values outside 0..2.  Host only,
 * no GPU work. */
int dg_mesh_set_fused_stage(dg_mesh* mesh, int fp64, int fp32, int pairs);

/* Cells per block of the schedule-2 vmult passes, as a multiplier tile
 * (1, 2 or 4) of the base count, for one precision (DG_FP64, DG_MIXED or
 * DG_MIXED_EXPLICIT for the FP32 vmult, DG_PAIRS); dg_mesh_autotune sets it
 * together with the schedule.  DG_ERR_ARG for other values.  Host only, no
 * GPU work. */
int dg_mesh_set_vmult_tile(dg_mesh* mesh, int precision, int tile);

/* Physical coordinates of all nodes: xyz[dim][cell][node] (device, FP64). */
int dg_mesh_node_coords(dg_ctx* ctx, const dg_mesh* mesh, double* xyz, void* stream);

/* Physics: gamma, g, f of eq. governing_equations_2 (f-plane, k = vertical
 * unit vector = last coordinate); variant R1/R2 (Section 3); penalty = 1
 * keeps the Rusanov term on rho e implicit at stage l (as a lagged-lambda
 * jump term added to D). */
typedef struct {
  double gamma, g, f;
  int variant;
  int penalty;
  int precision;             /* DG_FP64; DG_MIXED: Schur vmults inside the
                                Krylov solves run in FP32 (FP32 accumulation)
                                under FP64 iterative refinement; the outer
                                residual, orthogonalisation, reductions,
                                Schur right-hand side, velocity recovery and
                                explicit operator stay FP64;
                                DG_MIXED_EXPLICIT: DG_MIXED plus the explicit
                                operator in FP32 on perturbations (see
                                dg_mesh_set_background and imex_ark2_step);
                                DG_PAIRS (not in the paper; an emulation, not
                                IEEE FP64): the Schur vmults inside the
                                Krylov solves run on the FP32 pipe in pairs
                                of FP32 numbers (hi + lo, about 48
                                significant bits, about 1e-14 relative per
                                operation), everything else as DG_FP64;
                                plain FP64 GMRES, no refinement. */
  const double* f_cell;      /* optional device array, one Coriolis parameter
                                per cell (NULL: f everywhere); lets one mesh
                                carry several independent instances */
  double lambda_min;         /* not in the paper: floor (m/s, >= 0) of the
                                Rusanov coefficient of the non-stiff fluxes
                                (rho, rho u, rho kappa); 0 keeps the paper's
                                lambda = max(|u-.n|, |u+.n|).  At rest that
                                lambda vanishes and a cell-to-cell
                                checkerboard of vertical momentum, invisible
                                to the centred pressure flux, grows through
                                the explicit density at the buoyancy
                                frequency (about 9 % per step on the
                                planetary wave at dt = 10 s); 1 m/s damps it.
                                The stiff rho e Rusanov term and its implicit
                                counterpart keep |u.n|. */
} dg_phys;

/*
 * Explicit operator (stage rates), Section 3: weak residuals of the
 * non-stiff part f_NS (advection: rho u, rho u (x) u, kappa rho u with
 * Rusanov) and of the stiff part f_S (pressure with centred {p}, enthalpy
 * flux h rho u with centred flux and Rusanov on rho e, gravity -rho g k,
 * Coriolis -f rho k x u, -g rho k.u), multiplied by the inverse mass matrix.
 *  q     in : 5 x N
 *  f_ns  out: 5 x N   (rho, rho u, rho v, rho w, rho E rates)
 *  f_s   out: 4 x N   (rho u, rho v, rho w, rho E rates; the rho rate is 0)
 */
int dg_apply_explicit(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                      const double* q, double* f_ns, double* f_s, void* stream);

/*
 * Geostrophic imbalance (Section 4, planetary-scale inertia-gravity wave,
 * eq. egeo): E_geo = domain mean of |(1/rho) dp/dx - f v|, with the
 * scheme's own FP64 discrete pressure gradient and Coriolis term (the stiff
 * x-momentum rate of dg_apply_explicit, divided by rho at each node) and
 * the volume quadrature weights w det J; the domain measure is the sum of
 * the weights (x_max z_max on a flat box).  In 3D the x-momentum balance is
 * averaged over the volume.  q: device 5 x N; *e_geo: host.  Synchronises
 * `stream`.  phys->precision is ignored (always FP64).
 */
int dg_geostrophic_error(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                         const double* q, double* e_geo, void* stream);

/*
 * Background for the FP32 explicit operator (DG_MIXED_EXPLICIT).  q_bg
 * (device, 5 x N, FP64, e.g. the balanced hydrostatic state) is copied; its
 * rates F(q_bg) are computed once in FP64 (again whenever gamma, g, f or
 * f_cell change).  Afterwards, with phys->precision == DG_MIXED_EXPLICIT,
 * dg_apply_explicit and every stage of imex_ark2_step evaluate
 * F(q) = F(q_bg) + [F(q) - F(q_bg)], the difference in FP32 from
 * q' = q - q_bg (subtracted in FP64) with every nonlinear flux expanded
 * about the background so that no background-sized term cancels, and the
 * Rusanov term split as lambda/2 [q'] + (lambda - lambda_bg)/2 [q_bg] with
 * the background jumps and lambda_bg taken from FP64.  The background stays
 * until the mesh is destroyed.  Accuracy: F' to FP32 precision of F', but
 * after whole steps the perturbation fields carry errors of 1e-6 to 1e-4
 * relative L2 (the stiff explicit rates amplify the FP32 error of F').
 * Without a background, imex_ark2_step under DG_MIXED_EXPLICIT computes the
 * first-stage rates F(q^n) in FP64 and the later stages' rates as FP32
 * increments about q^n, which keeps the FP32 error proportional to the
 * change within one step; dg_apply_explicit then returns DG_ERR_ARG.
 */
int dg_mesh_set_background(dg_ctx* ctx, dg_mesh* mesh, const dg_phys* phys,
                           const double* q_bg, void* stream);

/*
 * Outer state of the far-field faces (DG_BC_FARFIELD; reading of the
 * non-reflecting upper boundary of Section 4.3).  q_far: device 5 x N nodal
 * state (e.g. the background atmosphere); its traces at the far-field face
 * points are stored (the array itself is not kept).  The explicit operator
 * uses them as the plus state of those faces in the same Rusanov and centred
 * fluxes as at an interior face (lambda = max(|u-.n|, |u_far.n|)).  In the
 * implicit stage system the outer state is known data: B, C and the
 * implicit Rusanov term keep their inner halves ({x} = x-/2, (h rho u)-.n/2,
 * lambda x-), and the outer halves move to the right-hand sides
 * (dg_schur_rhs subtracts M^{-1} b_far and M^{-1} g_far from the
 * predictors, dg_recover_velocity M^{-1} b_far).  Required before any
 * operator call on a mesh with far-field faces (else DG_ERR_ARG); a no-op
 * on a mesh without them.  DG_MIXED_EXPLICIT and ensembles are not
 * available with far-field faces (DG_ERR_UNSUPPORTED); the preconditioners
 * treat them as walls (they stay approximate inverses; the flexible GMRES
 * still solves the exact system).
 */
int dg_mesh_set_far_state(dg_ctx* ctx, dg_mesh* mesh, const double* q_far, void* stream);

/*
 * Rayleigh damping (sponge) layers of the orography tests (Section 4, eq.
 * damping).  With layers set, every evaluation of the explicit operator on
 * this mesh (dg_apply_explicit, each stage of imex_ark2_step, host-driven or
 * graph) adds -lambda(x) (q - q_bar) to the non-stiff rates f_NS of all five
 * conserved fields.  lambda = lambda_bar sin^2(pi/2 (z - z_b)/(z_t - z_b))
 * for z >= z_b, 0 below; lateral layers (x_layers / y_layers = 1, y in 3D
 * only) ramp the same way over their width from lo + width down to lo and
 * from hi - width up to hi; where layers overlap the largest lambda
 * applies; ramp arguments are clipped to [0, 1].  The damping is explicit:
 * one ARK2 step multiplies a pure relaxation by the explicit stability
 * polynomial R(-lambda dt), |R| < 1 up to lambda dt of about 2.5 (the
 * paper uses lambda_bar dt = 1.2).
 * q_bar: 5 x N device state, copied; s == NULL switches the layers off.
 * Applied by dg_apply_explicit_noalloc too; not applied by ensembles.
 */
typedef struct {
  double lambda_bar;               /* 1/s */
  double z_b, z_t;                 /* top layer: zero below z_b, lambda_bar at z_t */
  int x_layers;                    /* 1: layers inside both ends of [x_lo, x_hi] */
  double x_lo, x_hi, x_width;
  int y_layers;                    /* 1: the same in y (3D) */
  double y_lo, y_hi, y_width;
} dg_sponge;
int dg_mesh_set_sponge(dg_ctx* ctx, dg_mesh* mesh, const dg_sponge* s, const double* q_bar, void* stream);

/* Coefficients frozen during one Picard iteration of stage l (device,
 * N each; u_lag 3 x N): rho^(n,l), p^(n,l,k), u^(n,l,k); a_dt = at_ll dt. */
typedef struct {
  const double* rho;
  const double* p_lag;
  const double* u_lag;
  double a_dt;
} dg_implicit_coeffs;

/*
 * Schur-complement vmult, Section 3 (R1 / R2 pressure systems), scaled by
 * D^{-1} (D = M / (gamma-1), the diagonal mass term):
 *   R2: y = D^{-1} [ D + P - (C^(k) + M_g)(A + R)^{-1} B ] x
 *   R1: y = D^{-1} [ D + P - C^(k) A^{-1} B ] x
 * B: centred weak gradient times a_dt; A: rho-weighted mass; R = beta A J,
 * beta = a_dt f; C: weak divergence of h rho u with h rho = gamma p_lag /
 * (gamma - 1); M_g = a_dt g rho k.; P: implicit Rusanov jump term
 * a_dt/(2(gamma-1)) lambda^(k) [.][.] (zero when phys->penalty == 0).
 *  x in: N, y out: N (must not alias x).
 */
int dg_apply_implicit(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                      const dg_implicit_coeffs* cf, const double* x, double* y,
                      void* stream);

/*
 * Right-hand side of the scaled pressure system from the stage vectors
 * m_hat (3 x N, nodal momentum predictor = M^{-1} f) and e_hat (N, nodal
 * energy predictor = M^{-1} g):
 *   R2: rhs = D^{-1} [ g - k^(k) - (C + M_g)(A + R)^{-1} (f - f_g) ]
 *   R1: rhs = D^{-1} [ g - M_g u^(k) - k^(k) - C A^{-1} (f - R u^(k) - f_g) ]
 */
int dg_schur_rhs(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                 const dg_implicit_coeffs* cf, const double* m_hat,
                 const double* e_hat, double* rhs, void* stream);

/* Velocity recovery once p is known (u out: 3 x N):
 *   R2: u = (A + R)^{-1} (f - f_g - B p)
 *   R1: u = A^{-1} (f - f_g - R u^(k) - B p) */
int dg_recover_velocity(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                        const dg_implicit_coeffs* cf, const double* m_hat,
                        const double* p, double* u, void* stream);

/* Restarted GMRES(restart) with classical Gram-Schmidt (a second pass when
 * the first cancels |w| by more than 1e3) and FP64 device reductions on the
 * scaled Schur system; stops when
 * ||b - S x||_2 <= rtol ||b||_2.  x in: initial guess, out: solution (best
 * iterate and DG_ERR_NOT_CONVERGED after maxit).  Synchronises `stream`.
 * With phys->precision == DG_MIXED the solve is iterative refinement: the
 * residual r = b - S x is formed with the FP64 vmult, a correction d with
 * S d ~ r is found by GMRES whose vmults run in FP32 (to relative residual
 * inner_rtol, default 1e-4 when 0), x += d, until the FP64 test above
 * holds; maxit bounds the inner iterations in total.
 *
 * precond (not in the paper, whose GMRES is unpreconditioned):
 *   DG_PRECOND_NONE  (0) plain GMRES as above;
 *   DG_PRECOND_VLINE (1) right preconditioning by the vertical-line solve:
 *     the part of S that couples the nodes of one vertical line of cells
 *     (chains joined by conforming faces of the last reference direction
 *     that end in walls at both ends) -- vertical gradient and divergence
 *     through the K_dd metric entry and the z normals, the vertical faces'
 *     penalty, gravity -- factored in FP32 once per dg_gmres_solve call and
 *     once per stage of imex_ark2_step (from the first Picard iterate; block Thomas,
 *     2n x 2n blocks in the unknowns x and w_z of a cell line) and applied
 *     once per Arnoldi step in flexible form (the vectors Z_j = P^{-1} V_j
 *     are kept, restart x N more doubles, and x += Z y); lines of chains cut
 *     by a 2:1 face or a periodic column are left as the identity.  The
 *     stopping test is still on the unpreconditioned residual b - S x.
 *     Also in graph mode (the factorisation is captured once per stage).
 *   DG_PRECOND_CELL (2) block Jacobi with the exact diagonal cell blocks of
 *     S (the cell's own volume and face terms plus, through every
 *     conforming neighbour, the term the face flux of the gradient brings
 *     back through the divergence's face flux; 2:1 faces keep only their
 *     own half), inverted in FP32 per cell; same flexible GMRES, setup and
 *     graph support as DG_PRECOND_VLINE.  For meshes whose stiff part the
 *     vertical lines miss (columns cut by 2:1 faces); measured: 30 % fewer
 *     iterations on a 2D refined mesh, no gain on the 3D refined hill.  Degree <= 3 in 3D
 *     (blocks of up to 64 x 64), any supported degree in 2D; otherwise
 *     DG_ERR_UNSUPPORTED.
 *   other values: DG_ERR_ARG. */
enum { DG_PRECOND_NONE = 0, DG_PRECOND_VLINE = 1, DG_PRECOND_CELL = 2 };

/* z = P^{-1} r for the preconditioner P of kind `precond`
 * (DG_PRECOND_VLINE or DG_PRECOND_CELL) built from the frozen coefficients
 * cf (r, z: N, device, not aliased); the phys precision field is ignored
 * (P is always factored in FP32 from the FP64 coefficients).  Exposed to
 * test and inspect the preconditioners. */
int dg_precond_apply(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                     const dg_implicit_coeffs* cf, int precond, const double* r, double* z,
                     void* stream);
typedef struct {
  double rtol;
  int restart, maxit;
  double inner_rtol;
  int precond;
} dg_gmres_opts;
typedef struct { int iters; double relres; int refinements; } dg_gmres_info;
int dg_gmres_solve(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                   const dg_implicit_coeffs* cf, const double* b, double* x,
                   const dg_gmres_opts* opts, dg_gmres_info* info, void* stream);

/*
 * One ARK2 IMEX step (Section 3): stages 2 and 3 take rho explicitly, then
 * the Picard loop (initial guess = previous stage; stop when
 * max(||dp||/||p||, ||du||/||u||) < picard_rtol, or exactly picard_fixed
 * iterations if > 0) around the Schur solve and the velocity recovery;
 * final update y^{n+1} = y^n + dt sum_l b_l (F_NS,l + F_S,l).
 *  q in/out: 5 x N (device).  Synchronises `stream` to fill info.
 */
typedef struct {
  double picard_rtol;
  int picard_maxit, picard_fixed;
  dg_gmres_opts gmres;
  int graph;   /* 1: device-driven step (not in the paper): the Givens
                  rotations and every stopping test run on the GPU, the loops
                  are CUDA-graph while nodes, and the whole step is captured
                  once per (mesh, q, dt, phys, opts) and replayed as one graph
                  launch; the first call for a configuration also runs one
                  host-driven step on a copy of q to size the workspace.  Same
                  arithmetic as graph = 0 up to the rounding of the Givens
                  updates.  Not available under dg_profile_begin
                  (DG_ERR_UNSUPPORTED). */
} dg_step_opts;
typedef struct {
  int picard_iters[3];
  int gmres_iters_total;
  double max_relres;
  int refinements_total;   /* DG_MIXED: FP64 residual sweeps over all solves */
} dg_step_info;
int imex_ark2_step(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                   double* q, double dt, const dg_step_opts* opts,
                   dg_step_info* info, void* stream);

/*
 * Ensembles: many independent instances (meshes of any size, dim 2 or 3,
 * degree 1..4, each with its own Coriolis parameter) advanced together.
 * Instances sharing (dim, degree) are merged into one device mesh (disjoint
 * union of cells and faces) so that each kernel of a step covers all of
 * them in one launch; the Coriolis parameter is carried per cell.  Within a
 * group the Schur solves and Picard loops run jointly (norms over the
 * group), and all instances of a group must share dt.
 *  dg_ensemble_create: descs[n] as for dg_mesh_create (host, copied),
 *    f_inst[n] host Coriolis parameters.  The ensemble owns device state.
 *  dg_ensemble_set_state / get_state: copy instance i's state (device,
 *    5 x N_i, same layout as for a single mesh) into / out of the ensemble.
 *  dg_ensemble_step: one ARK2 step of every group (imex_ark2_step with the
 *    per-cell f), dt_inst[n] host; info sums iterations over the groups.
 */
typedef struct dg_ensemble dg_ensemble;
int dg_ensemble_create(dg_ctx* ctx, const dg_mesh_desc* descs, const double* f_inst, int n,
                       dg_ensemble** out);
void dg_ensemble_destroy(dg_ensemble* ens);
int dg_ensemble_info(const dg_ensemble* ens, int* n_groups, int64_t* total_nodes);
int dg_ensemble_instance_nodes(const dg_ensemble* ens, int i, int64_t* n_nodes);
int dg_ensemble_set_state(dg_ensemble* ens, int i, const double* q, void* stream);
int dg_ensemble_get_state(dg_ensemble* ens, int i, double* q, void* stream);
int dg_ensemble_step(dg_ensemble* ens, const dg_phys* phys, const double* dt_inst,
                     const dg_step_opts* opts, dg_step_info* info, void* stream);

/*
 * Launch accounting (no counterpart in the paper; used to measure the hot
 * path).  Between begin and end every kernel launch of `mesh` is counted
 * per kernel class; classes whose bit is set in time_mask are also
 * bracketed by CUDA events on the launching stream.  dg_profile_end
 * synchronises on the last event and fills out[k] for k < min(max_out,
 * DG_KERNEL_CLASSES) with the class name, launch count, number of timed
 * launches and their summed device time in ms.
 */
enum { DG_KERNEL_CLASSES = 18 };
typedef struct {
  char name[32];
  int64_t launches;
  int64_t timed_launches;
  double total_ms;
} dg_kernel_stat;
int dg_profile_begin(dg_mesh* mesh, uint32_t time_mask);
int dg_profile_end(dg_mesh* mesh, dg_kernel_stat* out, int max_out, int* n_out);

/*
 * Allocation-free explicit operator (the paper has no counterpart: this
 * exists for callers that must not allocate device memory while they run,
 * e.g. a service that reserves its memory up front and forbids allocation
 * in its steady state, or a framework that owns every device allocation
 * and rejects raw cudaMalloc, which may also synchronise the device).
 * Same arguments, results and layout as dg_apply_explicit (damping layers
 * set by dg_mesh_set_sponge included), which instead grows per-mesh
 * workspace with cudaMalloc on its first call on a mesh.  phys->precision
 * DG_FP64 and DG_MIXED both run the FP64 explicit kernels, as
 * dg_apply_explicit does; DG_MIXED_EXPLICIT returns DG_ERR_UNSUPPORTED.
 *  - Scratch comes from one fixed array of 2^22 doubles (32 MiB) of device
 *    memory in the library image; every GPU that loads the library holds it
 *    until the process exits.  A mesh needs 14 doubles per face-point slot
 *    (n_elem * 2 dim * (r+1)^(dim-1) slots) plus 9 per hanging point;
 *    larger meshes are rejected with DG_ERR_ARG and a message naming the
 *    sizes.  The call makes no cudaMalloc / cudaFree and calls no
 *    allocating library routine.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (the current device must be the context's); make
 *    that first call before any stream capture.
 *  - All calls share the one array and every scratch value is written
 *    before it is read (nothing needs clearing between calls), so two calls
 *    that can overlap on the GPU (different streams, or different threads)
 *    race on it: order them on one stream or synchronise between them.
 */
int dg_apply_explicit_noalloc(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* phys,
                              const double* q, double* f_ns, double* f_s, void* stream);

/*
 * FMA-throughput probe (no counterpart in the paper; it measures the
 * arithmetic roof that the FP64 and FP32 cell kernels are bound by).
 * Launches, on the context's device (which must be current), a grid that
 * fills every SM with threads each running 8 independent chains of
 * x <- x * a + b for `iters` rounds in FP64 (bits = 64) or FP32
 * (bits = 32); two untimed launches, then one launch timed with CUDA events
 * on `stream`.  *tflops = 2 flops x chains x iters x threads / time;
 * *ms (may be NULL) = that launch's time.  Allocates and frees a small
 * device buffer; synchronises `stream`.  Suggested iters: 8192 (FP64),
 * 524288 (FP32), a few tens of ms each on GB300.
 */
int dg_probe_fma(dg_ctx* ctx, int bits, int iters, double* tflops, double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DGIMEX_H */
