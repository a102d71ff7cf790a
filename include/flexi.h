/*
 * flexi.h -- C ABI of the GB300 (sm_103a) DGSEM library libflexi_gb300.so.
 *
 * The library evaluates the semi-discrete DGSEM operator of the compressible
 * Navier-Stokes equations on hexahedral meshes (Krais et al., "FLEXI: A high
 * order discontinuous Galerkin framework for hyperbolic-parabolic conservation
 * laws", Sec. 3.1, Eq. semiDiscrete with BR1 lifting, Eq. discreteGradient),
 * advances it with the Williamson low-storage explicit Runge-Kutta scheme
 * (Sec. 3.4; Carpenter-Kennedy 4(5) coefficients) and provides the discrete
 * adjoint of both.  Every stage runs in hand-written CUDA kernels on one GPU.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  - n = N + 1 nodes per direction; per element n^3 nodes ("DOF" per variable,
 *    Sec. 5.6 PID definition).
 *  - Solution arrays (U, Ut, dU, adjoints) are DEVICE pointers owned by the
 *    caller, contiguous, layout [K][5][k][j][i] (i fastest), conserved variables
 *    (rho, rho u, rho v, rho w, rho E); element type double for precision
 *    FLEXI_FP64 and float for the FP32 forms.
 *  - Element-local sides: 0: xi1=-1, 1: xi1=+1, 2: xi2=-1, 3: xi2=+1,
 *    4: xi3=-1, 5: xi3=+1.  Side-local face coordinates (p, q) are the two
 *    remaining volume indices in increasing direction order.  An orientation
 *    code o in 0..7 maps a face node (p, q) of one element to (p', q') of the
 *    neighbour: (a,b) = o&1 ? (q,p) : (p,q); p' = o&2 ? N-a : a;
 *    q' = o&4 ? N-b : b  (master/slave side systems and flips, Sec. 5.1).
 *  - Calls that take a `stream` (a cudaStream_t, NULL = default stream) only
 *    enqueue work; they return before the GPU finishes.  Conditions found on
 *    the device (non-physical states) are latched in a device status word and
 *    reported by the next flexi_reduce or flexi_query(FLEXI_Q_STATUS).
 *  - Errors are returned as flexi_status codes; nothing is thrown across the
 *    ABI and nothing exits the process.  flexi_strerror gives the text.
 *  - A context belongs to the CUDA device that was current at flexi_mesh_init.
 *    Every call that launches work or copies data returns FLEXI_EINVAL, before
 *    touching the GPU, when another device is current in the calling thread.
 *  - No call allocates device buffers after flexi_mesh_init (flexi_rk_run_host
 *    stages through buffers allocated there); flexi_rk_run instantiates a CUDA
 *    graph, a driver resource, when it first replays a step.
 */
#ifndef FLEXI_GB300_H
#define FLEXI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flexi_ctx flexi_ctx;

typedef enum {
  FLEXI_OK = 0,
  FLEXI_EINVAL = -1,        /* bad argument (null pointer, size out of range, bad enum) */
  FLEXI_ENOMEM = -2,        /* device or host allocation failed in flexi_mesh_init */
  FLEXI_ECUDA = -3,         /* a CUDA runtime call failed (launch, copy, sync) */
  FLEXI_EMESH = -4,         /* inconsistent connectivity or non-positive Jacobian */
  FLEXI_ENONPHYSICAL = -5,  /* rho <= 0 or p <= 0 (or NaN) seen on a face since the last check */
  FLEXI_EUNSUPPORTED = -6   /* valid request this build does not implement (e.g. N > 7) */
} flexi_status;

enum { FLEXI_NODES_GAUSS = 0, FLEXI_NODES_LOBATTO = 1 };
/* Riemann solvers (Sec. 2.2 names Roe, HLL-type and Rusanov fluxes): ROE_SMOOTH
 * replaces |lambda| by (lambda^2 + delta^2)/(2 delta) below delta = 0.1 c (C^1
 * operator); RUSANOV is the local Lax-Friedrichs flux. */
enum { FLEXI_RIEMANN_ROE = 0, FLEXI_RIEMANN_HLLC = 1, FLEXI_RIEMANN_ROE_SMOOTH = 2, FLEXI_RIEMANN_RUSANOV = 3,
       FLEXI_RIEMANN_EC = 4 /* entropy conservative: the EC two-point flux below, no dissipation */ };
/* Arithmetic forms: FP64; FP32 storage+flux math with FP32 line sweeps; FP32
 * with the D-matrix line sweeps on tensor cores in TF32 or BF16, each operand
 * split into three terms of the narrow type (six products, FP32 accumulation). */
enum { FLEXI_FP64 = 0, FLEXI_FP32 = 1, FLEXI_FP32_TF32 = 2, FLEXI_FP32_BF16 = 3 };
/* Volume integral (Sec. 3.3): STANDARD is the weak form of Eq. semiDiscrete; KEP is
 * the split form of Eq. semiDiscreteSplit on Gauss-Lobatto nodes, 2 sum_a D_ia
 * F#(U_i, U_a) with Pirozzoli's kinetic-energy-preserving two-point flux (the
 * flux of the paper's NACA 64418 computation, Sec. 7.1) and metric terms averaged
 * over each pair; EC uses Chandrashekar's entropy-conservative two-point flux
 * (logarithmic means of rho and beta = rho/(2p)) instead; with FLEXI_RIEMANN_EC at
 * the faces and mu = 0 the discrete entropy is conserved.  Viscous fluxes stay in
 * the standard form. */
enum { FLEXI_SPLIT_STANDARD = 0, FLEXI_SPLIT_KEP = 1, FLEXI_SPLIT_EC = 2 };
/* Boundary kinds (Sec. 2.2: boundary conditions enter weakly through the outer
 * state of the numerical flux; the inner lifted gradients are used outside):
 * EXACT: the exact state FLEXI_EXACT_* at the face nodes (Dirichlet; the default);
 * OUTFLOW: the inner state (extrapolation, supersonic outflow);
 * SLIP_WALL: the inner state with its normal velocity reversed (inviscid wall). */
enum { FLEXI_BC_EXACT = 0, FLEXI_BC_OUTFLOW = 1, FLEXI_BC_SLIP_WALL = 2 };
/* Lifting (Sec. 3.2; Bassi & Rebay): BR1 is Eq. discreteGradient, its gradient used in the
 * volume integral and, averaged, in the viscous face flux.  BR2 keeps that volume gradient,
 * but the viscous face flux takes on each side the broken gradient (the BR1 gradient minus
 * the lifting r_f = (1/J) l_hat(+-1) (U* - U_e) n s_hat of every face) plus eta_br2 times
 * the face's own lifting (FP64 / FP32, standard volume integral). */
enum { FLEXI_LIFTING_BR1 = 0, FLEXI_LIFTING_BR2 = 1 };
/* Exact states for exact-state boundary sides (and the manufactured source term). */
enum { FLEXI_EXACT_TGV = 0, FLEXI_EXACT_FREESTREAM = 1, FLEXI_EXACT_MANUFACTURED = 2 };

typedef struct {
  int N;          /* polynomial degree, 1..7 */
  int Ngeo;       /* geometry degree of the node coordinates, 1..N */
  int node_type;  /* FLEXI_NODES_* */
  int riemann;    /* FLEXI_RIEMANN_* */
  int precision;  /* FLEXI_FP64 / FLEXI_FP32 / FLEXI_FP32_TF32 / FLEXI_FP32_BF16 */
  int bc_exact;   /* FLEXI_EXACT_* used on every exact-state (FLEXI_BC_EXACT) side */
  int source;     /* 1: add the manufactured-solution source term */
  int split_form; /* FLEXI_SPLIT_*; KEP and EC need FLEXI_NODES_LOBATTO and FP64 or FP32 */
  double gamma, Pr, mu; /* ideal gas, constant viscosity (Stokes' hypothesis) */
  double Ma;            /* Mach number of the Taylor-Green exact state */
  int adjoint;          /* 1: also allocate the discrete adjoint's scratch (volume gradients
                           and face adjoints, about 37 words per DOF); 0: adjoint calls
                           return FLEXI_EUNSUPPORTED */
  int lifting;          /* FLEXI_LIFTING_* */
  double eta_br2;       /* BR2 penalty factor (>= 0), used with FLEXI_LIFTING_BR2 */
} flexi_params;

/* Geometry and connectivity (Sec. 3.1 mapping and curl-form metrics, Eq.
 * contravariantBasisVectorsCurl; Sec. 5.1 sides).
 *   coords: HOST pointer, double [K][Ngeo+1][Ngeo+1][Ngeo+1][3], physical node
 *           coordinates at the Gauss-Lobatto points of each element, in the
 *           element-local index order [k][j][i].
 *   conn:   HOST pointer, int32 [K][6][3]: (neighbour element, neighbour local
 *           side, orientation code this-side -> neighbour-side), or
 *           (-1 - bc_id, -1, 0) on a boundary side (kind set by flexi_set_bc;
 *           exact state by default).
 * Computes on the device: x at the solution nodes, curl-form metrics Ja, 1/J,
 * face normals and surface elements; allocates every buffer later calls use.
 * Returns FLEXI_EMESH for asymmetric connectivity or J <= 0, FLEXI_EINVAL for
 * bad sizes or parameters, FLEXI_EUNSUPPORTED for the split form with Gauss
 * nodes or a tensor-core form.  On success *out owns everything; free it with
 * flexi_destroy.  The call synchronises `stream`. */
flexi_status flexi_mesh_init(flexi_ctx **out, const flexi_params *p, int K, const double *coords,
                             const int32_t *conn, void *stream);

/* Non-conforming meshes (Sec. "Non-conforming meshes", mortar method): a big side
 * is cut at the middle of its reference square into two halves along its first
 * face coordinate p (type 1), along q (type 2) or into four quarters (type 3).
 *   conn:    as for flexi_mesh_init, except that every side on such an interface
 *            has (FLEXI_CONN_MORTAR, m, pos): m the mortar row, pos = -1 for the
 *            big side, else the small side's position.
 *   mortars: HOST pointer, int32 [M][15]: (big element, big local side, type,
 *            then for pos = 0..3: small element, small local side, orientation
 *            code mapping the small side's (p, q) to the node (p', q') of its
 *            sub-square of the big side, rescaled to 0..N; -1 -1 -1 where the
 *            type has only two positions).  pos = a (type 1), b (type 2) or
 *            a + 2b (type 3), a / b = 0 for the lower, 1 for the upper half
 *            along p / q of the big side's frame.
 * Per stage the big element's solution U and lifted gradients are interpolated
 * to the small sides (I^L, I^U), the numerical and BR1 lifting fluxes are
 * computed there and L2-projected back (P^L, P^U).  Returns FLEXI_EMESH for
 * inconsistent mortar rows; otherwise as flexi_mesh_init.  The discrete adjoint
 * covers mortar meshes. */
#define FLEXI_CONN_MORTAR (-1073741824)
flexi_status flexi_mesh_init_mortar(flexi_ctx **out, const flexi_params *p, int K, const double *coords,
                                    const int32_t *conn, int M, const int32_t *mortars, void *stream);

/* Boundary kind of every side with boundary id bc_id (conn value -1 - bc_id).
 * Returns FLEXI_EINVAL for an unknown kind or an id no boundary side carries.
 * Synchronous (copies a small table to the device); call it between time steps. */
flexi_status flexi_set_bc(flexi_ctx *ctx, int bc_id, int kind);

/* Ut = L(U, t): the semi-discrete right-hand side, Eq. semiDiscrete with the
 * BR1 gradients of Eq. discreteGradient (steps: prolongation, lifting, face
 * fluxes, volume integral, surface integral, 1/J scaling).  U, Ut: device. */
flexi_status flexi_rhs(flexi_ctx *ctx, const void *U, void *Ut, double t, void *stream);

/* One LSERK4(5) step in place (Sec. 3.4, Williamson 2N form):
 *   for k = 1..5: dU = A_k dU + dt L(U, t + c_k dt); U = U + B_k dU.
 * U, dU: device, updated in place (dU is multiplied by A_1 = 0 first). */
flexi_status flexi_rk_step(flexi_ctx *ctx, void *U, void *dU, double t, double dt, void *stream);

/* nsteps steps of flexi_rk_step (times t0 + s dt), enqueued on `stream`.  The last
 * stage of each step but the last also writes the face states of the new U, so
 * that only the first step prolongs U (the same arithmetic: the results equal
 * those of nsteps flexi_rk_step calls bit for bit).  When one step does not
 * depend on t (no source term, no exact-state boundary with the time-dependent
 * manufactured state), stream is not the legacy NULL stream, kernel timing is off
 * and nsteps > 1, the first step runs eagerly and the rest replay a CUDA graph of
 * one step, captured once per (U, dU, dt, stream) and kept in the context; a later
 * call that reuses it prolongs the caller's U first.
 * U, dU: device, updated in place. */
flexi_status flexi_rk_run(flexi_ctx *ctx, void *U, void *dU, int nsteps, double t0, double dt, void *stream);

/* As flexi_rk_step, and also stores the five stage inputs U_{k-1} into
 * U_stages (device, [5][K][5][n^3]) for the adjoint. */
flexi_status flexi_rk_step_stages(flexi_ctx *ctx, void *U, void *dU, double t, double dt, void *U_stages,
                                  void *stream);

/* Discrete adjoint of one flexi_rk_step (reverse of the stage loop):
 *   for k = 5..1: lam_dU += B_k lamU; lamU += dt (dL/dU(U_{k-1}, t + c_k dt))^T lam_dU;
 *                 lam_dU = A_k lam_dU.
 * U_stages: device [5][K][5][n^3] as written by flexi_rk_step_stages; t: the
 * step's start time (exact-state boundaries are evaluated at the stage times of
 * the forward step).  lamU, lam_dU: device, updated in place.  Requires
 * flexi_params.adjoint = 1, FLEXI_FP64 or FLEXI_FP32, BR1 or BR2 lifting, the
 * standard or the split-form volume integral; every numerical flux (the Roe fluxes by a
 * hand-written reverse, HLLC, Rusanov and EC in forward mode); periodic meshes
 * and meshes with boundaries of every kind (the outer state's dependence on the
 * inner one is transposed; a source term does not depend on U) and mortar
 * meshes (FLEXI_EUNSUPPORTED for the tensor-core precisions). */
flexi_status flexi_adjoint_step(flexi_ctx *ctx, const void *U_stages, void *lamU, void *lam_dU, double t,
                                double dt, void *stream);

/* (dL/dU(U, t))^T lam: the adjoint of flexi_rhs alone.  All device pointers. */
flexi_status flexi_rhs_adjoint(flexi_ctx *ctx, const void *U, const void *lam, void *out, double t,
                               void *stream);

/* End-to-end convenience call on HOST memory: copies U_host (pinned or pageable,
 * layout as above) to the device state, runs nsteps steps from t0 with step dt as
 * flexi_rk_run does without a graph, and copies the result back into U_host.
 * Synchronous. */
flexi_status flexi_rk_run_host(flexi_ctx *ctx, void *U_host, int nsteps, double t0, double dt, void *stream);

/* Global FP64 reductions (Sec. 5.3: the only all-to-all operation is the global
 * time step).  out (HOST, 8 doubles): [0..4] integrals of the conserved
 * variables by the collocated quadrature (sum w_i w_j w_k J U), [5] kinetic
 * energy sum w J |m|^2/(2 rho), [6] dKE/dt if Ut != NULL (else 0), [7] the
 * largest stable dt of Eqs. CFLCondition/DFLCondition with CFL = DFL = cfl,
 * gamma_RK = 1 (reading).  Synchronises `stream`; returns FLEXI_ENONPHYSICAL if
 * the status word was set (and clears it). */
flexi_status flexi_reduce(flexi_ctx *ctx, const void *U, const void *Ut, double cfl, double *out, void *stream);

/* Allocation-free form of flexi_reduce, for callers that cannot allocate
 * device memory when they need the sums (an application whose own memory
 * manager owns all device memory, or a time loop that must not call
 * cudaMalloc/cudaFree because they synchronise the device).  It computes the
 * same 8 outputs as flexi_reduce (same layout, same FLEXI_ENONPHYSICAL report)
 * but keeps its per-element partial sums in a fixed array in the library's
 * static device memory instead of a context buffer, and calls no allocating
 * routine.  The paper has no counterpart of this call.
 *   - Limit: K <= FLEXI_NOALLOC_MAX_ELEMENTS elements; larger meshes return
 *     FLEXI_EINVAL.  One thread per node: n^3 <= 512 (N <= 7, the library's
 *     limit), else FLEXI_EUNSUPPORTED.  The static array (about 4.5 MiB) is held
 *     by every GPU that loads the library until the process exits.
 *   - The static array used is the one of the current device, which must be
 *     the context's (else FLEXI_EINVAL, before any launch).
 *   - The first call on a device looks up the array's device address (once per
 *     device); make that first call before any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU (several
 *     streams or host threads on one device) race on it.  Synchronises `stream`. */
#define FLEXI_NOALLOC_MAX_ELEMENTS 65536
flexi_status flexi_reduce_noalloc(flexi_ctx *ctx, const void *U, const void *Ut, double cfl, double *out,
                                  void *stream);

enum {
  FLEXI_Q_K = 0, FLEXI_Q_N = 1, FLEXI_Q_NSIDES = 2, FLEXI_Q_NBCSIDES = 3, FLEXI_Q_DOF = 4,
  FLEXI_Q_BYTES_PER_STAGE = 5, /* algorithmic HBM bytes of one RK stage (minimum-traffic schedule) */
  FLEXI_Q_FLOPS_PER_STAGE = 6, /* algorithmic floating-point operations of one RK stage */
  FLEXI_Q_STATUS = 7,          /* synchronises and returns (then clears) the device status word */
  FLEXI_Q_DEVICE_BYTES = 8,    /* device memory held by the context */
  FLEXI_Q_PRECISION = 9
};
flexi_status flexi_query(flexi_ctx *ctx, int what, int64_t *val);

/* Kernel timing: when enabled, every kernel launch of the library is bracketed
 * by CUDA events on its stream; flexi_kernel_times synchronises and returns,
 * per kernel class (0 lift+volume, 1 face flux, 2 surface+RK, 3 prolong,
 * 4 boundary, 5 adjoint, 6 reduce, 7 other), the summed milliseconds and the
 * launch counts since the last reset (arrays of 8).  */
flexi_status flexi_profile(flexi_ctx *ctx, int enable);
flexi_status flexi_kernel_times(flexi_ctx *ctx, double *ms, int64_t *count, int reset);

const char *flexi_strerror(flexi_status s);
void flexi_destroy(flexi_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FLEXI_GB300_H */
