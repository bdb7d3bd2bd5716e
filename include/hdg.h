/*
 * hdg.h -- C-ABI of the GB300 HDG linearize + condense library (libhdg.so).
 *
 * The library implements the data-parallel hot path of an implicit HDG
 * discretization of the compressible Navier-Stokes equations (Welter, Collin,
 * Nguyen, Peraire): at one Newton step of one DIRK stage it evaluates the
 * element residuals and their Jacobians at quadrature points (Sec. 2.1, 2.2,
 * eqs. hdg-weak, num-flux-hdg, fully-discrete-local), contracts them into the
 * element blocks, eliminates the interior unknowns (Q, U) by static
 * condensation (Sec. 2.5, eqs. newton-local-block, local-elimination,
 * schur-trace), scatters the condensed face blocks into a block-sparse trace
 * matrix, and provides the trace matvec and the interior recovery that GMRES
 * consumes (Sec. 3.2).
 *
 * Conventions shared by every call on quadrilateral / hexahedral handles
 * (tetrahedral handles, created by hdg_create_tet, use the packed layouts of
 * the tetrahedral section at the end of this header)
 * -----------------------------------------------------------------------
 *  d = 2 (quadrilaterals) or 3 (hexahedra), m = d + 2 conserved variables
 *  u = [rho, rho v_1..rho v_d, rho E]; degree p (1..3); element nodes are the
 *  tensor Gauss-Lobatto points, Np = (p+1)^d, node j = j1 + (p+1) j2 +
 *  (p+1)^2 j3; local face f = 2 r + s is the face xi_r = -1 (s = 0) or +1
 *  (s = 1); Nfp = (p+1)^(d-1) trace nodes per face, ordered in the face's
 *  canonical frame (origin at the corner with the smallest master vertex id,
 *  first axis towards the adjacent corner with the smaller id).
 *  Faces are numbered by first encounter scanning elements and local faces.
 *
 *  Device arrays (caller-owned, FP64, contiguous, row-major as written):
 *    U     [E][m][Np]          conserved state
 *    Q     [E][d][m][Np]       gradient, Q[e][k][a] = d u_a / d x_k
 *    UH    [F][m][Nfp]         single-valued trace
 *    Ustar [E][m][Np]          known DIRK stage data: the stage residual is
 *                              (1/a_ii) M (U - Ustar) + dt N(W)
 *    nu    [E][Np]             nodal artificial viscosity (frozen), or NULL
 *  Trace vectors x, y, g, dUH are [F][m][Nfp].
 *
 * Errors: every call returns HDG_OK (0) or a negative code; the handle keeps a
 * message (hdg_last_error).  Nothing aborts, exits or traps on the device.
 * Device work is asynchronous on the stream set with hdg_set_stream (default:
 * the legacy default stream); the caller synchronises.  Numerical failures
 * found on the device (zero pivot, non-finite values) are latched in a status
 * word that hdg_status() reads back.
 */
#ifndef HDG_H
#define HDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HDG_OK 0
#define HDG_EINVAL (-1)       /* bad argument */
#define HDG_ENOMEM (-2)       /* device or host allocation failed */
#define HDG_ECUDA (-3)        /* a CUDA runtime call failed */
#define HDG_ESINGULAR (-4)    /* zero pivot in an element interior block */
#define HDG_ENONFINITE (-5)   /* NaN / Inf in an element block */
#define HDG_ENOCONV (-6)      /* iterative solve did not converge */
#define HDG_EUNSUPPORTED (-7) /* mesh / degree / mode not supported */

#define HDG_QUAD 1
#define HDG_HEX 2

/* Arithmetic of the condensation path. */
#define HDG_PREC_FP64 0       /* everything in FP64 */
#define HDG_PREC_MIXED 1      /* FP64 pointwise terms, interior LU (with pivoting) and right-hand sides;
                                 FP32 contraction, off-diagonal blocks, Schur complement and trace blocks */
#define HDG_PREC_MIXED_TF32 2   /* as HDG_PREC_MIXED, Schur product S = Dt - W Z on tensor cores in TF32 */
#define HDG_PREC_MIXED_3XTF32 3 /* as HDG_PREC_MIXED, Schur product in 3xTF32 split precision on tensor cores */

typedef struct hdg_ctx* hdg_handle;

/* Mesh description, host memory, copied at create; the caller keeps ownership.
 * Elements are affine (parallelograms / parallelepipeds); vertices in tensor
 * order, vertex c = c1 + 2 c2 + 4 c3 at reference corner xi_r = 2 c_r - 1. */
typedef struct {
    int32_t dim;                  /* 2 or 3 */
    int32_t elem_type;            /* HDG_QUAD (dim 2) or HDG_HEX (dim 3) */
    int64_t n_elem;
    int64_t n_vert;
    const double* vert_xyz;       /* [n_vert][dim] */
    const int64_t* elem_vert;     /* [n_elem][2^dim] */
    const int64_t* periodic_map;  /* [n_vert] master vertex of each vertex, or NULL */
    const int32_t* bnd_tag;       /* [n_elem][2 dim] per local face: 0 interior / periodic; on faces with
                                     one element the boundary kind (Sec. 2.2; the forms are readings):
                                     1 far-field / supersonic inflow, bhat = uhat - u_b;
                                     2 supersonic outflow, bhat = uhat - u (extrapolated);
                                     3 isothermal no-slip wall, bhat = [fhat_rho; uhat_rhov;
                                       uhat_rhoE - uhat_rho c_v T_w];
                                     4 adiabatic no-slip wall, bhat = [fhat_rho; uhat_rhov; fhat_rhoE].
                                     NULL for a fully periodic mesh. */
} hdg_mesh;

/* Solver parameters (hdg_set_params).  tau: constant scalar stabilization of
 * eq. num-flux-hdg; visc_law 0: mu = 1/Re, 1: mu = C1 T^1.5 / (T + S) / Re
 * with T = gamma (gamma-1) M^2 e (eq. sutherland, eq. tgv-sutherland).
 * tau_mode 0: the constant tau; 1: the state-dependent stabilization
 * tau(uhat) = |vhat . n| + chat + mu(That) / h_K per face point (a wave speed
 * plus a viscous part over the element length h_K = |K|^{1/d}; the reading of
 * the paper's description), differentiated exactly in the Jacobians. */
typedef struct {
    double tau;
    int32_t visc_law;
    double suth_c1;
    double suth_s;
    int32_t precision;            /* HDG_PREC_* */
    int32_t tau_mode;             /* 0 constant tau, 1 state-dependent */
} hdg_params;

typedef struct {
    int32_t dim, p, m, Np, Nq, nf, Nfp, Nfq;
    int32_t n_u;                  /* m Np: interior U unknowns per element */
    int32_t n_q;                  /* d m Np */
    int32_t t;                    /* nf m Nfp: trace unknowns per element */
    int32_t block;                /* m Nfp: BSR block size */
    int64_t n_elem, n_faces, nnzb;
    int64_t device_bytes;         /* device memory held by the handle */
} hdg_sizes;

/* Build tables, connectivity, the BSR pattern and device storage (Sec. 2.2
 * spaces, Sec. 3.5 face partition).  Fails with HDG_EUNSUPPORTED for
 * non-affine elements, p outside 1..3 or boundary tags outside 0..4, and
 * HDG_EINVAL for inconsistent meshes (a face shared by more than two
 * elements, a degenerate periodic face, boundary tags 1..4 not marking
 * exactly the faces with a single element). */
int hdg_create(hdg_handle* out, const hdg_mesh* mesh, int p, double gamma, double Re,
               double Pr, double Mach);
/* Same as hdg_create without touching the GPU: connectivity and tables only;
 * device calls on such a handle return HDG_EINVAL. */
int hdg_create_host(hdg_handle* out, const hdg_mesh* mesh, int p, double gamma, double Re,
                    double Pr, double Mach);
int hdg_destroy(hdg_handle h);
const char* hdg_last_error(hdg_handle h);

int hdg_set_params(hdg_handle h, const hdg_params* prm);
/* The per-element storage of the condensed system (BSR values, the interior
 * rows kept for recovery, per-chunk trace rows) is allocated on the first
 * linearization in a precision, so a run in one precision never holds the
 * other's arrays (a mixed-form run of 98,304 hex p = 3 elements needs about
 * 230 GB; the FP64 arrays would add 370 GB).  hdg_reserve allocates the
 * storage of `precision` now, for callers that must not allocate later
 * (hdg_linearize_condense_static requires the FP64 storage reserved). */
int hdg_reserve(hdg_handle h, int precision);
int hdg_set_stream(hdg_handle h, void* cuda_stream);
/* Boundary data (host): tag 1, the state u_b [m] of the far-field / inflow
 * faces (trace equation <uhat - u_b, mu> = 0); tag 3, ub[0] = the wall
 * temperature T~_w (T~ = gamma M^2 p / rho, so T~_inf = 1).  Required before
 * linearizing a mesh with faces of that tag. */
int hdg_set_bc_state(hdg_handle h, int tag, const double* ub);
/* Nodal tag-1 data: ubf [F][m][Nfp] (device, canonical face-node order; only
 * the rows of tag-1 faces are read), copied into the handle on the stream;
 * it replaces the constant state (e.g. an inflow profile).  NULL returns to
 * the constant state. */
int hdg_set_bc_field(hdg_handle h, const double* ubf);
int hdg_query_sizes(hdg_handle h, hdg_sizes* out);

/* Host copies of the integer skeleton data (any pointer may be NULL):
 * f2e [F][2] elements of each face (-1 on the boundary), f2lf [F][2] local
 * faces, e2f [E][nf], perm [E][nf][Nfp] canonical index of each local face
 * node, bsr_rowptr [F+1], bsr_col [nnzb] (ascending within a row). */
int hdg_get_connectivity(hdg_handle h, int32_t* f2e, int32_t* f2lf, int32_t* e2f,
                         int32_t* perm, int32_t* bsr_rowptr, int32_t* bsr_col);

/* One Newton linearization of one DIRK stage at W = (Q, U, UH), followed by
 * static condensation of every element and assembly of the trace system
 * S dUH = g (eqs. newton-linearization, local-elimination, schur-trace).
 * Inputs are device pointers (layouts above); dt and a_ii enter the stage
 * residual of eq. fully-discrete-local.  The library keeps S (BSR), g and the
 * per-element factors needed by hdg_recover_interior.  res_norm (host,
 * optional): when not NULL it receives ||F(W)||_2, the FP64 norm of the stage
 * residual at the same W (eq. nonlinear-residual, as hdg_residual's norms[0],
 * whatever the handle's precision), and the call then synchronises the
 * stream; when NULL the call is asynchronous. */
int hdg_linearize_condense(hdg_handle h, const double* U, const double* Q, const double* UH,
                           const double* Ustar, const double* nu, double dt, double a_ii,
                           double* res_norm);

/* y = S x on the assembled trace operator (device pointers, [F][m][Nfp]; FP64
 * vectors).  FP64 system: FP64 products and sums.  Mixed system (FP32 blocks):
 * x is rounded to FP32 and the products are FP32; quad / hex handles sum each
 * block in FP32 and the blocks of a row in FP64, tetrahedral handles sum the
 * whole block row in FP32 (in a fixed order, so results are reproducible). */
int hdg_trace_matvec(hdg_handle h, const double* x, double* y);
/* Copy the condensed right-hand side g = sum_K (-R_uhat^K + C^K y^K) to g. */
int hdg_trace_rhs(hdg_handle h, double* g);
/* Interior recovery dW_K = -y_K - X_K dUH_K (eq. local-elimination) for every
 * element: dQ [E][d][m][Np], dU [E][m][Np] (device, caller-owned). */
int hdg_recover_interior(hdg_handle h, const double* dUH, double* dQ, double* dU);
/* Copy the BSR values: [nnzb][block][block], block column-major, i.e.
 * value (r, c) of block b at vals[(b * block + c) * block + r], r = a Nfp + k.
 * The values are FP64 after an FP64 linearization and FP32 (vals then points
 * to float storage of the same shape) after an HDG_PREC_MIXED one. */
int hdg_get_blocks(hdg_handle h, double* vals);
/* Per-element Schur complements S^K (eq. schur-trace) as well as the assembled
 * blocks: after this call every hdg_linearize_condense also writes, for every
 * element K, its t x t condensed block S^K = D - C A^{-1} B into SK (device,
 * caller-owned; NULL switches the output off).  Layout: quad / hex handles
 * [E][t][t] row-major, t = nf m Nfp; tetrahedral handles packed, element e's
 * t_e x t_e block at offset sum_{e' < e} t_{e'}^2.  Rows and columns follow the
 * element's local trace order (local face, component, face node; on quad / hex
 * faces the element's own node order, which hdg_get_connectivity's perm maps to
 * the canonical one; on tetrahedral faces the canonical order).  Values are
 * FP64 after an FP64 linearization and FP32 after a mixed one (SK then points to
 * float storage of the same shape).  Asynchronous on the handle's stream. */
int hdg_set_element_block_output(hdg_handle h, void* SK);
/* Read back the latched device status: HDG_OK, HDG_ESINGULAR or
 * HDG_ENONFINITE (synchronises the stream). */
int hdg_status(hdg_handle h);

/* FP64 stage residual F(W) = [R_q; R_u; R_uhat] at W = (Q, U, UH) (eq.
 * nonlinear-residual; R_uhat assembled over both sides of every face).
 * Optional device outputs Rq [E][d][m][Np], Ru [E][m][Np], Ruh [F][m][Nfp];
 * norms (host, optional) receives ||F||_2, ||(R_q, R_u)||_2, ||R_uhat||_2 and
 * then the call synchronises the stream.  Allocates its scratch on first use. */
int hdg_residual(hdg_handle h, const double* U, const double* Q, const double* UH, const double* Ustar,
                 const double* nu, double dt, double a_ii, double* Rq, double* Ru, double* Ruh, double* norms);
/* Q = Q_lift(U, Uhat): per element, the gradient for which the gradient
 * equations hold exactly (eq. hdg-grad with R_q = 0; R_q is linear in Q, so
 * Q_lift = M_K^{-1} (-(u, grad phi)_K + <uhat, phi n>_dK) component by
 * component).  U [E][m][Np], UH [F][m][Nfp] and Q [E][d][m][Np] are device
 * arrays; Q is written.  Asynchronous on the handle's stream. */
int hdg_lift_gradient(hdg_handle h, const double* U, const double* UH, double* Q);

/* Newton update W <- W + alpha dW (eq. newton-update) on device arrays. */
int hdg_update_state(hdg_handle h, double* U, double* Q, double* UH, const double* dU, const double* dQ,
                     const double* dUH, double alpha);
/* Artificial-viscosity field (Sec. 2.2, eq. av-coeffs) from the nodal state
 * U [E][m][Np] and gradient Q [E][d][m][Np] (device): at every node
 * s = sqrt(h_m / p) L(-div v) / c* * L(-div v)^2 / (L(-div v)^2 + |curl v|^2
 * + 1e-12), c* = sqrt(gamma p / rho), L = clamp to >= 0; nu_raw = c_av
 * min(max(s, 0), s_max); the elemental raw value is the maximum over the
 * element's nodes.  Smoothing: two passes of averaging to the (periodic
 * master) vertices with the element mean of its vertices in between, then
 * multilinear interpolation to the nodes.  Writes nu [E][Np] (device), the
 * field hdg_linearize_condense takes (frozen over a step).  Asynchronous. */
int hdg_av_field(hdg_handle h, const double* U, const double* Q, double c_av, double h_m, double s_max, double* nu);
/* Volume-integrated diagnostics (Sec. 5.1, eqs. tgv-kinetic-energy and
 * tgv-total-dissipation) with the volume quadrature: out (host, 4 doubles)
 * = (E_k, eps_S, eps_D, |Omega|), E_k = int rho v.v / (2 |Omega|),
 * eps_S = int mu~ |curl v|^2 / (Re |Omega|), eps_D = 4 int mu~ (div v)^2 /
 * (3 Re |Omega|), u and grad u from U and Q.  Fixed-order sums; synchronises. */
int hdg_tgv_diagnostics(hdg_handle h, const double* U, const double* Q, double* out);

/* Reduced-basis initial guess (Sec. 3.4, eq. rb-min).  A window of at most
 * nb_max (<= 20) accepted trace corrections W and their products Z = S W
 * (each taken with the trace operator current at insertion) lives on the
 * device.  hdg_rb_setup allocates and clears it (nb_max = 0 disables it);
 * when enabled, hdg_newton, hdg_newton_fixed and hdg_dirk_step start every
 * GMRES solve from the guess and insert the accepted correction afterwards.
 * hdg_rb_push inserts w (device [F][m][Nfp]) with z = S w (one matvec),
 * discarding the oldest column when full; hdg_rb_guess writes x0 = W c,
 * c = argmin ||g - Z c||_2, solved through the normal equations by
 * Cholesky with diagonal pivoting (pivots below 1e-13 of the largest
 * diagonal are dropped, so an empty window gives x0 = 0).  Asynchronous. */
int hdg_rb_setup(hdg_handle h, int nb_max);
int hdg_rb_push(hdg_handle h, const double* w);
int hdg_rb_guess(hdg_handle h, const double* g, double* x0);

/* Preconditioner used by hdg_gmres (precond != 0), hdg_newton,
 * hdg_newton_fixed and hdg_dirk_step: HDG_PC_BLOCKJACOBI (default) or
 * HDG_PC_SCHWARZ. */
#define HDG_PC_BLOCKJACOBI 1
#define HDG_PC_SCHWARZ 2
int hdg_set_preconditioner(hdg_handle h, int kind);
/* One-level additive Schwarz on element-centred face patches (Sec. 3.3,
 * eq. additive-schwarz): M^{-1} = sum_r R_r^T S_r^{-1} R_r, R_r the
 * restriction to the nf faces of element r, S_r = R_r S R_r^T (t x t, no
 * coarse space).  Setup factors every S_r (partial pivoting; FP64 for the
 * FP64 system, FP32 for the mixed one), on the stream; apply computes
 * y = M^{-1} x for device vectors x, y [F][m][Nfp] (distinct), summing the
 * patch corrections of a face in a fixed order (bitwise reproducible).
 * A zero or non-finite pivot sets the status read by hdg_status.
 * Tetrahedral handles: the patch of element r holds its four faces' blocks
 * (t = 60 .. 300 unknowns for face degrees 1..4); S_r is gathered from the
 * assembled blocks and factored in place by LU with partial pivoting in the
 * system's precision (P S_r = L U, row-major [t][t rounded up to 4]); the
 * factors take sum_r t_r^2 values (FP64: 42 GB on the 100,800-element mesh,
 * FP32: 21 GB), allocated on the first set-up; apply solves L U z = P R_r x
 * per patch in the factors' precision and sums the corrections of a face over
 * its elements in ascending element order. */
int hdg_schwarz_setup(hdg_handle h);
int hdg_schwarz_apply(hdg_handle h, const double* x, double* y);

/* Block-Jacobi preconditioner of the trace system: the inverse of every
 * diagonal block S_FF of the current S (the one-face special case of the
 * additive Schwarz method, eq. additive-schwarz), and y = M^{-1} x.  Hex and
 * quad handles: partial-pivot LU in FP64, kept in the system's storage
 * precision.  Tetrahedral handles: Gauss-Jordan with partial pivoting in the
 * system's precision (FP32 for the mixed form).  A zero or non-finite pivot
 * sets the handle's status (hdg_status). */
int hdg_blockjacobi_setup(hdg_handle h);
int hdg_blockjacobi_apply(hdg_handle h, const double* x, double* y);
/* Restarted GMRES(restart) on S x = b with FP64 Arnoldi (Sec. 3.2; classical
 * Gram-Schmidt with one reorthogonalisation, CGS2), left-preconditioned by
 * the selected preconditioner (hdg_set_preconditioner; block-Jacobi by
 * default) when precond != 0.
 * x holds the initial guess and receives the solution (device arrays
 * [F][m][Nfp]).  Stops when the preconditioned residual ||M^{-1}(b - S x)||
 * drops below rtol x ||M^{-1} b|| (so a good initial guess saves
 * iterations) or after max_iter iterations (HDG_ENOCONV).
 * iters / relres (host, optional) receive the iteration count and the final
 * relative preconditioned residual.  Workspace is allocated on first use. */
int hdg_gmres(hdg_handle h, const double* b, double* x, int restart, int max_iter, double rtol, int precond,
              int* iters, double* relres);

/* Newton iteration on the DIRK stage equations (eqs. newton-linearization,
 * newton-update with alpha = 1): repeat { F(W); linearize + condense;
 * block-Jacobi GMRES on S dUH = g (rtol gmres_rtol); recover; W += dW } until
 * ||F(W)||_2 <= tol (absolute, FP64) or max_newton linearizations.  U, Q, UH
 * are updated in place.  hist (host, optional, max_newton + 1 entries)
 * receives ||F|| before each iteration.  Returns HDG_ENOCONV if tol was not
 * reached.  Work arrays are allocated on first use. */
int hdg_newton(hdg_handle h, double* U, double* Q, double* UH, const double* Ustar, const double* nu, double dt,
               double a_ii, double tol, int max_newton, int restart, int max_gmres, double gmres_rtol,
               double* hist, int* newton_iters, int* gmres_iters);

/* Newton iterations with a fixed-length GMRES(m) (m iterations from zero,
 * block-Jacobi, Givens rotations and the triangular solve on the device): no
 * host synchronisation inside an iteration, so with use_graph != 0 one
 * iteration is captured once into a CUDA graph (on an internal stream) and
 * replayed n_newton times on the handle's stream; the graph is rebuilt when
 * the arguments change.  hist (host, optional, n_newton + 1 entries) receives
 * ||F|| before each iteration and after the last.  Synchronises at the end. */
int hdg_newton_fixed(hdg_handle h, double* U, double* Q, double* UH, const double* Ustar, const double* nu,
                     double dt, double a_ii, int n_newton, int m, int use_graph, double* hist);
/* One step of an s-stage DIRK method (Sec. 2.3, eqs. dirk-stage, dirk-update)
 * with Butcher matrix A [s][s] (row-major, lower triangular) and weights b [s];
 * the tableau must be stiffly accurate (b = last row of A), so that W^{n+1} is
 * the last stage.  Stage i solves the stage equations with
 * U* = U^n - a_ii sum_{j<i} d_ij (U^{n,j} - U^n), d = A^{-1}, by n_newton
 * fixed Newton iterations (as hdg_newton_fixed), starting from the previous
 * stage.  With use_graph != 0 the whole step (s stages x n_newton iterations)
 * is captured once as one CUDA graph and replayed.  U, Q, UH hold W^n on entry
 * and W^{n+1} on return; hist (host, optional, s (n_newton + 1) entries)
 * receives the residual norms.  A and b both NULL (with s = 3) select
 * Alexander's SDIRK3 (the tableau of hdg_sdirk3_tableau).  Synchronises at
 * the end. */
int hdg_dirk_step(hdg_handle h, double* U, double* Q, double* UH, const double* nu, double dt, int s,
                  const double* A, const double* b, int n_newton, int m, int use_graph, double* hist);

/* Alexander's three-stage, third-order, L-stable, stiffly accurate SDIRK
 * (the DIRK method the paper cites for its time stepping, Sec. 2.3): writes
 * the Butcher matrix A (host, [3][3] row-major, lower triangular) and the
 * weights b (host, [3], equal to the last row of A).  The diagonal gamma is
 * the root in (1/3, 1/2) of gamma^3 - 3 gamma^2 + 3 gamma / 2 - 1/6 = 0;
 * a21 = (1 - gamma) / 2, b1 = -(6 gamma^2 - 16 gamma + 1) / 4,
 * b2 = (6 gamma^2 - 20 gamma + 5) / 4.  Needs no handle. */
int hdg_sdirk3_tableau(double* A, double* b);

/* Autotuner (not from the paper).  Times every kernel variant that computes
 * the same quantities to the same accuracy on the caller's own inputs
 * (reps linearize + condense calls each, after one warm-up, CUDA events on
 * the handle's stream) and keeps the fastest for later calls:
 *  - FP64 form: the volume contraction as a dense GEMM (blocks64_mode 0)
 *    or by sum factorisation over the tensor-product basis (1), the
 *    elimination kernel's panel width (16 or 8 columns) and the residency it
 *    is compiled for (2 or 1 CTAs per SM), and the Schur product
 *    S = Dt - W Z inside the FP64 elimination (schur_mode 0) or on the BF16
 *    tensor cores by exact digit splitting of the FP64 factors (schur_mode 3:
 *    W and Z cut into 6..8 digits of 6..8 bits, products accumulated exactly
 *    in FP32, combined and subtracted in FP64; truncation below 2^-48 of the
 *    row / column scales); results agree to FP64 rounding level;
 *  - mixed form: the elimination as one fused kernel (at 2 or 3 CTAs per
 *    SM) or split into an FP64 LU (panel width 16 or 8) and two FP32
 *    triangular solves,
 *    the volume contraction as FP32 SIMT (blocks_mode 0) or
 *    3xTF32 tensor cores (1, 3-D), and, when requested as HDG_PREC_MIXED,
 *    the Schur product as FP32 SIMT (schur_mode 0) or 3xTF32 tensor cores
 *    (2) — all FP32-accurate; TF32 / 3xTF32 requested explicitly are kept;
 *  - tetrahedral handles: the elimination panel width (16 or 8 columns) of
 *    the persistent linearize + condense kernel (elim_nb; the other fields
 *    are zero; hdg_set_tuning reads elim_nb only).
 * out (host, optional) receives the choice and every candidate's time.
 * hdg_set_tuning applies a stored choice.  Both synchronise; the system
 * left assembled is that of the last candidate timed. */
typedef struct {
    int elim_nb, elim_minb, schur_mode;   /* the chosen variant */
    int blocks_mode, elim_mixed_minb, blocks64_mode, elim_mixed_split;
    int n_cand;                           /* candidates timed (<= 16) */
    int cand[16][7];                      /* (elim_nb, elim_minb, schur_mode, blocks_mode, elim_mixed_minb,
                                             blocks64_mode, elim_mixed_split) of each candidate */
    double ms[16];                        /* mean time of one linearize + condense, ms */
} hdg_tune;
int hdg_autotune(hdg_handle h, const double* U, const double* Q, const double* UH, const double* Ustar,
                 const double* nu, double dt, double a_ii, int reps, hdg_tune* out);
int hdg_set_tuning(hdg_handle h, const hdg_tune* t);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * every kernel launch (not from the paper: instrumentation for rooflines).
 * Kernel classes: HDG_K_POINT (A0/A1 quadrature-point fluxes and Jacobians),
 * HDG_K_BLOCKS (A2 contraction), HDG_K_ELIM (A3/A4 bordered elimination),
 * HDG_K_ASSEMBLE (A5), HDG_K_MATVEC (A6), HDG_K_RECOVER (A7), HDG_K_SCHUR
 * (the separate Schur product of the mixed form).
 * hdg_profile_read synchronises the stream, writes the accumulated
 * milliseconds [HDG_NK] and launch counts [HDG_NK] since the last read, and
 * clears them. */
#define HDG_K_POINT 0
#define HDG_K_BLOCKS 1
#define HDG_K_ELIM 2
#define HDG_K_ASSEMBLE 3
#define HDG_K_MATVEC 4
#define HDG_K_RECOVER 5
#define HDG_K_SCHUR 6
#define HDG_NK 7
int hdg_profile(hdg_handle h, int enable);
int hdg_profile_read(hdg_handle h, double* ms, int64_t* launches);

/* Peak-rate probes of the current device (not from the paper: the roofline
 * denominators, measured).  Each probe is a hand-written kernel that keeps
 * one arithmetic pipe busy with independent operations on register or
 * shared-memory data; tflops (host, 6 entries) receives the best of three
 * timed launches (CUDA events, after one warm-up) in TFLOP/s (TOP/s for
 * INT8): [0] FP64 FMA, [1] FP64 tensor MMA (mma.sync m8n8k4), [2] FP32 FMA,
 * [3] TF32 tcgen05.mma (128 x 256 x 8), [4] BF16 tcgen05.mma (128 x 256 x 16),
 * [5] INT8 mma.sync m16n8k32 (sm_103a has no tcgen05 INT8 kind).  ms (host,
 * optional, 6 entries) receives the launch times.  Allocates 256 bytes of
 * device memory for the call; synchronises the device's default stream. */
int hdg_measure_peaks(double* tflops, double* ms);

/* Allocation-free variant of hdg_linearize_condense (the paper has no
 * counterpart).  It is for callers that must not allocate device memory once
 * the handle exists: a host whose memory pool has taken the remaining HBM
 * after set-up, or a step loop that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree.  It builds the FP64 system only:
 * the same arguments, preconditions (tag-1 boundary state and tag-3 wall
 * temperature set where the mesh has such faces) and results as
 * hdg_linearize_condense on an HDG_PREC_FP64 handle (res_norm omitted); a
 * handle set to a mixed precision gets HDG_EUNSUPPORTED.  The FP64 system
 * storage must be reserved at set-up (hdg_reserve(h, HDG_PREC_FP64)), else
 * HDG_EINVAL.  The per-chunk scratch (trace rows, point coefficients and the
 * per-point stabilization) comes from a 64 MiB file-scope device array of the
 * library instead of the handle's scratch, so elements are condensed in
 * chunks of at most 64 MiB / (scratch of one element) (45 hex p=2, 15 hex
 * p=3 elements), whatever scratch budget the handle was created with.  The
 * call issues no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make it before any
 * stream capture.  Every call, from any handle, shares the one array: calls
 * whose GPU work overlaps (for example on two streams) race and corrupt each
 * other's results; serialise them.  Returns HDG_EINVAL if one element's
 * scratch exceeded the array (no supported (d, p) does). */
int hdg_linearize_condense_static(hdg_handle h, const double* U, const double* Q, const double* UH,
                                  const double* Ustar, const double* nu, double dt, double a_ii);

/* ------------------------------------------------------------------------
 * Tetrahedral meshes of per-element degree on quadratic geometry (the
 * batched workload of Sec. 4: curved anisotropic tetrahedra with a mix of
 * degrees).  Readings:
 *   element space: total degree p_K in 1..4 on each tetrahedron, nodal
 *     Lagrange basis on the equispaced lattice (i, j, k), i + j + k <= p_K,
 *     node at xi = -1 + 2 (i, j, k) / p_K, k slowest and i fastest, on the
 *     reference tetrahedron v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1),
 *     v3 = (-1,-1,1); local face f is opposite vertex f;
 *   trace space of a face: total degree p_F = max(p_L, p_R) (p_K on the
 *     boundary), Lagrange on the equispaced lattice (i, j) of the face in its
 *     canonical frame: vertices g0 < g1 < g2 by master id, node (i, j), j
 *     slowest, at barycentric weights ((p_F - i - j), i, j) / p_F;
 *   quadrature: collapsed Gauss-Jacobi rules with p_K + 2 points per
 *     collapsed direction in the element, p_F + 2 on a face (exact to degree
 *     2p + 3), face points placed in the canonical frame;
 *   geometry: the isoparametric 10-node quadratic map (vertices, then the
 *     midpoints of edges 01, 02, 03, 12, 13, 23), evaluated at every
 *     quadrature point of curved elements; straight-sided elements keep one
 *     affine record.
 * Packed device layouts (FP64):
 *   U, Ustar  per element [m][Np_e] back to back (offsets uoff, m = 5)
 *   Q         per element [3][m][Np_e] (offset 3 uoff)
 *   UH, g, x  per face [m][Nfp_F] back to back (offsets hoff)
 *   blocks    block b (row face F, column face G) at boff[b], bs_F x bs_G,
 *             bs = m Nfp, column-major: value (r, c) at boff[b] + c bs_F + r,
 *             r = a Nfp_F + l.
 * ---------------------------------------------------------------------- */
#define HDG_TET 3

typedef struct {
    int64_t n_elem;
    int64_t n_vert;
    const double* vert_xyz;       /* [n_vert][3] */
    const int64_t* elem_vert;     /* [n_elem][4], positively oriented */
    const int64_t* periodic_map;  /* [n_vert] master vertex, or NULL */
    const int32_t* bnd_tag;       /* [n_elem][4] per local face (kinds as for hdg_mesh), or NULL */
    const int32_t* elem_p;        /* [n_elem] degrees 1..4 */
    const double* geo;            /* [n_elem][10][3] quadratic nodes, or NULL for straight-sided elements */
} hdg_tet_mesh;

typedef struct {
    int64_t n_elem, n_faces, nnzb;
    int64_t n_u;                  /* sum of m Np_e: length of U (Q is 3 n_u) */
    int64_t n_trace;              /* sum of m Nfp_F: length of UH, g, x */
    int64_t n_vals;               /* sum of bs_F bs_G: length of the block values */
    int64_t n_curved;             /* elements with per-point geometry */
    int64_t device_bytes;
} hdg_tet_sizes;

/* Build tables, skeleton, geometry and device storage of a tetrahedral mesh.
 * HDG_EUNSUPPORTED for degrees outside 1..4; HDG_EINVAL for inconsistent
 * meshes (a face of more than two elements, repeated vertices, untagged
 * boundary faces, tagged interior faces, a non-positive Jacobian at a
 * quadrature point).  Supported calls on the handle: hdg_set_params (tau,
 * viscosity law, precision: any HDG_PREC_MIXED* selects the tetrahedral mixed
 * form: FP32 Jacobian terms and column variations, the contraction and the
 * Schur product S = Dt - W Z on the tensor cores in 3xTF32, FP32 triangular
 * solves for W and Z and FP32 trace blocks, with FP64 fluxes, lifting
 * operators, interior LU (pivoting) and right-hand sides), hdg_set_bc_state, hdg_set_stream, hdg_linearize_condense (packed
 * layouts; nu must be NULL), hdg_trace_matvec, hdg_trace_rhs,
 * hdg_recover_interior, hdg_get_blocks (FP32 values after a mixed
 * linearization), hdg_status, hdg_residual, hdg_update_state,
 * hdg_blockjacobi_setup / _apply, hdg_gmres, hdg_newton, hdg_newton_fixed,
 * hdg_dirk_step, hdg_rb_*, hdg_set_preconditioner, hdg_schwarz_setup /
 * _apply,
 * hdg_autotune / hdg_set_tuning (panel width), hdg_profile*, hdg_destroy; the
 * others return HDG_EUNSUPPORTED. */
int hdg_create_tet(hdg_handle* out, const hdg_tet_mesh* mesh, double gamma, double Re, double Pr, double Mach);
int hdg_create_tet_host(hdg_handle* out, const hdg_tet_mesh* mesh, double gamma, double Re, double Pr,
                        double Mach);
int hdg_tet_query(hdg_handle h, hdg_tet_sizes* out);
/* Host copies (any pointer may be NULL): uoff [E+1], hoff [F+1], face_p [F],
 * f2e [F][2] (-1 on the boundary), e2f [E][4], frame [E][4][3] (local
 * vertices of each face in canonical order), rowptr [F+1], col [nnzb]
 * (ascending), boff [nnzb+1]. */
int hdg_tet_layout(hdg_handle h, int64_t* uoff, int64_t* hoff, int32_t* face_p, int32_t* f2e, int32_t* e2f,
                   int32_t* frame, int32_t* rowptr, int32_t* col, int64_t* boff);
/* Reference tables (host): the element rule xq [Nq][3], wq [Nq] and basis
 * phi [Nq][Np], dphi [3][Nq][Np] of degree p; the face rule xs [Nfq][2],
 * ws [Nfq] and trace basis mu [Nfq][Nfp] of degree pF.  NULL skips. */
int hdg_tet_ref_tables(int p, double* xq, double* wq, double* phi, double* dphi);
int hdg_tri_ref_tables(int pF, double* xs, double* ws, double* mu);

/* ---- Partition-ready layout (Sec. 3.5) ------------------------------------
 * For a run over several GPUs, element-local work (linearization, condensation,
 * recovery) stays on the part that owns the element; parts exchange only trace
 * data of faces on part interfaces: the condensed blocks of those faces' rows
 * during assembly, and trace entries (the halo) in every matvec.  These calls
 * describe the layout on the host (quad, hex and tetrahedral handles, host-only
 * handles included); no call of the library communicates.
 *
 * hdg_partition: recursive coordinate bisection of the element centroids
 * (vertex means) into n_parts parts.  Each split cuts the longest extent of the
 * current element set (lowest axis on ties), ordered by (coordinate, element
 * id), at the element count of its first half of the parts; part q gets
 * E / n_parts elements, plus one for q < E mod n_parts.  elem_part [E] (host,
 * out).  HDG_EINVAL for n_parts outside 1..E or a NULL elem_part. */
int hdg_partition(hdg_handle h, int n_parts, int32_t* elem_part);

typedef struct {
    int64_t n_elem;             /* elements of the part */
    int64_t n_interior_elem;    /* of which none has a face on a part interface */
    int64_t n_faces;            /* faces the part owns: the owner of a face is the smaller part id of its elements */
    int64_t n_interface_faces;  /* faces between this part and another (owned or not) */
    int64_t n_halo_faces;       /* faces owned elsewhere whose trace entries the owned block rows reference */
} hdg_part_sizes;

/* Layout of part `part` under the partition elem_part [E] (any non-negative ids):
 * elems [n_elem] (interior elements first, then interface elements, ascending
 * ids within each), faces [n_faces] (owned, ascending), interface_faces and
 * interface_peer [n_interface_faces] (ascending faces, the other part),
 * halo_faces and halo_owner [n_halo_faces] (ascending faces, their owner).
 * Host arrays allocated by the caller from the sizes; any pointer may be NULL,
 * so a first call with NULL arrays returns the sizes.  HDG_EINVAL for a NULL
 * elem_part, part < 0 or a negative part id. */
int hdg_part_layout(hdg_handle h, const int32_t* elem_part, int part, hdg_part_sizes* sizes, int64_t* elems,
                    int64_t* faces, int64_t* interface_faces, int32_t* interface_peer, int64_t* halo_faces,
                    int32_t* halo_owner);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H */
