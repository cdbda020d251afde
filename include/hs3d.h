/*
 * hs3d -- GB300 (sm_103a) DGSEM residual and low-storage RK3 library for the
 * compressible Euler and Navier-Stokes equations on curvilinear hexahedra.
 *
 * The method is the one of the HORSES3D paper (arXiv 2206.09733):
 *   - conservation law u_t + div F_e = div F_v, u = (rho, rho v, rho e)
 *     (Sec. 3.2, Eq. compressibleNScompact; F_v of Eq. viscousfluxes);
 *   - mapped to the reference cube, J u_t + div_xi F~ = 0 with contravariant
 *     fluxes (Sec. 3.3, Eq. compressibleNScompact_transformed);
 *   - DGSEM weak form with a numerical flux at faces on Gauss-Lobatto nodes
 *     (Sec. 3.3, Eqs. NS2-NS5), Lax-Friedrichs / Roe / central surface
 *     fluxes and BR1 viscous terms (Sec. 3.3, list of fluxes);
 *   - Chandrashekar entropy-conservative split form (Sec. 3.5);
 *   - Williamson low-storage RK3 (Sec. 3.7).
 *
 * Conventions for every entry point:
 *   - All device arrays are FP64, contiguous, at least 16-byte aligned,
 *     element-major: u[e][v][k][j][i] with v = rho, rho v1, rho v2, rho v3,
 *     rho e and i the fastest (xi) index; n = N+1 nodes per direction.
 *     Elements of an ex*ey*ez box are numbered e = a + ex*(b + ey*c).
 *   - The caller owns state arrays (u, g, dudt); the library owns meshes,
 *     their geometry and scratch, and server slots.
 *   - Calls taking a `stream` (a cudaStream_t, NULL = legacy default stream)
 *     are stream-ordered and asynchronous; they enqueue work and return.
 *     The same mesh must not be used by two streams at once (its scratch is
 *     shared).
 *   - No exception crosses the ABI.  Every call returns an hs3d_status; on
 *     error hs3d_last_error() gives a thread-local message.  A CUDA error is
 *     reported as HS3D_ERR_CUDA.  Invalid arguments are rejected before any
 *     work is enqueued (HS3D_ERR_INVALID), unsupported combinations with
 *     HS3D_ERR_UNSUPPORTED.
 *   - There is no CPU fallback: without a usable GPU every compute call
 *     returns HS3D_ERR_CUDA.
 */
#ifndef HS3D_H
#define HS3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS3D_OK = 0,
    HS3D_PENDING = 1,            /* server: request not finished yet */
    HS3D_ERR_INVALID = -1,       /* bad argument or descriptor */
    HS3D_ERR_NOMEM = -2,         /* device or host allocation failed, or request larger than the budget */
    HS3D_ERR_CUDA = -3,          /* a CUDA call failed (no device, launch error, ...) */
    HS3D_ERR_TIMEOUT = -4,       /* a bounded wait ran out */
    HS3D_ERR_NONPHYSICAL = -5,   /* rho <= 0, p <= 0 or NaN detected in a state */
    HS3D_ERR_UNSUPPORTED = -6    /* valid but not implemented combination */
} hs3d_status;

/* physics */
enum { HS3D_EULER = 0, HS3D_NS = 1 };
/* surface (Riemann) flux, Sec. 3.3, each times the face scale |Ja^d|:
 *   LF        (F_L+F_R).n/2 - lambda [[u]]/2, lambda = max(|v_L.n| + c_L, |v_R.n| + c_R)
 *   ROE       Roe's flux (sqrt(rho) averages, no entropy fix); the wave strengths are
 *             formed from the jumps of rho, v, p with the averaged state, which is also
 *             Roe and Pike's construction (the two name the same flux)
 *   EC        central: Chandrashekar's entropy-conservative flux, no dissipation
 *   RUSANOV   as LF with lambda = max(|v_L.n|, |v_R.n|) + max(c_L, c_R)
 *   LDROE     low-dissipation Roe (L2Roe): the velocity jump in Roe's dissipation
 *             scaled by min(1, max(M_L, M_R)), M = |v|/c
 *   MATRIX    entropy-stable: Chandrashekar's flux minus matrix dissipation
 *             R|Lambda|T R^T [[w]] (scaled eigenvectors at the Chandrashekar averages,
 *             w the entropy variables) */
enum {
    HS3D_FLUX_LF = 0,
    HS3D_FLUX_ROE = 1,
    HS3D_FLUX_EC = 2,
    HS3D_FLUX_RUSANOV = 3,
    HS3D_FLUX_LDROE = 4,
    HS3D_FLUX_MATRIX = 5
};
/* volume term (Sec. 3.5): standard DGSEM, or a split form written as flux
 * differencing with a symmetric two-point flux F#(u_i, u_m).(Ja_i + Ja_m):
 *   EC         Chandrashekar's entropy-conservative, kinetic-energy-preserving flux
 *   KG         Kennedy-Gruber:  {rho}{v_a}, {rho}{v_a}{v} + {p}a, {rho}{v_a}{e} + {p}{v_a}
 *   PIROZZOLI  Pirozzoli:       as KG for mass and momentum, energy {rho}{v_a}{h}
 *   DUCROS     Ducros et al.:   {rho}{v_a}, {rho v}{v_a} + {p}a, {rho e + p}{v_a}
 *   MORINISHI  Morinishi:       {rho v_a}, {rho v_a}{v} + {p}a, {rho v_a}{|v|^2/2} + gamma/(gamma-1){p v_a}
 *   IR         entropy conserving (Ismail-Roe), from z = sqrt(rho/p)(1, v, p) and
 *              logarithmic means of z1 and z5
 * ({.} arithmetic mean of the two nodes, v_a = v.a, e = (rho e)/rho,
 * h = (rho e + p)/rho) */
enum {
    HS3D_VOL_STANDARD = 0,
    HS3D_VOL_EC = 1,
    HS3D_VOL_KG = 2,
    HS3D_VOL_PIROZZOLI = 3,
    HS3D_VOL_DUCROS = 4,
    HS3D_VOL_MORINISHI = 5,
    HS3D_VOL_IR = 6
};
/* explicit low-storage time integrator (Sec. 3.7): Williamson's three-stage
 * third-order scheme, or Carpenter and Kennedy's five-stage fourth-order
 * 2N-storage scheme (NASA TM 109112, 1994) */
enum { HS3D_TIME_RK3 = 0, HS3D_TIME_RK4 = 1 };
/* arithmetic: all FP64; or FP32 flux arithmetic on FP64-formed deviations
 * from a per-element reference state, with FP64 state, geometry and state
 * accumulation (MIXED32).  MIXED_TC is accepted and computes exactly as
 * MIXED32: the derivative-matrix contraction stays on the CUDA cores (the
 * part a TF32-split tensor-core product could take measured at most 4% of
 * the residual at N = 7; the float-float mass contraction needs more than
 * FP32 accuracy). */
enum { HS3D_FP64 = 0, HS3D_MIXED32 = 1, HS3D_MIXED_TC = 2 };
/* initial conditions */
enum { HS3D_IC_VORTEX = 0, HS3D_IC_TGV = 1 };
/* solution nodes (Sec. 3.3): Gauss-Lobatto, or Gauss-Legendre (standard
 * volume term only: the split forms need the Gauss-Lobatto summation-by-parts
 * property) */
enum { HS3D_NODES_LOBATTO = 0, HS3D_NODES_GAUSS = 1 };

/* Mesh of a periodic box [lo, hi] with ex*ey*ez hexahedra of degree N
 * (1 <= N <= 7) on Gauss-Lobatto nodes (Sec. 3.1, 3.3).  Every node is moved
 * by perturb_amp * (L_c/2pi) * sin(t_x) sin(t_y) sin(t_z), t = the unperturbed
 * position mapped linearly from [lo, hi] to [-pi, pi] (so on [-pi,pi]^3 the
 * displacement is exactly amp*sin(x)sin(y)sin(z) in every coordinate).
 * node_xyz, if not NULL, is a HOST FP64 array [E][3][n][n][n] of node
 * coordinates that replaces the generator (the box must still be periodic and
 * the faces of neighbouring elements must coincide).  periodic[] must be all
 * 1 (other boundaries: HS3D_ERR_UNSUPPORTED).
 * nodes: HS3D_NODES_LOBATTO (zero) or HS3D_NODES_GAUSS.  The element map is
 * always the degree-N interpolant through the Gauss-Lobatto points (generator
 * or node_xyz); on Gauss nodes the state, X, Ja and J live at the
 * Gauss-Legendre points: Ja^d is the curl-form metric polynomial evaluated
 * there, J = det(dX/dxi) of the map, the face metrics its values at the face
 * points. */
typedef struct {
    int ex, ey, ez;
    int N;
    double lo[3], hi[3];
    int periodic[3];
    double perturb_amp;
    const double *node_xyz;
    int nodes;
} hs3d_mesh_desc;

/* Solver configuration.  gamma: ratio of specific heats; Re, Pr: Reynolds and
 * Prandtl numbers (mu = 1/Re, kappa = mu gamma/((gamma-1) Pr), gas constant
 * 1, temperature T = p/rho); Ma: used only by initial conditions; cfl: the
 * convective CFL number of the time-step rule; time_scheme: HS3D_TIME_RK3
 * or HS3D_TIME_RK4, the integrator of hs3d_rk3_step/hs3d_rk3_run and of the
 * server (a zero-initialised struct selects RK3). */
typedef struct {
    int physics;
    int surface_flux;
    int volume_form;
    int precision;
    double gamma, Re, Pr, Ma, cfl;
    int time_scheme;
} hs3d_solver_cfg;

/* Initial condition.  VORTEX: isentropic vortex of strength beta centred at
 * (xc, yc) (uniform in z), free stream rho = p = 1 moving at Ma*sqrt(gamma)
 * along x, evaluated at time t (translated, nearest periodic image).
 * TGV: Taylor-Green vortex, p0 = 1/(gamma Ma^2), rho = p/p0. */
typedef struct {
    int kind;
    double gamma, Ma, beta, xc, yc, t;
} hs3d_ic;

typedef struct hs3d_mesh hs3d_mesh;
typedef struct hs3d_server hs3d_server;

/* Build a mesh on the current CUDA device: node coordinates, curl-form metric
 * terms Ja^d_c = J dxi_d/dx_c and J (Sec. 3.3), face normals, computed by GPU
 * kernels in FP64.  Synchronous.  The library owns all its memory;
 * HS3D_ERR_NOMEM if the device cannot hold it. */
hs3d_status hs3d_mesh_create(const hs3d_mesh_desc *desc, hs3d_mesh **out);
void hs3d_mesh_destroy(hs3d_mesh *mesh);

/* Elements, degree and device bytes held by the mesh (any pointer may be NULL). */
hs3d_status hs3d_mesh_info(const hs3d_mesh *mesh, int64_t *E, int *N, size_t *device_bytes);

/* Copy the mesh geometry into caller-owned DEVICE arrays (any may be NULL):
 * X [E][3][n3], Ja [E][3][3][n3], J [E][n3].  Stream-ordered. */
hs3d_status hs3d_mesh_geometry(const hs3d_mesh *mesh, double *X, double *Ja, double *J, void *stream);

/* Evaluate an initial condition at the mesh nodes into u (device). */
hs3d_status hs3d_init_state(const hs3d_mesh *mesh, const hs3d_ic *ic, double *u, void *stream);

/* Semi-discrete residual du/dt = -(V + S)/J (Sec. 3.3, Eq. NS5 in strong
 * form on Gauss-Lobatto nodes): volume term V (standard or split form),
 * surface term S lifted from the numerical fluxes, Jacobian scaling; for NS
 * the BR1 gradients and viscous fluxes.  u and dudt: device [E][5][n3],
 * distinct arrays.  Stream-ordered. */
hs3d_status hs3d_residual(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, const double *u, double *dudt,
                          void *stream);

/* One low-storage Runge-Kutta step (Sec. 3.7) of the scheme cfg->time_scheme
 * names: per stage k,
 *   g <- A_k g + dt R(u),  u <- u + B_k g,
 * Williamson RK3: A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15);
 * Carpenter-Kennedy RK4: five stages with their published A_k, B_k.
 * (The name keeps "rk3" for the default scheme.)  u and g: device
 * [E][5][n3] doubles, updated in place.  g is the stepper's register
 * (caller-owned scratch, need not be initialised): the FP64 path keeps it in
 * FP64; the mixed paths, whose increments dt R are FP32 quantities, keep it
 * as FP32 [E][5][n3] in the first half of the buffer (the state u always
 * accumulates in FP64).  dt > 0 is used
 * as given; dt <= 0 computes dt on the device from the state at the start of
 * the step:
 *   dt = min( cfl*8/(n^2 max_nodes sum_d (|Ja^d.v| + c|Ja^d|)/J),
 *             12/(n^4 max_nodes (mu/rho) sum_d (|Ja^d|/J)^2) )   (viscous term NS only).
 * Stream-ordered. */
hs3d_status hs3d_rk3_step(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, double *u, double *g, double dt,
                          void *stream);

/* nsteps steps as hs3d_rk3_step, replayed from a CUDA graph captured on
 * the first call for this (mesh, cfg, u, g, dt).  The mesh keeps the graphs of
 * the two most recently used (cfg, u, g, dt), so a caller alternating between
 * two state buffers replays without re-capture; a third combination replaces
 * the least recently used graph.  dt > 0: fixed; dt == 0: from the rule above,
 * with one pass over u before the first step for its dt maxima; dt < 0:
 * continue — when the previous hs3d_rk3_step / hs3d_rk3_run on this mesh
 * advanced this same u with the same cfg and nothing rewrote u, the mesh's
 * dt maxima or its FP32 shadow since (hs3d_init_state of u, hs3d_residual or
 * hs3d_dt of another state, hs3d_clock with reset, hs3d_autotune), the
 * maxima the last step left are used and that pass is skipped (the steps are
 * then exactly the steps of one longer run); otherwise as dt == 0.  The
 * library cannot see writes to u by the caller: a caller that changes u
 * between calls passes dt = 0.  Stream-ordered. */
hs3d_status hs3d_rk3_run(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, double *u, double *g, double dt,
                         int nsteps, void *stream);

/* dt of the rule above for state u, written to dt_out (DEVICE, 1 double). */
hs3d_status hs3d_dt(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, const double *u, double *dt_out,
                    void *stream);

/* Simulated time and step count accumulated by hs3d_rk3_step / hs3d_rk3_run on
 * this mesh since creation or the last reset (reset != 0 zeroes them).
 * Synchronises the stream. */
hs3d_status hs3d_clock(const hs3d_mesh *mesh, double *t, int64_t *steps, int reset, void *stream);

/* Quadrature diagnostics (FP64, fixed-order two-level reduction, so the
 * result is bitwise reproducible): out[0..4] = sum_e sum_ijk J w_i w_j w_k
 * f_v with f = dudt if given else u; if dudt is given out[5] = entropy rate
 * sum J w w w (w(u).dudt) with w = dS/du, S = -rho s, s = ln p - gamma ln rho
 * (Sec. 4.4, Eq. shock:entropy) and out[6] = sum |J w w w w_v dudt_v|.
 * out: DEVICE, 7 doubles.  Stream-ordered. */
hs3d_status hs3d_diagnostics(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, const double *u,
                             const double *dudt, double *out, void *stream);

/* The quadrature diagnostics of hs3d_diagnostics, for callers that cannot
 * allocate device memory: code running while a CUDA stream capture is
 * active (cudaMalloc is not allowed there), code inside a framework whose
 * memory pool owns all device memory, or real-time loops that must not
 * allocate or synchronise.  The paper has no counterpart; this is a library
 * convenience.  Allocates nothing: the caller passes every input (N, E,
 * gamma, the solution nodes the mesh was built on, HS3D_NODES_LOBATTO or
 * HS3D_NODES_GAUSS, whose quadrature weights the sums use, the Jacobian J
 * [E][n3] e.g. copied out by hs3d_mesh_geometry, the state u and optionally
 * dudt, all DEVICE FP64) and the DEVICE output out[7] (same meaning as
 * hs3d_diagnostics; the two give the same result on the same mesh).  The
 * per-block partial sums live in one fixed device array of 4096 slots, each
 * covering 2048 nodes, so E*(N+1)^3 may not exceed 8,388,608 nodes
 * (HS3D_ERR_INVALID beyond).  The array is compiled into the library: every
 * GPU that loads it holds the array (256 KB) until the process exits.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call reuses the same array and leaves its partial sums in it; each
 * call writes every slot it later reads, so nothing needs clearing, but two
 * calls that overlap on the GPU (other streams, other threads) race on the
 * array and give wrong results.  Stream-ordered. */
hs3d_status hs3d_diagnostics_noalloc(int N, int64_t E, double gamma, int nodes, const double *J, const double *u,
                                     const double *dudt, double *out, void *stream);

/* Autotuner: times every admissible launch shape (elements per CTA) of the
 * BR1-gradient and element kernels for this mesh and configuration on a
 * scratch state, keeps the fastest for (N, precision, kernel) for the rest of
 * the process, and writes the choices to the JSON file named by the
 * environment variable HS3D_TUNE_CACHE if set (read back at the next mesh
 * creation).  choice_out (HOST, 2 ints, may be NULL) receives [gradient,
 * element] elements per CTA.  Synchronous; allocates two scratch states.
 * Call it outside any stream capture. */
hs3d_status hs3d_autotune(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, int *choice_out, void *stream);

/* ---------------------------------------------------------------- per-element degree (Sec. 3.6) */

/* A periodic box as for hs3d_mesh_create whose elements carry their own
 * polynomial degree (Sec. 3.6, isotropic per element): degree is a HOST
 * array of E = ex*ey*ez ints in 1..7 in element order e = a + ex*(b + ey*c);
 * desc->N is ignored, desc->node_xyz must be NULL and desc->nodes
 * Gauss-Lobatto.  Faces between elements of degrees N_L and N_R are coupled
 * by a mortar of degree max(N_L, N_R) (the mortar method Sec. 3.6 names):
 * traces interpolated to its Gauss-Lobatto points, the numerical flux and
 * the BR1 interface value formed there, and each side given the L2
 * projection onto its degree (exact integrals).  Like the paper's, this
 * coupling does not keep entropy conservation across faces of different
 * degree.  Geometry (the rules for p-non-conforming faces Sec. 3.6 follows):
 * every element's map is the degree-Ngeo polynomial, Ngeo = max(1,
 * floor(Nmin/2)), interpolating the box map (with its perturbation) at the
 * element's degree-Ngeo Gauss-Lobatto points; its metric terms are the curl
 * form at the element's own degree, so the two sides of every face see the
 * same face metric and a uniform flow stays uniform.  Nmin = 1 requires
 * perturb_amp = 0 (HS3D_ERR_INVALID otherwise).  Synchronous. */
typedef struct hs3d_pmesh hs3d_pmesh;
hs3d_status hs3d_pmesh_create(const hs3d_mesh_desc *desc, const int *degree, hs3d_pmesh **out);

/* As hs3d_pmesh_create with a degree per element AND reference direction
 * (Sec. 3.6: P_x, P_y, P_z may differ, anisotropic p-adaptation): degree3 is
 * a HOST array of 3E ints in 1..7, element e's (P_x, P_y, P_z) at 3e.  Element
 * e has P_d + 1 Gauss-Lobatto nodes along d, node (i, j, k) at
 * i + n_x (j + n_y k), and its block [5][n_x n_y n_z] in element order (the
 * offsets of hs3d_pmesh_layout).  The face normal to d couples its two sides
 * with a mortar of degree max(P_L, P_R) in EACH tangential direction
 * separately (interpolation to, and L2 projection from, its points direction
 * by direction); its face metric is that of a side whose tangential degrees
 * are the mortar's (the minus side first), else the minus side's
 * interpolated, which is exact (Pmin = the smallest degree of the mesh over
 * elements and directions, Ngeo = max(1, floor(Pmin/2)) as above).  The dt
 * rule takes each direction's resolution inside the sum:
 *   dt = min( cfl*8 / max_nodes sum_d n_d^2 (|Ja^d.v| + c|Ja^d|)/J,
 *             12 / max_nodes (mu/rho) sum_d n_d^4 (|Ja^d|/J)^2 ).
 * When every element has equal degrees in its three directions this is
 * hs3d_pmesh_create with degree[e] = P_x of e.  Otherwise the mesh runs in
 * FP64 only (a mixed-precision cfg gives HS3D_ERR_UNSUPPORTED), and every
 * hs3d_pmesh_* call below applies.  Synchronous. */
hs3d_status hs3d_pmesh_create3(const hs3d_mesh_desc *desc, const int *degree3, hs3d_pmesh **out);
void hs3d_pmesh_destroy(hs3d_pmesh *pmesh);

/* State layout of the mesh: element e's block [5][n_e][n_e][n_e] (n_e its
 * degree + 1, v and i as in the conforming layout) starts offset[e] doubles
 * into the state array; offset (HOST, E+1 int64) also receives offset[E] =
 * the doubles a state array must hold.  Elements are stored grouped by
 * degree (ascending), in element order within a degree; each group starts at
 * a multiple of 160 doubles, and the gaps between groups are never read or
 * written.  (A mesh of hs3d_pmesh_create3 with per-direction degrees stores
 * its blocks [5][n_x n_y n_z] in element order, without gaps.)  Ngeo (may be
 * NULL) receives the geometry degree. */
hs3d_status hs3d_pmesh_layout(const hs3d_pmesh *pmesh, int64_t *offset, int *Ngeo);

/* Node coordinates and Jacobians into caller-owned DEVICE arrays (either may
 * be NULL): element e's X block [3][nodes_e] at 3*offset[e]/5, its J block
 * [nodes_e] at offset[e]/5 (arrays of 3*offset[E]/5 and offset[E]/5 doubles).
 * Stream-ordered. */
hs3d_status hs3d_pmesh_geometry(const hs3d_pmesh *pmesh, double *X, double *J, void *stream);

/* Initial condition at every element's nodes into u (device, the layout above). */
hs3d_status hs3d_pmesh_init_state(const hs3d_pmesh *pmesh, const hs3d_ic *ic, double *u, void *stream);

/* Residual du/dt = -(V + S)/J of every element (volume term at its own
 * degree, surface term from the mortar fluxes projected onto its faces), as
 * hs3d_residual.  u, dudt: device, the layout above, distinct.  Any
 * precision; Gauss-Lobatto nodes.  Stream-ordered. */
hs3d_status hs3d_pmesh_residual(const hs3d_pmesh *pmesh, const hs3d_solver_cfg *cfg, const double *u, double *dudt,
                                void *stream);

/* nsteps low-storage RK steps of cfg->time_scheme on u and g (device, the
 * layout above; g need not be initialised).  dt > 0: fixed; otherwise dt
 * of every step is the conforming rule per element with the element's own
 * n, minimised over the elements:
 *   dt = min_e min( cfl*8/(n_e^2 lam_c,e), 12/(n_e^4 lam_v,e) ),
 * the first step from a pass over u, the later ones from the maxima the
 * previous step's last stage reduced.  Steps after the first replay one
 * captured CUDA graph (kept for the last (cfg, u, g, dt)).  dt < 0:
 * continue -- when the previous hs3d_pmesh_run on this mesh advanced this
 * same u with the same cfg and neither hs3d_pmesh_init_state of u, a
 * mixed-precision hs3d_pmesh_residual of another state nor a clock reset
 * came between, every
 * step is a replay (the steps are exactly those of one longer run);
 * otherwise as dt = 0.  Writes to u by the caller are not seen: a caller
 * that changes u passes dt = 0.  Stream-ordered. */
hs3d_status hs3d_pmesh_run(const hs3d_pmesh *pmesh, const hs3d_solver_cfg *cfg, double *u, double *g, double dt,
                           int nsteps, void *stream);

/* Quadrature diagnostics of hs3d_diagnostics on the mesh with per-element
 * degrees (each element with its own Gauss-Lobatto weights): out[0..4] =
 * sum_e sum_ijk J w_i w_j w_k f_v (f = dudt if given, else u), out[5] the
 * entropy rate and out[6] its magnitude scale.  Each degree group reduces in
 * a fixed order and the groups are summed in a fixed order, so the result
 * is bitwise reproducible.  u, dudt: device, the layout above; out: DEVICE,
 * 7 doubles.  Stream-ordered. */
hs3d_status hs3d_pmesh_diagnostics(const hs3d_pmesh *pmesh, const hs3d_solver_cfg *cfg, const double *u,
                                   const double *dudt, double *out, void *stream);

/* Simulated time and steps of hs3d_pmesh_run since creation or the last
 * reset, as hs3d_clock. */
hs3d_status hs3d_pmesh_clock(const hs3d_pmesh *pmesh, double *t, int64_t *steps, int reset, void *stream);

/* ---------------------------------------------------------------- instrumentation */

/* One RK3 step exactly as hs3d_rk3_step, launched eagerly with CUDA events
 * between the kernels on `stream`; waits for the step and writes the device
 * time in milliseconds to the HOST array ms_out[5]: [0] dt rule (maxima +
 * finalize), [1] BR1 gradient kernels, [2] face kernels, [3] element
 * (volume + lift + RK) kernels, each summed over the stages, [4] the
 * whole step.  Not part of the method; used to attribute time to kernels. */
hs3d_status hs3d_rk3_step_profiled(const hs3d_mesh *mesh, const hs3d_solver_cfg *cfg, double *u, double *g,
                                   double dt, double *ms_out, void *stream);

/* Measured arithmetic throughput of this GPU from FMA-chain kernels (8
 * independent chains per thread, 8 CTAs of 256 threads per SM), written to
 * the HOST array tflops_out[2]: [0] FP64, [1] FP32, in TFLOP/s (an FMA counts
 * two flops).  The roofline denominators of ALU-bound kernels.  Synchronous. */
hs3d_status hs3d_alu_peaks(double *tflops_out, void *stream);

/* Self-check of the library's integer-pipe FP64->FP32 rounding (used by the
 * mixed path instead of the FP64-pipe conversion): over n DEVICE doubles,
 * counts (DEVICE, 4 x uint64) receives [0] results that differ bitwise from
 * the hardware round-to-nearest conversion (inputs in the FP32 normal range,
 * infinities, NaN), [1] FP32->FP64 widenings that differ from the hardware
 * one, [2] inputs below the FP32 normal range (flushed to zero by design),
 * [3] finite inputs of magnitude 2^-74 .. 2^127 whose integer-pipe low part
 * (x - hi rounded to FP32, the float-float split) differs bitwise from the
 * hardware rounding of the FP64 difference.  Stream-ordered. */
hs3d_status hs3d_check_rounding(const double *in, int64_t n, unsigned long long *counts, void *stream);

/* ---------------------------------------------------------------- serving */

/* A solve request: a mesh, a solver configuration, an initial condition and
 * a stopping rule (t_final > 0: integrate to exactly t_final, the last dt
 * clipped; else n_steps steps).  result_host, if not NULL, is a caller-owned
 * HOST buffer of E*5*n3 doubles that receives the final state; it must stay
 * valid until hs3d_poll reports the request finished. */
typedef struct {
    hs3d_mesh_desc mesh;
    hs3d_solver_cfg cfg;
    hs3d_ic ic;
    double t_final;
    int n_steps;
    double *result_host;
} hs3d_request;

/* Outcome and timing of a request (seconds since the server was created). */
typedef struct {
    hs3d_status status;      /* HS3D_OK when finished, HS3D_PENDING, or an error */
    double t_sim;            /* simulated time reached */
    int64_t steps;           /* RK steps taken */
    int64_t dof;             /* nodes of the request (E n^3) */
    double t_submit, t_admit, t_done;
    size_t device_bytes;     /* footprint charged to the budget */
} hs3d_result;

/* A continuous-batching server on the current device.  hbm_budget_bytes
 * bounds the device memory held by admitted requests (0: 90% of the free
 * memory at creation).  max_batch bounds the requests sharing one launch
 * (0: 256).  A host thread admits queued requests when the budget has room,
 * groups the admitted ones by (N, physics, fluxes, precision), runs one RK3
 * step per group with shared launches, retires finished requests and
 * immediately admits the next. */
hs3d_status hs3d_server_create(size_t hbm_budget_bytes, int max_batch, hs3d_server **out);
/* Stops the thread after the running step; unfinished requests are dropped. */
void hs3d_server_destroy(hs3d_server *server);
/* Launch design of the shared launches (takes effect at the next step):
 *   HS3D_LAUNCH_GRID (default): one CTA per tile of elements (faces), each
 *     finding its request by a binary search over the group's item table;
 *   HS3D_LAUNCH_PERSISTENT: a work table (the request of every element of a
 *     group, uploaded when the set of running requests changes) and a
 *     persistent grid per kernel (as many CTAs as are resident at once), whose
 *     CTAs walk the tiles with a stride of the grid size.
 * Both compute the same results bit for bit. */
enum { HS3D_LAUNCH_GRID = 0, HS3D_LAUNCH_PERSISTENT = 1 };
hs3d_status hs3d_server_set_launch_mode(hs3d_server *server, int mode);
/* Copies the request and queues it; never blocks on the GPU.  HS3D_ERR_NOMEM
 * if the request alone exceeds the budget, HS3D_ERR_INVALID for a bad
 * descriptor. */
hs3d_status hs3d_submit(hs3d_server *server, const hs3d_request *req, uint64_t *ticket);
/* Non-blocking: HS3D_PENDING until the request is finished, then its final
 * status; res (may be NULL) receives the timing record.  A finished ticket
 * can be polled again; unknown tickets give HS3D_ERR_INVALID. */
hs3d_status hs3d_poll(hs3d_server *server, uint64_t ticket, hs3d_result *res);
/* Counters: requests queued, running, finished; device bytes in use. */
hs3d_status hs3d_server_stats(hs3d_server *server, int64_t *queued, int64_t *running, int64_t *finished,
                              size_t *bytes_in_use);

/* Thread-local message of the last failing call on this thread. */
const char *hs3d_last_error(void);
/* Library version string. */
const char *hs3d_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HS3D_H */
