/*
 * dgw.h -- C ABI of the GB300 DG elastic-wave hot path.
 *
 * The library evaluates the semi-discrete upwind DG operator of a linear
 * Friedrichs system (the paper's Section 2, eq. LPDE: Q du/dt +
 * sum_k d_k(A_k u) = 0) on curvilinear hexahedra, and advances it with a
 * five-stage low-storage Runge-Kutta method.  Three systems are built
 * (dgw_config.system): velocity-stress elasticity (m = 9 unknowns, the
 * medium in Q; the hot path), scalar transport (m = 1, A_k = beta_k, Q = 1;
 * Section 6.1) and the linearized shallow-water system of
 * eq. linearizedShallow with Phi = 1 and no Coriolis force, friction or wind
 * stress (m = 3, u = (phi, Phi u, Phi v), Q = I, A_3 = 0; Section 6.2).  The numerical flux is the upwind HDG flux (eq. RiemannFluxBoth)
 * with the trace eliminated through the face conservation condition
 * (eq. HDGeqn, in the form of eq. iHDGtrace); the time scheme is the paper's
 * element-by-element explicit HDG scheme (Section 4.3) with LSRK(5,4) in place
 * of forward Euler.
 *
 * Conventions shared by every call
 * --------------------------------
 * N      polynomial degree per axis (1..7); n = N+1 GLL nodes per axis,
 *        Np = n^3 nodes per element, nf = n^2 nodes per face.
 * node   index i + n*(j + n*k) of reference node (r_i, s_j, t_k); r fastest.
 * faces  0: r=-1, 1: r=+1, 2: s=-1, 3: s=+1, 4: t=-1, 5: t=+1.
 * state  u[m][nel][Np], FP64.  Elastic: m = 9, fields (v1, v2, v3, s11, s22,
 *        s33, s23, s13, s12); transport: m = 1; shallow water: m = 3,
 *        (phi, Phi u, Phi v).  Below, [9] reads [m] for the other systems.
 *
 * Errors: every call returns a dgw_status and never aborts or throws.  A
 * failing call leaves a message retrievable with dgw_last_error(ctx).  Calls
 * on one context are not thread safe; distinct contexts are independent.
 * Device work is enqueued on the caller's stream (a cudaStream_t passed as
 * void*, NULL = legacy default stream).  Pointers to field buffers may be
 * device memory (the call is asynchronous on the stream) or host memory (the
 * call stages the data through context-owned device buffers and returns after
 * the copies back to the host have completed).  The library never frees
 * caller memory.
 */
#ifndef DGW_H
#define DGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgw_ctx dgw_ctx;

typedef enum {
  DGW_OK = 0,
  DGW_ERR_ARG = -1,         /* invalid argument (sizes, connectivity, J <= 0, material) */
  DGW_ERR_STATE = -2,       /* calls out of order: create -> mesh -> material -> compute */
  DGW_ERR_OOM = -3,         /* device allocation failed */
  DGW_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  DGW_ERR_UNSTABLE = -5,    /* non-finite energy */
  DGW_ERR_TIMEOUT = -6,     /* reserved for bounded device waits */
  DGW_ERR_UNSUPPORTED = -7  /* configuration or call not built */
} dgw_status;

enum { DGW_PRECISION_FP64 = 0, DGW_PRECISION_MIXED = 1, DGW_PRECISION_MIXED_TC_FP16 = 2, DGW_PRECISION_MIXED_TC_BF16 = 3 };
/* Boundary tags.  1 is the traction-free surface of the elastic system
 * (exterior state (v, -sigma)) and the reflecting wall of the shallow-water
 * system (exterior state (phi, q - 2 (q.n) n), q the momentum, n the
 * horizontal part of the unit normal); it is refused for transport.  2 is a
 * zero exterior state for every system (absorbing for elasticity, zero
 * inflow for transport). */
enum { DGW_BC_INTERIOR = 0, DGW_BC_FREE_SURFACE = 1, DGW_BC_WALL = 1, DGW_BC_ABSORBING = 2 };
enum { DGW_SYSTEM_ELASTIC = 0, DGW_SYSTEM_TRANSPORT = 1, DGW_SYSTEM_SHALLOW_WATER = 2 };

typedef struct {
  int N;          /* polynomial degree, 1..7 */
  int flux_tau;   /* 0: central flux (stabilisation dropped), 1: upwind HDG flux */
  int precision;  /* DGW_PRECISION_FP64: every operation in FP64.
                     DGW_PRECISION_MIXED: volume, flux and lift in FP32 with FP32
                     geometry; the Runge-Kutta registers and energy stay FP64.
                     DGW_PRECISION_MIXED_TC_FP16 / _BF16: as MIXED, with the
                     volume term's 1-D derivative contractions D u and
                     D (A(Ja^i) u) on the tensor cores: each operand split into
                     a 16-bit hi and lo part (FP16 with a power-of-two scale per
                     line group, or BF16), D_hi x_hi + D_hi x_lo + D_lo x_hi
                     accumulated in FP32.  Single solves only (not batches).
                     The MIXED forms are for the elastic system only. */
  double cfl;     /* CFL number used by dgw_dt_cfl */
  int system;     /* DGW_SYSTEM_*.  Transport and shallow water: FP64 only, no
                     material (Q = I), no point force, receivers, adjoint or
                     batches (those calls return DGW_ERR_UNSUPPORTED). */
  double beta[3]; /* transport velocity (DGW_SYSTEM_TRANSPORT); ignored otherwise */
} dgw_config;

/* ABI version of this header (bumped on any signature change). */
#define DGW_ABI_VERSION 10
int dgw_abi_version(void);

/* GLL nodes r[0..N] (ascending, r[0] = -1, r[N] = +1) and weights w[0..N]
 * that the library uses; node coordinates passed to dgw_mesh_upload must be
 * given at these reference positions.  r, w: host arrays of N+1 doubles,
 * caller-owned.  DGW_ERR_ARG if N is outside 1..7 or a pointer is NULL. */
dgw_status dgw_reference_nodes(int N, double* r, double* w);

/* Create a context on CUDA device `device`.  *out receives an opaque handle
 * that owns all geometry, material and scratch device memory; release it
 * with dgw_destroy.  DGW_ERR_ARG for a bad config, DGW_ERR_CUDA if the device
 * cannot be used. */
dgw_status dgw_create(dgw_ctx** out, int device, const dgw_config* cfg);

/* Free every resource of the context (NULL is accepted). */
dgw_status dgw_destroy(dgw_ctx* ctx);

/* Mesh and skeleton (Section 2: elements K_j, faces of the skeleton, outward
 * normals n^- and n^+ = -n^-).  All arrays are host, caller-owned, read
 * during the call only:
 *   x      [nel][Np][3] physical coordinates of the element nodes at the
 *          reference positions of dgw_reference_nodes; faces shared by two
 *          elements must carry coincident nodes;
 *   etoe   [nel][6] neighbour element across each local face, -1 on a
 *          physical boundary (periodic meshes list the periodic neighbour);
 *   etof   [nel][6] the neighbour's local face (ignored where etoe = -1);
 *   orient [nel][6] face-node permutation 0..7: own face-local (a, b) (a along
 *          the lower-numbered tangential axis) meets neighbour (a', b') with
 *          (a1, b1) = (o & 1) ? (b, a) : (a, b), a' = (o & 2) ? N - a1 : a1,
 *          b' = (o & 4) ? N - b1 : b1;
 *   bc     [nel][6] DGW_BC_INTERIOR where etoe >= 0, otherwise
 *          DGW_BC_FREE_SURFACE / DGW_BC_WALL (see the boundary tags above) or
 *          DGW_BC_ABSORBING (exterior state 0).
 * The call computes the curl-form metric terms, Jacobians, face normals and
 * face stabilisation matrices on the device.  DGW_ERR_ARG (message names the
 * element) if the connectivity is not symmetric, a tag is inconsistent, or
 * J <= 0 at some node; nel * Np must be below 2^31.  May be called again to
 * replace the mesh (material must then be uploaded again).  For transport and
 * shallow water the context is ready for compute calls after this call. */
dgw_status dgw_mesh_upload(dgw_ctx* ctx, int64_t nel, const double* x, const int64_t* etoe,
                           const int8_t* etof, const int8_t* orient, const int8_t* bc);

/* Per-element isotropic medium: density rho, Lame parameters lam and mu (host
 * [nel] arrays, caller-owned).  The medium enters only the time weight
 * Q = diag(rho I, C_V^{-1}).  DGW_ERR_ARG unless rho > 0, mu > 0 and
 * lam > -2/3 mu everywhere.  DGW_ERR_STATE before dgw_mesh_upload.
 * DGW_ERR_UNSUPPORTED for transport and shallow water (Q = I). */
dgw_status dgw_material_upload(dgw_ctx* ctx, const double* rho, const double* lam, const double* mu);

/* rhs = L(u) = Q^{-1} [ split-form volume term + lifted upwind flux
 * difference ] for every element (the explicit HDG right-hand side, Section
 * 4.3, with the flux of eq. RiemannFluxBoth).  u: [9][nel][Np] input, rhs:
 * [9][nel][Np] output, both FP64, must not overlap.  t is the stage time (no
 * time-dependent terms are active; kept for sources). */
dgw_status dgw_rhs(dgw_ctx* ctx, const double* u, double* rhs, double t, void* stream);

/* One fused LSRK stage s (0..4):  res <- a_s res + dt L(u_in);
 * u_out <- u_in + b_s res (the explicit HDG scheme of Section 4.3, with the
 * five-stage low-storage Runge-Kutta method of Carpenter and Kennedy in place
 * of forward Euler).  u_in and u_out must be distinct buffers (the
 * face gather reads neighbours of u_in while u_out is written); res is read
 * and written in place.  Device pointers only. */
dgw_status dgw_stage(dgw_ctx* ctx, const double* u_in, double* u_out, double* res, int stage,
                     double t, double dt, void* stream);

/* dgw_stage followed by the discrete energy of u_out (as dgw_energy, in
 * FP64), accumulated inside the same kernel from the values it writes, so the
 * state is not read a second time.  energy_out: host double; synchronises the
 * stream.  The reduction order differs from dgw_energy's (agreement to
 * rounding).  DGW_ERR_UNSTABLE if the energy is not finite. */
dgw_status dgw_stage_energy(dgw_ctx* ctx, const double* u_in, double* u_out, double* res, int stage,
                            double t, double dt, double* energy_out, void* stream);

/* nsteps LSRK(5,4) steps of size dt from time t0, in place on u and res
 * (the explicit scheme of Section 4.3, five dgw_stage calls per step).
 * The first stage does not read the register (a_0 = 0), so the incoming
 * contents of res never matter; on return res holds the register of the last
 * stage.  res may be NULL: the context keeps the register in its own device
 * buffer.  Uses a context-owned second state buffer for the stage ping-pong
 * and copies the final state back into u.  Host buffers (u or res not device
 * memory) are staged through context buffers: u is copied in and out, res
 * only out (and not at all for nsteps = 0); the call then synchronises
 * `stream`. */
dgw_status dgw_step(dgw_ctx* ctx, double* u, double* res, double t0, double dt, int nsteps,
                    void* stream);

/* dgw_step whose last stage also accumulates the discrete energy of the new
 * state (as dgw_stage_energy; E as in dgw_energy), so advancing a state and
 * reading its energy costs no second pass over it; with host buffers, no
 * second upload.
 * nsteps >= 1; energy_out: host double; synchronises `stream`.
 * DGW_ERR_UNSTABLE if the energy is not finite. */
dgw_status dgw_step_energy(dgw_ctx* ctx, double* u, double* res, double t0, double dt, int nsteps,
                           double* energy_out, void* stream);

/* Discrete energy E = 1/2 sum_K sum_nodes w J u^T Q u, accumulated in FP64
 * with a fixed reduction order (bit-reproducible for a given mesh).
 * energy_out: host double.  Synchronises the stream.  DGW_ERR_UNSTABLE if E
 * is not finite (the value is still written). */
dgw_status dgw_energy(dgw_ctx* ctx, const double* u, double* energy_out, void* stream);

/* Point force F R(t) delta(x - x_s) in the velocity equations (the forcing f
 * of eq. LPDE): x_s is the image of the reference point xi[3] (in [-1,1]^3)
 * of `element`, F = force[3], and R is the Ricker wavelet
 * (1 - 2 (pi f0 (t - t0))^2) exp(-(pi f0 (t - t0))^2).  It is projected by
 * collocation, F R(t) l_j(xi) / (w_j J_j), added to the right-hand side of
 * that element at the stage times t + c_s dt of dgw_rhs/dgw_stage/dgw_step
 * (whose t arguments are the step start times).  element = -1 removes the
 * source.  DGW_ERR_STATE before mesh and material (material sets rho of the
 * source element: upload material first, set the source after).  Elastic
 * contexts only (DGW_ERR_UNSUPPORTED otherwise). */
dgw_status dgw_source_set(dgw_ctx* ctx, int64_t element, const double* xi, const double* force, double f0,
                          double t0);

/* Adjoint of nsteps LSRK steps of size dt that start at time t0 from the
 * forward state u_ckpt (device [9][nel][Np]; the register at a step start is
 * irrelevant, a_0 = 0).  lam_u, lam_res (device, distinct): the adjoint state
 * after the steps on entry, at t0 on return.  grad_mat (device [3][nel]:
 * rho, lambda, mu per element) is incremented by sum over stages of
 * dt w_s^T (dL/dm) u_{s-1} -- the contribution of these steps to the
 * gradient of any functional of the states -- including the medium's effect
 * on Q^{-1}, on the face impedances of the stabilisation and on the point
 * force.  The transpose uses L^T = (M Q) L_rev (M Q)^{-1}, L_rev the operator
 * with A_k -> -A_k (the upwind stabilisation of eq. RiemannFluxBoth is
 * symmetric and unchanged).  Stage inputs are recomputed from u_ckpt (once;
 * scratch as for dgw_adjoint_traces).
 * Adjoint sources between steps need either nsteps = 1 per call with
 * dgw_receivers_adjoint between calls, or dgw_adjoint_traces.
 * Elastic FP64 contexts only (DGW_ERR_UNSUPPORTED otherwise). */
dgw_status dgw_adjoint_step(dgw_ctx* ctx, double* lam_u, double* lam_res, double* grad_mat, const double* u_ckpt,
                            double t0, double dt, int nsteps, void* stream);

/* dgw_adjoint_step for a misfit of receiver traces: the adjoint of the nsteps
 * steps from the checkpoint u_ckpt (the state at t0), where before the
 * transpose of step k (k = nsteps-1 down to 0) lam_u += S^T g_traces[k], S the
 * receiver sampling of dgw_receivers_sample applied to the state after step k.
 * g_traces: device [nsteps][nrec][3], the misfit's derivative with respect to
 * the traces.  One call covers a whole checkpoint segment: the forward states
 * are recomputed once from u_ckpt, keeping every stage input and every
 * stage's operator output dt (K u + f) (before Q^{-1}), which the gradient
 * terms then read instead of applying the operator again: (3 + 10 nsteps)
 * state-sized device buffers of context scratch (released with the context).
 * If those do not fit, or the environment variable DGW_ADJOINT_LOW_MEMORY is
 * 1, only the stage inputs are kept ((3 + 5 nsteps) buffers) and the gradient
 * terms recompute the operator; DGW_ERR_OOM if even those do not fit (use
 * shorter segments).  Both adjoint calls share that scratch.
 * DGW_ERR_STATE without receivers; otherwise as dgw_adjoint_step. */
dgw_status dgw_adjoint_traces(dgw_ctx* ctx, double* lam_u, double* lam_res, double* grad_mat, const double* u_ckpt,
                              const double* g_traces, double t0, double dt, int nsteps, void* stream);

/* Receivers: velocity sampled at reference points xi[n][3] of elements[n]
 * (host arrays) with the element's Lagrange basis.  n = 0 removes them.
 * Elastic contexts only (DGW_ERR_UNSUPPORTED otherwise). */
dgw_status dgw_receivers_set(dgw_ctx* ctx, int n, const int64_t* elements, const double* xi);

/* out[n][3] (device) = velocity of u (device) at the receivers. */
dgw_status dgw_receivers_sample(dgw_ctx* ctx, const double* u, double* out, void* stream);

/* Transpose of dgw_receivers_sample: lam_u (device state) += S^T g, g device [n][3]. */
dgw_status dgw_receivers_adjoint(dgw_ctx* ctx, double* lam_u, const double* g, void* stream);

/* dt = cfl * h / (c_max * N^2) with h the smallest element edge length
 * (distance between adjacent element corner nodes) and c_max the largest
 * P-wave speed sqrt((lam + 2 mu) / rho); the CFL convention of the paper's
 * time-dependent transport experiments (Section 6.1).  The N^2 scaling
 * understates the stiffness of the elastic operator at low degree: with the
 * upwind flux and LSRK(5,4), a rough state (random nodal values, warped and
 * rotated elements, heterogeneous medium) grows without bound at CFL 0.5 for
 * N = 1 and 2; the stable limits measured there are about 0.125-0.15 (N = 1)
 * and 0.45-0.5 (N = 2), while N = 3 to 7 are stable at 0.5.  Set cfg.cfl
 * accordingly for N <= 2. */
dgw_status dgw_dt_cfl(dgw_ctx* ctx, double* dt_out);

/* ---- Batches: many solves advanced together (serving) -------------------
 * A batch advances solves of one degree N, precision and flux choice, each
 * owned by its own context (mesh, medium, point force), in lock step: every
 * launch of the batched stage kernel covers the elements of all of them (one
 * CTA per tile).  Not part of the paper (its runs are single solves); the
 * arithmetic per element is the one of dgw_stage. */
typedef struct dgw_batch dgw_batch;

/* Most solves in one batch (their descriptors are kernel parameters). */
#define DGW_BATCH_MAX_SOLVES 128

/* Create an empty batch for degree N, precision and flux_tau on `device`,
 * holding up to max_solves (1..DGW_BATCH_MAX_SOLVES) solves.  Records the
 * CUDA graph of two LSRK steps once. */
dgw_status dgw_batch_create(dgw_batch** out, int device, int N, int precision, int flux_tau, int max_solves);

/* Free the batch (not the contexts or buffers it referenced; NULL accepted). */
dgw_status dgw_batch_destroy(dgw_batch* b);

/* Make the batch advance n solves: ctxs[i] (same N, precision, flux, device;
 * mesh and material uploaded), u[i] and res[i] (distinct device buffers
 * [9][nel_i][Np], the state in and out and the LSRK register), step size
 * dt[i] and current time t0[i] (for the point force).  The context's second
 * state buffer serves as the stage ping-pong partner, so a context belongs to
 * at most one batch at a time.  Enqueues the upload of the times on `stream`
 * and rewrites the descriptors in the batch's graph: the new composition
 * applies to replays enqueued after this call (use the same stream for set
 * and run), replays already enqueued keep theirs; no synchronisation, no new
 * graph.  Call again whenever the set of solves changes, passing each
 * continuing solve's current time.  DGW_ERR_ARG beyond max_solves. */
dgw_status dgw_batch_set(dgw_batch* b, int n, dgw_ctx* const* ctxs, double* const* u, double* const* res,
                         const double* dt, const double* t0, void* stream);

/* Advance every solve of the batch by 2 * npairs LSRK steps (graph replays
 * enqueued on `stream`; asynchronous). */
dgw_status dgw_batch_run(dgw_batch* b, int npairs, void* stream);

/* Message of the last failing batch call (b may be NULL). */
const char* dgw_batch_last_error(const dgw_batch* b);

/* Discrete energy for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment convenience.  Some
 * callers cannot call cudaMalloc -- a host framework whose pool allocator
 * owns all device memory and caps it, a time loop that must not allocate once
 * it is running, code that only receives device pointers from another
 * library.  This entry point needs no context and allocates nothing: every
 * argument is the caller's device memory, and the reduction's scratch is a
 * fixed 512 KB array in the library's device module (held on every device
 * that loads the library until the process exits).
 *   N           degree 1..7; x, u at the nodes of dgw_reference_nodes(N)
 *   nel         1 .. DGW_ENERGY_STATIC_MAX_ELEMENTS (larger: DGW_ERR_ARG)
 *   x           device [nel][Np][3] node coordinates (J is computed from them)
 *   u           device [9][nel][Np] state
 *   rho,lam,mu  device [nel] medium (no validation of the values)
 *   energy_out  device pointer to one double; written when the work queued on
 *               `stream` (the current device's) completes.
 * Same value as dgw_energy on the same mesh to rounding.  The first call on
 * a device looks up the scratch array's device address; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: it assumes the device's primary context is not destroyed
 * (cudaDeviceReset) while the library is loaded.  All calls share the
 * scratch array: calls whose kernels overlap on the GPU (unordered streams)
 * race.  Every array must be device memory of the current device (or managed
 * memory); others are refused with DGW_ERR_ARG.  Errors:
 * dgw_last_error(NULL). */
#define DGW_ENERGY_STATIC_MAX_ELEMENTS (1 << 20)
dgw_status dgw_energy_static(int N, int64_t nel, const double* x, const double* u, const double* rho,
                             const double* lam, const double* mu, double* energy_out, void* stream);

/* ---- iHDG-II: the paper's locally implicit iteration ---------------------
 * The paper's iHDG-II algorithm (Section 3, Algorithm "The iHDG-II
 * approach"; eqs. iHDGlocal and iHDGtrace) for sigma u - L(u) = b with L the
 * upwind operator of the context (transport, shallow water, or the FP64
 * elastic operator without its point force): every element
 * solves its local problem with its own unknowns at iteration k+1 and its
 * neighbours' at k in the weighted trace,
 *     (sigma I - L_K^self) u_K^{k+1} = b_K + L_K^nbr(u^k),
 * L_K^self being L with the interior neighbour states zero.  Transport:
 * sigma = 0 is the steady equation (Section 4.1, forcing f); sigma = 1/dt
 * with b = u^m/dt + f is one implicit Euler step solved element by element
 * (Section 4.3, the locally implicit method).  Shallow water: sigma = 2/dt
 * with b = sigma u^m + L(u^m) (f = dgw_rhs of u^m) is one Crank-Nicolson
 * step (Section 6.2).  Elastic (FP64 contexts): sigma = 1/dt with
 * b = u^m/dt + f is one implicit Euler step, sigma = 2/dt with
 * b = sigma u^m + L(u^m) one Crank-Nicolson step, of du/dt = L(u) (L includes
 * Q^{-1}); a point force enters through f.  Degrees: transport N <= 4, shallow
 * water N <= 3, elastic N <= 3; the local block of m Np rows is inverted in
 * shared memory up to 125 rows and in global memory beyond. */

/* Build and invert sigma I - L_K^self for every element (device memory:
 * nel * (m Np)^2 doubles, about 1 MB per 8 elements for transport at N = 4).
 * sigma >= 0.  Elastic: nel * (9 Np)^2 doubles (2.65 MB per element at
 * N = 3); the local blocks are formed by applying the operator to unit vectors
 * in the elements of one colour of a greedy element colouring at a time.
 * DGW_ERR_UNSUPPORTED for mixed-precision contexts, beyond the degrees above,
 * and (elastic) for a mesh where an element is its own neighbour;
 * DGW_ERR_STATE before the mesh (elastic: before the material); DGW_ERR_ARG if
 * a local matrix is singular.  Synchronises `stream`. */
dgw_status dgw_ihdg_setup(dgw_ctx* ctx, double sigma, void* stream);

/* Iterate from the initial guess in u (device [m][nel][Np], overwritten with
 * the result) with b = sigma * u_prev + f (device [m][nel][Np] each; either may be
 * NULL for zero; neither may alias u) until ||u^k - u^{k-1}||_{L2} < tol (the
 * paper's eq. tolerancecriteriarelerror, L2 norm of the mass matrix) or
 * max_iter iterations.  *iterations receives the iterations done and
 * *last_change (may be NULL) the last ||u^k - u^{k-1}||.  Synchronises
 * `stream` once per iteration (the stopping test).  DGW_ERR_STATE before
 * dgw_ihdg_setup; DGW_ERR_UNSTABLE on a non-finite iterate. */
dgw_status dgw_ihdg_solve(dgw_ctx* ctx, const double* u_prev, const double* f, double* u, double tol, int max_iter,
                          int* iterations, double* last_change, void* stream);

/* ---- Checkpoint and resume ------------------------------------------------
 * The paper's runs are not restarted; these calls serve long solves and the
 * serving loop.  A checkpoint is a host byte buffer: an 80-byte header (magic,
 * ABI version, degree, fields, element count, step, time, a fingerprint of the
 * mesh and medium, an FNV-1a checksum of the payload), then u [m][nel][Np]
 * and, optionally, the Runge-Kutta register (FP64, the layout of the field
 * buffers).  Between steps the register is not needed (the first stage does
 * not read it); inside a step sequence driven by dgw_stage it is. */

/* Bytes of a checkpoint of this context's solve, with (with_res != 0) or
 * without the register.  DGW_ERR_STATE before the mesh. */
dgw_status dgw_state_bytes(dgw_ctx* ctx, int with_res, size_t* bytes);

/* Write a checkpoint of (u, res, t, step) into the host buffer buf (buf_bytes
 * at least dgw_state_bytes).  u, res: device or host field buffers; res NULL
 * leaves the register out.  Synchronises `stream`.  DGW_ERR_ARG for a short
 * buffer. */
dgw_status dgw_get_state(dgw_ctx* ctx, const double* u, const double* res, double t, int64_t step, void* buf,
                         size_t buf_bytes, void* stream);

/* Load a checkpoint written by dgw_get_state into u (and res, unless NULL)
 * and return its time and step (either pointer may be NULL).  The checkpoint
 * must come from a context on the same mesh and medium (same degree, system,
 * element count, connectivity, boundary tags, smallest edge, largest wave
 * speed and uploaded medium) with the same ABI, and its payload must match its checksum; otherwise
 * DGW_ERR_ARG and nothing is copied.  Synchronises `stream`. */
dgw_status dgw_set_state(dgw_ctx* ctx, const void* buf, size_t buf_bytes, double* u, double* res, double* t,
                         int64_t* step, void* stream);

/* ---- Debug build ----------------------------------------------------------
 * Built with -DDGW_DEBUG_CHECKS (paper_1711_01175_gb300.build.build(debug=True),
 * libdgw_debug.so; the Python binding loads it when the environment variable
 * DGW_DEBUG_CHECKS=1), the stage kernels of dgw_rhs, dgw_stage and dgw_step
 * check every state value they load (finite) and every neighbour index they
 * follow (inside the mesh), record the first failing element and count the
 * failures, and skip the read a bad index would make.  This call synchronises
 * the device, returns the first fault since the previous call (code 0: none,
 * 1: non-finite state, 2: neighbour index out of range; element: the element
 * being computed) and the number of failed checks, and clears them.  Release
 * builds return DGW_ERR_UNSUPPORTED.  Any pointer may be NULL. */
dgw_status dgw_debug_status(dgw_ctx* ctx, int* code, int64_t* element, int64_t* count);

/* Measurement helper; the paper has no counterpart.  The FP64 fused
 * multiply-add rate of CUDA device `device` in TFLOP/s (2 flops per DFMA):
 * eight independent DFMA chains per thread, 8 blocks of 256 threads per SM,
 * 4096 iterations, timed with CUDA events on the legacy stream (the best of
 * three launches after a warm-up).  It is the measured ceiling of the FP64
 * path, whose stage kernel is bound by the FP64 pipe.  Allocates and frees a
 * small device buffer and synchronises the device.  tflops: host double.
 * Errors: dgw_last_error(NULL). */
dgw_status dgw_probe_fp64_rate(int device, double* tflops);

/* Message of the last failing call on ctx (or of the last failing call
 * without a context when ctx is NULL).  Never NULL; owned by the library. */
const char* dgw_last_error(const dgw_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGW_H */
