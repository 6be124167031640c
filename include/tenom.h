/* tenom.h - C ABI of the GB300 (sm_103a) TENO-M library.
 *
 * Method: Li, Fu & Adams, "A low-dissipation shock-capturing framework with flexible
 * nonlinear dissipation control" (arXiv 2010.13289).  The library advances the
 * compressible Euler equations of an ideal gas on a uniform Cartesian grid
 * (Section 2, Eqs. conservationlaw-approximateEq, extended dimension by dimension as in
 * Section 4) with the conservative finite-difference form
 *     dU_i/dt = - sum_a (Fhat_{a,i+1/2} - Fhat_{a,i-1/2}) / dx_a ,
 * where every face flux Fhat is built by Roe-averaged characteristic decomposition,
 * local Lax-Friedrichs (Rusanov) splitting (Section 4), and, per characteristic field and
 * split side, the TENO-M reconstruction (Sections 2-3: Table 1 candidates, Eqs.
 * measureTENO/taukTENO indicators, Eqs. normalize/cut-off, Eq. mp_flux filtering of the
 * nonsmooth candidates by the MP or TVD5 limiter, Eq. reconstuction with w_k = d_k).
 * Time integration is the third-order SSP Runge-Kutta method (Section 4, CFL 0.4).
 *
 * Conventions for every entry point
 *   - All floating point is IEEE binary64 (double).
 *   - Grid arrays are caller-owned DEVICE pointers (any allocator, e.g. PyTorch), laid out
 *     structure-of-arrays [nvar][nz][ny][nx], x fastest, contiguous, 8-byte aligned, no
 *     ghost cells (boundary conditions are applied inside the library).  nvar = dim + 2:
 *     (rho, rho*u_1 .. rho*u_dim, E).  Unused trailing extents must be 1.
 *   - Face arrays of axis a have n_a + 1 entries along a (face f lies between cells f-1
 *     and f); same ordering otherwise.
 *   - Calls are asynchronous and ordered on the context's CUDA stream, unless stated.
 *   - Every call returns tenom_status; nothing aborts or throws across the ABI.  A CUDA
 *     error is returned as TENOM_E_CUDA; tenom_last_error(ctx) gives the text.
 *   - Non-physical states met by a kernel (rho <= 0, p <= 0, Roe c^2 <= 0, non-finite
 *     indicator) set bits in a sticky device status word; tenom_status_word() reads it.
 *   - A context may be used by one host thread at a time.
 */
#ifndef TENOM_H
#define TENOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TENOM_OK = 0,
  TENOM_E_INVALID = 1,      /* bad argument (null/misaligned pointer, bad size or option) */
  TENOM_E_CUDA = 2,         /* a CUDA runtime call failed */
  TENOM_E_NONPHYSICAL = 3,  /* device status word has a non-physical bit set */
  TENOM_E_TIMEOUT = 4,      /* a bounded device wait gave up */
  TENOM_E_UNSUPPORTED = 5   /* option combination not built */
} tenom_status;

enum { TENOM_BC_PERIODIC = 0, TENOM_BC_TRANSMISSIVE = 1 };     /* ghost fill: wrap / zero-gradient copy */
enum { TENOM_LIM_MP = 0, TENOM_LIM_TVD5 = 1, TENOM_LIM_VA = 2 };  /* Section 3.2 limiters */
enum { TENOM_CT_CONST = 0, TENOM_CT_ADAPTIVE = 1 };            /* C_T fixed, or TENO8A (Section 2.4) */
enum { TENOM_CURV_M4 = 0, TENOM_CURV_MM = 1 };                 /* MP curvature d_{i+1/2} (Section 3.2.2 / 4) */
enum { TENOM_W_TENOM = 0, TENOM_W_TENO = 1 };                  /* w_k = d_k (Sec. 3.3) / renormalised (Eq. weight_renormalize) */

/* Device status word bits */
enum { TENOM_ST_RHO = 1, TENOM_ST_P = 2, TENOM_ST_ROE = 4, TENOM_ST_NONFINITE = 8 };

/* Uniform Cartesian grid of the Euler initial-value problem (Section 2, Section 4). */
typedef struct tenom_grid {
  int dim;         /* 1, 2 or 3 */
  int n[3];        /* cells per axis (x, y, z); unused axes = 1 */
  double dx[3];    /* spacing per axis; unused axes ignored */
  int bc[3];       /* TENOM_BC_* per axis */
  double gamma;    /* ratio of specific heats */
} tenom_grid;

/* Reconstruction scheme.  Defaults (tenom_scheme_default): K = 6, MP, C_T = 1e-5 constant
 * (K = 8: adaptive C_T of TENO8A), mp_alpha = 1.25 (Eq. upper_limiter), mp_beta = 4
 * (Eq. large_curvature), M4 curvature (Eq. maximal_curvature), w_k = d_k with the
 * maximal-order d_k (Section 3.3 leaves the choice open). */
typedef struct tenom_scheme {
  int K;            /* 6 or 8 (Eq. rdistribution: candidates S_0..S_{K-3}) */
  int limiter;      /* TENOM_LIM_*: MP and TVD5 everywhere; VA (Van Albada, kappa = 1/3) for the
                       forward calls only -- the adjoint calls return TENOM_E_UNSUPPORTED and
                       tenom_batch_create rejects it */
  int ct_mode;      /* TENOM_CT_* */
  double ct_const;  /* C_T when ct_mode == TENOM_CT_CONST */
  double mp_alpha;
  double mp_beta;
  int mp_curv;      /* TENOM_CURV_* */
  int weights;      /* TENOM_W_* */
  double d[6];      /* optimal weights d_0..d_{K-3}; all zero = maximal-order default */
  int decisions;    /* TENOM_DECIDE_FILTERED (default): cutoff decisions certified in FP32 and
                       decided in FP64 where the FP32 bounds do not settle them (same outcome
                       as FP64); TENOM_DECIDE_FP64: FP64 only */
  int positivity;   /* TENOM_PP_OFF (default) or TENOM_PP_ON: the positivity-preserving flux
                       limiter that Section 4.4 applies (Hu, Adams & Shu 2013).  It belongs to a
                       forward-Euler stage of length dt, so it acts in the stepping calls
                       (tenom_rk3_step, tenom_advance, tenom_advance_host and the batched
                       steps: in every SSP-RK3 stage, with that step's dt); tenom_rhs,
                       tenom_rhs_noalloc and tenom_face_dump return the unlimited operator;
                       the adjoint calls return TENOM_E_UNSUPPORTED.  Per face of axis
                       a the high-order flux F^H is pulled towards the local Lax-Friedrichs flux
                       F^LF = (F(U_L) + F(U_R) - alpha (U_R - U_L))/2, alpha = max(|u_a| + c) of
                       the two cells: F = F^LF + theta (F^H - F^LF), theta in [0, 1] the product
                       of a density factor and a pressure factor chosen so that both one-sided
                       states U_L - mu F and U_R + mu F (mu = 2 dim dt/dx_a) keep density and
                       pressure >= min(1e-13, their value with F^LF); theta = 1 leaves F^H
                       untouched. */
} tenom_scheme;

enum { TENOM_PP_OFF = 0, TENOM_PP_ON = 1 };

enum { TENOM_DECIDE_FILTERED = 0, TENOM_DECIDE_FP64 = 1 };

typedef struct tenom_ctx tenom_ctx;

/* Fill *s with the defaults for K (6 or 8).  Host only. */
tenom_status tenom_scheme_default(tenom_scheme* s, int K);

/* Create a context for one grid and scheme.  stream: a cudaStream_t (NULL = legacy
 * default stream) on which every call of this context is ordered.  Allocates the
 * context's device workspace (stage buffer, face buffers, scalars) on the current device:
 * about (nvar * ncell * (1 + dim) + small) * 8 bytes.  On success *ctx owns it. */
tenom_status tenom_create(tenom_ctx** ctx, const tenom_grid* grid, const tenom_scheme* scheme, void* stream);

/* Free the context and its workspace (synchronises its stream first).  NULL is a no-op. */
tenom_status tenom_destroy(tenom_ctx* ctx);

/* Conserved state from primitives (rho, u_1..u_dim, p): U = (rho, rho u, p/(gamma-1) + rho|u|^2/2).
 * prim and U: device [nvar][ncell].  prim may not alias U. */
tenom_status tenom_init_state(tenom_ctx* ctx, const double* prim, double* U);

/* Semi-discrete operator dUdt = L(U) = - sum_a (Fhat_{a,i+1/2} - Fhat_{a,i-1/2})/dx_a
 * (Eq. approximateEq).  U, dUdt: device [nvar][ncell]; dUdt may not alias U. */
tenom_status tenom_rhs(tenom_ctx* ctx, const double* U, double* dUdt);

/* Stable step dt = cfl / max_i sum_a (|u_a| + c)_i / dx_a (Section 4), written to the
 * device double *dt_dev (no host synchronisation). */
tenom_status tenom_max_dt(tenom_ctx* ctx, const double* U, double cfl, double* dt_dev);

/* One SSP-RK3 step in place (Section 4): U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 * U <- 1/3 U + 2/3 (U2 + dt L(U2)).  dt read from the device double *dt_dev. */
tenom_status tenom_rk3_step(tenom_ctx* ctx, double* U, const double* dt_dev);

/* nsteps SSP-RK3 steps with dt = min(cfl/max signal speed, t_end - t) recomputed on the
 * device before each step; t is a device double advanced in place (steps after t reaches
 * t_end do nothing).  Pass t_end = +inf for unclipped steps. */
tenom_status tenom_advance(tenom_ctx* ctx, double* U, double* t_dev, double t_end, double cfl, int nsteps);

/* Host-buffer convenience: copy U_host (pinned or pageable, [nvar][ncell]) to the device,
 * run tenom_advance from t = *t_host, copy the state and t back, synchronise. */
tenom_status tenom_advance_host(tenom_ctx* ctx, const double* U_host_in, double* U_host_out, double* t_host,
                                double t_end, double cfl, int nsteps);

/* The positivity-preserving flux limiter of one forward-Euler stage of length *dt_dev
 * (Section 4.4; see tenom_scheme.positivity) applied in place to face fluxes Fhat of axis
 * `axis` (device [nvar][nface_a], layout of tenom_face_dump) at the state U (device
 * [nvar][ncell]).  The stepping calls apply the same kernel to their own fluxes when the
 * scheme asks for it; this call applies it whatever the scheme's flag, to fluxes the caller
 * supplies.  A face whose blend factors are both 1 is left bit for bit.  dt_dev <= 0 leaves
 * Fhat unchanged.  Returns TENOM_E_INVALID for a bad axis or pointer. */
tenom_status tenom_positivity_limit(tenom_ctx* ctx, const double* U, int axis, const double* dt_dev, double* Fhat);

/* Diagnostic face dump of axis a for parity checks: the same kernel as the solver writes
 * Fhat (device [nvar][nface_a]) and per face, field s and split side (0: f+, 1: f-) one
 * byte flags (device [nface_a][nvar][2]): bits 0..K-3 = delta_k of Eq. cut-off, bits 6-7 =
 * [beta] - 7 of Eq. cut-off_adjust when C_T is adaptive.  flags may be NULL. */
tenom_status tenom_face_dump(tenom_ctx* ctx, const double* U, int axis, double* Fhat, uint8_t* flags);

/* Decision statistics of the reconstruction at the state U (device [nvar][ncell]) on the
 * faces of axis `axis`, for logging (not part of a step): the face kernel's characteristic
 * sequences (f+ and f- of every field, Section 4) are examined instead of reconstructed,
 * and TENOM_NSTATS counters are ADDED to the caller-owned device array counters_dev (64-bit;
 * the caller zeroes it).  Per split side: [0] sides; [1] sides the certified FP32 cutoff
 * filter decided, [2] of which its decisions differ from the FP64 ones (rounding-decided);
 * [3] sides with every candidate smooth; [4 + k], k = 0..K-3: candidates k judged nonsmooth
 * (delta_k = 0, Eq. cut-off); [10] sides where the limiter runs (any nonsmooth candidate,
 * Eq. mp_flux); [11] nonsmooth candidates whose value the limiter changed; [12] decisions
 * within 1e-10 relative of the cutoff (|chi_k - C_T| <= 1e-10 C_T), [13] sides with one;
 * [14 + j]: adaptive exponent [beta] = 7 + j of TENO8A (Eq. cut-off_adjust), [18] sides
 * with beta within 1e-10 of an integer; [19] sides with a non-finite sum of gamma.
 * Stream-ordered.  Returns TENOM_E_INVALID for a bad axis or pointer. */
#define TENOM_NSTATS 20
tenom_status tenom_decision_stats(tenom_ctx* ctx, const double* U, int axis, unsigned long long* counters_dev);

/* ---------------------------------------------------------------- batched 1D problems
 * Many independent 1D Euler problems of uneven size advanced together (each problem as in
 * tenom_advance, on its own grid, time and CFL step).  State: one caller-owned device array
 * U[3][total] where problem j owns cells [off_j, off_j + n_j) (tenom_batch_layout).  Each RK
 * stage is one persistent kernel over a work list of (problem, face tile) items; a step is
 * captured once into a CUDA graph and replayed.  Problems whose time reached their t_end
 * are masked (their state is left untouched). */
typedef struct tenom_batch tenom_batch;

/* n[j], dx[j] (host arrays of nprob); bc[j] per problem (host, NULL = all transmissive);
 * scheme as for tenom_create (K = 6 or 8; MP or TVD5).  t_j = 0, t_end_j = +inf. */
tenom_status tenom_batch_create(tenom_batch** b, int nprob, const int* n, const double* dx, const int* bc,
                                double gamma, const tenom_scheme* scheme, void* stream);
tenom_status tenom_batch_destroy(tenom_batch* b);
/* off_host[nprob + 1] cell offsets and the total cell count. */
tenom_status tenom_batch_layout(const tenom_batch* b, long long* off_host, long long* total);
/* U = conserved state of prim (rho, u, p), both [3][total] device arrays. */
tenom_status tenom_batch_init_state(tenom_batch* b, const double* prim, double* U);
/* Set t_j and/or t_end_j from host arrays (NULL leaves them); synchronises. */
tenom_status tenom_batch_set_time(tenom_batch* b, const double* t_host, const double* t_end_host);
tenom_status tenom_batch_get_time(tenom_batch* b, double* t_host);
tenom_status tenom_batch_status_word(tenom_batch* b, int* status_host, int reset);
/* nsteps SSP-RK3 steps of every unfinished problem: per problem dt_j = min(cfl / max signal
 * speed_j, t_end_j - t_j); replays a CUDA graph of one step (rebuilt when U or cfl change). */
tenom_status tenom_batch_step(tenom_batch* b, double* U, double cfl, int nsteps);
/* The same step sequence launched directly on the stream (no graph). */
tenom_status tenom_batch_step_direct(tenom_batch* b, double* U, double cfl, int nsteps);
/* One persistent stage launch (1, 2, 3) with the current per-problem dt: stage 1 reads U and
 * writes the stage buffer, stage 3 writes U.  For drivers that sequence stages themselves. */
tenom_status tenom_batch_stage(tenom_batch* b, int stage, double* U);
/* Time the stage kernel for tiles of 64/128/256 faces and 1/2/4/8 resident CTAs per SM on
 * this batch and keep the fastest (writes the choice if the pointers are non-NULL). */
tenom_status tenom_batch_autotune(tenom_batch* b, double* U, int* tile, int* ctas_per_sm);
tenom_status tenom_batch_set_tiling(tenom_batch* b, int tile, int ctas_per_sm);

/* Size of the static device scratch of tenom_rhs_noalloc: 16 MiB, held on every GPU that
 * loads this library until the process exits. */
#define TENOM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* tenom_rhs without a context and without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate device memory
 * once they are running -- code living inside another framework's memory pool or
 * allocator hook, or a latency-critical loop that cannot accept the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It computes dUdt = L(U) for the given grid and
 * scheme, on `stream` (a cudaStream_t; NULL = legacy default stream), with the face-sweep
 * and flux-difference kernels of tenom_rhs.  One difference: tenom_rhs first computes the
 * cells' primitives (velocity, p, H, c, sqrt rho) once per cell into its context's
 * buffer, while this call has no such buffer and the face kernels form them for each
 * staged point of their tile; the two round alike except in the last bits, which can
 * flip a cutoff decision that rounding sets (a flat sequence at a zero-gradient boundary);
 * agreement to 1e-13 of each component's largest value is tested.  U and dUdt are caller-owned device arrays as for tenom_rhs; status_dev
 * is an optional caller-owned device int that receives TENOM_ST_* bits (ORed in, the
 * caller clears it); with NULL the bits go to a word inside the scratch and are not
 * reported.
 * Scratch: the face fluxes of every axis live in one file-scope static device array of
 * TENOM_NOALLOC_SCRATCH_BYTES; a grid needing more -- (dim+2) * sum_a nface_a * 8 bytes
 * plus 256 -- is rejected with TENOM_E_INVALID and a message on stderr (for 2D that is
 * about 260,000 cells).  The array's device address is looked up the first time the
 * entry point runs on a device (cudaGetSymbolAddress, with that device current); make
 * that first call before any stream capture.  Every call, on every stream and host
 * thread, shares the one array and it keeps the last call's contents, so calls whose
 * kernels overlap on the GPU race: order them on one stream or synchronise between them.
 * Returns TENOM_E_CUDA if a launch fails. */
tenom_status tenom_rhs_noalloc(const tenom_grid* grid, const tenom_scheme* scheme, const double* U, double* dUdt,
                               int* status_dev, void* stream);

/* ---------------------------------------------------------------- frozen-branch adjoint
 * Reverse-mode derivative of the solver with every branch fixed at the forward pass: the
 * cutoff flags delta_k (Eq. cut-off), the limiter selections (MP median / bounds, TVD5 slope),
 * the argmax of the LLF alpha and dt.  Because TENO-M assembles with constant weights
 * w_k = d_k (Section 3.3), no derivative flows through beta, tau, gamma or chi.  All arrays
 * are device [nvar][ncell] unless stated. */

/* Bytes of cutoff flags one stage records (all axes): sum_a nface_a * nvar * 2. */
size_t tenom_flags_bytes(const tenom_ctx* ctx);

/* Ubar = L'(U)^T w (vector-Jacobian product of tenom_rhs at U; flags decided at U). */
tenom_status tenom_rhs_vjp(tenom_ctx* ctx, const double* U, const double* w, double* Ubar);

/* tenom_rk3_step that also records the tape of the step: tape_states = [U1, U2] (2 * nvar *
 * ncell doubles) and tape_flags (3 * tenom_flags_bytes bytes), for tenom_rk3_step_adjoint_tape. */
tenom_status tenom_rk3_step_record(tenom_ctx* ctx, double* U, const double* dt_dev, double* tape_states,
                                   uint8_t* tape_flags);

/* Ubar_n = (dU^{n+1}/dU^n)^T Ubar_np1 for the step recorded from U_n (dt frozen).  Ubar_n
 * and Ubar_np1 must be distinct arrays. */
tenom_status tenom_rk3_step_adjoint_tape(tenom_ctx* ctx, const double* U_n, const double* tape_states,
                                         const uint8_t* tape_flags, const double* dt_dev, const double* Ubar_np1,
                                         double* Ubar_n);

/* ---- linearisation tape (faster reverse, larger tape) ----
 * The flags tape above makes every adjoint sweep rebuild the frozen linear reconstructions
 * (projection, limiter selections) from the stage state.  The linearisation tape stores
 * them instead: per face and characteristic field s (Section 4 projection, Eq. mp_flux
 * filtering, Eq. reconstuction assembly with w_k = d_k), with the frozen linear weights
 * op (f+) and om (f-, on the mirrored stencil), W_q = l_s . U_q, G_q = l_s . F_q,
 *   fs = f+ + f- = sum_q sigma_q G_q + (alpha_s / 2) delta_q W_q,
 *   sigma_q = (op_q + om_{K-1-q}) / 2,  delta_q = op_q - om_{K-1-q},
 * the record is (fs, omegaW = sum_q delta_q W_q, sigma_0..K-1, delta_0..K-1): 2K + 2 doubles.
 * Layout of one stage: axis after axis; inside axis a, [nvar][2K+2][nface_a] doubles
 * (face order as the face buffers of tenom_face_dump). */

/* Bytes one stage records: sum_a nface_a * nvar * (2K + 2) * 8. */
size_t tenom_lin_tape_bytes(const tenom_ctx* ctx);

/* dUdt = L(U) as tenom_rhs, also writing the linearisation of L at U to `lin`
 * (tenom_lin_tape_bytes bytes, caller-owned device memory, 8-byte aligned). */
tenom_status tenom_rhs_record(tenom_ctx* ctx, const double* U, double* dUdt, double* lin);

/* Ubar = L'(U)^T w from the linearisation tenom_rhs_record wrote at the same U. */
tenom_status tenom_rhs_vjp_lin(tenom_ctx* ctx, const double* U, const double* lin, const double* w, double* Ubar);

/* tenom_rk3_step recording tape_states = [U1, U2] (as tenom_rk3_step_record) and the
 * linearisation of its three stages, tape_lin (3 * tenom_lin_tape_bytes bytes). */
tenom_status tenom_rk3_step_record_lin(tenom_ctx* ctx, double* U, const double* dt_dev, double* tape_states,
                                       double* tape_lin);

/* As tenom_rk3_step_adjoint_tape, from a step recorded by tenom_rk3_step_record_lin. */
tenom_status tenom_rk3_step_adjoint_lin(tenom_ctx* ctx, const double* U_n, const double* tape_states,
                                        const double* tape_lin, const double* dt_dev, const double* Ubar_np1,
                                        double* Ubar_n);

/* tenom_rk3_step_adjoint_tape without a caller tape: records the step (flags) from U_n
 * internally first. */
tenom_status tenom_rk3_step_adjoint(tenom_ctx* ctx, const double* U_n, const double* dt_dev, const double* Ubar_np1,
                                    double* Ubar_n);

/* Sticky device status word (TENOM_ST_* bits); synchronises the stream.  reset != 0 clears it. */
tenom_status tenom_status_word(tenom_ctx* ctx, int* status_host, int reset);

/* Text of the last error of this context ("" if none).  Valid until the next call. */
const char* tenom_last_error(const tenom_ctx* ctx);

/* Measurement helper (not part of the method): average duration in ms of the face kernel
 * of axis a over the last tenom_rk3_step/tenom_advance calls, timed with CUDA events on
 * the context stream when timing is enabled.  enable != 0 turns timing on and resets. */
tenom_status tenom_kernel_timing(tenom_ctx* ctx, int enable, double* face_ms_per_launch, long long* launches);

/* FP64 pipe throughput probe (not part of the method): runs `iters` dependent-chain DFMA
 * iterations per thread on a grid of nblocks x 256 threads and writes the achieved
 * FLOP/s (2 per DFMA) to *flops.  Synchronises the stream. */
tenom_status tenom_fp64_peak(void* stream, int nblocks, int iters, double* flops);

/* Numerical self-check (not part of the method): for each x[i] (positive, normal) writes
 * out[6i..6i+5] = (two-step Newton-Raphson 1/x used by the kernels, CUDA's 1.0/x,
 * x * Newton 1/sqrt(x) used by the kernels, CUDA's sqrt(x), one-step Newton 1/x used where
 * only a comparison follows, the kernels' integer-pipe FP32 truncation of x (of -x for odd
 * i), widened back to double).  Device arrays; async. */
tenom_status tenom_check_fastmath(const double* x, double* out, long long n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TENOM_H */
