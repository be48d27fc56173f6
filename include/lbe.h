/*
 * lbe.h -- C ABI of the GB300 (sm_103a) CSF lattice Boltzmann library for
 * thermocapillary flow (Zheng, Zheng & Zhai, arXiv:1412.6238).
 *
 * One call of lbe_step advances, for every cell, the three coupled D2Q9
 * lattices of the paper by one time step:
 *   - the Cahn-Hilliard LBE for the order parameter c (Sec. II, Eq. 27 with
 *     the equilibrium of Eq. 21-22, c = sum g_i by Eq. 28),
 *   - the flow LBE forced by the continuous surface force (Sec. II, Eq. 12
 *     with Eq. 5, Eq. 6 and the moments of Eq. 13), the force being
 *     F = eps*alpha*|grad c|^2 (-sigma kappa n + grad_s sigma) + rho a
 *     (Eq. 3) with sigma(T) linear in T (Eq. aEq3),
 *   - the thermal LBE for T (Sec. III, Eq. aEq12 with h_eq of Eq. aEq9,
 *     T from Eq. aEq13, conductivity lambda = rho c_v c_s^2 tau_h, Eq. aEq14).
 * Problem statement (Sec. IV): periodic in x, no-slip walls with imposed
 * temperatures at the bottom and top; lattice units dx = dt = 1.
 *
 * Conventions
 *   - Cells x = 0..nx-1, y = 0..ny-1; arrays are [ny][nx], x fastest, y = 0 is
 *     the bottom row.  The walls lie half a cell outside the first and last
 *     rows (halfway bounce-back for f and g, anti-bounce-back for hbar; the
 *     paper names the boundary conditions but gives no scheme).
 *   - Phase c = 0 has viscosity eta1 and conductivity lam1, phase c = 1 has
 *     eta2 and lam2; both vary linearly in c in between.
 *   - sigma(T) = sigma0 - sigmaT (T - Tref); sigmaT here is MINUS the paper's
 *     d sigma / d T, so it is positive for the usual fluids.
 *   - Population state arrays are [27][ny][nx] doubles, planes f_0..f_8,
 *     g_0..g_8, hbar_0..hbar_8, velocity order 0 (0,0), 1 (1,0), 2 (0,1),
 *     3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1); they hold
 *     the pre-collision (post-streaming) populations of the current step.
 *
 * Ownership and errors
 *   - The library owns every device buffer it allocates.  Inputs are copied
 *     during the call; output buffers belong to the caller.
 *   - Every call returns an lbe_status; on failure lbe_last_error() gives a
 *     message.  A handle that returned LBE_ECUDA or LBE_ENAN stays usable
 *     only through lbe_set_state / lbe_load / lbe_destroy.
 *   - All work is ordered on one CUDA stream per handle (the caller's, or a
 *     private non-blocking stream when NULL is passed).  Waits on the host are
 *     bounded (LBE_TIMEOUT_MS environment variable, default 600000 ms) and
 *     return LBE_ETIMEOUT rather than blocking forever; the work stays
 *     enqueued and a later wait may still succeed.
 *   - The strip kernel's waits for its shared-memory copies are bounded too
 *     (2^22 polls).  A wait that runs out sets a device error word; the CTA
 *     issues no further copy, drains (bounded) the copies it has in flight
 *     and returns.  Every later call that waits (lbe_step with check_every,
 *     lbe_synchronize, lbe_fields, lbe_sums, lbe_get_state, lbe_save, the
 *     adjoint calls) then returns LBE_ECUDA, and the handle refuses to step
 *     until lbe_set_state or lbe_load gives it a new state (which clears the
 *     word).
 *   - Fault injection on the host, for tests (LBE_FAULT environment variable,
 *     read by lbe_init / lbe_init_batch): "alloc" makes the call fail as an
 *     out-of-memory would, before any device work; "withhold:<row>" makes the
 *     first strip-kernel step of the handle stage nothing for row <row> (its
 *     slot's barrier still expects the bytes) and give up a copy wait after
 *     2^12 polls, so that the path above runs without any GPU fault.
 */
#ifndef LBE_H
#define LBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBE_ABI_VERSION 2

typedef struct lbe_handle lbe_handle;

typedef enum {
  LBE_OK = 0,
  LBE_EINVAL = -1,   /* bad argument or parameter set (message says which) */
  LBE_ENOMEM = -2,   /* device or host allocation failed */
  LBE_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  LBE_ENAN = -4,     /* the periodic check found a NaN/Inf in the fields */
  LBE_ETIMEOUT = -5, /* a bounded host wait ran out */
  LBE_ESTATE = -6    /* call not valid in the handle's current state */
} lbe_status;

/* Population storage.  Arithmetic is FP64 for LBE_F64 and FP32 otherwise.
 * The deviation forms store f_i, g_i (i > 0) and hbar_i - w_i rho c_v T_r(y)
 * (T_r the linear conduction profile between the wall means) scaled by a
 * power of two in 16 bits; g_0 (which carries c) stays FP32.  LBE_F16MIX
 * keeps f (which carries the momentum, hence u) in FP32 and stores g_i
 * (i > 0) and the hbar deviations in FP16, the three populations of a
 * direction in one 8-byte word.  The FP32 and 16-bit forms also keep the low
 * part of g_0 (FP16), so that c = sum g_i is carried to about 1e-11. */
typedef enum {
  LBE_F64 = 0,     /* 216 B per cell per buffer (parity mode)              */
  LBE_F32 = 1,     /* 110 B per cell per buffer (27 fp32 + fp16 low part)  */
  LBE_F16DEV = 2,  /* 58 B per cell per buffer (26 fp16 + 1 fp32 + 1 fp16) */
  LBE_BF16DEV = 3, /* 58 B per cell per buffer (26 bf16 + 1 fp32 + 1 fp16) */
  LBE_F16MIX = 4   /* 76 B per cell per buffer (10 fp32 + 18 fp16)         */
} lbe_storage;

/* Parameters of one instance, lattice units.  Validity (LBE_EINVAL
 * otherwise): nx >= 1, ny >= 2, rho > 0, rho2 >= 0, cv > 0, eta1,
 * eta2 > 0, lam1, lam2 >= 0 (> 0 with interp = 1), eps > 0,
 * tau_g > 1/2, mobility >= 0, eta_n > 0, interp and wall_mid 0 or 1,
 * -1 <= cos_wet <= 1, dissip 0 or 1 (1 with FP64 or FP32 storage), reserved 0,
 * and 0 < omega < 2 for every relaxation rate at c = 0 and c = 1.  Layout
 * change from ABI version 1: rho2, interp, wall_mid, cos_wet, dissip and
 * reserved appended. */
typedef struct {
  int32_t nx, ny;       /* cells; periodic in x, walls in y           */
  int32_t storage;      /* lbe_storage; must be equal for all instances */
  int32_t check_every;  /* FP64 sums + NaN scan every k steps of lbe_step
                           (then lbe_step waits for the stream); 0 = off */
  double rho, cv;       /* density of phase c = 0, specific heat       */
  double eta1, eta2;    /* dynamic viscosity of phase c=0, c=1         */
  double lam1, lam2;    /* conductivity of phase c=0, c=1              */
  double sigma0, sigmaT, Tref; /* sigma = sigma0 - sigmaT (T - Tref)   */
  double eps, beta;     /* interface parameter and free-energy coefficient,
                           E_0 = beta c^2 (c-1)^2 (Sec. II)            */
  double tau_g;         /* CH relaxation time; omega_g = 1/tau_g        */
  double mobility;      /* M = Gamma (tau_g - 1/2) (Eq. 16)            */
  double ax, ay;        /* body acceleration (force rho a)             */
  double eta_n;         /* n = grad c / sqrt(|grad c|^2 + eta_n^2)      */
  double rho2;          /* density of phase c = 1; 0 (or rho): uniform.
                           A density varying with c, rho(c) = rho + c
                           (rho2 - rho), brings in the grad(rho c_s^2)
                           source of Eq. 12, the pressure correction
                           (dt/2) u.grad(rho c_s^2) of Eq. 13 and
                           grad(rho c_s^2) in the thermal force of Eq. aEq4;
                           it needs FP64 storage (LBE_EINVAL otherwise) and
                           is not covered by lbe_adjoint                  */
  /* Boundary and property variants the paper leaves open (0: off; none is
     covered by lbe_adjoint, which then returns LBE_EINVAL):              */
  int32_t interp;       /* eta(c), lambda(c): 0 linear, 1 harmonic
                           1/((1-c)/a + c/b)                              */
  int32_t wall_mid;     /* 1: the anti-bounce-back of hbar on a diagonal
                           link takes the wall temperature where the link
                           crosses the wall, (T_w(x) + T_w(x -+ 1))/2     */
  double cos_wet;       /* cos of the contact angle of phase 1 at both
                           walls (0: neutral, mirror ghost rows of c).  The
                           ghost rows of c gain the flux (sqrt(2 beta)/eps)
                           cos(theta) c (1 - c) of a cubic wall energy
                           (Young's law)                                  */
  int32_t dissip;       /* 1: keep the pressure-work / viscous-dissipation
                           term -fbar_i q_i of Eq. aEq7 that Eq. aEq8 drops
                           (fbar from the f lattice, q_i = (xi_i - u).
                           (xi_i.grad) u; the velocity gradients from a
                           pass of their own before each step); FP64 or
                           FP32 storage, on the tile kernel               */
  int32_t reserved;     /* 0 */
} lbe_params;

/* Initial and boundary data of one instance (host pointers, copied). */
typedef struct {
  const double* c0;   /* [ny][nx] initial order parameter            */
  const double* T0;   /* [ny][nx] initial temperature                */
  const double* Tbot; /* [nx] wall temperature at y = -1/2            */
  const double* Ttop; /* [nx] wall temperature at y = ny - 1/2        */
} lbe_init_fields;

/* Field mask bits for lbe_fields. */
#define LBE_FIELD_C 1u
#define LBE_FIELD_P 2u
#define LBE_FIELD_UX 4u
#define LBE_FIELD_UY 8u
#define LBE_FIELD_T 16u

int32_t lbe_abi_version(void);

/* Create a handle holding one instance and set its state to the
 * equilibrium of Sec. II/III at rest: u = 0, p = 0, c = c0, T = T0
 * (f_i = 0, g_i = g_eq(c0, mu(c0), 0) with mu from the discrete Laplacian,
 * hbar_i = w_i rho c_v T0).  stream: a cudaStream_t or NULL. */
lbe_status lbe_init(const lbe_params* params, const lbe_init_fields* init,
                    void* stream, lbe_handle** out);

/* Same for n independent instances (params[n], init[n]) of possibly
 * different sizes and parameters, advanced together by one persistent
 * kernel launch per step. */
lbe_status lbe_init_batch(int32_t n, const lbe_params* params,
                          const lbe_init_fields* init, void* stream,
                          lbe_handle** out);

/* Enqueue nsteps time steps of every instance on the handle's stream
 * (replayed from a captured CUDA graph).  Returns after enqueueing when
 * check_every == 0; otherwise runs the FP64 NaN/Inf scan every check_every
 * steps, waits for the stream and returns LBE_ENAN if any was found. */
lbe_status lbe_step(lbe_handle* h, int64_t nsteps);

/* Bounded wait until all work on the handle's stream is done. */
lbe_status lbe_synchronize(lbe_handle* h);

/* Macroscopic fields of one instance at the current step: c = sum g_i
 * (Eq. 28), p = sum f_i (Eq. 13), u = sum xi_i f_i/(rho c_s^2) + F/(2 rho)
 * (Eq. 13 with the c_s^2 of the Eq. 12 source), T = sum hbar_i / (rho c_v)
 * (Eq. aEq13).  dst[0..4] receive c, p, ux, uy, T for the bits set in mask
 * (entries for unset bits are ignored), each [ny][nx] contiguous, on the
 * device (on_device = 1) or in host memory (0), as double (dtype 0) or
 * float (dtype 1).  Waits for completion. */
lbe_status lbe_fields(lbe_handle* h, int32_t instance, uint32_t mask,
                      void* const dst[5], int32_t on_device, int32_t dtype);

/* FP64 diagnostics of one instance: out[0] = sum c, out[1] = sum p,
 * out[2] = sum_i,x hbar_i, out[3] = ||u^n - u^(n-1)||_2 / ||u^n||_2 (the
 * per-step velocity residual, 0 before the first step), out[4] = number of
 * non-finite values among c, p, ux, uy, T.  Deterministic.  Waits. */
lbe_status lbe_sums(lbe_handle* h, int32_t instance, double out[5]);

/* Copy the pre-collision population state of one instance to / from a
 * [27][ny][nx] double array (device memory if on_device, else host).
 * Setting a state converts it to the handle's storage and clears a
 * LBE_ENAN / LBE_ECUDA condition.  Both wait for completion. */
lbe_status lbe_get_state(lbe_handle* h, int32_t instance, double* pops,
                         int32_t on_device);
lbe_status lbe_set_state(lbe_handle* h, int32_t instance, const double* pops,
                         int32_t on_device);

/* Checkpoint: write every instance's parameters, walls, step count and
 * state to a file / restore them into a handle of the same layout. */
lbe_status lbe_save(lbe_handle* h, const char* path);
lbe_status lbe_load(lbe_handle* h, const char* path);

/* Step-kernel choice (autotuner hook).  Kernel ids 0 .. lbe_num_tiles()-1:
 * ids whose shape has ty > 0 are the tile kernel with TX x TY cells per CTA
 * (any storage; FP64 provides id 0 only); ids 7 and 8 (ty == 0) are the
 * strip kernel with 128 output columns per CTA marching over rows, staging
 * each row's pulled populations in shared memory with bulk copies (16/32-bit
 * and F16MIX storages, every instance at least 4 columns wide; the default
 * there).  They differ in who refreshes the periodic ghost columns (4 copies
 * of the edge cells at each end of a stored row): with 7 a second kernel
 * after the step, with 8 the step itself (the owner of an edge cell stores
 * it twice); both give bitwise the same state.  The default is 8 when the
 * instances are narrow (cells-weighted mean of at most 8 strips of 128
 * columns), else 7.  Ids 5 and 6 are retired and rejected.
 * grid_ctas: persistent grid size (0 = resident CTAs x SMs, -1 = one CTA per
 * work item).  seg_rows > 0: rows per strip work item, items taken
 * round-robin; < 0: balanced: the strips of all instances laid end to end
 * and cut into one contiguous range of rows per CTA, marched in pieces of
 * at most -seg_rows rows; 0: automatic (balanced ranges when the instances
 * differ in size, else items with the row count chosen from the wave
 * count, at most 96).  LBE_EINVAL for a kernel the handle cannot use.
 * lbe_get_tile() reports {kernel id, grid CTAs, seg rows, work items}. */
int32_t lbe_num_tiles(void);
lbe_status lbe_tile_shape(int32_t tile_id, int32_t* tx, int32_t* ty);
lbe_status lbe_set_tile(lbe_handle* h, int32_t tile_id, int32_t grid_ctas, int32_t seg_rows);
lbe_status lbe_get_tile(const lbe_handle* h, int32_t out[4]);

/* ---- Discrete adjoint (gradients of a drop-migration observable).
 *
 * The observable of a state Q is the phase-1 centroid velocity of the
 * migration problem (Sec. IV.C):
 *   l(Q) = sum_x c(x) u_y(x) / sum_x c(x)
 * with c, u_y the fields of Q as lbe_fields computes them (u includes the
 * half-step force, Eq. 13).  The loss of a run of N steps from Q_0 is the mean
 * of l over the last `window` states:  L = (1/W) sum_{n=N-W+1..N} l(Q_n).
 * The gradient is the discrete adjoint of the FP64 step: the transposed
 * streaming (bounce-back and anti-bounce-back included), the transposed
 * collision of all three lattices (Eq. 12, 27, aEq12) with the force of Eq. 3
 * and sigma(T) of Eq. aEq3, and the transposed isotropic stencils with their
 * ghost-row rules, propagated backward over the run.  Parameters:
 *   theta = (sigmaT, eta2/eta1, lam2/lam1), the ratios varied with eta1 and
 *   lam1 fixed.  The initial state is the equilibrium of lbe_init at u = 0, so
 *   hbar_i(x, 0) = w_i rho c_v T0(x) and dL/dT0(x) = rho c_v sum_i w_i
 *   dL/dhbar_i(x, 0). */
typedef struct {
  int64_t steps;       /* N >= 1 steps from the handle's current state      */
  int64_t window;      /* 1 <= W <= N: states averaged into the loss          */
  int64_t ckpt_every;  /* k >= 1: spacing of the stored checkpoints; the
                          backward recomputes each segment of k steps from
                          its checkpoint and keeps k + 1 FP64 states          */
} lbe_adjoint_spec;

/* Forward N steps from the handle's current state (the handle's storage and
 * kernel; checkpoints of the raw storage every k steps), then the backward
 * sweep over the recomputed states (kept as FP64).  The backward arithmetic
 * follows the forward's: FP64 for an LBE_F64 handle; FP32 per-cell products
 * for the other storages, whose trajectory is an FP32 one (the adjoint
 * vectors and the parameter sums stay FP64; the loss is always FP64).
 * Outputs (each may be NULL):
 *   loss     host double: L
 *   grad     host double[3]: dL/dsigmaT, dL/d(eta2/eta1), dL/d(lam2/lam1)
 *   dT0      [ny][nx] doubles: dL/dT0
 *   dQ0      [27][ny][nx] doubles: dL/dQ_0 (adjoint of the starting state)
 * dT0 and dQ0 are device pointers if on_device, else host.  The handle must
 * hold one instance.  On return the handle holds the state after the N steps
 * (steps_done advanced by N).  Device memory used during the call:
 * about (k + 1 + 2) * 27 + 30 doubles per cell plus N/k raw checkpoints; it is
 * allocated and freed inside the call (LBE_ENOMEM if it does not fit).
 * Waits. */
lbe_status lbe_adjoint(lbe_handle* h, const lbe_adjoint_spec* spec, double* loss,
                       double grad[3], double* dT0, double* dQ0, int32_t on_device);

/* One adjoint step at an explicit state, for tests and custom losses (FP64
 * arithmetic whatever the storage).  With
 * Q = Q_n ([27][ny][nx] device doubles, instance 0's parameters) and
 * a_next = dL/dQ_{n+1} (device, same layout):
 *   a_out = (dQ_{n+1}/dQ_n)^T a_next + wl * dl/dQ_n          (device)
 *   grad[0..2] += a_next^T dQ_{n+1}/dtheta + wl * dl/dtheta  (host)
 * a_next may be NULL (taken as zero: the last state of a run).  Waits. */
lbe_status lbe_adjoint_step(lbe_handle* h, const double* Q, const double* a_next, double wl,
                            double* a_out, double grad[3]);

/* l(Q) of a [27][ny][nx] device state with instance 0's parameters.  Waits. */
lbe_status lbe_observable(lbe_handle* h, const double* Q, double* out);

/* Introspection. */
int64_t lbe_steps_done(const lbe_handle* h);
void* lbe_stream(const lbe_handle* h);         /* the cudaStream_t used   */
int32_t lbe_num_instances(const lbe_handle* h);
int64_t lbe_state_bytes(const lbe_handle* h); /* both population buffers */

void lbe_destroy(lbe_handle* h);

/* Allocation-free FP64 sums.  The paper has no counterpart: this is a library
 * service for callers that cannot let the library allocate device memory (a
 * framework whose caching allocator owns the device memory, a per-step
 * monitoring loop where cudaMalloc/cudaFree would synchronize the device, a
 * process with a fixed device-memory budget).  It computes what lbe_sums
 * computes, but from caller-provided fields and without a handle:
 *   cur[0..4]  device pointers to c, p, ux, uy, T of one state, n values each
 *   prev       NULL, or device pointers whose [2] and [3] (ux, uy) are the
 *              previous step's velocity (for the residual; other entries unused)
 *   rho_cv     rho * c_v, so that out[2] = rho c_v sum T = sum of hbar
 *   out        device pointer to 5 doubles: sum c, sum p, sum hbar, residual
 *              ||u - u_prev|| / ||u|| (0 without prev), non-finite count
 *   stream     cudaStream_t the two kernels are enqueued on (asynchronous).
 * Its only scratch is a static 384 KiB device array inside the library, held
 * by every GPU that loads it until the process exits (or the device is
 * reset); n must be at most
 * 33,554,432 (LBE_EINVAL otherwise, message from lbe_last_error(NULL)).  No
 * call allocates or frees memory.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current, so
 * make that first call before any stream capture; a call made while another
 * driver context is current on the device looks the address up again for
 * that context.  A cudaDeviceReset after the first call is not supported (the
 * module is reloaded and the cached address may be stale).  All calls on a
 * device share the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialized by the caller. */
lbe_status lbe_sums_fields_noalloc(const double* const cur[5], const double* const prev[5],
                                   int64_t n, double rho_cv, double* out, void* stream);

/* Last error message of the handle (or of this thread if h is NULL). */
const char* lbe_last_error(const lbe_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LBE_H */
