/*
 * sbiem.h -- C ABI of the GB300 spectral boundary integral element method
 * (sBIEM) for a mildly non-planar 2D in-plane (mode II) fault, after Romanet &
 * Ozawa, "Fully dynamic earthquake cycle simulations on a non-planar fault
 * using the spectral boundary integral element method" (arXiv 2107.03550).
 *
 * One handle = one periodic fault of N elements on one GPU.  Every step of
 * the time integration runs in the library's own sm_103a CUDA kernels; the
 * host only validates arguments, enqueues launches and copies results out.
 *
 * Conventions shared by all entry points
 *   - Host pointers are plain C arrays in element order i = 0..N-1 (element
 *     centres x_i = -L/2 + (i + 1/2) dx, L = N dx, periodic).  Inputs are
 *     copied; the caller keeps ownership of every buffer it passes.
 *   - Outputs are written into caller-owned host buffers; a NULL output
 *     pointer skips that output.
 *   - The handle owns all device memory it allocates (through the allocator
 *     given in sbiem_params, else cudaMalloc) and frees it in sbiem_destroy.
 *   - Return value: SBIEM_OK (0) or a negative SBIEM_ERR_* code;
 *     sbiem_strerror() gives a message, sbiem_last_error() adds detail.
 *   - A handle is bound to the CUDA device that was current at creation and
 *     to one stream (default: a non-blocking stream of its own; see
 *     sbiem_set_stream); it is not thread-safe.
 */
#ifndef SBIEM_H
#define SBIEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define SBIEM_OK                 0
#define SBIEM_ERR_INVALID       -1  /* bad argument (N, dt, parameters, NULL input) */
#define SBIEM_ERR_NOMEM         -2  /* device allocation failed */
#define SBIEM_ERR_CUDA          -3  /* a CUDA runtime call failed */
#define SBIEM_ERR_NEWTON        -4  /* friction Newton iteration cap hit (Sec. 3.2 failure) */
#define SBIEM_ERR_OPENING       -5  /* sigma_load + sigma_el <= 0 on a sliding element (Sec. 3.2) */
#define SBIEM_ERR_STATE         -6  /* theta <= 0 with the explicit state update (Sec. 3.2) */
#define SBIEM_ERR_DTMIN         -7  /* failure at dt = dt_min in the adaptive run (Sec. 3.2) */
#define SBIEM_ERR_UNSUPPORTED   -8  /* valid request outside what this build implements */
#define SBIEM_ERR_WAIT          -9  /* a device-side wait ran past its iteration limit (the
                                       step is rejected; the CUDA context stays usable) */

/* bit flags of the device status word (sbiem_status) */
#define SBIEM_FLAG_NEWTON   1u
#define SBIEM_FLAG_OPENING  2u
#define SBIEM_FLAG_STATE    4u
#define SBIEM_FLAG_WAIT     8u  /* a bounded device wait (copy completion) gave up */

typedef struct sbiem_s* sbiem_t;

typedef void* (*sbiem_alloc_fn)(size_t bytes, void* user);
typedef void  (*sbiem_free_fn)(void* ptr, void* user);

/*
 * Parameters of one fault.  Table 1 names; Sec. 3.1 truncation; Sec. 3.2
 * minimum time step.  Fill with sbiem_default_params() first.
 */
typedef struct sbiem_params {
  int64_t N;            /* elements; a power of two, 16 <= N <= 2^20          */
  double  dx;           /* element size Delta s (m)                            */
  double  mu;           /* shear modulus (Pa)                                  */
  double  cs, cp;       /* shear and dilatational wave speeds (m/s), cp > cs   */
  double  beta_min;     /* dt_min = beta_min dx / cs (Sec. 3.2), default 0.25  */
  double  eta_w;        /* truncation parameter eta (Sec. 3.1), default 1;
                           0: the quasi-dynamic limit (Appendix, Quasi-dynamic
                           BIEM): no history, no current-interval kernel term,
                           static stiffness plus radiation damping            */
  double  kc_L;         /* k_c * eta * Omega (Sec. 3.1), default 200           */
  double  kcN_L;        /* the normal-traction kernel's own k_c * eta * Omega:
                           the second cutting plane Sec. 3.1 proposes for the
                           slower-converging normal kernel; each field's
                           weights are zero past its own window, the rings
                           keep the longer one.  0 (default): kc_L, the
                           paper's single plane                               */
  int32_t kc_units;     /* 0: k_c in rad/m (default); 1: in cycles/m           */
  int32_t precision;    /* 0: FP64 throughout (default); 1: FP32 history
                           convolution and FFTs, FP64 state and Newton        */
  int32_t state_law;    /* 0: aging law integrated exactly at constant Vbar
                           over the step (default); 1: explicit
                           theta + thetadot dt as printed in Sec. 3.3          */
  int32_t newton_maxit; /* Newton iteration cap per solve, default 50          */
  int32_t quadrature;   /* kernel weights of the history and current-interval
                           integrals: 0 (default) the midpoint rule of Sec.
                           3.3, w_{n,j} = dt_min C(k_n, (j + 1/2) dt_min);
                           1 the integral of C(k_n, tau) over each interval
                           [j dt_min, (j + 1) dt_min] (six-point
                           Gauss-Legendre); the two differ by O(dt^2).  With
                           1 the FP32 sweep streams its weights           */
  double  newton_tol;   /* |delta ln V| convergence tolerance, default 1e-12   */
  double  f0, V0;       /* reference friction and slip rate (Eq. momentum)     */
  sbiem_alloc_fn alloc_fn; /* optional device allocator (NULL: cudaMalloc)     */
  sbiem_free_fn  free_fn;  /* matching free (NULL: cudaFree)                   */
  void*   alloc_user;      /* passed to alloc_fn / free_fn                     */
} sbiem_params;

/* Fill p with the defaults listed above (N = 0: the caller must set N, dx,
 * mu, cs, cp, f0, V0). */
void sbiem_default_params(sbiem_params* p);

/*
 * sbiem_create -- set up one fault (Sec. 3; geometry Sec. 2.2).
 *
 * h:          fault profile x2 = h(x_i) (m); used only when kappa is NULL, in
 *             which case kappa = h'' by spectral differentiation on the device.
 * kappa:      curvature h''(x_i) (1/m), or NULL.
 * a, b, Dc:   rate-and-state parameters per element (Eq. momentum, aging law).
 * sigma_load: compressive normal load per element (Pa), > 0.
 * tau_load:   shear load per element (Pa), or NULL for the load in equilibrium
 *             with the initial state: sigma f(V_init, theta_init) + mu/(2cs) V.
 * tau_load_rate: d tau_load / dt per element (Pa/s), or NULL for zero.
 * prescribed: per element 0 = frictional, 1 = slip rate prescribed (the
 *             null-slip-rate zones of Sec. 4, plate-rate loading); NULL = none.
 * V_presc:    prescribed slip rate (m/s); may be NULL when prescribed is NULL.
 * V_init, theta_init: initial slip rate (> 0 on frictional elements) and
 *             state (> 0).
 * On success *out receives the handle.  Slip starts at zero; history is empty.
 * Errors: SBIEM_ERR_INVALID, SBIEM_ERR_NOMEM, SBIEM_ERR_CUDA.
 */
int sbiem_create(sbiem_t* out, const sbiem_params* p,
                 const double* h, const double* kappa,
                 const double* a, const double* b, const double* Dc,
                 const double* sigma_load, const double* tau_load,
                 const double* tau_load_rate,
                 const uint8_t* prescribed, const double* V_presc,
                 const double* V_init, const double* theta_init);

/* Free every device buffer of the handle.  NULL is accepted. */
void sbiem_destroy(sbiem_t s);

/* Bind the handle to a CUDA stream (cudaStream_t passed as void*; NULL is the
 * legacy default stream).  All later work of the handle is enqueued there.
 * A new handle uses a non-blocking stream of its own. */
int sbiem_set_stream(sbiem_t s, void* cuda_stream);

/*
 * sbiem_step -- one accepted time step of length dt (Sec. 3.3): predictor,
 * tractions from the spectral formulas with the truncated history
 * convolution (Sec. 3.1), Newton for the slip rate, then the same with the
 * averaged slip rate and state rate, then the history push.
 * dt must be m * dt_min for an integer m >= 1 (the history is kept on the
 * dt_min grid).  Synchronizes with the stream to read the status.
 * Errors: SBIEM_ERR_INVALID (dt), SBIEM_ERR_NEWTON, SBIEM_ERR_OPENING,
 * SBIEM_ERR_STATE -- on these the fault state is left as it was before the
 * step.
 */
int sbiem_step(sbiem_t s, double dt);

/*
 * sbiem_enqueue -- enqueue nsteps steps of length dt without synchronizing
 * (a captured CUDA graph of one step is replayed nsteps times).  A step that
 * fails sets the device status word; it and every later step then leave the
 * state untouched.  Read the outcome with sbiem_status().
 */
int sbiem_enqueue(sbiem_t s, double dt, int64_t nsteps);

/* Kernels one replay of the step graph of sbiem_enqueue launches for steps
 * of dt (a power of two times dt_min; the graph is captured if it is not
 * yet).  The prologue sweep of a new sequence is not counted. */
int sbiem_step_kernels(sbiem_t s, double dt, int64_t* kernels);

/* Synchronize and read the device status bits (SBIEM_FLAG_*) and the number of
 * committed steps; clear != 0 resets the status word (state is unaffected). */
int sbiem_status(sbiem_t s, uint32_t* flags, int64_t* steps_done, int clear);

/*
 * sbiem_run -- adaptive time integration up to t_end by step doubling
 * (Sec. 3.2): dt = m dt_min with m a power of two (m <= 2^30, <= m_max).  A
 * trial advances once by dt (not committed) and twice by dt/2; the error is
 * eps = max_i |delta_full - delta_halves| (slip).  eps <= eps0: the
 * two-half-step state is kept and m becomes the largest power of two <=
 * 0.9 (eps0/eps)^(1/3) m, at most 2m.  eps > eps0 or a failure (Newton cap,
 * opening, state): the state and the overwritten history slots are restored
 * and m is at least halved.  At m = 1 a single step is taken and its error
 * is ignored; a failure there returns SBIEM_ERR_DTMIN with the state at the
 * start of that step.  Stops after max_steps accepted steps.
 * Outputs (host, may be NULL): accepted steps, the next m, the time reached,
 * and m_hist[k] = m of accepted step k (caller buffer of max_steps int64).
 * The first call allocates the snapshot buffers (about the ring size).
 */
int sbiem_run(sbiem_t s, double t_end, double eps0, int64_t m0, int64_t m_max,
              int64_t max_steps, int64_t* steps_done, int64_t* m_next, double* t_reached,
              int64_t* m_hist);

/*
 * Output of sbiem_run while it runs (the slip history of a cycle, the
 * rupture front, V_max ...): after every `every`-th accepted step, and after
 * the last accepted step of the run, the library copies the committed slip
 * and slip rate to page-locked host buffers it owns and calls
 *   cb(user, step, t, m, delta, V, N)
 * with step = accepted steps so far in this run, t = simulated time, m = that
 * step's length in dt_min; delta and V (N doubles each) are valid during the
 * call only.  A nonzero return stops the run after that step (sbiem_run then
 * returns SBIEM_OK with the steps done so far).  cb = NULL removes the
 * callback.  Errors: SBIEM_ERR_INVALID (every < 1), SBIEM_ERR_NOMEM.
 */
typedef int (*sbiem_output_fn)(void* user, int64_t step, double t, int64_t m, const double* delta,
                               const double* V, int64_t N);
int sbiem_set_output(sbiem_t s, sbiem_output_fn cb, void* user, int64_t every);

/*
 * sbiem_step_host -- a step driven from host memory: copies tau_load (N
 * doubles, replaces the shear load) host->device, runs one step and copies the
 * new slip rate V (N doubles) device->host.  Either pointer may be NULL.
 * Host buffers should be pinned for asynchronous copies: with page-locked
 * buffers, once a sequence of steps of one length is under way (after the
 * first such call), the copies, the step and the read of the status word
 * run as one CUDA graph (captured for that step length and pointer pair)
 * with one synchronization per step.  Errors as sbiem_step.
 */
int sbiem_step_host(sbiem_t s, double dt, const double* tau_load, double* V_out);

/* Copy the committed state to host buffers (N doubles each): slip delta,
 * slip rate V, state theta, and the elastic traction changes tau_el and
 * sigma_el (compression positive) of the last pass of the last step; *t is
 * the simulated time.  Synchronizes. */
int sbiem_get_state(sbiem_t s, double* delta, double* V, double* theta,
                    double* tau_el, double* sigma_el, double* t);

/* Replace the committed state (any pointer NULL keeps that field).
 * Prescribed elements keep V = V_presc whatever V holds for them.  The
 * spectral running sums F[delta], F[kappa delta] are recomputed. */
int sbiem_set_state(sbiem_t s, const double* delta, const double* V,
                    const double* theta);

/* Number of modes (N/2 + 1) and per-mode window lengths M_n (Sec. 3.1):
 * M must hold N/2 + 1 int64.  The history of mode n holds M_n - 1 slots. */
int sbiem_windows(sbiem_t s, int64_t* M);

/* Load / read the history rings (Sec. 3.3, last paragraph).  Layout: for
 * each mode n = 0..N/2 in turn, M_n - 1 complex values (re, im interleaved,
 * FP64), newest first: first the shear field F[Vbar], then (a second array)
 * the normal field F[kappa Vbar].  Length of each array: 2 * sum_n (M_n - 1)
 * doubles.  The spectral convention is F[f]_n = sum_i f_i exp(-2 pi i n i/N). */
int sbiem_set_history(sbiem_t s, const double* hist_T, const double* hist_N);
/* The same from device memory: hist_T, hist_N are device arrays in the
 * layout above, FP64 (values_fp32 = 0) or FP32 (values_fp32 = 1) re/im
 * pairs, converted to the handle's precision on the device (for rings of
 * hundreds of millions of slots).  Synchronizes the handle's stream. */
int sbiem_set_history_device(sbiem_t s, const void* hist_T, const void* hist_N, int32_t values_fp32);
int sbiem_get_history(sbiem_t s, double* hist_T, double* hist_N);

/* Checkpoint / restart.  sbiem_save writes to `path` (binary, little endian,
 * this library's own format "SBIEMCK3") the parameters, the per-element
 * inputs (kappa, a, b, Dc, loads, prescribed mask and rates), the committed
 * state (delta, V, theta), the time, the step count and the history rings;
 * it synchronizes the handle's stream.  sbiem_load creates a new handle from
 * such a file; `alloc` (or NULL) supplies only the allocator fields
 * (alloc_fn, free_fn, alloc_user).  A loaded handle continues bitwise like
 * the saved one (after a save both recompute their next history sums).  Errors: SBIEM_ERR_INVALID (bad path or file),
 * SBIEM_ERR_NOMEM, SBIEM_ERR_CUDA. */
int sbiem_save(sbiem_t s, const char* path);
/* The handle's parameters (a copy; the allocator fields as given). */
int sbiem_get_params(sbiem_t s, sbiem_params* out);
int sbiem_load(sbiem_t* out, const char* path, const sbiem_params* alloc);

/*
 * Timing probe.  sbiem_probe_enable(s, nslots) with nslots >= 1 makes every
 * later step record four CUDA events on the handle's stream (as event-record
 * nodes inside the step graph as well): at the start of the step, before and
 * after the history convolution kernel, and at the end of the step.  Step k
 * (counted from the call) uses event slot k mod nslots, so nslots steps can
 * be enqueued back to back and read afterwards.  nslots = 0 disables the
 * probe.  sbiem_probe_read synchronizes on the slot's last event and returns
 * the elapsed milliseconds of that step and of its history convolution.
 * Enabling or disabling rebuilds the step graph.
 */
int sbiem_probe_enable(sbiem_t s, int nslots);
int sbiem_probe_read(sbiem_t s, int slot, float* ms_step, float* ms_history);

/*
 * sbiem_history_sums -- run the truncated history convolution alone (Sec. 3.1
 * window, Sec. 3.3 step (2), midpoint weights) on the current rings:
 *   A^T_n = sum_{j=m}^{M_n-1} w^T_{n,j} H^T_n[j-m],  A^N_n likewise,
 * for the history shift m >= 1 (a step of m dt_min).  AT and AN receive
 * N/2 + 1 complex values each (re, im interleaved, FP64) in caller-owned host
 * memory.  The state is not modified.  Synchronizes.
 * Errors: SBIEM_ERR_INVALID (NULL, m < 1), SBIEM_ERR_CUDA.
 */
int sbiem_history_sums(sbiem_t s, int64_t m, double* AT, double* AN);

/*
 * sbiem_history_sums_noalloc -- the history convolution of
 * sbiem_history_sums for callers that cannot allocate device memory.  The
 * paper has no counterpart; this entry point exists for library users.
 *
 * Who needs it: callers that must not allocate device memory themselves or
 * through a library.  A host application that owns every byte of the GPU
 * (a simulation framework handing out slices of one fixed arena, or a
 * process held to a hard device-memory budget) cannot let a library grow its
 * footprint behind its back; a real-time loop cannot take cudaMalloc's
 * latency, its device-wide synchronization or its locks in the middle of a
 * step.  Such a caller keeps the history in its own buffers and needs only
 * the sums.
 *
 * Inputs (device pointers, caller-owned, not modified):
 *   ring     nslots history slots in the library's layout: per slot the
 *            shear value F[Vbar] then the normal value F[kappa Vbar], complex,
 *            FP64 (32 bytes per slot) or FP32 (16 bytes) per `precision`;
 *   weights  per lag the pair (w^T, w^N), FP64 (16 bytes) or FP32 (8 bytes);
 *   ring_off[n], w_off[n] (int64, nmodes entries) start slot / weight of mode n;
 *   R[n] = M_n - 1 (int32, slots of mode n), M[n] = M_n (int32, weights of
 *   mode n), head[n] (int32, ring position of the newest slot of mode n,
 *   0 <= head[n] < R[n], 0 where R[n] = 0; the slot of the i-th newest value
 *   is (head[n] + i) mod R[n]).
 * Outputs: AT, AN (device, nmodes complex FP64 each, re/im interleaved).
 * m: the history shift (a step of m dt_min), m >= 1.  stream: cudaStream_t or
 * NULL.
 *
 * Scratch: one static device array of about 3.8 MB that every GPU loading
 * the library holds until exit; it bounds the sizes to nmodes <=
 * SBIEM_NOALLOC_MAX_MODES (N <= 65536) and to
 * sum_n ceil(R[n] / 2048) <= SBIEM_NOALLOC_MAX_CHUNKS.  Larger inputs return
 * SBIEM_ERR_INVALID.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Each call clears the counters it needs, but every call shares the
 * one array: calls that overlap on the GPU (several streams, or several host
 * threads) race, so serialize them on one stream.  The call synchronizes the
 * stream once (to read the chunk count) and returns with the sums enqueued.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 */
#define SBIEM_NOALLOC_MAX_MODES  32769
#define SBIEM_NOALLOC_MAX_CHUNKS 65536
int sbiem_history_sums_noalloc(int64_t nmodes, int32_t precision, int64_t m,
                               const void* ring, const void* weights,
                               const int64_t* ring_off, const int64_t* w_off,
                               const int32_t* R, const int32_t* M, const int32_t* head,
                               double* AT, double* AN, void* stream);

/* sbiem_history_enqueue -- enqueue the history convolution of
 * sbiem_history_sums on the handle's stream without synchronizing or copying
 * (for timing the kernel with events on that stream).  The sums land in the
 * handle's A^T, A^N: exactly the sums the next step of m dt_min needs, so
 * that step takes them instead of sweeping again.
 * Two kernels run: the bulk-async sweep (chunk partial sums) and the
 * per-mode finish.  `sweep_done` (a cudaEvent_t, or NULL) is recorded on the
 * stream between the two, so the sweep alone can be timed. */
int sbiem_history_enqueue(sbiem_t s, int64_t m);
int sbiem_history_enqueue_marked(sbiem_t s, int64_t m, void* sweep_done);

/* sbiem_read_probe -- a measurement helper, not a step of the method: read
 * `bytes` bytes of device memory at `data` once with coalesced 128-bit loads
 * (4 CTAs of 256 threads per SM, eight loads in flight per thread) and sum
 * them as float4s; `sink` (device, one float) is written only if the sum
 * equals a sentinel, which keeps the loads.  It gives the bandwidth a plain
 * read of that many bytes reaches, the ceiling beside which the history
 * sweep's fraction of the large-copy peak is read (fixed launch and ramp
 * costs weigh on reads of tens of MB).  `data` must be 16-byte aligned and
 * `bytes` a multiple of 16; enqueued on `stream` (a cudaStream_t, NULL: the
 * legacy stream), no synchronization.  Errors: SBIEM_ERR_INVALID for a null
 * or misaligned pointer or size, SBIEM_ERR_CUDA for a failed launch. */
int sbiem_read_probe(const void* data, int64_t bytes, float* sink, void* stream);

/* ------------------------------------------------------------- ensembles
 * A batch advances many faults together (independent realizations of uneven
 * N): one launch of the history convolution covers the chunks of every
 * member, and per group of equal N one launch of each pass kernel handles
 * all members of the group (the groups run as parallel branches of one CUDA
 * graph per step).  Members keep their own state, read with sbiem_get_state
 * after sbiem_batch_status; they must share the device and the precision.
 * A member whose step fails stops committing (its own status word) while the
 * others go on.  The history convolution is one bulk-async sweep over the
 * members' chunk tables laid end to end (statically partitioned over the
 * CTAs) and the per-(member, mode) sums, in one persistent cooperative
 * launch with a grid barrier (bounded: see sbiem_batch_set_wait_limit)
 * between the two.
 *
 * sbiem_batch_create: n member handles (not owned); they must share the
 *   device and the precision.  chunk_slots: the lags per chunk of the
 *   batch's own chunk table (0: the members' length; else the chunk length
 *   of a sweep shape, 256/512/1024 FP64 or 512/1024/2048 FP32).  Errors:
 *   SBIEM_ERR_INVALID, SBIEM_ERR_NOMEM.
 * sbiem_batch_enqueue: nsteps steps of each member's dt_min, asynchronous.
 * sbiem_batch_status: synchronize; per member (caller order) status flags
 *   and committed steps (arrays of n, may be NULL).
 * Members share weights: with equal dx, c_s, c_p, dt_min, quadrature and
 *   precision, mode n of N has the wavenumber of mode n 2^p of 2^p N and so
 *   the same weights as far as both windows reach; with one cutting plane a
 *   member whose every window is no longer than a larger member's reads a
 *   prefix of that member's weight runs (members of equal N and windows read
 *   one copy).  The sweep then copies ring slots under an L2 evict-first
 *   policy so that the shared weight runs stay in L2.
 * sbiem_batch_tune: autotuner -- times the batched history convolution for
 *   every sweep shape (with the batch's chunk table of that shape's chunk
 *   length, built once per length), each weight form
 *   (streamed, or evaluated on chip for the modes with s step up to 1/256,
 *   1/64 or 1/32 when the members share c_s, c_p and dt_min) and 1 .. (occupancy
 *   limit) resident sweep CTAs per SM, reps timed launches each (median), and
 *   keeps the fastest.  It then chooses the history form (one persistent
 *   launch or two launches, sbiem_batch_set_persistent) and the overlap
 *   together: for each form, the sweep alone followed by the passes, and
 *   the overlapped step's two branches timed together (the next step's
 *   sweep beside the passes) for 1 .. (occupancy limit) sweep CTAs per SM;
 *   the fastest candidate is kept (a new batch steps without overlap).
 *   Returns the chunk length, the CTAs per SM chosen and the sweep's time
 *   (sbiem_batch_get_sweep gives the rest).  The committed state is not
 *   changed.
 * sbiem_batch_set_overlap: overlap on (1) or off (0) by hand; *on_out (may
 *   be NULL) gets the setting in force before the call.  Results agree
 *   either way up to summation order.
 */
typedef struct sbiem_batch_s* sbiem_batch_t;
/* sbiem_batch_set_wait_limit: polls of the persistent history launch's grid
 *   barrier before a CTA gives up (default SBIEM_WAIT_LIMIT_DEFAULT); a CTA
 *   that gives up flags every member SBIEM_FLAG_WAIT, so that step is
 *   rejected for all of them with nothing committed.  0 gives up at once: a
 *   way to exercise the path without any fault.  Synchronizes; the step
 *   graph is rebuilt. */
int sbiem_batch_create(sbiem_batch_t* out, int n, const sbiem_t* members, int64_t chunk_slots);
void sbiem_batch_destroy(sbiem_batch_t b);
int sbiem_batch_set_stream(sbiem_batch_t b, void* cuda_stream);
int sbiem_batch_enqueue(sbiem_batch_t b, int64_t nsteps);
int sbiem_batch_status(sbiem_batch_t b, uint32_t* flags, int64_t* steps_done);
int sbiem_batch_tune(sbiem_batch_t b, int reps, int64_t* chunk_slots, int* blocks_per_sm, float* ms);
int sbiem_batch_set_overlap(sbiem_batch_t b, int on, int* on_out);
int sbiem_batch_set_wait_limit(sbiem_batch_t b, int64_t polls);
/* sbiem_batch_get_sweep: the batch's history-convolution configuration; any
 *   pointer may be NULL.  shape: sweep shape (as sbiem_get_sweep);
 *   gen_ds_max: largest s step of a mode whose weights are evaluated on chip
 *   (0: every weight streamed); ctas_per_sm: resident CTAs per SM of the
 *   persistent launch; overlap: 1 when the next step's sweep runs beside the
 *   passes; distinct_weights: weight arrays read (members sharing one count
 *   once); persistent: 1 for the one-launch form, 0 for the two-launch form.
 * sbiem_batch_set_persistent: the history convolution as one persistent
 *   cooperative launch (1, the default) or as a sweep launch followed by a
 *   per-(member, mode) sum launch (0, no grid barrier).  Results are bitwise
 *   equal either way.  *on_out (may be NULL) gets the form in force before
 *   the call.  Synchronizes; the step graph is rebuilt. */
int sbiem_batch_get_sweep(sbiem_batch_t b, int32_t* shape, double* gen_ds_max, int32_t* ctas_per_sm,
                          int32_t* overlap, int32_t* distinct_weights, int32_t* persistent);
int sbiem_batch_set_persistent(sbiem_batch_t b, int on, int* on_out);

/* ------------------------------------------------ learned Newton initial guess
 * A 5 -> 64 -> 64 -> 1 perceptron (GELU = x Phi(x)) predicts ln V* - ln V_prev
 * of the friction Newton solve (Eq. momentum) from the features
 * (ln V_prev, ln theta, tau/sigma, a, b) of an element.  Parameter vector
 * (FP32, SBIEM_MLP_PARAMS + SBIEM_MLP_NORM values): W1[64][5], b1[64],
 * W2[64][64], b2[64], W3[64], b3, then in_mean[5], in_std[5], out_mean,
 * out_std (features are normalized as (f - mean)/std, the output is
 * out_mean + out_std * y).  The deployed network runs in BF16 with FP32
 * accumulation (warp mma.sync); its guess starts Newton only when it is
 * finite, inside the solve's bracket and at least 0.1 away from ln V_prev
 * (where the previous slip rate is a poor start), otherwise ln V_prev does,
 * so the converged slip rates are those of plain Newton to its tolerance.
 */
#define SBIEM_MLP_PARAMS 4609
#define SBIEM_MLP_NORM   12
/* Deploy a network in the handle's Newton kernel (NULL: plain Newton). */
int sbiem_set_mlp(sbiem_t s, const float* params);
/* Record (features, converged ln V) rows of later Newton solves into a device
 * buffer of capacity rows (0 disables); rows beyond capacity are dropped. */
int sbiem_harvest_enable(sbiem_t s, int64_t capacity);
/* Copy up to max_rows harvested rows of 6 floats (ln V_prev, ln theta,
 * tau/sigma, a, b, ln V*) to rows_out; *rows = rows stored; reset != 0
 * restarts the buffer. */
int sbiem_harvest_read(sbiem_t s, float* rows_out, int64_t max_rows, int64_t* rows, int reset);
/* Network evaluation on the GPU for n raw feature rows X[n][5] (host) ->
 * out[n] predicted residuals (host).  Allocates its own device buffers. */
int sbiem_mlp_predict(const float* params, const float* X, int64_t n, float* out);
/* Mean-squared-error loss over normalized inputs X[n][5] and targets t[n]
 * and its gradient with respect to the SBIEM_MLP_PARAMS weights (FP32, own
 * forward / backward kernels, fixed-order reduction). */
int sbiem_mlp_grad(const float* params, const float* X, const float* t, int64_t n, float* grad, float* loss);
/* Train on n harvested rows (host, 6 floats each): normalization from the
 * data, seeded initialization, Adam (lr) on shuffled batches for `epochs`
 * passes, all on the GPU; writes SBIEM_MLP_PARAMS + SBIEM_MLP_NORM values
 * to params and the last batch's loss to *final_loss. */
int sbiem_mlp_train(const float* samples, int64_t n, int epochs, int batch, float lr, uint64_t seed,
                    float* params, float* final_loss);

/* Device-side quantities of the last step: Newton iterations (sum, max over
 * elements and passes). */
int sbiem_newton_stats(sbiem_t s, int64_t* iters_sum, int32_t* iters_max);
/* Running totals of Newton iterations and solves (every pass of every step,
 * trial and rejected steps of sbiem_run included) since creation or the last
 * reset (reset != 0 zeroes them after reading).  Synchronizes. */
int sbiem_newton_totals(sbiem_t s, int64_t* iters, int64_t* solves, int reset);

/* Bytes the history convolution must read per step (rings, plus the
 * weights unless the sweep evaluates them on chip) and the total device
 * footprint of the handle. */
int sbiem_footprint(sbiem_t s, int64_t* history_bytes_per_step, int64_t* device_bytes);

/*
 * History sweep configuration (Sec. 3.3 step (2) runs unchanged; only its
 * launch shape and where its weights come from change).
 *   shape: lags per chunk x stages in flight; the chunk length is fixed at
 *     creation (shape 3: 2048 lags FP32, 1024 FP64, two stages), so only
 *     shapes of that chunk length are accepted (0 and 2, or 1, or 3 and 4;
 *     shape 4 is shape 3's chunk in one stage).
 *   gen_ds_max (FP32 form only): where the weights come from.  The
 *     midpoint weights w_{n,j} = dt_min C(s) at s = (j + 1/2) ds_n,
 *     ds_n = c_s k_n dt_min, depend on the mode only through ds_n; modes
 *     with ds_n <= gen_ds_max evaluate them on chip from a
 *     piecewise-polynomial table of C^T, C^N (pieces of width 1/4 in s,
 *     each with a degree-5 polynomial valid over 1.5 piece widths, built in
 *     FP64 from the library's kernel route, rounded to FP32, read through
 *     L1; a thread evaluates eight consecutive lags from one piece), so for
 *     them the sweep reads only ring slots; the other modes stream the
 *     materialized weights with the slots.  0 streams every mode's weights;
 *     modes with ds up to 1/64 evaluate in blocks of eight lags, modes
 *     above it (up to 1/32, the largest step a four-lag block allows;
 *     larger values are taken as 1/32) in blocks of four.  1/64 is the
 *     default of a new FP32 handle whenever its windows' s range fits the
 *     table (k_c L <= about 340 rad); table_err is the
 *     table's largest error relative to dt_min max|C| (-1: no table).
 *   ctas_per_sm: resident sweep CTAs per SM (0: as many as fit).
 *   lag_ctas_per_sm (get only): the same for the next step's sweep that
 *     sbiem_enqueue runs beside the passes.
 * sbiem_set_sweep synchronizes and rebuilds the step graphs.  sbiem_tune is
 * the autotuner: it times `reps` launches (median, after one untimed) of the
 * history convolution for every shape of the handle's chunk length, the
 * thresholds 0, 1/512, 1/256, 1/128, 1/64 and 1/32, and 1 .. (occupancy limit)
 * CTAs per SM, and keeps the fastest; then, in the FP32 form with N <=
 * 16384 (one-launch passes), it times the next step's sweep (the overlapped
 * form of sbiem_enqueue) together with the two passes it runs beside, for
 * 1 .. (occupancy limit) sweep CTAs per SM, and keeps the fastest; in the
 * FP32 form with N > 16384 it times the best setting of each shape over
 * real overlapped steps, each undone after its timing (state and the
 * overwritten ring slots restored), and keeps the fastest step.  Nothing is committed while it times; the committed state is
 * unchanged.  Errors: SBIEM_ERR_INVALID, SBIEM_ERR_UNSUPPORTED
 * (gen_ds_max > 0 without a table), SBIEM_ERR_CUDA.
 */
int sbiem_get_sweep(sbiem_t s, int32_t* shape, double* gen_ds_max, int32_t* ctas_per_sm, int32_t* lag_ctas_per_sm,
                    double* table_err);

/*
 * sbiem_set_wait_limit -- polls (mbarrier try_wait calls) the history sweep
 * makes while it waits for a stage's bulk copy before it gives up (default
 * SBIEM_WAIT_LIMIT_DEFAULT).  On giving up the sweep sets SBIEM_FLAG_WAIT,
 * waits at the default limit for every copy it has in flight, and returns;
 * the step is then rejected (SBIEM_ERR_WAIT, committed state unchanged) and
 * the CUDA context stays usable.  polls = 0 gives up at the first wait: a
 * way to exercise that path without any fault.  Synchronizes and rebuilds
 * the step graphs.  Errors: SBIEM_ERR_INVALID (negative), SBIEM_ERR_CUDA.
 */
#define SBIEM_WAIT_LIMIT_DEFAULT 4194304
int sbiem_set_wait_limit(sbiem_t s, int64_t polls);
int sbiem_set_sweep(sbiem_t s, int32_t shape, double gen_ds_max, int32_t ctas_per_sm);
int sbiem_tune(sbiem_t s, int reps, int32_t* shape, double* gen_ds_max, int32_t* ctas_per_sm, float* ms);
/* sbiem_set_lag_sweep -- resident CTAs per SM of the next step's sweep that
 * sbiem_enqueue runs beside the passes (the value sbiem_tune chooses; 0:
 * the built-in rule, which sbiem_set_sweep also restores), clamped to the
 * occupancy limit.  Synchronizes and rebuilds the step graphs.  Errors:
 * SBIEM_ERR_INVALID (NULL handle, negative), SBIEM_ERR_CUDA. */
int sbiem_set_lag_sweep(sbiem_t s, int32_t lag_ctas_per_sm);

/*
 * sbiem_kernel_values -- host FP64 evaluation of the convolution kernels
 * C^T_II (Eq. Ct, Sec. 2.3) and C^N_II (Sec. 2.4) at n points s = c_s |k| t
 * (s >= 0) for r = c_s / c_p, by the library's own route (the one its
 * weight tables are built from).  No GPU work.  Returns SBIEM_ERR_INVALID on
 * NULL pointers, negative s or r outside (0, 1).
 */
int sbiem_kernel_values(const double* s, int64_t n, double r, double* cT, double* cN);

/* Static message for an SBIEM_* code; sbiem_last_error() returns the detail
 * of the last failure on the calling thread. */
const char* sbiem_strerror(int code);
const char* sbiem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SBIEM_H */
