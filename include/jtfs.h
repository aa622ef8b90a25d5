/*
 * jtfs.h -- C ABI of the GB300 (sm_103a) joint time-frequency scattering
 * library: the JTFS transform Phi(x), its adjoint, the metamer loss
 * E(y) = ||Phi(y) - Phi_target||^2 with its gradient, and an Adam metamer step.
 *
 * Method: Lostanlen & Han, "Musical Metamerism with Time-Frequency
 * Scattering".  Section, equation and listing references below are to that
 * paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: 0 on success, a negative JTFS_ERR_* code otherwise; no C++
 *   exception crosses this boundary.  jtfs_error_string() names a code.
 * - Device pointers: every float* / void* data argument of the compute calls
 *   (x, phi, dphi, dx, y, phi_target, loss, dy, adam_m, adam_v, workspace) is a
 *   pointer to GPU global memory owned by the caller.  Arrays are dense and
 *   row-major; pointers to float data must be 16-byte aligned.  The library
 *   never frees or retains them beyond the call.
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every compute call only enqueues work, ordered on that stream
 *   (some of it on the plan's own streams, forked from and joined back to it,
 *   see below), and returns without synchronising; errors that only a
 *   finished kernel can reveal are not reported by the call.
 * - Workspace: compute calls need a caller-allocated device scratch buffer of
 *   at least jtfs_workspace_bytes(plan) bytes (256-byte aligned).  Its content
 *   on entry is ignored; calls sharing one workspace must not overlap in time.
 * - A plan is immutable after creation and may be shared by several streams
 *   provided each uses its own workspace.  Besides its tables it owns three
 *   CUDA streams and four events, created with it on its device: a call forks
 *   the independent launches of the second-order frequential stage onto those
 *   streams and joins them back to the caller's stream before the next stage
 *   (which keeps every call asynchronous and capturable in a CUDA graph); with
 *   stage events registered (jtfs_profile_stage) the launches stay in order on
 *   the caller's stream.
 * - Device-side errors: a kernel cannot return a code, so the two failures
 *   only a running kernel sees -- a non-finite loss (JTFS_ERR_NONFINITE) and a
 *   tensor-core barrier wait that ran out (JTFS_ERR_TIMEOUT) -- set a status
 *   word in device memory, and jtfs_status() (a synchronising call) returns
 *   and clears it.  Call it after a run of compute calls, e.g. once per
 *   descent, before trusting their results.
 */
#ifndef JTFS_H
#define JTFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define JTFS_OK             0
#define JTFS_ERR_ARG       -1  /* invalid argument (NULL pointer, bad value) */
#define JTFS_ERR_SHAPE     -2  /* unsupported sizes (N, T, F, filterbank)   */
#define JTFS_ERR_WORKSPACE -3  /* workspace NULL or misaligned              */
#define JTFS_ERR_CUDA      -4  /* a CUDA runtime call failed                */
#define JTFS_ERR_NOMEM     -5  /* host or device allocation failed          */
#define JTFS_ERR_NODEVICE  -6  /* plan was created host-only                */
#define JTFS_ERR_TOOBIG    -7  /* plan needs more scratch than the fixed
                                  array of jtfs_forward_noalloc holds       */
#define JTFS_ERR_NONFINITE -8  /* a loss evaluated since the last
                                  jtfs_status was NaN or infinite           */
#define JTFS_ERR_TIMEOUT   -9  /* a tensor-core kernel gave up waiting on one
                                  of its barriers since the last jtfs_status;
                                  the outputs of that call are invalid      */

/* Plan flags. */
#define JTFS_PLAN_HOST_ONLY 1u /* build the tables on the host only; compute
                                  calls then fail with JTFS_ERR_NODEVICE.   */
/* Unpooled outputs (§3.3-§3.5 with average_local / average_local_fr off):
 * JTFS_PLAN_UNPOOLED_T: the zeroth-order block is x itself ([N]); the
 *   second order is |Y2_fr| *_n1 phi_F at time stride 2^j2 (no phi_T), the
 *   block of n2 being [1+2K][R_out][N / 2^j2]; the first order keeps S1 at
 *   stride T.  Plans where some first-order j1 exceeds log2 T are refused
 *   (JTFS_ERR_SHAPE): their second-order rows would need U1 at stride j1.
 * JTFS_PLAN_UNPOOLED_F: frequential stride 2^j for every beta (phi_F
 *   included) and no phi_F averaging: each path has N_fr / 2^j rows instead
 *   of R_out (first and second order).
 * Phi's path order is unchanged; jtfs_phi_size gives the new size. */
#define JTFS_PLAN_UNPOOLED_T 4u
#define JTFS_PLAN_UNPOOLED_F 8u

typedef struct jtfs_plan_s* jtfs_plan_t;

/*
 * Create a plan: filterbanks and the multirate schedule of one JTFS
 * configuration, plus (unless JTFS_PLAN_HOST_ONLY) their device tables on the
 * current CUDA device.
 *
 *   N      samples per clip, a power of two, 16 <= N <= 2^20; periodic boundary.
 *   J, Q   first-order filterbank (§3.1 generator): octaves and filters per
 *          octave (constant-Q part), Q-1 constant-bandwidth filters below.
 *   Q2     filters per octave of the second-order time filterbank (same J).
 *   J_fr, Q_fr  frequential filterbank along the n1 axis (§3.4), spun to +/-.
 *   T      time averaging scale and output stride (power of two, <= N);
 *          phi_T has sigma = 0.1/T cycles/sample (§2.2).
 *   F      frequency averaging scale (>= 1); phi_F has sigma = 0.1/F
 *          cycles/bin, output stride 2^floor(log2 F) along n1.
 *   batch  clips per call (>= 1).
 *
 * Derived quantities (per clip): N1 first-order filters; N_fr = next power
 * of two >= N1 + 2^(J_fr+1) (frequential FFT length, rows zero-padded on the
 * right, §3.4 listing); R_out = N_fr / 2^floor(log2 F) pooled rows;
 * n_frames = N / T.
 *
 * On success *out owns host memory and, unless host-only, device memory;
 * release it with jtfs_plan_destroy.  Errors: JTFS_ERR_ARG (out NULL),
 * JTFS_ERR_SHAPE (sizes outside the ranges above or an empty filterbank),
 * JTFS_ERR_CUDA / JTFS_ERR_NOMEM (device table upload failed).
 */
int jtfs_plan(jtfs_plan_t* out, int64_t N, int J, int Q, int Q2, int J_fr,
              int Q_fr, int64_t T, int F, int batch, uint32_t flags);

/* Release a plan (NULL is accepted).  Device memory is freed synchronously. */
int jtfs_plan_destroy(jtfs_plan_t plan);

/*
 * Phi layout (main algorithm, §3.5): per clip a flat float vector of
 * jtfs_phi_size(plan) entries,
 *   [ S0 : n_frames ]
 *   [ first order : (1+K) paths x R_out rows x n_frames ]
 *   [ second order: for each active n2 ascending, (1+2K) paths x R_out x n_frames ]
 * where K is the number of frequential wavelets before spinning, the first
 * path of each group is the beta = 0 (phi_F) path, then +xi_n (n ascending),
 * then (second order only) -xi_n.  An n2 is active when some first-order
 * filter has j1 < j2.  Batched arrays are [batch][phi_size].
 * Returns the size, or a negative error code if plan is NULL.
 */
int64_t jtfs_phi_size(jtfs_plan_t plan);

/*
 * Path metadata, one entry per path of Phi in its order (§3.5's yields):
 *   order     0 zeroth order (S0, or x itself unpooled in time), 1 first-order
 *             frequential path (|S1 * psi_beta| * phi_F), 2 second-order path;
 *   n2        second-order time filter index (order 2), else -1;
 *   beta_idx  frequential filter: 0 phi_F, 1..K +xi_n, K+1..2K -xi_n (order 1
 *             uses 0..K), -1 for order 0;
 *   spin      sign of the frequential centre frequency (0 for phi_F and order 0);
 *   offset    first float of the path's block inside one clip's Phi; the block
 *             is rows x frames and ends where the next path starts (the last
 *             one at jtfs_phi_size).
 * Arrays (host, any may be NULL) need as many entries as the return value:
 * the number of paths, 1 + (1 + K) + n_active (1 + 2K).  Host-only plans answer
 * too.  Errors: JTFS_ERR_ARG for a NULL plan.
 */
int jtfs_path_meta(jtfs_plan_t plan, int32_t* order, int32_t* n2, int32_t* beta_idx,
                   int32_t* spin, int64_t* offset);

/* Bytes of device workspace one compute call needs (0 if plan is NULL). */
size_t jtfs_workspace_bytes(jtfs_plan_t plan);

/*
 * Plan inspection (host memory, no device access).
 * jtfs_plan_info fills info[0..count) with, in order:
 *   N, J, Q, Q2, J_fr, Q_fr, T, F, batch, N1, N2, K, N_fr, log2 T,
 *   floor(log2 F), R_out, n_frames, n_active, phi_size
 * and returns the number of values available (19), or JTFS_ERR_ARG.
 */
int jtfs_plan_info(jtfs_plan_t plan, int64_t* info, int count);

/*
 * jtfs_plan_filters copies one filterbank: which = 0 first-order time
 * (psi^{tm,1}), 1 second-order time (psi^{tm,2}), 2 frequential (psi^{fr,1},
 * positive spin), 3 the two low-pass filters (phi_T then phi_F, xi = 0).
 * xi and sigma are in cycles per sample (per bin for the frequential axis);
 * j is the largest dyadic subsampling with 2^j (xi + 3 sigma) <= 1/2.
 * Writes min(count, size) entries to each non-NULL array and returns the
 * filterbank size, or JTFS_ERR_ARG.
 */
int jtfs_plan_filters(jtfs_plan_t plan, int which, double* xi, double* sigma,
                      int32_t* j, int count);

/*
 * jtfs_plan_schedule copies one of the plan's work tables, for inspection
 * and tests (the paper has no counterpart: these are this library's launch
 * schedules), as int64 into out[0 .. min(n, size)) (host memory) and returns
 * the table's size in values (call with out = NULL, n = 0 to size it):
 *   which = 0: the gradient gather onto the U1 rows, per block of 256
 *              samples: (row, block in the row, log2 of the row's length);
 *   which = 1: the banded phi_T adjoint on the tensor cores, per CTA:
 *              (clip, active group, first of its 128 rows, first sample);
 *   which = 2: per active second-order group: (level s2, rows, n1max,
 *              reach W of the banded phi_T average or 0 when dense, samples
 *              per CTA of its tensor-core banded adjoint or 0, K atoms of its
 *              tensor-core frequential forward or 0 for the FFT kernels, the
 *              same for the adjoint).
 * Works on host-only plans.  Errors: JTFS_ERR_ARG (NULL plan, bad which,
 * n < 0, out NULL with n > 0).
 */
int64_t jtfs_plan_schedule(jtfs_plan_t plan, int which, int64_t* out, int64_t n);

/*
 * Forward transform, Eqs. (1)-(5) with the multirate schedule of §3.2-§3.5:
 *   x   [batch][N] float32 (device), real audio clips.
 *   phi [batch][phi_size] float32 (device), output, layout as above.
 * Errors: JTFS_ERR_ARG (NULL pointer), JTFS_ERR_NODEVICE, JTFS_ERR_WORKSPACE,
 * JTFS_ERR_CUDA (launch failure).
 */
int jtfs_forward(jtfs_plan_t plan, const float* x, float* phi, void* workspace,
                 void* stream);

/*
 * Adjoint (vector-Jacobian product) of jtfs_forward at x, §2.3 Eqs. (6)-(8):
 *   dx = J_Phi(x)^T dphi.  Recomputes every intermediate from x.
 *   x    [batch][N] float32 (device); dphi [batch][phi_size] float32 (device);
 *   dx   [batch][N] float32 (device), output (overwritten).
 * The modulus derivative at 0 is taken as 0.  Errors as jtfs_forward.
 */
int jtfs_backward(jtfs_plan_t plan, const float* x, const float* dphi,
                  float* dx, void* workspace, void* stream);

/*
 * Metamer loss and gradient (§1.2, §2.3):
 *   loss[b] = sum_i (Phi(y)[b][i] - phi_target[b][i])^2   (float32 [batch])
 *   dy[b]   = d loss[b] / d y[b]                            ([batch][N])
 * y and phi_target as for jtfs_forward; loss and dy are device outputs.
 * dy may be NULL (loss only).  Errors as jtfs_forward.
 */
int jtfs_loss_grad(jtfs_plan_t plan, const float* y, const float* phi_target,
                   float* loss, float* dy, void* workspace, void* stream);

/*
 * One metamer descent step with Adam (beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-8, bias-corrected with the 1-based step index `step`) on y, in
 * place.  The paper refines y by additive gradient steps (§2.3); Adam is the
 * optimiser this library's workloads use.
 *   y, adam_m, adam_v  [batch][N] float32 (device), updated in place;
 *                      m and v must start at zero before step 1.
 *   phi_target         [batch][phi_size] float32 (device).
 *   loss_out           [batch] float32 (device): loss at the y given on entry.
 * Errors as jtfs_forward, plus JTFS_ERR_ARG for step < 1 or lr <= 0.
 */
int metamer_step(jtfs_plan_t plan, float* y, const float* phi_target,
                 float* adam_m, float* adam_v, int step, float lr,
                 float* loss_out, void* workspace, void* stream);

/*
 * metamer_step_counted -- metamer_step with the 1-based Adam step index read
 * from device memory (`step`, one int32) and incremented there by the call,
 * so that one recorded call replays as successive steps from a CUDA graph
 * (the §2.3 descent repeated with no host involvement).  The bias
 * corrections are computed on the device in double from that index, as
 * metamer_step computes them on the host, so the iterates of the two calls
 * agree.  Arguments and errors
 * otherwise as metamer_step (step must hold >= 1; it is not checked on the
 * host).
 */
int metamer_step_counted(jtfs_plan_t plan, float* y, const float* phi_target,
                         float* adam_m, float* adam_v, int32_t* step, float lr,
                         float* loss_out, void* workspace, void* stream);

/*
 * Reconstruction variant of §2.3: the paper starts the descent from coloured
 * Gaussian noise whose power spectral density follows the target's
 * first-order scattering S1x(t, lambda), and refines it by momentum updates
 * whose step size follows the "bold driver" heuristic.
 *
 * jtfs_coloured_init -- initial signal of that descent.  With Psi_l the
 * first-layer filtering of band l decimated to its U1 rate (§3.2), P_l the
 * phi_T pooling that turns U1 into S1 (Eq. (4)) and ^T real adjoints:
 *   y~ = sum_l c_l Psi_l^T ( A_l . Psi_l w ),   A_l = 2^(lT-k1) P_l^T S1x(., l),
 *   y0 = y~ ||x|| / ||y~||   per clip (y0 = 0 where y~ = 0),
 * c_l = 2^(k1+1) / sqrt(mean over the N bins of psi_hat_l^6) (so band l of y~
 * has E|Psi_l y~|^2 = A_l^2 for a slowly varying envelope; jtfs_init_gains
 * returns c_l 2^(lT-k1)).  y~ is linear in w, so y0 is Gaussian given the
 * target, with local power in band l proportional to S1x^2.
 *   x        [batch][N] float32 (device): the target clips.
 *   w_noise  [batch][N] float32 (device): white Gaussian noise drawn by the
 *            caller (the library draws no random numbers).
 *   y0       [batch][N] float32 (device), written; may not alias x or w_noise.
 * All three 16-byte aligned.  Uses the workspace like jtfs_forward; errors
 * as jtfs_forward.
 */
int jtfs_coloured_init(jtfs_plan_t plan, const float* x, const float* w_noise,
                       float* y0, void* workspace, void* stream);

/* Entries of jtfs_init_gains' table (per first-order filter n1, c_l 2^(lT-k1));
 * returns the count (N1), writes min(count, n) floats to out if out != NULL
 * (JTFS_ERR_ARG if n < count).  Host-only plans answer too. */
int64_t jtfs_init_gains(jtfs_plan_t plan, float* out, int64_t n);

/*
 * metamer_step_momentum -- one evaluation of the momentum descent of §2.3
 * with the bold-driver step size, on every clip, in place:
 *   u_n = m u_{n-1} - mu_n grad E(y_n),   y_{n+1} = y_n + u_n.
 * Per clip, E(y_n) is compared with E_acc, the loss at the last accepted
 * point.  E <= E_acc accepts y_n: mu grows by 1.1 (not at the first
 * evaluation), E_acc = E, g_acc = grad E(y_n), and the momentum step is
 * taken.  Otherwise (E increased, or is NaN) y_n is rejected: mu halves, y
 * returns to the accepted point (y_n - u_{n-1}), the momentum is dropped and
 * the step -mu * g_acc is taken from there.  Every decision is made on the
 * device, so the call can be captured in a CUDA graph.
 *   y, u, g_acc  [batch][N] float32 (device), updated in place; u and g_acc
 *                start at zero.
 *   state        [batch][4] float32 (device, 16-byte aligned), updated in
 *                place: (mu, E_acc, 1 if the last evaluation was accepted
 *                else 0, evaluations so far).  Start with (mu0, +inf, 0, 0);
 *                §2.3 uses mu0 = 0.1.
 *   m            momentum in [0, 1) (§2.3: 0.9).
 *   loss_out     [batch] float32 (device): E at the y given on entry.
 * Errors as jtfs_forward, plus JTFS_ERR_ARG for m outside [0, 1).
 */
int metamer_step_momentum(jtfs_plan_t plan, float* y, const float* phi_target,
                          float* u, float* g_acc, float* state, float m,
                          float* loss_out, void* workspace, void* stream);

/* The update of metamer_step_momentum alone, from a loss [batch] and
 * gradient g [batch][n] already computed (n a power of two). */
int jtfs_momentum_update(float* y, float* u, float* g_acc, const float* g,
                         float* state, const float* loss, int batch, int64_t n,
                         float m, void* stream);

/*
 * jtfs_forward_noalloc -- the forward transform of jtfs_forward, for callers
 * that cannot allocate device memory: code that runs where cudaMalloc is not
 * allowed or not available to it (for example a real-time audio callback
 * that must not block on the allocator, or a plug-in whose host owns all
 * device memory and hands it only a stream).  It takes no workspace and
 * allocates nothing; it is an addition of this library, with no counterpart
 * in the paper.
 *
 * Scratch: a fixed array of JTFS_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into
 * the library, so every GPU that loads the library holds those 32 MiB until
 * the process exits.  Plans whose jtfs_workspace_bytes() exceed it are
 * rejected with JTFS_ERR_TOOBIG before any work is enqueued (the 8192-sample
 * single-clip plan needs about 10 MiB).
 *   x   [batch][N] float32 (device), phi [batch][phi_size] float32 (device),
 *   as for jtfs_forward; results are identical to jtfs_forward's.
 * Set-up: the first call on each device looks up the array's device address
 * (a runtime query, no allocation); make that first call before starting any
 * stream capture.  The device that was current when the plan was created must
 * be current.
 * Sharing: all calls on a device use the same array and leave their data in
 * it.  The forward pass writes every scratch byte before reading it, so no
 * clearing is needed, but calls that can overlap on the GPU (different
 * streams, different threads) race on the array and corrupt each other's
 * results; serialise them.
 * Errors: JTFS_ERR_ARG, JTFS_ERR_NODEVICE, JTFS_ERR_TOOBIG, JTFS_ERR_CUDA.
 */
#define JTFS_NOALLOC_SCRATCH_BYTES (32u << 20)
int jtfs_forward_noalloc(jtfs_plan_t plan, const float* x, float* phi,
                         void* stream);

/*
 * Ragged batches: clips of any lengths solved together.
 *
 * A clip of length L is zero-padded on the right to N = the next power of
 * two >= max(L, T) (the padding of §3.2 with the periodic boundary), its Phi
 * is computed at that N and only the first ceil(L/T) frames of every row are
 * kept (the crop's adjoint fills zeros).  Clips are grouped by N; each group
 * runs on its own plan, all on the caller's stream.
 *
 * Packed layouts (all device, float32):
 *   samples: clip b occupies [sample_off[b], sample_off[b+1]), L_b samples;
 *   Phi:     clip b occupies [phi_off[b], phi_off[b+1]) as rows x ceil(L_b/T)
 *            frames, rows in the order of the Phi layout above (S0 is one row).
 */
typedef struct jtfs_batch_s* jtfs_batch_t;

/*
 * Create a ragged batch of `count` clips (1 <= count, 1 <= lengths[b] <= 2^20);
 * other parameters as jtfs_plan.  flags: JTFS_PLAN_HOST_ONLY, and
 * JTFS_BATCH_REFLECT for the padding "on both sides" of §3.2 in place of
 * zeros on the right: each clip is mirrored (edge samples not repeated) over
 * P samples on each side, P = ceil(sqrt(ln(1000)/2) / (pi sigma_min)) with
 * sigma_min the narrowest Fourier width among the first- and second-order
 * filters and phi_T (where the slowest time envelope falls below 1e-3),
 * padded to n = next power of two >= L + 2P with p0 = T floor((n-L)/(2T))
 * samples on the left; Phi keeps the ceil(L/T) frames from frame p0/T on, and
 * the gradient sums every mirrored copy back onto its sample.  Padded lengths
 * must stay <= 2^20 (JTFS_ERR_SHAPE otherwise).  The unpooled flags are
 * refused (JTFS_ERR_ARG): the crop indexes Phi as rows x frames.  Errors as
 * jtfs_plan.
 */
#define JTFS_BATCH_REFLECT 2u
/* The same call under the name of a plan for clips of uneven lengths. */
int jtfs_plan_ragged(jtfs_batch_t* out, const int64_t* lengths, int count, int J,
                     int Q, int Q2, int J_fr, int Q_fr, int64_t T, int F,
                     uint32_t flags);
int jtfs_batch_create(jtfs_batch_t* out, const int64_t* lengths, int count, int J,
                      int Q, int Q2, int J_fr, int Q_fr, int64_t T, int F,
                      uint32_t flags);
int jtfs_batch_destroy(jtfs_batch_t batch);

/* Host arrays of count+1 offsets (may be NULL); returns the number of clips. */
int jtfs_batch_layout(jtfs_batch_t batch, int64_t* sample_off, int64_t* phi_off);

/* Bytes of device workspace the batch calls need (0 if batch is NULL). */
size_t jtfs_batch_workspace_bytes(jtfs_batch_t batch);

/* Phi of every clip (cropped), packed.  Errors as jtfs_forward. */
int jtfs_batch_forward(jtfs_batch_t batch, const float* x, float* phi,
                       void* workspace, void* stream);

/*
 * One Adam metamer step on every clip (as metamer_step), with the 1-based step
 * index read from, and then incremented in, device memory (`step`, one int32)
 * so that repeated calls can be recorded once and replayed.  y, adam_m, adam_v
 * are packed samples; loss [count] receives each clip's loss at the y given on
 * entry.  Errors as metamer_step.
 */
int jtfs_batch_metamer_step(jtfs_batch_t batch, float* y, const float* phi_target,
                            float* adam_m, float* adam_v, int32_t* step,
                            float lr, float* loss, void* workspace,
                            void* stream);

/*
 * Autotuning.  A plan has six execution choices that change no result
 * beyond rounding:
 *   choice[0]  wide column tiles (1) or narrow ones (0) for the second-order
 *              frequential forward kernel;
 *   choice[1]  time samples per CTA of the phi_T averaging forward
 *              (1024, 2048 or 4096);
 *   choice[2]  points per CTA of the batched small FFTs (1024 .. 8192);
 *   choice[3]  second-order frequential scattering of the path groups with at
 *              most 64 rows n1 on the tensor cores (1) or on the FFT kernels
 *              (0); reads 0, and setting 1 has no effect, for plans whose
 *              shape the tensor-core kernels do not handle (R_out not 16 or
 *              32, no such group);
 *   choice[4]  time pooling of the second order (dense groups) on the tensor
 *              cores (1) or on the FMA kernels (0); reads 0 for plans whose
 *              frame count (N / T) is not 32, 64 or 128.
 *   choice[5]  time-axis FFTs of the first and second layers (§3.2-§3.3) on
 *              the in-place radix-16 engine (1: every size up to 2^13 of a
 *              stage in one launch, 2^14 .. 2^16 on clusters of 2-8 CTAs
 *              exchanging through distributed shared memory) or on the
 *              batched / four-step kernels (0, which choice[2] tunes).
 * jtfs_set_tuning takes n = 3 .. 6 (later choices unchanged).
 * jtfs_autotune times jtfs_loss_grad on the caller's y and phi_target (device
 * arrays as for jtfs_loss_grad; loss [batch] and dy [batch][N] are scratch
 * outputs) for each candidate, one choice at a time, keeps the fastest, and
 * writes the choices to choice[0..n) (host, may be NULL).  It synchronises
 * the stream (it is a set-up call, not a hot-path one).  jtfs_set_tuning
 * applies saved choices; jtfs_get_tuning reads the current ones.  All return
 * the number of choices (6) or an error code.  Not thread-safe with concurrent
 * compute calls on the same plan.
 */
int jtfs_autotune(jtfs_plan_t plan, const float* y, const float* phi_target,
                  float* loss, float* dy, void* workspace, void* stream,
                  int64_t* choice, int n);
int jtfs_set_tuning(jtfs_plan_t plan, const int64_t* choice, int n);
int jtfs_get_tuning(jtfs_plan_t plan, int64_t* choice, int n);

/*
 * Learned initialiser layers.  The paper has no such network: it refines a
 * noise initialisation (Sec. 2.3); this decoder proposes the initial waveform
 * from the target's Phi instead.  A layer is a transposed 1-D convolution with
 * stride 2, kernel 9, padding 4 and output padding 1, mapping x [B][T][Ci] to
 * z [B][2T][Co] (activations channels-last):
 *   z[b][t][co] = bias[co] + sum over (ci, u, k) with t = 2u - 4 + k of x[b][u][ci] W[ci][co][k],
 * W [Ci][Co][9] float32 (the master copy).  BF16 tensors are uint16_t bit
 * patterns.  Hidden layers have Co = 128 and run on the tensor cores (BF16
 * operands, FP32 accumulation); the output layer (Ci = 128, Co = 1) runs on
 * the FMA units.  Input widths are padded to Cip = jtfs_convt_padded_channels(Ci)
 * (a multiple of 128) with zero channels.  All pointers are device pointers,
 * 16-byte aligned; calls are asynchronous on `stream`.
 *   jtfs_convt_pack_input      x [B][T][Cip] bf16 = phi [B][C][T] * row_scale[c] (zero for c >= C)
 *   jtfs_convt_pack_weights    wf [256][5 Cip] bf16, wf[(p, co)][(j, ci)] = W[ci][co][2j + p] (0 if 2j+p > 8);
 *                              wd [128][9 x 128] bf16, wd[ci][(k, co)] = W[ci][co][k] (only for Ci = 128;
 *                              may be NULL).  Call after every update of W.
 *   jtfs_convt_forward         z (float32, may be NULL) and h = GELU(z) (bf16, may be NULL) from x [B][T][Cip]
 *   jtfs_convt_backward_data   g_prev[b][u][ci] = (sum over k, co of g[b][2u-4+k][co] W[ci][co][k]) * GELU'(zprev[b][u][ci])
 *                              (the GELU' factor only when zprev != NULL), from g [B][2T][128] bf16;
 *                              writes float32 and/or bf16 (either may be NULL); Ci = Co = 128
 *   jtfs_convt_backward_weight dW [Ci][128][9] (float32) = sum over b, u of x[b][u][ci] g[b][2u-4+k][co],
 *                              split over positions with a fixed-order reduction; workspace of
 *                              jtfs_convt_weight_workspace_bytes(B, Cip, Co, T) bytes
 *   jtfs_convt_bias_grad       db [128] = column sums of g [rows][128] (float32); workspace of
 *                              jtfs_convt_bias_workspace_bytes(rows) bytes
 *   jtfs_convt_out_forward     y [B][2T] (float32) from x [B][T][128] bf16, w [128][1][9], bias [1]
 *   jtfs_convt_out_backward_data   as jtfs_convt_backward_data for the output layer, from dy [B][2T] float32
 *   jtfs_convt_out_backward_weight dw [128][1][9] and db [1] (db may be NULL); workspace of
 *                              jtfs_convt_out_workspace_bytes(B, T) bytes
 *   jtfs_decoder_error         1 if a tensor-core kernel gave up waiting on one of its barriers since the
 *                              last call (its outputs are then invalid), else 0; synchronous; clears the flag
 *   jtfs_cast_bf16             round-to-nearest float32 -> bf16
 *   jtfs_adam_update           Adam (0.9, 0.999, 1e-8, bias-corrected, 1-based step) on float32
 *                              parameters, also writing their bf16 copy if param_bf16 != NULL
 * Errors: JTFS_ERR_ARG (NULL pointer, unsupported width, misaligned pointer,
 * sizes < 1 or too large), JTFS_ERR_CUDA.
 */
int jtfs_convt_padded_channels(int C);
int jtfs_convt_pack_input(const float* phi, const float* row_scale, uint16_t* x,
                          int B, int C, int T, void* stream);
int jtfs_convt_pack_weights(const float* w, uint16_t* wf, uint16_t* wd, int Ci,
                            int Co, void* stream);
int jtfs_convt_forward(const uint16_t* x, const uint16_t* wf, const float* bias,
                       float* z, uint16_t* h, int B, int Cip, int Co, int T,
                       void* stream);
int jtfs_convt_backward_data(const uint16_t* g, const uint16_t* wd,
                             const float* zprev, float* g_prev,
                             uint16_t* g_prev_bf16, int B, int Ci, int Co,
                             int T, void* stream);
size_t jtfs_convt_weight_workspace_bytes(int B, int Cip, int Co, int T);
int jtfs_convt_backward_weight(const uint16_t* x, const uint16_t* g, float* dw,
                               int B, int Ci, int Cip, int Co, int T,
                               void* workspace, void* stream);
size_t jtfs_convt_bias_workspace_bytes(int64_t rows);
int jtfs_convt_bias_grad(const float* g, float* db, int64_t rows, int Co,
                         void* workspace, void* stream);
int jtfs_convt_out_forward(const uint16_t* x, const float* w, const float* bias,
                           float* y, int B, int Ci, int T, void* stream);
int jtfs_convt_out_backward_data(const float* dy, const float* w,
                                 const float* zprev, float* g_prev,
                                 uint16_t* g_prev_bf16, int B, int Ci, int T,
                                 void* stream);
size_t jtfs_convt_out_workspace_bytes(int B, int T);
int jtfs_convt_out_backward_weight(const uint16_t* x, const float* dy, float* dw,
                                   float* db, int B, int Ci, int T,
                                   void* workspace, void* stream);
int jtfs_decoder_error(void);
int jtfs_cast_bf16(const float* x, uint16_t* y, int64_t n, void* stream);
int jtfs_adam_update(float* param, const float* grad, float* m, float* v,
                     uint16_t* param_bf16, int64_t n, float lr, int step,
                     void* stream);

/*
 * Measurement hooks (host-side bookkeeping; not thread-safe).
 *
 * jtfs_profile_stage registers `count` CUDA events (cudaEvent_t passed as
 * void*, created by the caller) for one stage: every later launch of that
 * stage's kernel records events[2i] just before and events[2i+1] just after
 * it on the stream of the call, for i = 0, 1, ... until count/2 launches are
 * recorded.  events = NULL or count = 0 clears the registration.  Stages:
 */
#define JTFS_STAGE_FREQ2_FWD 0 /* second-order frequential scattering, modulus,
                                  phi_F averaging (§3.4, Eq. (5))           */
#define JTFS_STAGE_FREQ2_ADJ 1 /* its adjoint (§2.3, Eq. (7))                */
#define JTFS_STAGE_POOL_FWD  2 /* second-order phi_T averaging (Eq. (5))     */
#define JTFS_STAGE_POOL_ADJ  3 /* its adjoint (Eq. (6))                      */
#define JTFS_STAGE_FREQ2_FWD_TC 4 /* the tensor-core launches inside stage 0  */
#define JTFS_STAGE_FREQ2_ADJ_TC 5 /* the tensor-core launches inside stage 1  */
#define JTFS_STAGE_COUNT     6
int jtfs_profile_stage(jtfs_plan_t plan, int stage, void** events, int count);

/*
 * Number of kernel launches one call makes: call = 0 jtfs_forward,
 * 1 jtfs_backward, 2 jtfs_loss_grad (with gradient), 3 metamer_step.
 * Returns the count or JTFS_ERR_ARG.
 */
int64_t jtfs_launch_count(jtfs_plan_t plan, int call);

/*
 * Tensor-core second-order frequential scattering (§3.4, the modulus of
 * Eq. (2), phi_F of Eq. (5), and the adjoint of §2.3 / Eq. (7)).  Per time
 * column of a path group with n1max <= 64 rows, the filtering along n1 by
 * psi_beta (decimated by 2^k) is a product with a fixed complex matrix H_beta
 * [N_fr / 2^k][n1max] and the phi_F averaging after the modulus a product with
 * a fixed real matrix P_k [R_out][N_fr / 2^k]; the kernels run both on BF16
 * tensor cores with hi/lo-split operands and FP32 accumulation.
 *
 * jtfs_tc_error: 1 if a tensor-core frequential kernel gave up waiting on one
 * of its barriers since the last call (its outputs are then invalid), else 0;
 * synchronous; clears the flag.  JTFS_ERR_CUDA if the flag cannot be read.
 *
 * jtfs_tc_table copies, as float (hi + lo of the BF16 split), one of the
 * plan's operand tables into out[0 .. n) (host memory) and returns the number
 * of floats the table has (call with out = NULL to size it):
 *   which = 0: H, [rows][128]: row 2 (off_beta + r) + x, column 2 n + y holds
 *              the coefficient of (re, im)[y] of Y2[n] in (re, im)[x] of
 *              Z_beta[r], n < 64; off_beta = sum of N_fr / 2^k over earlier
 *              filters (filter order of the Phi layout);
 *   which = 1: P, [log2 F + 1][R_out][N_fr]: P_k[ro][r], zero for r >= N_fr / 2^k.
 * Works on host-only plans.  Errors: JTFS_ERR_ARG (NULL plan, bad which),
 * JTFS_ERR_SHAPE (the plan has no tensor-core groups).
 */
int jtfs_tc_error(void);
int64_t jtfs_tc_table(jtfs_plan_t plan, int which, float* out, int64_t n);
/*
 * jtfs_tc_error_info: the first tensor-core wait that expired since the last
 * call, as info[0 .. min(n, 4)): CTA index (-1: none), thread, byte offset of
 * the barrier in the CTA's shared memory, phase parity waited for.
 * Synchronous; clears the record; returns 4 or JTFS_ERR_CUDA.
 */
int jtfs_tc_error_info(int64_t* info, int n);

/*
 * jtfs_status -- the device-side status of every call enqueued on this
 * device since the previous jtfs_status: synchronises `stream` (void* as
 * elsewhere), then reads and clears the status word.
 *   JTFS_ERR_TIMEOUT    a tensor-core kernel (frequential scattering, time
 *                       pooling or decoder layer) gave up on a barrier wait;
 *                       the call that launched it produced invalid outputs.
 *   JTFS_ERR_NONFINITE  a loss (jtfs_loss_grad, metamer_step*, the batch
 *                       step) was NaN or infinite: §2.3's loss is finite for
 *                       finite inputs, so y or the target held NaN / Inf.
 *   JTFS_OK             neither.
 * TIMEOUT is reported in preference to NONFINITE.  The word is per device,
 * not per stream: a call on another stream that has not finished may set it
 * later.  Also clears what jtfs_tc_error / jtfs_decoder_error report.
 * JTFS_ERR_CUDA if the stream or the word cannot be read.
 */
int jtfs_status(void* stream);

/*
 * jtfs_set_wait_limit -- for tests of the error path: the number of polls
 * every later bounded barrier wait of the tensor-core kernels makes before
 * giving up (polls >= 0; 0 makes every such wait give up at once), or the
 * default bound (about 0.3 s) again for polls < 0.  Waits that drain copies
 * and MMAs before a CTA exits keep their full bound, so a kernel that gives
 * up still leaves no copy or MMA in flight.  Synchronous; affects every plan
 * on the current device.  Returns JTFS_OK or JTFS_ERR_CUDA.
 */
int jtfs_set_wait_limit(int64_t polls);

/* Static description of an error code (never NULL). */
const char* jtfs_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* JTFS_H */
