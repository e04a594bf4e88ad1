/*
 * cbessfm.h -- C-ABI of the GB300 (sm_103a) CB-ESSFM digital backpropagation library.
 *
 * The library implements the coupled-band enhanced split-step Fourier method of
 * "A New Twist on Low-Complexity Digital Backpropagation" (Civelli, Jana, Forestieri,
 * Secondini): overlap-and-save blocks (Sec. III-A, Fig. 2) of a dual-polarization field, two
 * full-band FFTs, a DEMUX into N_sb subbands, N_st steps of {GVD, NLPR} (Figs. 3-4) with the
 * nonlinear phase of Eq. (NLPR-multiband-2pol), asymmetric steps with splitting ratio rho
 * (Sec. III-C), a final GVD, MUX and two inverse FFTs.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units are SI.  A 4D sample is four float32 values (x.re, x.im, y.re, y.im), 16 bytes,
 *    16-byte aligned; a field is [batch][n_samples] such samples, contiguous.
 *  - The input is one period of a periodic sequence: overlap-and-save blocks wrap circularly.
 *  - Taps are the *effective* filter coefficients w[s][i][l][m + N_c] applied as
 *        theta_i[k] = sum_l sum_{m=-N_c}^{N_c} w[s][i][l][m + N_c] * P_l[(k - m) mod N']
 *    with P_l = |x_l|^2 + |y_l|^2 (the 3/2 XPM degeneracy factor of Eq. (NLPR-multiband-2pol)
 *    is folded into w[s][i][l] for l != i).  The rotation is exp(+j theta_i) on both
 *    polarizations and the GVD of subband bin f is exp(+j 2 pi^2 beta2 dz f^2) (Sec. III-A).
 *  - Device pointers are CUDA device addresses owned by the caller unless stated otherwise.
 *    The plan owns its device tables.  Every call is asynchronous on `stream` (a cudaStream_t;
 *    NULL is the legacy default stream) unless stated otherwise.
 *  - Errors: every call returns a cbessfm_status; nothing aborts and no C++ exception crosses
 *    the ABI.  cbessfm_last_error() returns a thread-local message for the last failure.
 *  - A plan is read-only during launches, so concurrent launches with one plan on different
 *    streams are safe; cbessfm_set_coeffs / cbessfm_set_ratio must not race with launches that
 *    use the plan.
 */
#ifndef CBESSFM_H_
#define CBESSFM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so this header does not need the CUDA headers. */
typedef struct CUstream_st* cbessfm_stream;

typedef enum {
    CBESSFM_OK = 0,
    CBESSFM_ERR_INVALID_ARG = 1,     /* a parameter is out of range or a pointer is NULL      */
    CBESSFM_ERR_UNSUPPORTED = 2,     /* valid, but not supported by this build (size limits)   */
    CBESSFM_ERR_ALIAS = 3,           /* output overlaps input                                  */
    CBESSFM_ERR_CUDA = 4,            /* a CUDA runtime call failed                             */
    CBESSFM_ERR_OOM = 5,             /* device or host allocation (or a host resource) failed  */
    CBESSFM_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up (see get_status)    */
    CBESSFM_ERR_NOT_IMPLEMENTED = 7
} cbessfm_status;

/* Fiber link being backpropagated (Sec. II-A, Eq. (NLSE); Sec. IV-A). */
typedef struct {
    double beta2;        /* group-velocity dispersion, s^2/m (e.g. -21.7e-27)                 */
    double gamma;        /* nonlinear coefficient, 1/(W m); informational (taps carry it)     */
    double alpha;        /* power attenuation, 1/m; informational (taps carry it)             */
    double span_length;  /* m                                                                 */
    int    n_spans;      /* link length = n_spans * span_length                               */
    double sample_rate;  /* full-band sampling rate R, Hz                                     */
} cbessfm_link;

typedef enum {
    CBESSFM_C64 = 0,     /* complex64 input/output (float4 per 4D sample)                    */
    CBESSFM_F16x4 = 1,   /* four fp16 per 4D sample, FP32 arithmetic inside                 */
    CBESSFM_BF16x4 = 2   /* four bf16 per 4D sample, FP32 arithmetic inside                 */
} cbessfm_storage;

typedef struct cbessfm_plan cbessfm_plan;

/*
 * cbessfm_plan_create -- build a DBP plan (Sec. III-A; asymmetric steps Sec. III-C).
 *   link      host pointer to the link description; L_step = n_spans * span_length / steps.
 *   bands     N_sb >= 1 subbands.
 *   steps     N_st >= 0 steps (0 = dispersion compensation over the whole link, EDC).
 *   ratio     splitting ratio rho in [0, 1]: first GVD (1 - rho) L_step, interior GVDs L_step,
 *             last GVD rho L_step.
 *   coeffs    host float array [steps][bands][bands][ntaps] of effective taps (may be NULL when
 *             steps == 0); copied into the plan.
 *   ntaps     2 N_c + 1, odd, 1 <= ntaps <= n_fft / 2.
 *   n_fft     N' = per-subband FFT size, a power of two in [16, 2048]; block N = bands * N'.
 *   overlap   N'_ov = per-subband overlap, even, 0 <= overlap < n_fft; N_ov = bands * N'_ov
 *             samples are shared by neighbouring blocks, N_ov / 2 dropped on each side
 *             (Sec. III-A, Fig. 2).
 *   storage   sample storage type of in/out.
 *   out       receives the plan.
 * Synchronous.  Builds the FP64-derived tables (GVD phases reduced modulo 2 pi, FFT twiddles)
 * on the current device.  Returns INVALID_ARG for out-of-range values, UNSUPPORTED when the
 * block does not fit one SM's shared memory: complex64 plans take up to 5 subbands at
 * n_fft = 1024 or 2048, 10 at 512 and 16 at 256 or less, for any ntaps.  These checks run
 * before the first CUDA call.
 */
cbessfm_status cbessfm_plan_create(const cbessfm_link* link, int bands, int steps, double ratio,
                                   const float* coeffs, int ntaps, int n_fft, int overlap,
                                   cbessfm_storage storage, cbessfm_plan** out);

/* Release the plan and its device tables.  Synchronous; NULL is accepted. */
cbessfm_status cbessfm_plan_destroy(cbessfm_plan* plan);

/*
 * cbessfm_set_coeffs -- replace the taps (layout as in plan_create).
 *   on_device = 0: `coeffs` is a host array (the call synchronizes the copy);
 *   on_device = 1: a device array, copied asynchronously on `stream`.
 */
cbessfm_status cbessfm_set_coeffs(cbessfm_plan* plan, const float* coeffs, int on_device,
                                  cbessfm_stream stream);

/* cbessfm_set_ratio -- change rho (Sec. III-C); rebuilds the first and last GVD tables with an
 * FP64 kernel on `stream`. */
cbessfm_status cbessfm_set_ratio(cbessfm_plan* plan, double ratio, cbessfm_stream stream);

/*
 * cbessfm_backpropagate -- run the DBP chain (Sec. III-A) on `batch` independent sequences.
 *   in, out    device arrays [batch][n_samples] 4D samples in the plan's storage type; out
 *              must not overlap in (ALIAS).
 *   n_samples  L >= 1 samples per sequence (one period); any length, blocks wrap circularly.
 * One kernel launch: each CTA stages its overlap-and-save blocks into shared memory and runs
 * the whole chain on chip.  Staging uses bulk copies of the Tensor Memory Accelerator, except
 * that 16-bit samples use coalesced loads where a copy would not start on a 16-byte boundary
 * (odd L or an odd block start).
 * Errors: INVALID_ARG for a NULL plan or buffer, in/out not 16-byte aligned, or n_samples or
 * batch < 1; ALIAS when out overlaps in; UNSUPPORTED beyond 2^31 - 1 blocks in one call; CUDA
 * when the launch fails.  A bounded in-kernel wait that gives up is reported later by
 * cbessfm_get_status.
 */
cbessfm_status cbessfm_backpropagate(const cbessfm_plan* plan, const void* in, void* out,
                                     int64_t n_samples, int batch, cbessfm_stream stream);

/*
 * Differentiation form.  The paper fits its taps offline with finite-difference gradients
 * (Sec. III-B); these calls give the exact gradient of a real loss L with respect to every
 * step's taps, the splitting ratio and the input, so the taps and rho can be trained on the
 * device.  Gradient convention for complex data: G = dL/dRe + j dL/dIm, stored like a
 * complex64 field.  Plans with 16-bit storage take and return their input and output fields in
 * that storage; the checkpoints, grad_out and grad_in are complex64 for every storage type (the
 * forward widens its input into the workspace and narrows its complex64 result into `out`, so
 * the gradients are those of the chain at the storage-rounded input).
 *
 * cbessfm_grad_workspace_size -- bytes of device workspace (caller-allocated, 256-byte aligned)
 *   holding, per overlap-and-save block, n_steps + 2 checkpoints of the block's field, two
 *   block-sized scratch fields of the adjoint and the per-block partial gradients, and for
 *   16-bit plans two complex64 copies of the whole input/output.
 */
cbessfm_status cbessfm_grad_workspace_size(const cbessfm_plan* plan, int64_t n_samples, int batch,
                                           size_t* bytes);

/*
 * cbessfm_backpropagate_checkpointed -- cbessfm_backpropagate that also stores, in `workspace`,
 * the spectrum after the first GVD, each step's time samples before its rotation and the
 * spectrum after the last GVD of every block (the adjoint recomputes the rest of each step).
 */
cbessfm_status cbessfm_backpropagate_checkpointed(const cbessfm_plan* plan, const void* in, void* out,
                                                  int64_t n_samples, int batch, void* workspace,
                                                  size_t ws_bytes, cbessfm_stream stream);

/*
 * cbessfm_grad -- adjoint of the checkpointed forward whose workspace is passed (same plan, taps,
 * ratio, n_samples and batch; the workspace must not have been reused in between).
 *   grad_out     device [batch][n_samples] G of the output (kept samples; gradient is zero on
 *                samples the forward did not produce).
 *   grad_coeffs  device double [steps][bands][bands][ntaps]: dL/dw, summed over blocks in FP64.
 *   grad_ratio   device double scalar dL/drho, or NULL.
 *   grad_in      device [batch][n_samples] G of the input (overwritten), or NULL.
 * Per block the adjoint walks the steps backwards: conjugate GVD, inverse transforms, and the
 * adjoint of the rotation, the coupled-band FIR (transposed taps) and the intensity.  dL/drho
 * (the ratio enters only the first and the last GVD, Sec. III-C) is accumulated as one term per
 * step built from exp(j theta) - 1, which keeps its FP32 error at the level of the other
 * gradients on long links where the two end terms nearly cancel.  With the per-polarization NLPR
 * (cbessfm_set_nlpr_mode, Eqs. (NLPR_polx/poly)) the phase gradients of the two polarizations
 * enter as their sum S and difference D: the FIR adjoint runs over S with all taps and over D
 * with the coupling taps (i != l) at 1/3, and the tap gradient adds sum_k D_i[k] (Px_l -
 * Py_l)[k - m] / 3 for i != l; the plan's mode must be the one of the checkpointed forward.
 */
cbessfm_status cbessfm_grad(const cbessfm_plan* plan, const void* grad_out, double* grad_coeffs,
                            double* grad_ratio, void* grad_in, void* workspace, size_t ws_bytes,
                            int64_t n_samples, int batch, cbessfm_stream stream);

/*
 * Batched form: many independent jobs, each with its own plan (subbands, steps, taps, N',
 * overlap, storage), input, output and length, in one persistent launch per group of jobs that
 * share N', the subband count and the storage type.  Within a group, CTAs claim work items of
 * consecutive overlap-and-save blocks from a device counter, longest jobs first.
 */
typedef struct {
    const cbessfm_plan* plan;   /* plan of this job; must outlive the batch                      */
    const void* in;             /* device [n_samples] samples in the plan's storage type          */
    void* out;                  /* device [n_samples]; must not overlap in                        */
    int64_t n_samples;          /* one period of this job's sequence                              */
} cbessfm_job;

typedef struct cbessfm_batch cbessfm_batch;

/*
 * cbessfm_batch_create -- validate the jobs, build and upload the work list.  Synchronous.
 * The batch owns its device descriptors (allocated here).  Job buffers are referenced, not
 * copied: run() processes whatever they hold at the time.  Every job's plan must have been
 * created on the current device, where the batch then runs (else CBESSFM_ERR_INVALID_ARG).
 */
cbessfm_status cbessfm_batch_create(const cbessfm_job* jobs, int njobs, cbessfm_batch** out);

/*
 * cbessfm_batch_run -- process every job: one counter reset and one persistent kernel per group,
 * asynchronous on `stream`.  The groups after the first run on streams the batch owns, forked
 * from `stream` and joined back into it by events, so one group's CTAs take over the SMs that
 * another group's finished CTAs free; the call returns with all of them ordered before later
 * work on `stream`.  It issues no host synchronization and no allocation, so it can be captured
 * into a CUDA graph and replayed.
 */
cbessfm_status cbessfm_batch_run(const cbessfm_batch* batch, cbessfm_stream stream);

/* Number of launch groups and work items of the batch. */
cbessfm_status cbessfm_batch_info(const cbessfm_batch* batch, int* n_groups, long long* n_items);

/* Release the batch (synchronizes the device first).  NULL is accepted. */
cbessfm_status cbessfm_batch_destroy(cbessfm_batch* batch);

/*
 * cbessfm_batch_run_noalloc -- the batched form for callers that cannot allocate device memory
 * when they run, e.g. a receiver's real-time DSP thread that must not wait on the allocator, a
 * process whose device memory is reserved up front and capped, or a plugin host that forbids
 * allocation inside its callbacks.  The paper has no counterpart: this is a deployment variant
 * of cbessfm_batch_run, computing the same chain with the same per-block arithmetic.
 *   jobs, njobs  as for cbessfm_batch_create; 1 <= njobs <= 64, all jobs with the same n_fft and
 *                bands and complex64 storage (else CBESSFM_ERR_UNSUPPORTED with a message);
 *                in/out are the caller's device buffers; every job's plan must have been
 *                created on the current device (else CBESSFM_ERR_INVALID_ARG).
 * The work list and counter live in one static device array of 21,248 bytes that every
 * GPU loading the library holds until exit; nothing is allocated by the call.  The first call on
 * a device looks up that array's device address and sets the kernel's shared-memory limit, so
 * make the first call before any stream capture.  The descriptors are copied from host stack
 * memory with cudaMemcpyAsync, so each call blocks the calling thread until the stream's
 * earlier work has finished; a caller that must not wait uses cbessfm_batch_create / _run.  All
 * calls share the array and it keeps the last call's contents (the call clears the counter
 * itself): calls that overlap on the GPU, from two streams or two threads, race and must be
 * ordered by the caller.  A staging wait that runs out (cbessfm_set_wait_limit) is reported,
 * as for cbessfm_batch_run, by cbessfm_get_status on the job's plan, not by this call's return.
 */
cbessfm_status cbessfm_batch_run_noalloc(const cbessfm_job* jobs, int njobs,
                                         cbessfm_stream stream);

/*
 * cbessfm_analytic_taps -- the CB-ESSFM coefficients of Sec. II-D, for use as plan taps.
 * For every subband separation d = l - i and tap m in [-N_c, N_c]:
 *   c_d[m] = (1/R'^2) double integral over mu, nu in [d R' - R'/2, d R' + R'/2] of
 *            K(mu, nu) exp(j 2 pi (mu - nu) m / R')        (Eq. ESSFM_coefficients_general, P = 1)
 * with R' = sample_rate / bands and the closed-form Volterra kernel of one step
 * (Eq. kernel_analytic) built from link->beta2, link->gamma and link->alpha (1/m, power), the
 * step length L = n_spans * span_length / steps and spans_per_step identical spans per step.
 * The double integral is a grid x grid midpoint rule, evaluated in FP64 on the current device.
 *   spans_per_step  1 for a step of one span or less (the step then starts at power
 *                   step_power[s] and decays over L); k > 1 for steps of k whole spans
 *                   (steps * k must equal n_spans).
 *   step_power      host [steps]: the reference power P of each step, in the units in which the
 *                   field's |u|^2 is given (1 for a field already in sqrt(W) at a span start).
 *   ntaps           odd, <= 1023; grid in [ntaps, 4096] (quadrature points per axis).
 *   taps            host out [steps][bands][bands][ntaps]: effective taps
 *                   w[s][i][l][m + N_c] = step_power[s] Re c_{l-i}[m], times 3/2 for l != i
 *                   (Eq. NLPR-multiband-2pol); the NLPR is a real phase, so the real part is kept.
 *   response        host out [2 bands - 1][ntaps][2] (re, im) of c_d[m] for d = -(bands-1) ..
 *                   bands-1, or NULL.
 * Synchronous (allocates and frees a small device buffer).  The paper also fits the taps
 * numerically (Sec. III-B); these analytic ones are the starting point for that.
 */
cbessfm_status cbessfm_analytic_taps(const cbessfm_link* link, int bands, int steps,
                                     int spans_per_step, const double* step_power, int ntaps,
                                     int grid, double* taps, double* response);

/*
 * cbessfm_backpropagate_host -- cbessfm_backpropagate of fields in host memory, with the
 * transfers overlapped.  The batch is copied into `dev_in` in groups of realizations (at most 64
 * groups) on a host-to-device stream; the chain kernel runs in launches of
 * `launch_blocks` OLS blocks of the flattened (realization, block) list, each launch waiting
 * only for the groups it reads; each group is copied from `dev_out` to `host_out` on a
 * device-to-host stream once its last block is computed.  The copy streams and the second
 * compute stream are owned by the plan (created at the first call).  The paper has no counterpart; the chain and its result are
 * those of cbessfm_backpropagate, bit for bit.
 *   host_in, host_out  [batch][n_samples] samples in the plan's storage type; page-locked
 *                      memory (cudaHostAlloc / pinned tensors) lets the copies overlap.
 *   dev_in, dev_out    device buffers of the same size (caller-owned, must not overlap).
 *   launch_blocks      OLS blocks per launch, rounded up to whole CTAs of the plan; 0 = one
 *                      CTA per SM per launch, the launches alternating between `stream` and a
 *                      second compute stream owned by the plan so that two are in flight
 *                      (with CBESSFM_PIPELINE_STREAMS=1 in the environment: all launches on
 *                      `stream`, one wave of resident CTAs first and two waves after).
 * Asynchronous: completion is ordered on `stream` (synchronize it before reading host_out).
 * Calls on one plan are serialized on the host; concurrent calls with one plan wait for each
 * other's enqueueing, not for the device.  Errors: CBESSFM_ERR_INVALID_ARG for NULL buffers,
 * n_samples or batch < 1, launch_blocks < 0, or realizations that do not span a multiple of
 * 16 bytes (batch > 1); the checks of cbessfm_backpropagate otherwise.
 */
cbessfm_status cbessfm_backpropagate_host(cbessfm_plan* plan, const void* host_in, void* host_out,
                                          void* dev_in, void* dev_out, int64_t n_samples,
                                          int batch, int launch_blocks, cbessfm_stream stream);

/*
 * Streamed form (per-step overlap-and-save).  The chain's operators are regrouped into one
 * pass per step over the whole sequence: pass s runs [GVD((1 - rho) L_step), for s = 0 only],
 * the step's NLPR, and GVD(L_step) (GVD(rho L_step) for the last step), each pass with its own
 * overlap-and-save blocks of the plan's N and N_ov (DEMUX and MUX inside every block, as in
 * cbessfm_backpropagate), the field going through device memory between passes.  A pass's
 * overlap must then cover one step's dispersion, not the whole link's; the price is N_st
 * launches and N_st reads and writes of the field.  The paper runs the whole chain per block;
 * this form computes the same operator sequence with a different block decomposition, so the
 * two agree where both overlaps cover their memory.
 * cbessfm_streamed_workspace_size -- bytes of device workspace for the intermediate fields
 *   (0, 1 or 2 fields of n_samples * batch complex64 4D samples, each rounded up to 256 bytes;
 *   2 for 16-bit plans from two steps on).
 * cbessfm_backpropagate_streamed -- in, out and workspace must not overlap; asynchronous on
 *   `stream`.  With steps <= 1 it is cbessfm_backpropagate.  The fields between passes are
 *   complex64 for every storage type: a 16-bit plan's input is widened into the workspace
 *   first and the last pass's result is narrowed (round to nearest) into `out`.
 */
cbessfm_status cbessfm_streamed_workspace_size(const cbessfm_plan* plan, int64_t n_samples,
                                               int batch, size_t* bytes);
cbessfm_status cbessfm_backpropagate_streamed(const cbessfm_plan* plan, const void* in, void* out,
                                              void* workspace, size_t ws_bytes, int64_t n_samples,
                                              int batch, cbessfm_stream stream);

/*
 * cbessfm_set_nlpr_mode -- 0 (default): the NLPR of Eq. (NLPR-multiband-2pol), one phase for
 * both polarizations of a subband (intensity |x|^2 + |y|^2, XPM weighted by the effective taps).
 * 1: the full-complexity form of Eqs. (NLPR_polx), (NLPR_poly), a phase per polarization with
 * co-polarized XPM twice as effective as cross-polarized XPM.  The taps keep their meaning
 * (w_il = (3/2) c_il for l != i), so with equal intensities in x and y both forms agree; the
 * FIR index is [k - m] in both.  The per-polarization form needs shared memory for a second set
 * of intensity rows: CBESSFM_ERR_UNSUPPORTED (plan unchanged) if they do not fit, and for
 * FP16/BF16 storage.  cbessfm_batch_* and the gradients run both modes (the per-polarization
 * adjoint needs further rows of shared memory: CBESSFM_ERR_UNSUPPORTED from
 * cbessfm_backpropagate_checkpointed / cbessfm_grad where they do not fit, e.g. 5 subbands of
 * N' = 1024); cbessfm_batch_run_noalloc supports mode 0 only.  Synchronous with respect to the
 * host, not to the device: do not call while launches of the plan are in flight.
 */
cbessfm_status cbessfm_set_nlpr_mode(cbessfm_plan* plan, int per_polarization);

/*
 * cbessfm_set_wait_limit -- bound of the forward chain kernels' waits for the bulk copies (TMA)
 * that stage each overlap-and-save block into shared memory, in SM clock cycles.  No part of the
 * paper: a guard against a copy that never completes.  cycles > 0: the bound; 0: one
 * non-blocking test per wait; < 0: the default (4e9 cycles, about 2 s, never reached by a live
 * copy).  A wait that runs out sets bit 0 of the plan's status word (cbessfm_get_status then
 * returns CBESSFM_ERR_TIMEOUT); the CTA then waits, with the default bound, for its copies in
 * flight to land and returns without writing its blocks' output.  Applies to launches made
 * after the call (plain, host-pipelined, streamed, checkpointed, and batches created after it).
 * Synchronous with respect to the host; CBESSFM_ERR_INVALID_ARG for a NULL plan.
 */
cbessfm_status cbessfm_set_wait_limit(cbessfm_plan* plan, long long cycles);

/*
 * cbessfm_get_status -- synchronize `stream`, then read and clear the plan's device status word
 * (bit 0: a bounded wait for a shared-memory copy gave up -> CBESSFM_ERR_TIMEOUT).
 */
cbessfm_status cbessfm_get_status(const cbessfm_plan* plan, cbessfm_stream stream);

/*
 * cbessfm_measure_fp32_peak -- a measurement utility, not an operation of the paper: the FP32
 * fused multiply-add rate of the current device, the denominator of the chain kernels' ALU
 * roofline.  A kernel of independent FFMA chains fills every SM (2048 threads each) and is
 * timed with CUDA events on `stream`; *flops = 2 x FFMA lane operations per second of the
 * fastest of `repeats` launches (1..1000; one untimed launch runs first), *sm_count = the
 * device's SM count.  Synchronous: it waits for `stream`.  CBESSFM_ERR_INVALID_ARG for NULL
 * outputs or repeats out of range, CBESSFM_ERR_CUDA if a launch or event call fails.
 */
cbessfm_status cbessfm_measure_fp32_peak(int repeats, double* flops, int* sm_count,
                                         cbessfm_stream stream);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char* cbessfm_last_error(void);

/* Library version string. */
const char* cbessfm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CBESSFM_H_ */
