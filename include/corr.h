/*
 * corr.h -- C ABI of gbcorr, an FX spectral correlator for one GB300 GPU.
 *
 * The method is the software spectral correlator of Prasad & Subrahmanya
 * ("Software Spectral Correlator for the 44-Element Ooty Radio Telescope"):
 * every antenna's real sample stream is transformed to spectral channels by
 * an FFT (the F-engine), and for every channel every pair of antennas is
 * cross-multiplied and accumulated to the required cadence (the X-engine),
 * giving the cross power spectra (Sec. 1 of the paper).
 *
 * Conventions shared by every call
 * --------------------------------
 *  N       antennas (elements), 1 <= N <= CORR_MAX_N.
 *  K       transform length in real samples, a power of two in [16, 4096];
 *          the paper uses K = 512 (Sec. 4).
 *  C       = K/2 channels, k = 0 .. K/2-1: DC kept, the Nyquist bin dropped
 *          (Sec. 1: K channels per 2K-point transform).
 *  P       = N(N+1)/2 outputs per channel: every pair i <= j including the
 *          autocorrelations, in row-major upper-triangle order,
 *          p(i, j) = i*N - i*(i-1)/2 + (j - i).
 *
 *  Input samples: 4-bit two's-complement integers in [-8, 7], two per byte,
 *  the earlier sample in the low nibble (Sec. 1: 4-bit quantisation).  Bytes
 *  are grouped in frames of K samples of *every* antenna (Sec. 2.2: a frame
 *  holds contiguous samples from all elements): layout
 *  [n/K frames][N antennas][K/2 bytes], frame-major.
 *
 *  Transform: X_i[s,k] = sum_{n<K} x_i[s*K+n] exp(-2 pi i k n / K), forward
 *  and unnormalised (Sec. 4).  Optional correction (Sec. 2.1):
 *  Y_i[s,k] = g_i exp(-2 pi i k tau_i / K) X_i[s,k] -- a complex gain g_i and
 *  a delay tau_i (samples, any real value) applied to antenna i.
 *
 *  Output: V_ij[k] = sum_s Y_i[s,k] conj(Y_j[s,k]), the raw sum over the
 *  n_spec spectra pushed since the last dump (divide by n_spec for a mean),
 *  laid out [P][C] as interleaved complex (re, im).
 *
 * Memory, streams and errors
 * --------------------------
 *  Pointers may be host or device memory unless stated otherwise; the
 *  library detects which.  The caller owns every buffer it passes; the handle
 *  owns its workspaces.  Work is queued on the handle's stream (its own
 *  non-blocking stream unless corr_set_stream gave another).  corr_push
 *  returns once its work is queued; a device input buffer must stay valid
 *  and unchanged until the next corr_dump or corr_sync.  (The F-engine
 *  launches of consecutive pushes alternate between two internal streams,
 *  each starting after the work queued on the handle's stream before its
 *  push; the handle's stream waits for them before the X-engine, a dump or
 *  any call that changes what they read.)  Every call returns CORR_OK or a
 *  negative corr_status; on error the accumulated state is unchanged unless
 *  stated, and corr_last_error(h) returns a one-line message (for errors of
 *  corr_create, call corr_last_error(NULL) on the same thread).  One handle
 *  must not be used from two host threads at once.
 */
#ifndef GBCORR_CORR_H
#define GBCORR_CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CORR_MAX_N 512

typedef struct corr_s* corr_t;

/* X-engine input precision. */
enum corr_dtype {
    /* FP32-accurate: the F-engine splits each spectrum value, pre-scaled by a
       power of two per antenna, into two FP16 terms hi + lo (~22 significant
       bits); the X-engine runs on the tensor cores (kind::f16, hi hi^T +
       hi lo^T + lo hi^T, FP32 accumulation) and divides the scale out. */
    CORR_FP32 = 0,
    /* Spectra scaled per (antenna, channel) and cast to FP16 / FP8-E4M3 before
       the tensor-core X-engine; FP32 accumulation; descaled at the flush.
       This is the paper's float-to-short-complex conversion with prescaling
       (Sec. 4) moved to tensor-core types. */
    CORR_FP16 = 1,
    CORR_FP8E4M3 = 2,
    /* FP32 spectra and an FP32 X-engine on the CUDA cores (no tensor cores). */
    CORR_FP32_SIMT = 3
};

enum corr_status {
    CORR_OK = 0,
    CORR_EINVAL = -1,    /* bad argument or size                          */
    CORR_ENOMEM = -2,    /* device or host allocation failed              */
    CORR_ECUDA = -3,     /* a CUDA call failed (message has the CUDA error) */
    CORR_ETIMEOUT = -4,  /* a bounded device-side wait gave up            */
    CORR_ESTATE = -5,    /* call not valid in the handle's current state  */
    CORR_EUNSUPPORTED = -6 /* valid request this build cannot serve       */
};

/* Create a correlator for N antennas, K-point transforms and X-engine
 * precision dtype.  Allocates the workspaces on the current CUDA device.
 * *out is set to NULL on failure. */
int corr_create(corr_t* out, int N, int K, int dtype);

/* Queue later work on `stream` (a cudaStream_t of the handle's device; NULL
 * means the legacy default stream).  Waits for the handle's queued work
 * first. */
int corr_set_stream(corr_t h, void* stream);

/* Capacity of the spectra workspace in frames, rounded up to a multiple of
 * 128; default 8192 (halved while the workspace would exceed 2 GiB, not below
 * 2048).  Pushes are transformed by the F-engine as they arrive and collected
 * in the workspace; the X-engine runs when it is full, at a push whose frame
 * count is not a multiple of 128, and at corr_dump / corr_sync.  Reallocates
 * the workspace; only valid with nothing pushed since the last dump. */
int corr_set_chunk(corr_t h, int64_t max_spectra);

/* Tile choices of the tensor-core X-engine (no counterpart in the paper; the
 * autotuner in paper_1102_0148_gb300/tune.py picks them): `window` = spectra
 * accumulated in TMEM before the epilogue adds them up in FP32 (a multiple
 * of 32, of 128 for FP8; 0 = 256 in FP32 mode, 512 for FP16
 * (1024 above 64 antennas), 2048 for FP8), `stages` = depth of the shared-memory
 * operand ring (2..16, clipped to what shared memory holds; 0 = automatic),
 * `split` = ranges of spectra per channel and antenna-block pair into which
 * a pass is cut (1..64, partials combined in a fixed order inside the
 * launch; 0 = chosen by the planner), `atoms` = k-tiles (32 spectra, 128 for
 * FP8) carried by one pipeline stage (1..8; 0 = as many as leave three
 * stages, up to 256 spectra).  The window is rounded up to whole stages.  CORR_EINVAL for
 * CUDA-core handles or out-of-range values. */
int corr_set_tiles(corr_t h, int window, int stages, int split, int atoms);

/* Per-antenna corrections of Sec. 2.1.  gains: N complex values as 2N floats
 * (re, im); delays: N floats, in samples.  Either may be NULL (gain 1,
 * delay 0); both NULL switches corrections off.  Host or device memory; the
 * values are copied before return.  Takes effect for spectra pushed later.
 * Every gain must be finite with |g| = 0 or 2^-40 <= |g| <= 2^40, every
 * delay finite; otherwise CORR_EINVAL and nothing changes.  (In CORR_FP32
 * mode each antenna's spectra enter the FP16 planes pre-scaled by the power
 * of two sigma_i = 2^floor(log2(2^15 / (8 K |g_i|))), which bounds every
 * scaled value by 2^15 for any 4-bit input and is divided out exactly; when
 * the gains change sigma, frames already pushed are cross-multiplied first.) */
int corr_set_corrections(corr_t h, const float* gains, const float* delays);

/* Pre-cast scales of a CORR_FP16 / CORR_FP8E4M3 handle (Sec. 4: the
 * conversion to a narrower type is preceded by prescaling).  Spectrum Y_i[k]
 * enters the tensor cores as s_i[k] Y_i[k]; every visibility is divided by
 * s_i[k] s_j[k] before it is accumulated, so the scales change only the
 * rounding, never the expected value.  By default the library picks the
 * power of two nearest (in log2) to t / sqrt(P_i[k] / 2), P = mean |Y|^2,
 * t = 64 (FP16) or 16 (FP8):
 * P from a 256-frame estimation pass before the first push, then from the
 * autocorrelations V_ii[k] / n_spec of each dumped integration.
 * corr_set_scales: `scales` = [N][C] floats (host or device) fixes the scales
 * until corr_set_scales(h, NULL) returns to the automatic choice.
 * corr_get_scales: copy the current scales to `scales` ([N][C] floats);
 * CORR_ESTATE before any are known.  Both: CORR_EINVAL on other dtypes. */
int corr_set_scales(corr_t h, const float* scales);
int corr_get_scales(corr_t h, float* scales);

/* Coarse delay tracking (the streaming form's integer sample shift; the
 * paper only mentions a phase correction before accumulation, Sec. 2.1):
 * every later push correlates y_i[t] = x_i[t - delays[i]] instead of x_i,
 * t counting the samples of the stream pushed into this handle.  delays: N
 * int32 in [0, K] (host or device), NULL or all zero = off.  The samples
 * before a push come from the end of the previous one (the stream's history,
 * carried on the device and in corr_save_state); when the delays are turned
 * on the history starts from zeros.  Frames already pushed keep the old
 * delays.  corr_grad applies them to its own samples from a zero history;
 * batches (corr_batch_*) reject handles with delays set (CORR_EINVAL). */
int corr_set_sample_delays(corr_t h, const int32_t* delays);

/* Correlate n samples per antenna (n a multiple of K, n >= 0) and add them
 * to the running integration.  `samples` holds n/K frames in the layout
 * above (n*N/2 bytes).  Host memory is staged through the handle's pinned
 * buffers; device memory is read in place.  With the fused F/X-engine on
 * (corr_set_fused) device-memory pushes are recorded and queued as one
 * launch at the next corr_dump, corr_dump_async, corr_sync or call that
 * changes what they read (or when 262144 frames wait); their buffers must
 * stay valid until then, as for every device push. */
int corr_push(corr_t h, const uint8_t* samples, int64_t n);

/* Fused F/X-engine (no counterpart in the paper's two-core design, Sec. 3):
 * for K = 512, CORR_FP32 and N <= 44 the transform and the cross-multiply
 * run as one persistent kernel per run of device-memory pushes, every SM
 * holding F-engine and X-engine warps, the spectra passed through a ring of
 * workspace slots that stays in L2 instead of a workspace in HBM.  Off by
 * default: on a GB300 at N = 44 the separate F- and X-engine launches are
 * faster (2.35 against 3.65 ms per 1 s integration at 35 MS/s).
 * corr_set_fused(h, 1) turns it on (allocating its ~69 MB ring on the first
 * call), CORR_EUNSUPPORTED where it is not served (other K, N or dtype, or a
 * device without cooperative launches); (h, 0) turns it off.  Pushes from
 * host memory, corr_grad and handles with sample delays use the separate
 * launches.  corr_get_fused: *on = 1 when device pushes go to the fused
 * launch. */
int corr_set_fused(corr_t h, int on);
int corr_get_fused(corr_t h, int* on);

/* Finish the integration: write V to `vis` ([P][C] complex64, or complex128
 * when vis_fp64 != 0), store the number of spectra summed in *n_spec (may be
 * NULL), and reset the accumulators.  Synchronises the handle's stream.
 * Accumulation across pushes is in FP64 on the device. */
int corr_dump(corr_t h, void* vis, int64_t* n_spec, int vis_fp64);

/* As corr_dump, but queued on the handle's stream without waiting for it
 * (no counterpart in the paper: it lets a streaming caller start pushing the
 * next integration while this one is still being reduced and copied out).
 * `vis` must be device memory or page-locked host memory (CORR_EINVAL
 * otherwise); it is complete once corr_sync (or a later corr_dump) returns,
 * and must not be read or reused before that.  *n_spec is set at once.  A
 * device-side error of the queued work is reported by that later call. */
int corr_dump_async(corr_t h, void* vis, int64_t* n_spec, int vis_fp64);

/* Wait for the handle's queued work; reports device-side errors. */
int corr_sync(corr_t h);

/* Release everything the handle owns.  NULL is a no-op. */
void corr_destroy(corr_t h);

/* Message of the last failed call on h (or, when h is NULL, of this thread's
 * last failed corr_create or corr_correlate_noalloc).  Never NULL; valid
 * until the next call. */
const char* corr_last_error(corr_t h);

/* Sizes of a handle: any pointer may be NULL. */
int corr_info(corr_t h, int* N, int* K, int* C, int* P, int* dtype);

/* Gradient of a real loss L(V) with respect to the per-antenna gains and
 * delays applied in the F-engine (Sec. 2.1), at (gains, delays) -- N complex
 * values as 2N floats and N floats, NULL meaning 1 and 0 -- for the
 * visibilities of `samples` (n samples per antenna, layout as corr_push).
 * grad_vis = dL/dRe V + i dL/dIm V, [P][C] complex64 (grad_fp64 = 0) or
 * complex128 (PyTorch's convention for complex tensors).  Writes
 * grad_gains = dL/dRe g + i dL/dIm g (2N floats) and grad_delays = dL/dtau
 * (N floats).  Every buffer may be host or device memory.
 * The uncorrected visibilities R are recomputed from the samples pass by pass
 * (spectra are never stored) into a separate accumulator, so the running
 * integration is untouched; then V_ij = a_i conj(a_j) R_ij gives the
 * gradient in closed form, in FP64.  Synchronises the handle's stream. */
int corr_grad(corr_t h, const uint8_t* samples, int64_t n, const float* gains,
              const float* delays, const void* grad_vis, int grad_fp64, float* grad_gains,
              float* grad_delays);

/* Checkpoint / resume of a running integration (no counterpart in the
 * paper).  corr_state_bytes: size of the state; corr_save_state waits for
 * the handle's work and copies its FP64 accumulators, spectrum count and
 * (FP16 / FP8) scales into the host buffer `buf`; corr_load_state restores
 * them into a handle of the same N, K and dtype (CORR_EINVAL otherwise), so
 * pushing the rest of the integration and dumping gives what one handle
 * would have given. */
int corr_state_bytes(corr_t h, size_t* bytes);
int corr_save_state(corr_t h, void* buf);
int corr_load_state(corr_t h, const void* buf);

/* Allocation-failure test hook (no counterpart in the paper): every device
 * allocation a handle, batch or plan makes goes through one helper; while
 * the environment variable CORR_TEST_FAIL_ALLOC holds a positive integer k,
 * the k-th allocation counted since the variable last changed value fails
 * as if the device were out of memory.  The call that made it returns
 * CORR_ENOMEM with nothing half-allocated and the handle still usable.
 * (corr_correlate_noalloc allocates nothing and is not affected.) */

/* Test hook for the failure path (no counterpart in the paper).  kind 1: in
 * the next tensor-core X-engine launch, the first work item of CTA 0 never
 * receives its first operand tile, so the MMA thread's bounded wait expires
 * after wait_limit_s seconds (0.001..10).  kind 2: in the next fused
 * F/X-engine launch the first chunk never counts as complete, so every
 * CTA's producer wait expires after wait_limit_s (or stops when another CTA
 * records its status); the F-engine warps stop at their next task.  The kernel then records a status
 * word, drains its own copies, frees its tensor memory and returns; the
 * next corr_dump / corr_sync reports CORR_ETIMEOUT and the handle stays
 * usable.  No GPU fault, trap or hang is involved. */
int corr_test_fault(corr_t h, int kind, double wait_limit_s);

/* Kernel classes reported by corr_profile_read. */
enum corr_kernel {
    CORR_KERNEL_FENGINE = 0, /* unpack + correction + FFT + corner turn    */
    CORR_KERNEL_XENGINE = 1, /* cross-multiply-accumulate                  */
    CORR_KERNEL_REDUCE = 2,  /* FP64 accumulation of the X-engine partials */
    CORR_KERNEL_DUMP = 3,    /* accumulator -> [P][C] output               */
    CORR_KERNEL_FUSED = 4,   /* fused F/X-engine (corr_set_fused)          */
    CORR_KERNEL_COUNT = 5
};

/* Instrumentation (no counterpart in the paper): while enabled, every kernel
 * the handle launches is bracketed by a pair of CUDA events on the handle's
 * stream.  The F-engine launches of consecutive pushes overlap on the side
 * streams, so each run of them (up to the next X-engine pass or other call
 * that waits for them) is bracketed as a whole: ms[CORR_KERNEL_FENGINE] is
 * the span of those runs and launches[] still counts every launch.
 * corr_profile_read waits for the handle's stream, writes for each class
 * c < n the number of launches (launches[c]) and their summed event-to-event
 * time in milliseconds (ms[c]) since the last read, and clears the
 * counters.  Either output may be NULL. */
int corr_profile_enable(corr_t h, int on);
int corr_profile_read(corr_t h, int64_t* launches, double* ms, int n);

/* F-engine only, for inspection: transform n samples per antenna (after
 * the handle's corrections) and write the spectra Y to `spectra` as
 * [N][n/K][C] complex64 (device memory).  Leaves the integration untouched;
 * n/K must not exceed the chunk size.  Synchronises the handle's stream. */
int corr_debug_spectra(corr_t h, const uint8_t* samples, int64_t n, float* spectra);

/* ------------------------------------------------------------------------
 * Batches: several correlators ("modes", e.g. sub-arrays with different N
 * and K) whose X-engine work runs as ONE persistent tensor-core launch per
 * pass (no counterpart in the paper, whose correlator serves one mode).
 * All modes share the X-engine precision (CORR_FP32, CORR_FP16 or
 * CORR_FP8E4M3) and one non-blocking stream owned by the batch; each mode
 * keeps its own workspace and FP64 accumulators.  Per pass index the
 * F-engine of every mode that has that pass is queued (the modes' F-engines
 * run side by side on their handles' side streams), then one launch covers
 * all of their X-engine work.  With each mode's chunk at least its
 * push size (corr_batch_set_chunk), a push is exactly one X-engine launch.
 *
 * corr_batch_create  n_modes in [1, 4]; N[m], K[m] as corr_create.
 * corr_batch_push    samples[m]: device buffer of n[m] samples per antenna of
 *                    mode m (layout as corr_push); n[m] may be 0.
 * corr_batch_dump    vis[m] as corr_dump (host or device); n_spec may be NULL.
 * corr_batch_capture one push of these device buffers plus a dump into the
 *                    device buffers vis[m], run once eagerly and then
 *                    recorded as a CUDA graph; the buffers' contents may
 *                    change between replays, their addresses may not.
 * corr_batch_replay  launch the recorded graph (asynchronous): every replay
 *                    writes one complete integration per mode into vis[m];
 *                    n_spec[m] (may be NULL) receives the spectra per mode.
 *                    CORR_ESTATE when frames were pushed since the last dump.
 * corr_batch_sync    wait for the batch stream; reports device-side errors.
 * corr_batch_handle  the corr_t of mode m (corrections, scales, profiling;
 *                    not to be destroyed or given another stream).
 * corr_batch_get_stream  the batch's cudaStream_t.
 * corr_batch_set_chunk / corr_batch_set_tiles  as corr_set_chunk /
 *                    corr_set_tiles for every mode; discard a recorded graph.
 * corr_batch_set_one_launch  on = 1: each pass runs the F-engines of all its
 *                    modes as one launch (a persistent kernel of 768-thread
 *                    CTAs, three 256-thread sub-blocks for K = 512, 1024 and
 *                    other K, 512 threads for K = 2048 / 4096), so a step is
 *                    one F-engine and one X-engine launch; on = 0 (the
 *                    default): one launch per mode, side by side.  On a
 *                    GB300 the single launch is ~15% slower on the batching
 *                    workload (its union kernel is held to 80 registers and
 *                    spills); results are the same.  Switching discards a
 *                    recorded graph.
 * Errors: as the single-mode calls; corr_batch_last_error(b) has the message
 * (corr_last_error(NULL) for corr_batch_create). */
typedef struct corr_batch_s* corr_batch_t;

int corr_batch_create(corr_batch_t* out, int n_modes, const int* N, const int* K, int dtype);
int corr_batch_set_chunk(corr_batch_t b, int64_t max_spectra);
int corr_batch_set_tiles(corr_batch_t b, int window, int stages, int split, int atoms);
int corr_batch_set_one_launch(corr_batch_t b, int on);
int corr_batch_push(corr_batch_t b, const uint8_t* const* samples, const int64_t* n);
int corr_batch_dump(corr_batch_t b, void* const* vis, int64_t* n_spec, int vis_fp64);
int corr_batch_capture(corr_batch_t b, const uint8_t* const* samples, const int64_t* n,
                       void* const* vis, int vis_fp64);
int corr_batch_replay(corr_batch_t b, int64_t* n_spec);
int corr_batch_sync(corr_batch_t b);
int corr_batch_handle(corr_batch_t b, int mode, corr_t* out);
int corr_batch_get_stream(corr_batch_t b, void** stream);
void corr_batch_destroy(corr_batch_t b);
const char* corr_batch_last_error(corr_batch_t b);

/* One-shot correlation that allocates no memory (the paper has no
 * counterpart; it exists for callers that must not allocate: a real-time
 * acquisition loop in which cudaMalloc/cudaFree could synchronise the device
 * and stall it, or a process whose device memory is all owned by another
 * allocator).
 *
 * Correlates n samples per antenna of `samples` (device memory, layout as
 * for corr_push, n a multiple of K) and writes V, summed over all n/K
 * spectra, to `vis` (device memory, [P][C] complex64), with the FP32
 * CUDA-core kernels of a CORR_FP32_SIMT handle and no corrections.  Work is
 * queued on `stream` (a cudaStream_t; NULL = legacy default stream) and the
 * call returns without waiting for it.
 *
 * Scratch: every intermediate buffer lives in one 32 MiB array compiled into
 * the library (each GPU that loads the library holds it until the process
 * exits).  Configurations whose scratch for one 128-frame pass exceeds it --
 * K*8 + N(N+1)/2 * K/2 * 24 + 128 * K * N * 4 bytes, each term rounded up to
 * 256 -- are rejected with CORR_EINVAL and a message stating both sizes
 * (N = 44, K = 512 fits).  The first call on each device looks up the
 * array's device address with cudaGetSymbolAddress while that device is
 * current; make that first call before any stream capture.  The address is
 * kept with the CUDA context it belongs to; after a device reset the first
 * call in the new context looks it up again (so, again, before any capture
 * in that context).  All calls share
 * the one array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.
 * Errors: CORR_EINVAL (arguments or size), CORR_ECUDA; message from
 * corr_last_error(NULL). */
int corr_correlate_noalloc(const uint8_t* samples, int64_t n, int N, int K, float* vis,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBCORR_CORR_H */
