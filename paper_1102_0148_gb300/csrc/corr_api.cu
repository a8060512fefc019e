// C ABI of gbcorr (declared in include/corr.h): handle lifecycle, workspace
// plan, the push loop that drives F-engine -> X-engine -> FP64 reduction per
// workspace pass, and the dump.
#include "corr_internal.h"
#include "fx_fused.h"
#include "xengine_tc.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

using namespace gbcorr;

namespace {

// Default workspace of the tensor-core handles: as many frames as fit in
// 8 GiB, at most 131072 (a 1 s integration at 35 MS/s and K = 512 is one
// pass; the X-engine's per-pass costs shrink with the pass) and at least
// 2048.  The CUDA-core X-engine keeps 8192 frames within 2 GiB (its FP32
// partials grow with the pass).
constexpr int64_t kDefaultChunk = 8192;
constexpr int64_t kMaxTcChunk = 131072;
constexpr int64_t kMinDefaultChunk = 2048;
constexpr size_t kDefaultWorkspaceBytes = (size_t)2 << 30;
constexpr size_t kTcWorkspaceBytes = (size_t)8 << 30;
constexpr int64_t kSimtSplit = 256;   // fewest frames per SIMT X-engine split (sizes the partials)
constexpr int kHostStages = 16;        // device staging buffers for host input
constexpr size_t kStageBytes = (size_t)32 << 20;   // ~32 MB each

thread_local std::string g_create_error = "no error";

}  // namespace

struct corr_s {
    int N = 0, K = 0, C = 0, P = 0, dtype = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;
    int64_t cap = 0;             // frames per workspace pass (multiple of kSpecPad)
    int spec_type = SPEC_F32;
    bool use_tc = false;
    void* spec = nullptr;
    float2* twiddle = nullptr;   // W_K^m, m in [0, K)
    float2* corr_tab = nullptr;  // [N][C]
    bool corr_on = false;
    float2* gains_dev = nullptr;
    float* delays_dev = nullptr;
    float* scale = nullptr;      // [N][C] pre-cast scales (FP16 / FP8)
    // [2][N] pre-scales sigma_i of the two-plane FP16 split (CORR_FP32): row 0
    // for unit gains (uncorrected passes), row 1 for the current corrections
    float* split = nullptr;
    std::vector<float> split_host;   // row 1 as last uploaded
    const float* fill_split = nullptr;   // sigma table of the frames waiting in the workspace
    float scale_target = 1.0f;   // rms of each real part after scaling
    bool scales_ready = false;   // scale[] holds valid values
    bool scales_user = false;    // set by corr_set_scales (not updated at dumps)
    double2* acc = nullptr;      // [C][P]
    double2* acc_raw = nullptr;  // [C][P] uncorrected visibilities for corr_grad
    float2* grad_buf = nullptr;  // device staging for corr_grad's inputs and outputs
    void* grad_scratch = nullptr; // corr_grad's factor table and partial sums
    float2* partial = nullptr;   // [max_split][C][P]
    int max_split = 0;
    int* status = nullptr;       // device-side error word
    // host-input staging ring: copies run ahead of the F-engine by up to
    // kHostStages - 1 chunks of stage_frames frames
    uint8_t* stage[kHostStages] = {};
    cudaEvent_t stage_free[kHostStages] = {};
    cudaEvent_t stage_full[kHostStages] = {};
    int64_t stage_frames = 0;
    int stage_next = 0;
    // F-engine launches of consecutive pushes alternate between two side
    // streams, so one launch's last CTAs run beside the next one's first.
    // The handle's stream waits for them (join_fengines) before anything
    // that reads the workspace or changes what the F-engine reads.
    cudaStream_t f_stream[2] = {};
    cudaEvent_t f_done[2] = {};
    cudaEvent_t f_fork = nullptr;
    bool f_pending[2] = {false, false};
    int f_next = 0;
    cudaStream_t f_last = nullptr;   // stream of the latest F-engine launch
    cudaEvent_t f_span = nullptr;    // profiling: start of the open run of side launches
    // coarse integer sample delays (corr_set_sample_delays)
    bool sdelay_on = false;
    int* sdelay = nullptr;          // [N] samples, device
    std::vector<int> sdelay_host;   // the same, for checkpoints
    uint8_t* hist[2] = {};          // [N][K/2] last frame of the stream so far (ping-pong)
    int hist_cur = 0;
    // delayed chunks, alternately: [cap][N][K/2] each; shift_free[b] follows
    // the F-engine launch that last read buffer b
    uint8_t* shifted[2] = {};
    cudaEvent_t shift_free[2] = {};
    int shift_cur = 0;
    int64_t shifted_frames = 0;
    void* vis_dev = nullptr;
    int64_t n_spec = 0;
    bool acc_zero = true;        // acc holds zeros (created, or dumped since its last pass)
    // partial slot 0 holds the integration so far, the pass result of a
    // multi-block mode that went into a zero accumulator, and acc still holds
    // zeros: a dump reads the slot directly, anything else that needs acc or
    // the partials first reduces it into acc (settle_partial)
    bool part_pending = false;
    int64_t fill = 0;            // frames waiting in the workspace for the X-engine
    double2* fill_acc = nullptr; // accumulator those frames belong to
    TcPlan* tc = nullptr;
    // fused F/X-engine (K = 512, FP32 mode, N <= 44): device-input pushes
    // wait here and run as one persistent launch at the next flush
    FxPlan* fx = nullptr;
    bool fx_on = false;
    std::vector<FxSegment> fx_pending;
    int64_t fx_pending_blocks = 0;
    // instrumentation: CUDA event pairs per kernel class
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[CORR_KERNEL_COUNT];
    int64_t prof_launches[CORR_KERNEL_COUNT] = {};
    double prof_ms[CORR_KERNEL_COUNT] = {};
    cudaEvent_t ev_open = nullptr;
    std::string err = "no error";
};

namespace {

int set_err(corr_t h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define CUDA_TRY(h, call)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err((h), e_ == cudaErrorMemoryAllocation ? CORR_ENOMEM : CORR_ECUDA, \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                           __LINE__);                                                     \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int spec_type_for(int dtype) {
    if (dtype == CORR_FP16) return SPEC_F16;
    if (dtype == CORR_FP8E4M3) return SPEC_F8;
    if (dtype == CORR_FP32) return SPEC_F16X2;
    return SPEC_F32;
}

void free_workspace(corr_t h) {
    cudaFree(h->spec);
    h->spec = nullptr;
    cudaFree(h->partial);
    h->partial = nullptr;
}

int alloc_workspace(corr_t h, int64_t cap) {
    cap = (cap + kSpecPad - 1) / kSpecPad * kSpecPad;
    const size_t eb = (size_t)spec_elem_bytes(h->spec_type);
    const size_t spec_bytes = (size_t)spec_planes(h->spec_type) * h->C * 2 * h->N * cap * eb;
    // FP32 partials: one per split of at least 256 frames for the CUDA-core
    // X-engine (its launch picks the split count up to this), at
    // most 8 slots for the tensor cores (their planner's limit)
    int max_split = (int)((cap + kSimtSplit - 1) / kSimtSplit);
    if (h->use_tc) max_split = std::min(max_split, 8);
    void* spec = nullptr;
    float2* part = nullptr;
    cudaError_t e = dev_malloc(&spec, spec_bytes);
    if (e == cudaSuccess) e = dev_malloc((void**)&part, (size_t)max_split * h->C * h->P * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemsetAsync(spec, 0, spec_bytes, h->stream);
    if (e != cudaSuccess) {
        cudaFree(spec);
        cudaFree(part);
        return set_err(h, CORR_ENOMEM, "workspace allocation of %zu bytes failed: %s", spec_bytes,
                       cudaGetErrorString(e));
    }
    free_workspace(h);
    h->spec = spec;
    h->partial = part;
    h->cap = cap;
    h->max_split = max_split;
    if (h->use_tc) {
        int rc = tc_plan_update(h->tc, h->spec, h->cap, h->N, h->C, h->spec_type, h->err);
        if (rc != CORR_OK) return rc;
    }
    return CORR_OK;
}

int check_status(corr_t h) {
    int st = 0;
    CUDA_TRY(h, cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        CUDA_TRY(h, cudaMemset(h->status, 0, sizeof(int)));
        if (h->tc) tc_reset(h->tc);
        return set_err(h, CORR_ETIMEOUT, "a bounded device-side wait gave up (code %d)", st);
    }
    return CORR_OK;
}

cudaEvent_t prof_event(corr_t h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Bracket one kernel launch with events on the handle's stream (when enabled).
void prof_begin(corr_t h) {
    if (!h->prof_on) return;
    h->ev_open = prof_event(h);
    if (h->ev_open) cudaEventRecord(h->ev_open, h->stream);
}

void prof_end(corr_t h, int cls) {
    if (!h->prof_on || !h->ev_open) return;
    cudaEvent_t e = prof_event(h);
    if (!e) return;
    cudaEventRecord(e, h->stream);
    h->ev_pending[cls].emplace_back(h->ev_open, e);
    h->ev_open = nullptr;
    h->prof_launches[cls] += 1;
}

// Make the handle's stream wait for the F-engine launches on the side
// streams.  With profiling on, the run of side launches since the last join
// is timed as one span on the handle's stream (launches overlap, so the
// average launch duration is the span over the launch count).
int join_fengines(corr_t h) {
    for (int j = 0; j < 2; ++j)
        if (h->f_pending[j]) {
            CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->f_done[j], 0));
            h->f_pending[j] = false;
        }
    if (h->f_span) {
        cudaEvent_t e = prof_event(h);
        if (e) {
            cudaEventRecord(e, h->stream);
            h->ev_pending[CORR_KERNEL_FENGINE].emplace_back(h->f_span, e);
        } else {
            h->ev_pool.push_back(h->f_span);
        }
        h->f_span = nullptr;
    }
    return CORR_OK;
}

// Wait on the host for the side streams (before freeing what they read).
int sync_fengines(corr_t h) {
    for (int j = 0; j < 2; ++j)
        if (h->f_stream[j]) CUDA_TRY(h, cudaStreamSynchronize(h->f_stream[j]));
    return join_fengines(h);
}

bool narrow(corr_t h) { return h->spec_type == SPEC_F16 || h->spec_type == SPEC_F8; }

// First scales of a narrow-type handle: transform a short prefix of the
// first pass (at most 256 frames, written into the still unused workspace as
// FP32 spectra) and set s[i][k] from its mean power.
int estimate_scales(corr_t h, const uint8_t* din, int64_t S) {
    const size_t ws = (size_t)spec_planes(h->spec_type) * h->C * 2 * h->N * h->cap *
                      spec_elem_bytes(h->spec_type);
    int64_t S_est = S < 256 ? S : 256;
    const int64_t fit = (int64_t)(ws / ((size_t)h->N * h->C * sizeof(float2)));
    if (S_est > fit) S_est = fit;
    if (S_est < 1) return set_err(h, CORR_EINVAL, "chunk too small to estimate scales");
    int jrc = join_fengines(h);
    if (jrc != CORR_OK) return jrc;
    FengineArgs fa{};
    fa.in = din;
    fa.N = h->N;
    fa.K = h->K;
    fa.S = S_est;
    fa.S_pad = S_est;
    fa.twiddle = h->twiddle;
    fa.corr = h->corr_on ? h->corr_tab : nullptr;
    fa.debug_out = static_cast<float2*>(h->spec);
    CUDA_TRY(h, launch_fengine(fa, h->stream));
    CUDA_TRY(h, launch_scales_from_spectra(static_cast<const float2*>(h->spec), h->N, S_est, h->C,
                                           h->scale_target, h->scale, h->stream));
    h->scales_ready = true;
    return CORR_OK;
}

// S frames rounded up to whole kSpecPad-frame blocks (the padding frames are zero).
int64_t pad_frames(int64_t S) { return (S + kSpecPad - 1) / kSpecPad * kSpecPad; }

// Two-plane pre-scales of a pass (CORR_FP32 handles; nullptr otherwise):
// unit gains for uncorrected passes, the current corrections' otherwise.
const float* split_table(corr_t h, bool raw) {
    if (!h->split) return nullptr;
    return raw || !h->corr_on ? h->split : h->split + h->N;
}

// F-engine of S frames at `din` (device) into the workspace from frame `off`,
// queued on the next side stream after the work already on the handle's
// stream; raw = true skips the per-antenna corrections (the uncorrected
// visibilities corr_grad needs).
// The F-engine arguments of S frames at din into workspace frame `off`.
FengineArgs fengine_args(corr_t h, const uint8_t* din, int64_t S, bool raw, int64_t off) {
    FengineArgs fa{};
    fa.in = din;
    fa.N = h->N;
    fa.K = h->K;
    fa.S = S;
    fa.S_pad = pad_frames(S);
    fa.twiddle = h->twiddle;
    fa.corr = (h->corr_on && !raw) ? h->corr_tab : nullptr;
    fa.spec = h->spec;
    fa.s_base = off;
    fa.plane_stride = (int64_t)h->C * 2 * h->N * h->cap;
    fa.spec_type = h->spec_type;
    fa.scale = (h->spec_type == SPEC_F16 || h->spec_type == SPEC_F8) ? h->scale : nullptr;
    fa.split = split_table(h, raw);
    fa.debug_out = nullptr;
    return fa;
}

int fengine_pass(corr_t h, const uint8_t* din, int64_t S, bool raw, int64_t off) {
    if (narrow(h) && !h->scales_ready) {
        int rc = estimate_scales(h, din, S);
        if (rc != CORR_OK) return rc;
    }
    const FengineArgs fa = fengine_args(h, din, S, raw, off);
    const int j = h->f_next;
    cudaStream_t st = h->f_stream[j];
    if (h->prof_on && !h->f_span) {
        h->f_span = prof_event(h);
        if (h->f_span) cudaEventRecord(h->f_span, h->stream);
    }
    CUDA_TRY(h, cudaEventRecord(h->f_fork, h->stream));
    CUDA_TRY(h, cudaStreamWaitEvent(st, h->f_fork, 0));
    CUDA_TRY(h, launch_fengine(fa, st));
    CUDA_TRY(h, cudaEventRecord(h->f_done[j], st));
    h->f_pending[j] = true;
    h->f_next = j ^ 1;
    h->f_last = st;
    if (h->f_span) h->prof_launches[CORR_KERNEL_FENGINE] += 1;
    return CORR_OK;
}

// A pass result left in partial slot 0 goes into the (zero) accumulator
// before the next launch that writes the partials or uses acc.
int settle_partial(corr_t h) {
    if (!h->part_pending) return CORR_OK;
    h->part_pending = false;
    h->acc_zero = false;
    prof_begin(h);
    CUDA_TRY(h, launch_reduce_partials(h->partial, 1, (int64_t)h->C * h->P, h->acc, h->stream,
                                       true));
    prof_end(h, CORR_KERNEL_REDUCE);
    return CORR_OK;
}

// FP64 reduction of a tensor-core launch's partials, when it wrote any.
int finish_tc_run(corr_t h, const TcRun& run, double2* acc) {
    if (run.direct) {           // single-block modes added into acc themselves
        if (acc == h->acc) h->acc_zero = false;
        return CORR_OK;
    }
    // a multi-block mode's pass result covers every (k, p) in slot 0: the
    // first pass of an integration stays there until a dump reads it or
    // settle_partial stores it; later passes are added
    if (acc == h->acc && h->acc_zero && run.n_split == 1) {
        h->part_pending = true;
        return CORR_OK;
    }
    const bool assign = acc == h->acc && h->acc_zero;
    if (acc == h->acc) h->acc_zero = false;
    prof_begin(h);
    CUDA_TRY(h, launch_reduce_partials(h->partial, run.n_split, (int64_t)h->C * h->P, acc,
                                       h->stream, assign));
    prof_end(h, CORR_KERNEL_REDUCE);
    return CORR_OK;
}

// X-engine half of a pass over the S_pad frames in the workspace -> `acc`.
int xengine_pass(corr_t h, int64_t S_pad, double2* acc) {
    int src = settle_partial(h);         // the launch overwrites the partials
    if (src != CORR_OK) return src;
    if (h->use_tc) {
        prof_begin(h);
        TcRun run{};
        run.S_pad = S_pad;
        run.partial = h->partial;
        run.acc = acc;
        run.scale = h->scale;
        run.split = h->fill_split;
        run.status = h->status;
        TcPlan* plans[1] = {h->tc};
        int rc = tc_launch(plans, 1, &run, h->stream, h->err);
        if (rc != CORR_OK) return rc;
        prof_end(h, CORR_KERNEL_XENGINE);
        return finish_tc_run(h, run, acc);
    } else {
        XengineArgs xa{};
        xa.spec = h->spec;
        xa.N = h->N;
        xa.C = h->C;
        xa.S_pad = S_pad;
        xa.spec_type = h->spec_type;
        xa.max_split = h->max_split;
        xa.partial = h->partial;
        xa.scale = nullptr;
        xa.status = h->status;
        prof_begin(h);
        CUDA_TRY(h, launch_xengine_simt(xa, h->stream));
        prof_end(h, CORR_KERNEL_XENGINE);
        const bool assign = acc == h->acc && h->acc_zero;
        if (acc == h->acc) h->acc_zero = false;
        prof_begin(h);
        CUDA_TRY(h, launch_reduce_partials(h->partial, xa.n_split, (int64_t)h->C * h->P, acc,
                                           h->stream, assign));
        prof_end(h, CORR_KERNEL_REDUCE);
    }
    return CORR_OK;
}

// The fused launch over the device-input pushes waiting for it.
int fx_flush(corr_t h) {
    if (h->fx_pending.empty()) return CORR_OK;
    int src = settle_partial(h);         // the fused kernel adds into acc
    if (src != CORR_OK) return src;
    prof_begin(h);
    int rc = fx_launch(h->fx, h->fx_pending.data(), (int)h->fx_pending.size(), h->twiddle,
                       split_table(h, false), h->corr_on ? h->corr_tab : nullptr, h->acc, h->status,
                       h->stream, h->err);
    h->acc_zero = false;
    h->fx_pending.clear();
    h->fx_pending_blocks = 0;
    if (rc != CORR_OK) return rc;
    prof_end(h, CORR_KERNEL_FUSED);
    return CORR_OK;
}

// Whether device-input pushes of this handle go to the fused launch.
bool fx_usable(corr_t h) { return h->fx && h->fx_on && !h->sdelay_on; }

// Record S frames of device input for the next fused launch (launching the
// waiting ones first when the block table would overflow).
int fx_append(corr_t h, const uint8_t* din, int64_t S) {
    const int64_t rec = (int64_t)h->N * (h->K / 2);
    while (S > 0) {
        const int64_t room = (int64_t)kFxMaxBlocks - h->fx_pending_blocks;
        if (room <= 0) {
            int rc = fx_flush(h);
            if (rc != CORR_OK) return rc;
            continue;
        }
        const int64_t take = std::min<int64_t>(S, room * 32);
        h->fx_pending.push_back(FxSegment{din, take});
        h->fx_pending_blocks += (take + 31) / 32;
        din += take * rec;
        S -= take;
    }
    return CORR_OK;
}

// X-engine over the frames waiting in the workspace (and the fused launch
// over the pushes waiting for it).
int flush(corr_t h) {
    int frc = fx_flush(h);
    if (frc != CORR_OK) return frc;
    int jrc = join_fengines(h);
    if (jrc != CORR_OK) return jrc;
    if (h->fill == 0) return CORR_OK;
    const int64_t f = h->fill;
    h->fill = 0;
    return xengine_pass(h, f, h->fill_acc);
}

// F-engine of S frames into the workspace after the frames already waiting
// there; the X-engine runs once the workspace is full, or at once when S is
// not a multiple of the 128-frame padding (the padding must stay at the end).
int stage_frames(corr_t h, const uint8_t* din, int64_t S, bool raw, double2* acc) {
    const float* split = split_table(h, raw);
    if (h->fill > 0 && (acc != h->fill_acc || split != h->fill_split)) {
        int rc = flush(h);
        if (rc != CORR_OK) return rc;
    }
    if (narrow(h) && !h->scales_ready) {
        int rc = flush(h);                       // the estimate uses the workspace
        if (rc == CORR_OK) rc = estimate_scales(h, din, S);
        if (rc != CORR_OK) return rc;
    }
    h->fill_acc = acc;
    h->fill_split = split;
    int rc = fengine_pass(h, din, S, raw, h->fill);
    if (rc != CORR_OK) return rc;
    const bool whole = S % kSpecPad == 0;
    h->fill += whole ? S : pad_frames(S);
    if (!whole || h->fill >= h->cap) return flush(h);
    return CORR_OK;
}

// Two delayed-chunk buffers of `cap` frames each (the F-engine of one chunk
// may still read its buffer while the next chunk is delayed into the other).
int alloc_shifted(corr_t h) {
    if (h->shifted_frames >= h->cap) return CORR_OK;
    int rc = sync_fengines(h);              // queued launches may read the old buffers
    if (rc != CORR_OK) return rc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const size_t bytes = (size_t)h->cap * h->N * (h->K / 2);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->shifted[b]);
        h->shifted[b] = nullptr;
    }
    h->shifted_frames = 0;
    for (int b = 0; b < 2; ++b) {
        CUDA_TRY(h, dev_malloc((void**)&h->shifted[b], bytes));
        if (!h->shift_free[b])
            CUDA_TRY(h, cudaEventCreateWithFlags(&h->shift_free[b], cudaEventDisableTiming));
    }
    h->shifted_frames = h->cap;
    return CORR_OK;
}

// Release the host-input staging ring (buffers and their events).
void free_stages(corr_t h) {
    for (int b = 0; b < kHostStages; ++b) {
        cudaFree(h->stage[b]);
        h->stage[b] = nullptr;
        if (h->stage_free[b]) cudaEventDestroy(h->stage_free[b]);
        if (h->stage_full[b]) cudaEventDestroy(h->stage_full[b]);
        h->stage_free[b] = h->stage_full[b] = nullptr;
    }
    h->stage_next = 0;
}

// Transform n samples (host or device memory) into the workspace, running the
// X-engine into `acc` whenever it fills up.
int process_samples(corr_t h, const uint8_t* samples, int64_t n, bool raw, double2* acc) {
    const int64_t frames = n / h->K;
    const int64_t rec = (int64_t)h->N * (h->K / 2);
    const bool host = !is_device_ptr(samples);
    // (the fused F-engine reads 16 bytes per lane: 16-byte aligned input only)
    if (!host && !raw && acc == h->acc && fx_usable(h) &&
        (reinterpret_cast<uintptr_t>(samples) & 15) == 0)
        return fx_append(h, samples, frames);
    if (host && !h->stage[0]) {
        // ~32 MB per buffer (whole 128-frame blocks), 16 of them: the copies
        // (~205 GB/s from pinned host memory) can run ~2.5 ms ahead of the
        // F-engine, across an X-engine pass of a whole integration.  All or
        // nothing: a failure releases the buffers made so far.
        h->stage_frames = std::max<int64_t>(
            kSpecPad, std::min<int64_t>(h->cap, (int64_t)(kStageBytes / rec)) / kSpecPad * kSpecPad);
        for (int b = 0; b < kHostStages; ++b) {
            cudaError_t e = dev_malloc((void**)&h->stage[b], (size_t)(h->stage_frames * rec));
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&h->stage_free[b], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&h->stage_full[b], cudaEventDisableTiming);
            if (e != cudaSuccess) {
                cudaGetLastError();
                free_stages(h);
                return set_err(h, e == cudaErrorMemoryAllocation ? CORR_ENOMEM : CORR_ECUDA,
                               "host-input staging buffers: %s", cudaGetErrorString(e));
            }
        }
    }
    if (h->sdelay_on) {                         // the pass may have grown since
        int rc = alloc_shifted(h);
        if (rc != CORR_OK) return rc;
    }
    for (int64_t f0 = 0; f0 < frames;) {
        if (h->fill > 0 && (acc != h->fill_acc || split_table(h, raw) != h->fill_split)) {
            int rc = flush(h);
            if (rc != CORR_OK) return rc;
        }
        const int64_t room = h->cap - h->fill;
        int64_t S = frames - f0 < room ? frames - f0 : room;
        if (host && S > h->stage_frames) S = h->stage_frames;
        const uint8_t* din = samples + f0 * rec;
        int b = 0;
        if (host) {
            b = h->stage_next;
            h->stage_next = (b + 1) % kHostStages;
            CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->stage_free[b], 0));
            CUDA_TRY(h, cudaMemcpyAsync(h->stage[b], din, (size_t)(S * rec), cudaMemcpyHostToDevice,
                                        h->copy_stream));
            CUDA_TRY(h, cudaEventRecord(h->stage_full[b], h->copy_stream));
            CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->stage_full[b], 0));
            din = h->stage[b];
        }
        int sb = -1;
        if (h->sdelay_on) {
            // the stream's history feeds pushes only; corr_grad's samples
            // (raw) start from zeros and leave it untouched
            const uint8_t* hin = raw ? nullptr : h->hist[h->hist_cur];
            uint8_t* hout = raw ? nullptr : h->hist[h->hist_cur ^ 1];
            sb = h->shift_cur;
            h->shift_cur ^= 1;
            CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->shift_free[sb], 0));
            CUDA_TRY(h, launch_sample_delay(din, S, h->N, h->K, h->sdelay, hin, hout, h->shifted[sb],
                                            h->stream));
            if (!raw) h->hist_cur ^= 1;
            din = h->shifted[sb];
        }
        int rc = stage_frames(h, din, S, raw, acc);
        if (rc != CORR_OK) return rc;
        if (sb >= 0) CUDA_TRY(h, cudaEventRecord(h->shift_free[sb], h->f_last));
        if (host) CUDA_TRY(h, cudaEventRecord(h->stage_free[b], h->f_last));
        f0 += S;
    }
    return CORR_OK;
}

void destroy_impl(corr_t h) {
    if (!h) return;
    for (int j = 0; j < 2; ++j)
        if (h->f_stream[j]) cudaStreamSynchronize(h->f_stream[j]);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    free_workspace(h);
    cudaFree(h->twiddle);
    cudaFree(h->corr_tab);
    cudaFree(h->gains_dev);
    cudaFree(h->delays_dev);
    cudaFree(h->scale);
    cudaFree(h->split);
    cudaFree(h->acc);
    cudaFree(h->acc_raw);
    cudaFree(h->grad_buf);
    cudaFree(h->grad_scratch);
    cudaFree(h->status);
    cudaFree(h->vis_dev);
    cudaFree(h->sdelay);
    cudaFree(h->hist[0]);
    cudaFree(h->hist[1]);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->shifted[b]);
        if (h->shift_free[b]) cudaEventDestroy(h->shift_free[b]);
    }
    free_stages(h);
    if (h->tc) tc_plan_destroy(h->tc);
    if (h->fx) fx_plan_destroy(h->fx);
    for (auto& v : h->ev_pending)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->f_span) cudaEventDestroy(h->f_span);
    for (int j = 0; j < 2; ++j) {
        if (h->f_done[j]) cudaEventDestroy(h->f_done[j]);
        if (h->f_stream[j]) cudaStreamDestroy(h->f_stream[j]);
    }
    if (h->f_fork) cudaEventDestroy(h->f_fork);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
}

}  // namespace

void gbcorr::set_global_error(const char* msg) { g_create_error = msg; }

namespace {
std::mutex g_alloc_mu;
std::string g_alloc_env;     // value of CORR_TEST_FAIL_ALLOC the count belongs to
long g_alloc_count = 0;      // allocations since it last changed
}  // namespace

cudaError_t gbcorr::dev_malloc(void** p, size_t bytes) {
    const char* env = getenv("CORR_TEST_FAIL_ALLOC");
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        const std::string v = env ? env : "";
        if (v != g_alloc_env) {
            g_alloc_env = v;
            g_alloc_count = 0;
        }
        const long k = v.empty() ? 0 : strtol(v.c_str(), nullptr, 10);
        if (k > 0 && ++g_alloc_count == k) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

extern "C" {

int corr_create(corr_t* out, int N, int K, int dtype) {
    if (!out) return set_err(nullptr, CORR_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > CORR_MAX_N)
        return set_err(nullptr, CORR_EINVAL, "N=%d outside [1, %d]", N, CORR_MAX_N);
    if (K < 16 || K > 4096 || (K & (K - 1)))
        return set_err(nullptr, CORR_EINVAL, "K=%d is not a power of two in [16, 4096]", K);
    if (dtype < CORR_FP32 || dtype > CORR_FP32_SIMT)
        return set_err(nullptr, CORR_EINVAL, "unknown dtype %d", dtype);

    corr_t h = new (std::nothrow) corr_s();
    if (!h) return set_err(nullptr, CORR_ENOMEM, "host allocation failed");
    h->N = N;
    h->K = K;
    h->C = K / 2;
    h->P = N * (N + 1) / 2;
    h->dtype = dtype;
    h->spec_type = spec_type_for(dtype);
    h->use_tc = dtype != CORR_FP32_SIMT;
    h->scale_target = dtype == CORR_FP8E4M3 ? 16.0f : 64.0f;

    auto bail = [&](int rc) {
        g_create_error = h->err;
        destroy_impl(h);
        return rc;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return set_err(nullptr, CORR_ECUDA, "no CUDA device available");
    }
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(set_err(h, CORR_ECUDA, "stream creation failed"));
    h->own_stream = true;
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(set_err(h, CORR_ECUDA, "stream creation failed"));
    for (int j = 0; j < 2; ++j)
        if (cudaStreamCreateWithFlags(&h->f_stream[j], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->f_done[j], cudaEventDisableTiming) != cudaSuccess)
            return bail(set_err(h, CORR_ECUDA, "stream creation failed"));
    if (cudaEventCreateWithFlags(&h->f_fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(set_err(h, CORR_ECUDA, "event creation failed"));
    h->f_last = h->stream;

    if (h->use_tc) {
        int rc = tc_plan_create(&h->tc, N, h->C, h->spec_type, h->err);
        if (rc != CORR_OK) return bail(rc);
    }
    // the fused F/X-engine is off until corr_set_fused(h, 1) makes its plan

    // Twiddles W_K^m = exp(-2 pi i m / K), from an exact integer angle in FP64.
    std::vector<float2> tw(K);
    for (int m = 0; m < K; ++m) {
        const double th = 2.0 * M_PI * (double)m / (double)K;
        tw[m] = make_float2((float)std::cos(th), (float)-std::sin(th));
    }
    const size_t acc_bytes = (size_t)h->C * h->P * sizeof(double2);
    if (dev_malloc((void**)&h->twiddle, K * sizeof(float2)) != cudaSuccess ||
        dev_malloc((void**)&h->acc, acc_bytes) != cudaSuccess ||
        dev_malloc((void**)&h->status, sizeof(int)) != cudaSuccess ||
        dev_malloc((void**)&h->corr_tab, (size_t)N * h->C * sizeof(float2)) != cudaSuccess ||
        dev_malloc((void**)&h->gains_dev, (size_t)N * sizeof(float2)) != cudaSuccess ||
        dev_malloc((void**)&h->delays_dev, (size_t)N * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return bail(set_err(h, CORR_ENOMEM, "device allocation failed"));
    }
    if (h->spec_type == SPEC_F16 || h->spec_type == SPEC_F8) {
        if (dev_malloc((void**)&h->scale, (size_t)N * h->C * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return bail(set_err(h, CORR_ENOMEM, "device allocation failed"));
        }
    }
    if (h->spec_type == SPEC_F16X2) {
        h->split_host.assign(2 * (size_t)N, split_scale_for(1.0, K));
        if (dev_malloc((void**)&h->split, 2 * (size_t)N * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return bail(set_err(h, CORR_ENOMEM, "device allocation failed"));
        }
        if (cudaMemcpy(h->split, h->split_host.data(), 2 * (size_t)N * sizeof(float),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(set_err(h, CORR_ECUDA, "initialisation copy failed"));
        h->split_host.resize(N);
    }
    if (cudaMemcpy(h->twiddle, tw.data(), K * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemsetAsync(h->acc, 0, acc_bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess)
        return bail(set_err(h, CORR_ECUDA, "initialisation copy failed"));
    if (h->scale) {
        std::vector<float> ones((size_t)N * h->C, 1.0f);
        if (cudaMemcpy(h->scale, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return bail(set_err(h, CORR_ECUDA, "initialisation copy failed"));
    }
    const size_t per_frame = (size_t)spec_planes(h->spec_type) * h->C * 2 * h->N *
                             spec_elem_bytes(h->spec_type);
    int64_t chunk = kDefaultChunk;
    if (h->use_tc) {
        chunk = (int64_t)(kTcWorkspaceBytes / per_frame) / kSpecPad * kSpecPad;
        chunk = std::max(kMinDefaultChunk, std::min(kMaxTcChunk, chunk));
    } else {
        while (chunk > kMinDefaultChunk && (size_t)chunk * per_frame > kDefaultWorkspaceBytes)
            chunk /= 2;
    }
    int rc = alloc_workspace(h, chunk);
    if (rc != CORR_OK) return bail(rc);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(set_err(h, CORR_ECUDA, "initialisation failed"));
    *out = h;
    return CORR_OK;
}

int corr_set_stream(corr_t h, void* stream) {
    if (!h) return CORR_EINVAL;
    int frc = fx_flush(h);
    if (frc != CORR_OK) return frc;
    int jrc = join_fengines(h);
    if (jrc != CORR_OK) return jrc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (h->own_stream) {
        cudaStreamDestroy(h->stream);
        h->own_stream = false;
    }
    h->stream = static_cast<cudaStream_t>(stream);
    return CORR_OK;
}

int corr_set_chunk(corr_t h, int64_t max_spectra) {
    if (!h) return CORR_EINVAL;
    if (max_spectra < 1 || max_spectra > (int64_t)1 << 24)
        return set_err(h, CORR_EINVAL, "chunk of %lld spectra outside [1, 2^24]",
                       (long long)max_spectra);
    if (h->n_spec != 0)
        return set_err(h, CORR_ESTATE, "chunk size can only change between integrations");
    int jrc = sync_fengines(h);
    if (jrc != CORR_OK) return jrc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return alloc_workspace(h, max_spectra);
}

int corr_set_fused(corr_t h, int on) {
    if (!h) return CORR_EINVAL;
    if (on && !h->fx) {
        if (!fx_supported(h->N, h->K, h->spec_type))
            return set_err(h, CORR_EUNSUPPORTED,
                           "the fused F/X-engine serves K = 512, CORR_FP32, N <= %d", kFxMaxN);
        std::string ferr;
        const int rc = fx_plan_create(&h->fx, h->N, ferr);
        if (rc != CORR_OK) return set_err(h, rc, "%s", ferr.c_str());
    }
    int frc = fx_flush(h);
    if (frc != CORR_OK) return frc;
    h->fx_on = on != 0;
    return CORR_OK;
}

int corr_get_fused(corr_t h, int* on) {
    if (!h || !on) return CORR_EINVAL;
    *on = h->fx && h->fx_on ? 1 : 0;
    return CORR_OK;
}

int corr_set_tiles(corr_t h, int window, int stages, int split, int atoms) {
    if (!h) return CORR_EINVAL;
    if (!h->use_tc) return set_err(h, CORR_EINVAL, "tile choices apply to tensor-core handles");
    return tc_set_tiles(h->tc, window, stages, split, atoms, h->err);
}

// Checkpoint layout: header, FP64 accumulator [C][P], pre-cast scales [N][C]
// (narrow types only).
struct StateHeader {
    uint64_t magic;
    int32_t N, K, dtype, scales_ready;
    int64_t n_spec;
    int32_t sample_delays, reserved;   // 1: delays [N] int32 and the stream history follow
};
constexpr uint64_t kStateMagic = 0x32726f6362677242ull;   // arbitrary tag

size_t state_bytes(corr_t h) {
    return sizeof(StateHeader) + (size_t)h->C * h->P * sizeof(double2) +
           (narrow(h) ? (size_t)h->N * h->C * sizeof(float) : 0) +
           (h->sdelay_on ? (size_t)h->N * sizeof(int32_t) + (size_t)h->N * (h->K / 2) : 0);
}

// Turn the coarse sample delays on with `d` (host, N entries) or off (all
// zero); the stream history starts from zeros when they are turned on.
int apply_sample_delays(corr_t h, const int* d) {
    bool any = false;
    for (int i = 0; i < h->N; ++i) any |= d[i] != 0;
    if (!any) {
        h->sdelay_on = false;
        return CORR_OK;
    }
    const size_t hb = (size_t)h->N * (h->K / 2);
    if (!h->sdelay) {
        // all or nothing: a failure releases what was made
        int* sd = nullptr;
        uint8_t* hs[2] = {};
        cudaError_t e = dev_malloc((void**)&sd, h->N * sizeof(int));
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = dev_malloc((void**)&hs[b], hb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(sd);
            cudaFree(hs[0]);
            cudaFree(hs[1]);
            return set_err(h, e == cudaErrorMemoryAllocation ? CORR_ENOMEM : CORR_ECUDA,
                           "sample-delay buffers: %s", cudaGetErrorString(e));
        }
        h->sdelay = sd;
        h->hist[0] = hs[0];
        h->hist[1] = hs[1];
    }
    int arc = alloc_shifted(h);
    if (arc != CORR_OK) return arc;
    if (!h->sdelay_on) {
        CUDA_TRY(h, cudaMemsetAsync(h->hist[h->hist_cur], 0, hb, h->stream));
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->sdelay, d, h->N * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));    // d may be a caller's temporary
    h->sdelay_host.assign(d, d + h->N);
    h->sdelay_on = true;
    return CORR_OK;
}

int corr_state_bytes(corr_t h, size_t* bytes) {
    if (!h || !bytes) return CORR_EINVAL;
    *bytes = state_bytes(h);
    return CORR_OK;
}

int corr_save_state(corr_t h, void* buf) {
    if (!h || !buf) return CORR_EINVAL;
    int frc = flush(h);
    if (frc == CORR_OK) frc = settle_partial(h);
    if (frc != CORR_OK) return frc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int rc = check_status(h);
    if (rc != CORR_OK) return rc;
    StateHeader hd{kStateMagic, h->N, h->K, h->dtype, h->scales_ready ? 1 : 0, h->n_spec,
                   h->sdelay_on ? 1 : 0, 0};
    unsigned char* p = static_cast<unsigned char*>(buf);
    memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t ab = (size_t)h->C * h->P * sizeof(double2);
    CUDA_TRY(h, cudaMemcpy(p, h->acc, ab, cudaMemcpyDeviceToHost));
    p += ab;
    if (narrow(h)) {
        CUDA_TRY(h, cudaMemcpy(p, h->scale, (size_t)h->N * h->C * sizeof(float),
                               cudaMemcpyDeviceToHost));
        p += (size_t)h->N * h->C * sizeof(float);
    }
    if (h->sdelay_on) {
        memcpy(p, h->sdelay_host.data(), h->N * sizeof(int32_t));
        p += h->N * sizeof(int32_t);
        CUDA_TRY(h, cudaMemcpy(p, h->hist[h->hist_cur], (size_t)h->N * (h->K / 2),
                               cudaMemcpyDeviceToHost));
    }
    return CORR_OK;
}

int corr_load_state(corr_t h, const void* buf) {
    if (!h || !buf) return CORR_EINVAL;
    StateHeader hd;
    memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kStateMagic) return set_err(h, CORR_EINVAL, "not a correlator state");
    if (hd.N != h->N || hd.K != h->K || hd.dtype != h->dtype)
        return set_err(h, CORR_EINVAL, "state of N=%d K=%d dtype=%d does not fit this handle",
                       (int)hd.N, (int)hd.K, (int)hd.dtype);
    int frc = flush(h);                  // pending frames are replaced with the state
    if (frc != CORR_OK) return frc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof hd;
    const size_t ab = (size_t)h->C * h->P * sizeof(double2);
    h->acc_zero = false;
    h->part_pending = false;
    CUDA_TRY(h, cudaMemcpy(h->acc, p, ab, cudaMemcpyHostToDevice));
    p += ab;
    if (narrow(h)) {
        if (hd.scales_ready) {
            CUDA_TRY(h, cudaMemcpy(h->scale, p, (size_t)h->N * h->C * sizeof(float),
                                   cudaMemcpyHostToDevice));
            h->scales_ready = true;
        }
        p += (size_t)h->N * h->C * sizeof(float);
    }
    if (hd.sample_delays) {
        std::vector<int> d(h->N);
        memcpy(d.data(), p, h->N * sizeof(int32_t));
        p += h->N * sizeof(int32_t);
        int rc = apply_sample_delays(h, d.data());
        if (rc != CORR_OK) return rc;
        CUDA_TRY(h, cudaMemcpy(h->hist[h->hist_cur], p, (size_t)h->N * (h->K / 2),
                               cudaMemcpyHostToDevice));
    } else {
        h->sdelay_on = false;
    }
    h->n_spec = hd.n_spec;
    return CORR_OK;
}

int corr_test_fault(corr_t h, int kind, double wait_limit_s) {
    if (!h) return CORR_EINVAL;
    if (kind == 2) {
        if (!h->fx || !h->fx_on)
            return set_err(h, CORR_EINVAL, "the fused-launch fault needs the fused F/X-engine on");
        int frc = flush(h);
        if (frc != CORR_OK) return frc;
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return fx_test_withhold(h->fx, wait_limit_s, h->err);
    }
    if (kind != 1) return set_err(h, CORR_EINVAL, "unknown fault kind %d", kind);
    if (!h->use_tc) return set_err(h, CORR_EINVAL, "the withheld-copy fault needs a tensor-core handle");
    int jrc = sync_fengines(h);
    if (jrc != CORR_OK) return jrc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return tc_test_withhold(h->tc, wait_limit_s, h->err);
}

int corr_set_sample_delays(corr_t h, const int32_t* delays) {
    if (!h) return CORR_EINVAL;
    std::vector<int> d(h->N, 0);
    if (delays) {
        if (is_device_ptr(delays)) {
            CUDA_TRY(h, cudaMemcpy(d.data(), delays, h->N * sizeof(int32_t), cudaMemcpyDeviceToHost));
        } else {
            memcpy(d.data(), delays, h->N * sizeof(int32_t));
        }
        for (int i = 0; i < h->N; ++i)
            if (d[i] < 0 || d[i] > h->K)
                return set_err(h, CORR_EINVAL, "sample delay %d of antenna %d is outside [0, K=%d]",
                               d[i], i, h->K);
    }
    int frc = flush(h);                  // frames already pushed keep the old delays
    if (frc != CORR_OK) return frc;
    return apply_sample_delays(h, d.data());
}

int corr_set_corrections(corr_t h, const float* gains, const float* delays) {
    if (!h) return CORR_EINVAL;
    // Host copies, to check the values and to derive the two-plane pre-scales.
    std::vector<float> gh, th;
    if (gains) {
        gh.resize(2 * (size_t)h->N);
        CUDA_TRY(h, cudaMemcpy(gh.data(), gains, gh.size() * sizeof(float), cudaMemcpyDefault));
        for (int i = 0; i < h->N; ++i) {
            const double a = std::hypot((double)gh[2 * i], (double)gh[2 * i + 1]);
            if (!std::isfinite(a) || a > kGainMax || (a > 0.0 && a < kGainMin))
                return set_err(h, CORR_EINVAL,
                               "gain %d has modulus %g: gains must be finite, 0 or within "
                               "[2^-40, 2^40]", i, a);
        }
    }
    if (delays) {
        th.resize(h->N);
        CUDA_TRY(h, cudaMemcpy(th.data(), delays, th.size() * sizeof(float), cudaMemcpyDefault));
        for (int i = 0; i < h->N; ++i)
            if (!std::isfinite(th[i]))
                return set_err(h, CORR_EINVAL, "delay %d is not finite", i);
    }
    // launches already queued keep the old tables; pushes waiting for the
    // fused launch are run with them now
    int frc0 = fx_flush(h);
    if (frc0 != CORR_OK) return frc0;
    int jrc = join_fengines(h);
    if (jrc != CORR_OK) return jrc;
    // Frames already pushed keep the old corrections and pre-scales: with new
    // pre-scales they are cross-multiplied first.
    if (h->split) {
        std::vector<float> sn(h->N, split_scale_for(1.0, h->K));
        if (gains)
            for (int i = 0; i < h->N; ++i)
                sn[i] = split_scale_for(std::hypot((double)gh[2 * i], (double)gh[2 * i + 1]), h->K);
        const bool on = gains || delays;
        const bool changed = sn != h->split_host || on != h->corr_on;
        if (changed && h->fill > 0 && h->fill_split != h->split) {
            int frc = flush(h);
            if (frc != CORR_OK) return frc;
        }
        if (sn != h->split_host) {
            CUDA_TRY(h, cudaMemcpyAsync(h->split + h->N, sn.data(), h->N * sizeof(float),
                                        cudaMemcpyHostToDevice, h->stream));
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            h->split_host = sn;
        }
    }
    if (!gains && !delays) {
        h->corr_on = false;
        return CORR_OK;
    }
    if (gains)
        CUDA_TRY(h, cudaMemcpyAsync(h->gains_dev, gains, (size_t)h->N * sizeof(float2),
                                    cudaMemcpyDefault, h->stream));
    if (delays)
        CUDA_TRY(h, cudaMemcpyAsync(h->delays_dev, delays, (size_t)h->N * sizeof(float),
                                    cudaMemcpyDefault, h->stream));
    CUDA_TRY(h, launch_correction_table(gains ? h->gains_dev : nullptr,
                                        delays ? h->delays_dev : nullptr, h->N, h->K, h->corr_tab,
                                        h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->corr_on = true;
    return CORR_OK;
}

int corr_push(corr_t h, const uint8_t* samples, int64_t n) {
    if (!h) return CORR_EINVAL;
    if (n < 0 || n % h->K)
        return set_err(h, CORR_EINVAL, "n=%lld is not a non-negative multiple of K=%d",
                       (long long)n, h->K);
    if (n == 0) return CORR_OK;
    if (!samples) return set_err(h, CORR_EINVAL, "samples is NULL");
    int rc = process_samples(h, samples, n, false, h->acc);
    if (rc != CORR_OK) return rc;
    h->n_spec += n / h->K;
    return CORR_OK;
}

int corr_grad(corr_t h, const uint8_t* samples, int64_t n, const float* gains,
              const float* delays, const void* grad_vis, int grad_fp64, float* grad_gains,
              float* grad_delays) {
    if (!h) return CORR_EINVAL;
    if (n < 0 || n % h->K)
        return set_err(h, CORR_EINVAL, "n=%lld is not a non-negative multiple of K=%d",
                       (long long)n, h->K);
    if (!samples || !grad_vis || !grad_gains || !grad_delays)
        return set_err(h, CORR_EINVAL, "NULL buffer");
    const size_t CPb = (size_t)h->C * h->P;
    if (!h->acc_raw) CUDA_TRY(h, dev_malloc((void**)&h->acc_raw, CPb * sizeof(double2)));
    // device staging: gains (N float2), delays (N float), outputs (N float2 + N float),
    // and the incoming gradient when it is host memory
    const size_t gv_bytes = CPb * (grad_fp64 ? sizeof(double2) : sizeof(float2));
    if (!h->grad_buf)
        CUDA_TRY(h, dev_malloc((void**)&h->grad_buf, 4 * (size_t)h->N * sizeof(float2) +
                                                     CPb * sizeof(double2)));
    if (!h->grad_scratch)
        CUDA_TRY(h, dev_malloc(&h->grad_scratch, grad_scratch_bytes(h->N, h->K)));
    float2* g_dev = h->grad_buf;
    float* t_dev = reinterpret_cast<float*>(g_dev + h->N);
    float2* gg_dev = g_dev + 2 * h->N;
    float* gt_dev = reinterpret_cast<float*>(gg_dev + h->N);
    void* gv_dev = g_dev + 4 * h->N;
    if (gains)
        CUDA_TRY(h, cudaMemcpyAsync(g_dev, gains, h->N * sizeof(float2), cudaMemcpyDefault, h->stream));
    if (delays)
        CUDA_TRY(h, cudaMemcpyAsync(t_dev, delays, h->N * sizeof(float), cudaMemcpyDefault, h->stream));
    const void* gv = grad_vis;
    if (!is_device_ptr(grad_vis)) {
        CUDA_TRY(h, cudaMemcpyAsync(gv_dev, grad_vis, gv_bytes, cudaMemcpyHostToDevice, h->stream));
        gv = gv_dev;
    }
    int frc = flush(h);                  // the running integration's pending frames
    if (frc != CORR_OK) return frc;
    CUDA_TRY(h, cudaMemsetAsync(h->acc_raw, 0, CPb * sizeof(double2), h->stream));
    if (n > 0) {
        int rc = process_samples(h, samples, n, true, h->acc_raw);
        if (rc == CORR_OK) rc = flush(h);
        if (rc != CORR_OK) return rc;
    }
    CUDA_TRY(h, launch_grad(h->acc_raw, gv, grad_fp64, gains ? g_dev : nullptr,
                            delays ? t_dev : nullptr, h->N, h->K, gg_dev, gt_dev,
                            h->grad_scratch, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(grad_gains, gg_dev, h->N * sizeof(float2), cudaMemcpyDefault,
                                h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(grad_delays, gt_dev, h->N * sizeof(float), cudaMemcpyDefault,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_status(h);
}

namespace {

// The dump kernels of the integration on stream st: the next integration's
// scales from this one's autocorrelations (when `scales`), then vis[p][k],
// from the accumulator (which is then cleared) or from a pass result still
// in partial slot 0 (the accumulator is zero already).
cudaError_t dump_ops(corr_t h, void* vis, int vis_fp64, bool scales, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (h->part_pending) {
        if (scales)
            e = launch_scales_from_partial(h->partial, h->N, h->C, h->P, h->n_spec,
                                           h->scale_target, h->scale, st);
        if (e == cudaSuccess) e = launch_dump_partial(h->partial, h->C, h->P, vis, vis_fp64, st);
        h->part_pending = false;
    } else {
        if (scales)
            e = launch_scales_from_autos(h->acc, h->N, h->C, h->P, h->n_spec, h->scale_target,
                                         h->scale, st);
        if (e == cudaSuccess) e = launch_dump(h->acc, h->C, h->P, vis, vis_fp64, st);
    }
    h->acc_zero = true;
    return e;
}

// Queue the dump of the integration into `vis` on the handle's stream.
int enqueue_dump(corr_t h, void* vis, int vis_fp64, bool dev) {
    int frc = flush(h);
    if (frc != CORR_OK) return frc;
    const size_t bytes = (size_t)h->C * h->P * (vis_fp64 ? sizeof(double2) : sizeof(float2));
    void* out = vis;
    if (!dev) {
        if (!h->vis_dev) CUDA_TRY(h, dev_malloc(&h->vis_dev, (size_t)h->C * h->P * sizeof(double2)));
        out = h->vis_dev;
    }
    // the next integration is scaled from this one's autocorrelations
    const bool scales = narrow(h) && !h->scales_user && h->n_spec > 0;
    prof_begin(h);
    CUDA_TRY(h, dump_ops(h, out, vis_fp64, scales, h->stream));
    if (scales) h->scales_ready = true;
    prof_end(h, CORR_KERNEL_DUMP);
    if (!dev) CUDA_TRY(h, cudaMemcpyAsync(vis, out, bytes, cudaMemcpyDeviceToHost, h->stream));
    return CORR_OK;
}

}  // namespace

int corr_dump(corr_t h, void* vis, int64_t* n_spec, int vis_fp64) {
    if (!h) return CORR_EINVAL;
    if (!vis) return set_err(h, CORR_EINVAL, "vis is NULL");
    int rc = enqueue_dump(h, vis, vis_fp64, is_device_ptr(vis));
    if (rc != CORR_OK) return rc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    rc = check_status(h);
    if (n_spec) *n_spec = h->n_spec;
    h->n_spec = 0;
    return rc;
}

int corr_dump_async(corr_t h, void* vis, int64_t* n_spec, int vis_fp64) {
    if (!h) return CORR_EINVAL;
    if (!vis) return set_err(h, CORR_EINVAL, "vis is NULL");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, vis) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, CORR_EINVAL, "corr_dump_async needs device or page-locked host memory");
    }
    const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (!dev && at.type != cudaMemoryTypeHost)
        return set_err(h, CORR_EINVAL, "corr_dump_async needs device or page-locked host memory");
    int rc = enqueue_dump(h, vis, vis_fp64, dev);
    if (rc != CORR_OK) return rc;
    if (n_spec) *n_spec = h->n_spec;
    h->n_spec = 0;
    return CORR_OK;
}

int corr_sync(corr_t h) {
    if (!h) return CORR_EINVAL;
    int frc = flush(h);
    if (frc != CORR_OK) return frc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_status(h);
}

void corr_destroy(corr_t h) { destroy_impl(h); }

const char* corr_last_error(corr_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int corr_info(corr_t h, int* N, int* K, int* C, int* P, int* dtype) {
    if (!h) return CORR_EINVAL;
    if (N) *N = h->N;
    if (K) *K = h->K;
    if (C) *C = h->C;
    if (P) *P = h->P;
    if (dtype) *dtype = h->dtype;
    return CORR_OK;
}

int corr_set_scales(corr_t h, const float* scales) {
    if (!h) return CORR_EINVAL;
    if (!narrow(h)) return set_err(h, CORR_EINVAL, "scales apply to CORR_FP16 / CORR_FP8E4M3 handles");
    int frc = flush(h);                  // waiting frames were cast with the old scales
    if (frc != CORR_OK) return frc;
    if (!scales) {
        h->scales_user = false;
        h->scales_ready = false;
        return CORR_OK;
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->scale, scales, (size_t)h->N * h->C * sizeof(float),
                                cudaMemcpyDefault, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->scales_user = true;
    h->scales_ready = true;
    return CORR_OK;
}

int corr_get_scales(corr_t h, float* scales) {
    if (!h) return CORR_EINVAL;
    if (!narrow(h)) return set_err(h, CORR_EINVAL, "scales apply to CORR_FP16 / CORR_FP8E4M3 handles");
    if (!scales) return set_err(h, CORR_EINVAL, "scales is NULL");
    if (!h->scales_ready) return set_err(h, CORR_ESTATE, "no scales yet: push data or set them");
    CUDA_TRY(h, cudaMemcpyAsync(scales, h->scale, (size_t)h->N * h->C * sizeof(float),
                                cudaMemcpyDefault, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CORR_OK;
}

int corr_profile_enable(corr_t h, int on) {
    if (!h) return CORR_EINVAL;
    int jrc = join_fengines(h);          // closes an open span of side launches
    if (jrc != CORR_OK) return jrc;
    h->prof_on = on != 0;
    return CORR_OK;
}

int corr_profile_read(corr_t h, int64_t* launches, double* ms, int n) {
    if (!h) return CORR_EINVAL;
    if (n < 0) return set_err(h, CORR_EINVAL, "n < 0");
    int jrc = join_fengines(h);
    if (jrc != CORR_OK) return jrc;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (int c = 0; c < CORR_KERNEL_COUNT; ++c) {
        for (auto& pr : h->ev_pending[c]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) h->prof_ms[c] += t;
            else cudaGetLastError();
            h->ev_pool.push_back(pr.first);
            h->ev_pool.push_back(pr.second);
        }
        h->ev_pending[c].clear();
    }
    for (int c = 0; c < n && c < CORR_KERNEL_COUNT; ++c) {
        if (launches) launches[c] = h->prof_launches[c];
        if (ms) ms[c] = h->prof_ms[c];
    }
    for (int c = 0; c < CORR_KERNEL_COUNT; ++c) {
        h->prof_launches[c] = 0;
        h->prof_ms[c] = 0.0;
    }
    return CORR_OK;
}

int corr_debug_spectra(corr_t h, const uint8_t* samples, int64_t n, float* spectra) {
    if (!h) return CORR_EINVAL;
    if (n < 0 || n % h->K)
        return set_err(h, CORR_EINVAL, "n=%lld is not a non-negative multiple of K=%d",
                       (long long)n, h->K);
    const int64_t S = n / h->K;
    if (S > h->cap) return set_err(h, CORR_EINVAL, "n/K=%lld exceeds the chunk size %lld",
                                   (long long)S, (long long)h->cap);
    if (S == 0) return CORR_OK;
    if (!samples || !spectra) return set_err(h, CORR_EINVAL, "NULL buffer");
    if (!is_device_ptr(samples) || !is_device_ptr(spectra))
        return set_err(h, CORR_EINVAL, "corr_debug_spectra needs device buffers");
    FengineArgs fa{};
    fa.in = samples;
    fa.N = h->N;
    fa.K = h->K;
    fa.S = S;
    fa.S_pad = S;
    fa.twiddle = h->twiddle;
    fa.corr = h->corr_on ? h->corr_tab : nullptr;
    fa.debug_out = reinterpret_cast<float2*>(spectra);
    CUDA_TRY(h, launch_fengine(fa, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CORR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct corr_batch_s {
    int n = 0;
    corr_t h[kMaxTcModes] = {};
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_frames[kMaxTcModes] = {};
    bool one_f = false;          // a pass's F-engines as one multi-mode launch
    std::string err = "no error";
};

namespace {

int batch_err(corr_batch_t b, int code, const char* msg) {
    b->err = msg;
    return code;
}

int batch_from_handle(corr_batch_t b, int m, int rc) {
    b->err = std::string("mode ") + std::to_string(m) + ": " + b->h[m]->err;
    return rc;
}

void batch_free_graph(corr_batch_t b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

int batch_check(corr_batch_t b, const uint8_t* const* samples, const int64_t* n) {
    for (int m = 0; m < b->n; ++m)
        if (b->h[m]->sdelay_on)
            return batch_err(b, CORR_EINVAL, "a mode has sample delays set; batches do not apply them");
    if (!samples || !n) return batch_err(b, CORR_EINVAL, "NULL argument");
    for (int m = 0; m < b->n; ++m) {
        if (n[m] < 0 || n[m] % b->h[m]->K)
            return batch_err(b, CORR_EINVAL, "a sample count is not a non-negative multiple of K");
        if (n[m] > 0 && !is_device_ptr(samples[m]))
            return batch_err(b, CORR_EINVAL, "batch pushes take device buffers");
    }
    return CORR_OK;
}

// Queue every pass of every mode: per pass index, the F-engine of each mode
// that has that pass, then one tensor-core launch over all of them.
int batch_enqueue(corr_batch_t b, const uint8_t* const* samples, const int64_t* n) {
    int64_t frames[kMaxTcModes], passes = 0;
    for (int m = 0; m < b->n; ++m) {
        frames[m] = n[m] / b->h[m]->K;
        passes = std::max(passes, (frames[m] + b->h[m]->cap - 1) / b->h[m]->cap);
    }
    for (int64_t pi = 0; pi < passes; ++pi) {
        TcPlan* plans[kMaxTcModes];
        TcRun runs[kMaxTcModes];
        int idx[kMaxTcModes];
        int na = 0;
        FengineArgs fas[kMaxTcModes];
        for (int m = 0; m < b->n; ++m) {
            corr_t h = b->h[m];
            const int64_t f0 = pi * h->cap;
            if (f0 >= frames[m]) continue;
            const int64_t S = std::min(h->cap, frames[m] - f0);
            const int64_t rec = (int64_t)h->N * (h->K / 2);
            if (b->one_f) {
                if (narrow(h) && !h->scales_ready) {
                    int rc = estimate_scales(h, samples[m] + f0 * rec, S);
                    if (rc != CORR_OK) return batch_from_handle(b, m, rc);
                }
                fas[na] = fengine_args(h, samples[m] + f0 * rec, S, false, 0);
            } else {
                int rc = fengine_pass(h, samples[m] + f0 * rec, S, false, 0);
                if (rc != CORR_OK) return batch_from_handle(b, m, rc);
            }
            TcRun r{};
            r.S_pad = pad_frames(S);
            r.partial = h->partial;
            r.acc = h->acc;
            r.scale = h->scale;
            r.split = split_table(h, false);
            r.status = h->status;
            plans[na] = h->tc;
            runs[na] = r;
            idx[na++] = m;
        }
        corr_t h0 = b->h[idx[0]];
        if (b->one_f) {
            // every mode's F-engine of this pass in one launch
            prof_begin(h0);
            cudaError_t fe = launch_fengine_multi(fas, na, b->stream);
            if (fe != cudaSuccess) {
                cudaGetLastError();
                return batch_err(b, CORR_ECUDA, (std::string("multi-mode F-engine launch: ") +
                                                 cudaGetErrorString(fe)).c_str());
            }
            prof_end(h0, CORR_KERNEL_FENGINE);
        } else {
            // the modes' F-engines run side by side; the launch waits for all
            for (int a = 0; a < na; ++a) {
                int rc = join_fengines(b->h[idx[a]]);
                if (rc != CORR_OK) return batch_from_handle(b, idx[a], rc);
            }
        }
        // one tensor-core launch over all of them (it overwrites their partials)
        for (int a = 0; a < na; ++a) {
            int src = settle_partial(b->h[idx[a]]);
            if (src != CORR_OK) return batch_from_handle(b, idx[a], src);
        }
        prof_begin(h0);
        int rc = tc_launch(plans, na, runs, b->stream, b->err);
        if (rc != CORR_OK) return rc;
        prof_end(h0, CORR_KERNEL_XENGINE);
        for (int a = 0; a < na; ++a) {
            rc = finish_tc_run(b->h[idx[a]], runs[a], b->h[idx[a]]->acc);
            if (rc != CORR_OK) return batch_from_handle(b, idx[a], rc);
        }
    }
    for (int m = 0; m < b->n; ++m) b->h[m]->n_spec += frames[m];
    return CORR_OK;
}

}  // namespace

extern "C" {

int corr_batch_create(corr_batch_t* out, int n_modes, const int* N, const int* K, int dtype) {
    if (!out) return set_err(nullptr, CORR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_modes < 1 || n_modes > kMaxTcModes || !N || !K)
        return set_err(nullptr, CORR_EINVAL, "a batch holds 1 to %d modes", kMaxTcModes);
    if (dtype != CORR_FP32 && dtype != CORR_FP16 && dtype != CORR_FP8E4M3)
        return set_err(nullptr, CORR_EINVAL, "a batch runs on the tensor cores (FP32, FP16, FP8)");
    corr_batch_t b = new (std::nothrow) corr_batch_s();
    if (!b) return set_err(nullptr, CORR_ENOMEM, "host allocation failed");
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return set_err(nullptr, CORR_ECUDA, "stream creation failed");
    }
    for (int m = 0; m < n_modes; ++m) {
        int rc = corr_create(&b->h[m], N[m], K[m], dtype);
        if (rc == CORR_OK) rc = corr_set_stream(b->h[m], b->stream);
        if (rc != CORR_OK) {
            std::string msg = std::string("mode ") + std::to_string(m) + ": " +
                              corr_last_error(b->h[m] ? b->h[m] : nullptr);
            b->n = m + 1;
            corr_batch_destroy(b);
            return set_err(nullptr, rc, "%s", msg.c_str());
        }
        b->n = m + 1;
    }
    *out = b;
    return CORR_OK;
}

int corr_batch_set_chunk(corr_batch_t b, int64_t max_spectra) {
    if (!b) return CORR_EINVAL;
    batch_free_graph(b);
    for (int m = 0; m < b->n; ++m) {
        int rc = corr_set_chunk(b->h[m], max_spectra);
        if (rc != CORR_OK) return batch_from_handle(b, m, rc);
    }
    return CORR_OK;
}

int corr_batch_set_tiles(corr_batch_t b, int window, int stages, int split, int atoms) {
    if (!b) return CORR_EINVAL;
    batch_free_graph(b);
    for (int m = 0; m < b->n; ++m) {
        int rc = corr_set_tiles(b->h[m], window, stages, split, atoms);
        if (rc != CORR_OK) return batch_from_handle(b, m, rc);
    }
    return CORR_OK;
}

int corr_batch_set_one_launch(corr_batch_t b, int on) {
    if (!b) return CORR_EINVAL;
    if (on != 0 && on != 1) return batch_err(b, CORR_EINVAL, "on must be 0 or 1");
    if (b->one_f != (on == 1)) batch_free_graph(b);   // a recorded step has the other form
    b->one_f = on == 1;
    return CORR_OK;
}

int corr_batch_handle(corr_batch_t b, int mode, corr_t* out) {
    if (!b || !out || mode < 0 || mode >= b->n) return CORR_EINVAL;
    *out = b->h[mode];
    return CORR_OK;
}

int corr_batch_get_stream(corr_batch_t b, void** stream) {
    if (!b || !stream) return CORR_EINVAL;
    *stream = b->stream;
    return CORR_OK;
}

int corr_batch_push(corr_batch_t b, const uint8_t* const* samples, const int64_t* n) {
    if (!b) return CORR_EINVAL;
    int rc = batch_check(b, samples, n);
    if (rc != CORR_OK) return rc;
    return batch_enqueue(b, samples, n);
}

int corr_batch_dump(corr_batch_t b, void* const* vis, int64_t* n_spec, int vis_fp64) {
    if (!b || !vis) return CORR_EINVAL;
    for (int m = 0; m < b->n; ++m) {
        int rc = corr_dump(b->h[m], vis[m], n_spec ? &n_spec[m] : nullptr, vis_fp64);
        if (rc != CORR_OK) return batch_from_handle(b, m, rc);
    }
    return CORR_OK;
}

int corr_batch_capture(corr_batch_t b, const uint8_t* const* samples, const int64_t* n,
                       void* const* vis, int vis_fp64) {
    if (!b || !vis) return CORR_EINVAL;
    int rc = batch_check(b, samples, n);
    if (rc != CORR_OK) return rc;
    for (int m = 0; m < b->n; ++m)
        if (!is_device_ptr(vis[m])) return batch_err(b, CORR_EINVAL, "captured dumps take device buffers");
    batch_free_graph(b);
    // One eager step first: scales, kernel attributes and buffers are settled
    // outside the capture.
    rc = batch_enqueue(b, samples, n);
    if (rc == CORR_OK) rc = corr_batch_dump(b, vis, nullptr, vis_fp64);
    if (rc != CORR_OK) return rc;
    bool prof[kMaxTcModes];
    for (int m = 0; m < b->n; ++m) {
        prof[m] = b->h[m]->prof_on;
        b->h[m]->prof_on = false;
    }
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        rc = batch_enqueue(b, samples, n);
        for (int m = 0; rc == CORR_OK && m < b->n; ++m) {
            corr_t h = b->h[m];
            e = dump_ops(h, vis[m], vis_fp64, narrow(h) && !h->scales_user, b->stream);
            if (e != cudaSuccess) rc = CORR_ECUDA;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e2 != cudaSuccess && rc == CORR_OK) {
            rc = CORR_ECUDA;
            e = e2;
        }
        b->graph = g;
        if (rc == CORR_OK) {
            e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e != cudaSuccess) rc = CORR_ECUDA;
        }
    } else {
        rc = CORR_ECUDA;
    }
    for (int m = 0; m < b->n; ++m) {
        b->h[m]->prof_on = prof[m];
        b->graph_frames[m] = n[m] / b->h[m]->K;
        b->h[m]->n_spec = 0;
    }
    if (rc != CORR_OK) {
        cudaGetLastError();
        batch_free_graph(b);
        if (rc == CORR_ECUDA)
            return batch_err(b, rc, (std::string("graph capture: ") + cudaGetErrorString(e)).c_str());
        return rc;
    }
    return CORR_OK;
}

int corr_batch_replay(corr_batch_t b, int64_t* n_spec) {
    if (!b) return CORR_EINVAL;
    if (!b->exec) return batch_err(b, CORR_ESTATE, "no captured step: call corr_batch_capture");
    // a replay is one whole integration per mode: frames pushed eagerly since
    // the last dump would be lost or miscounted
    for (int m = 0; m < b->n; ++m)
        if (b->h[m]->n_spec > 0 || b->h[m]->fill > 0)
            return batch_err(b, CORR_ESTATE, "frames pushed since the last dump: dump before replaying");
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess)
        return batch_err(b, CORR_ECUDA, (std::string("graph launch: ") + cudaGetErrorString(e)).c_str());
    for (int m = 0; n_spec && m < b->n; ++m) n_spec[m] = b->graph_frames[m];
    return CORR_OK;
}

int corr_batch_sync(corr_batch_t b) {
    if (!b) return CORR_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return batch_err(b, CORR_ECUDA, cudaGetErrorString(cudaGetLastError()));
    for (int m = 0; m < b->n; ++m) {
        int rc = check_status(b->h[m]);
        if (rc != CORR_OK) return batch_from_handle(b, m, rc);
    }
    return CORR_OK;
}

void corr_batch_destroy(corr_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_graph(b);
    for (int m = 0; m < b->n; ++m) corr_destroy(b->h[m]);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* corr_batch_last_error(corr_batch_t b) { return b ? b->err.c_str() : corr_last_error(nullptr); }

}  // extern "C"
