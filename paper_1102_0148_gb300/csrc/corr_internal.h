// Internal declarations shared by the gbcorr translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cmath>
#include <cstdint>
#include <string>

#include "corr.h"

namespace gbcorr {

// Element type of the corner-turned spectra workspace.
//   SPEC_F32    one FP32 plane (CUDA-core X-engine)
//   SPEC_F16    one FP16 plane of scaled values (precision form)
//   SPEC_F8     one FP8-E4M3 plane of scaled values (precision form)
//   SPEC_F16X2  two FP16 planes, hi = fp16(sigma_i x) and lo = fp16(sigma_i x - hi)
//               with the antenna's power-of-two pre-scale sigma_i (below):
//               ~22 significant bits, the FP32-accurate tensor-core input
enum SpecType { SPEC_F32 = 0, SPEC_F16 = 1, SPEC_F8 = 2, SPEC_F16X2 = 3 };

inline int spec_elem_bytes(int t) {
    return t == SPEC_F32 ? 4 : ((t == SPEC_F16 || t == SPEC_F16X2) ? 2 : 1);
}
inline int spec_planes(int t) { return t == SPEC_F16X2 ? 2 : 1; }

// Row of the corner-turned workspace holding plane (0 = Re, 1 = Im) of
// antenna i: 2 i + plane, the real and imaginary rows of an antenna side by
// side.  Antennas are grouped in blocks of 64 (the X-engine's tiles): block b
// occupies rows 128 b .. 128 b + 2 nb - 1, nb = min(64, N - 64 b).  With the
// rows of one antenna adjacent, an F-engine CTA's two rows of a channel and
// plane are one contiguous run of whole 128-byte lines (2 x 64 bytes for the
// 32-frame FP16 tiles below).
__host__ __device__ __forceinline__ int spec_row(int plane, int i, int N) {
    (void)N;
    return 2 * i + plane;
}

// Pre-scale of the two-plane FP16 split (SPEC_F16X2), one power of two per
// antenna.  A 4-bit input bounds every transform value, |X[k]| <= 8K (all
// samples -8), and a correction keeps |Y| = |a_i[k]| |X| = |g_i| |X|, so
//   sigma_i = 2^floor(log2(2^15 / (8 K |g_i|)))
// puts every sigma_i |Y| at or below 2^15, half the FP16 range limit (65504),
// whatever the gain, while the typical value (rms ~ sqrt(K) 2 |g_i|) stays
// hundreds of times above the FP16 subnormal range.  Powers of two make the
// scaling and the descaling by 1/(sigma_i sigma_j) in the X-engine exact.
// The exponent is clamped to [-60, 60] (zero gain takes 2^60).
constexpr double kSplitBound = 32768.0;
constexpr int kSplitExpMax = 60;
inline float split_scale_for(double gabs, int K) {
    if (!(gabs > 0.0)) return ldexpf(1.0f, kSplitExpMax);
    int e = (int)floor(log2(kSplitBound / (8.0 * K * gabs)));
    e = e < -kSplitExpMax ? -kSplitExpMax : (e > kSplitExpMax ? kSplitExpMax : e);
    return ldexpf(1.0f, e);
}
// Gains accepted by corr_set_corrections: 0 or 2^-40 <= |g| <= 2^40 (finite),
// so the descaled visibilities stay inside the FP32 range.
constexpr double kGainMin = 9.094947017729282e-13;   // 2^-40
constexpr double kGainMax = 1099511627776.0;         // 2^40

// Spectra are padded with zero frames up to a multiple of this many frames,
// so every X-engine tile along the spectrum axis is whole.
constexpr int kSpecPad = 128;

// Workspace layout, tile-major along the spectra: frames come in tiles of T
// = 32 (FP32: 128-byte rows; FP16 and the FP16 pair: 64-byte rows, the
// X-engine's 64-byte-swizzled k-tile) or 128 (FP8: 128-byte rows), and
// element (k, r, s) of a plane sits at ((s / T * C + k) * 2N + r) * T + s % T.
// One (tile, channel) holds all 2N rows contiguously, so the X-engine reads a
// k-tile of a channel as one block and an F-engine CTA's 32 frames of an
// antenna fill whole tile rows.  Planes (SPEC_F16X2) are plane_stride =
// C * 2N * cap elements apart.
inline __host__ __device__ int spec_tile_shift(int t) {
    return t == SPEC_F8 ? 7 : 5;
}
__host__ __device__ __forceinline__ int64_t spec_off(int k, int r, int64_t s, int N, int C,
                                                     int tshift) {
    return ((((s >> tshift) * C + k) * (2 * N) + r) << tshift) + (s & ((1 << tshift) - 1));
}

// Arguments of one F-engine pass over S frames of one input buffer.
struct FengineArgs {
    const uint8_t* in;       // [S][N][K/2] packed bytes (device)
    int N, K;
    int64_t S;               // frames to transform
    int64_t S_pad;           // frames written (>= S; the extra ones are zero)
    const float2* twiddle;   // W_K^m = exp(-2 pi i m / K), m in [0, K)
    const float2* corr;      // [N][K/2] correction a_i[k], or nullptr
    // Corner-turned workspace (spec_off): row r = spec_row(plane, antenna),
    // frames s_base .. s_base + S_pad - 1 of it written by this pass.
    void* spec;
    int64_t s_base;
    int64_t plane_stride;    // elements from the hi plane to the lo plane (SPEC_F16X2)
    int spec_type;
    const float* scale;      // [N][K/2] pre-cast scale (FP16/FP8 only)
    const float* split;      // [N] pre-scale sigma_i of the two-plane split (SPEC_F16X2 only)
    // Debug layout instead: float2 [N][S][K/2] (spec is ignored when set).
    float2* debug_out;
    // Set by launch_fengine: the K = 512 grid runs antenna fastest
    // (blockIdx.x = antenna) unless its frame blocks exceed gridDim.y's limit.
    int ant_x;
};

cudaError_t launch_fengine(const FengineArgs& a, cudaStream_t st);
// The F-engines of n modes (1 <= n <= 4, one workspace element type, no
// debug output) as one launch: each mode's frames as its own kernel would
// transform them.
cudaError_t launch_fengine_multi(const FengineArgs* modes, int n, cudaStream_t st);

// Coarse integer delays on the packed stream: out = in delayed by delays[i]
// samples (0..K) per antenna, S frames [S][N][K/2].  The frame before the
// chunk comes from hist_in ([N][K/2], zeros when NULL); the chunk's last
// frame is copied to hist_out when it is not NULL.
cudaError_t launch_sample_delay(const uint8_t* in, int64_t S, int N, int K, const int* delays,
                                const uint8_t* hist_in, uint8_t* hist_out, uint8_t* out,
                                cudaStream_t st);

// Correction table a[i][k] = g_i exp(-2 pi i k tau_i / K), computed in FP64.
cudaError_t launch_correction_table(const float2* gains, const float* delays, int N, int K,
                                    float2* table, cudaStream_t st);

// SIMT X-engine over one workspace pass: partial[split][k][p] (FP32 complex).
struct XengineArgs {
    const void* spec;        // FP32 workspace (spec_off), frames from 0
    int N, C;
    int64_t S_pad;           // frames present (multiple of kSpecPad)
    int spec_type;
    int max_split;           // partial slots available ([max_split][C][P])
    int64_t s_per_split;     // set by the launch: frames per split (multiple of 32)
    int n_split;             // set by the launch: splits (<= max_split)
    float2* partial;         // [n_split][C][P]
    const float* scale;      // [N][C] pre-cast scales (FP16/FP8), else nullptr
    int* status;             // device status word (bounded waits)
};

// Chooses the split of the pass (a.s_per_split, a.n_split) and launches.
cudaError_t launch_xengine_simt(XengineArgs& a, cudaStream_t st);

// acc[k][p] += sum over splits of partial[split][k][p], in a fixed order (FP64);
// assign: acc is known to hold zeros, acc[k][p] = that sum without reading it.
cudaError_t launch_reduce_partials(const float2* partial, int n_split, int64_t CP,
                                   double2* acc, cudaStream_t st, bool assign = false);

// vis[p][k] = acc[k][p] as complex64 (fp64 == 0) or complex128; then acc = 0.
cudaError_t launch_dump(double2* acc, int C, int P, void* vis, int fp64, cudaStream_t st);
// The same from a pass result still in partial slot 0 (part[k][p], FP32),
// with the accumulator already zero: nothing is cleared.
cudaError_t launch_dump_partial(const float2* part, int C, int P, void* vis, int fp64,
                                cudaStream_t st);

// Pre-cast scales s[i][k] = target / sqrt(P/2) from spectra Y[N][S][C] or from
// the autocorrelations of the FP64 accumulator acc[C][P] (or of a pass result
// in partial slot 0) over n_spec spectra.
cudaError_t launch_scales_from_spectra(const float2* Y, int N, int64_t S, int C, float target,
                                       float* scale, cudaStream_t st);
cudaError_t launch_scales_from_autos(const double2* acc, int N, int C, int P, int64_t n_spec,
                                     float target, float* scale, cudaStream_t st);
cudaError_t launch_scales_from_partial(const float2* part, int N, int C, int P, int64_t n_spec,
                                       float target, float* scale, cudaStream_t st);

// Gradient of a real loss of V with respect to the gains and delays, from the
// uncorrected visibilities R ([C][P] FP64) and G = dL/dRe V + i dL/dIm V
// ([P][C], complex64 or complex128).
cudaError_t launch_grad(const double2* R, const void* G, int G_fp64, const float2* gains,
                        const float* delays, int N, int K, float2* grad_g, float* grad_tau,
                        void* scratch, cudaStream_t st);
size_t grad_scratch_bytes(int N, int K);   // device scratch launch_grad needs

// Message returned by corr_last_error(NULL) on this thread.
void set_global_error(const char* msg);

// cudaMalloc for every device allocation of a handle or plan.  Test hook:
// while the environment variable CORR_TEST_FAIL_ALLOC holds a positive
// integer k, the k-th allocation counted since the variable last changed
// value fails with cudaErrorMemoryAllocation (nothing is allocated).
cudaError_t dev_malloc(void** p, size_t bytes);

}  // namespace gbcorr
