// Per-antenna, per-channel pre-cast scales for the FP16 / FP8 X-engine inputs.
//
// Paper: Sec. 4 -- the F-engine output is converted to a narrower type before
// the cross-multiply, and the precision lost in the conversion is offset by
// prescaling.  Here the scale of antenna i, channel k is chosen so that the
// real and imaginary parts of the scaled spectrum have a target rms:
//   s_i[k] = 2^round(log2(target / sqrt(P_i[k] / 2))),   P_i[k] = mean |Y_i[s,k]|^2,
// with P taken from the autocorrelation V_ii[k] / n_spec of the previous
// integration, or, before the first one, from a short estimation pass.  The
// X-engine divides each visibility by s_i s_j, so the scales never bias V.
// Scales are powers of two: scaling and descaling are then exact, and the
// integer-valued DC channel stays exactly representable in FP16.
#include "corr_internal.h"

namespace gbcorr {
namespace {

__device__ __forceinline__ float scale_for(double power, float target) {
    // power = mean |Y|^2; a silent channel keeps scale 1
    if (!(power > 0.0)) return 1.0f;
    const double e = rint(log2((double)target / sqrt(power * 0.5)));
    return (float)exp2(fmin(fmax(e, -60.0), 60.0));
}

__global__ void scales_from_spectra_kernel(const float2* Y, int N, int64_t S, int C, float target,
                                           float* scale) {
    const int64_t total = (int64_t)N * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / C);
        const int k = (int)(e - (int64_t)i * C);
        double p = 0.0;
        for (int64_t s = 0; s < S; ++s) {
            const float2 y = Y[((int64_t)i * S + s) * C + k];
            p += (double)y.x * y.x + (double)y.y * y.y;
        }
        scale[e] = scale_for(p / (double)S, target);
    }
}

// acc: the FP64 accumulator, or (float2) a pass result still in partial slot 0
template <typename T>
__global__ void scales_from_autos_kernel(const T* acc, int N, int C, int P, int64_t n_spec,
                                         float target, float* scale) {
    const int64_t total = (int64_t)N * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / C);
        const int k = (int)(e - (int64_t)i * C);
        const int p = i * N - i * (i - 1) / 2;      // pair (i, i)
        scale[e] = scale_for((double)acc[(int64_t)k * P + p].x / (double)n_spec, target);
    }
}

int blocks_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_scales_from_spectra(const float2* Y, int N, int64_t S, int C, float target,
                                       float* scale, cudaStream_t st) {
    scales_from_spectra_kernel<<<blocks_for((int64_t)N * C), 256, 0, st>>>(Y, N, S, C, target, scale);
    return cudaGetLastError();
}

cudaError_t launch_scales_from_autos(const double2* acc, int N, int C, int P, int64_t n_spec,
                                     float target, float* scale, cudaStream_t st) {
    scales_from_autos_kernel<double2><<<blocks_for((int64_t)N * C), 256, 0, st>>>(
        acc, N, C, P, n_spec, target, scale);
    return cudaGetLastError();
}

cudaError_t launch_scales_from_partial(const float2* part, int N, int C, int P, int64_t n_spec,
                                       float target, float* scale, cudaStream_t st) {
    scales_from_autos_kernel<float2><<<blocks_for((int64_t)N * C), 256, 0, st>>>(
        part, N, C, P, n_spec, target, scale);
    return cudaGetLastError();
}

}  // namespace gbcorr
