// Backward of the visibilities with respect to the per-antenna gains and
// delays applied in the F-engine (Sec. 2.1: a phase per stream applied before
// accumulation).
//
// With a_n[k] = g_n exp(-2 pi i k tau_n / K) and X the uncorrected spectra,
// every output is V_ij[k] = sum_s a_i X_i conj(a_j X_j) = a_i conj(a_j) R_ij[k],
// R the uncorrected visibilities (recomputed pass by pass from the samples by
// the F- and X-engine with corrections off -- spectra are never stored).
// For a real loss L and the incoming gradient G = dL/dRe V + i dL/dIm V
// (PyTorch's convention), dL = sum_p Re(conj(G_p) dV_p) gives
//   dL = sum_m Re(da_m B_m),  B_m[k] = sum_n F_mn[k] conj(a_n[k]) R_mn[k],
//   F_mn = conj(G_mn) (n > m),  G_nm (n < m),  2 Re G_mm (n = m),
// with R_mn = conj(R_nm) below the diagonal.  Hence grad_a_m = conj(B_m) and
//   grad_g_m   = sum_k grad_a_m[k] exp(+2 pi i k tau_m / K),
//   grad_tau_m = sum_k Re(conj(grad_a_m[k]) (-2 pi i k / K) a_m[k]).
// One CTA per antenna m; threads over channels; FP64 throughout; the sums
// over k are block reductions in a fixed order (deterministic).
#include "corr_internal.h"

namespace gbcorr {
namespace {

constexpr int kGradThreads = 256;

__device__ __forceinline__ double2 cmulD(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjD(double2 a) { return make_double2(a.x, -a.y); }

template <typename GT>
__device__ __forceinline__ double2 gload(const void* G, int64_t idx) {
    const GT v = static_cast<const GT*>(G)[idx];
    return make_double2((double)v.x, (double)v.y);
}

template <typename GT>
__global__ void __launch_bounds__(kGradThreads) grad_kernel(const double2* R, const void* G,
                                                            const float2* gains,
                                                            const float* delays, int N, int K,
                                                            float2* grad_g, float* grad_tau) {
    const int m = blockIdx.x;
    const int C = K / 2;
    const int P = N * (N + 1) / 2;
    double gg_re = 0.0, gg_im = 0.0, gt = 0.0;
    const double tau_m = delays ? (double)delays[m] : 0.0;
    const double2 g_m = gains ? make_double2(gains[m].x, gains[m].y) : make_double2(1.0, 0.0);
    for (int k = threadIdx.x; k < C; k += kGradThreads) {
        double2 B = make_double2(0.0, 0.0);
        for (int n = 0; n < N; ++n) {
            const double tau_n = delays ? (double)delays[n] : 0.0;
            const double2 g_n = gains ? make_double2(gains[n].x, gains[n].y) : make_double2(1.0, 0.0);
            double sn, cs;
            sincospi(-2.0 * (double)k * tau_n / (double)K, &sn, &cs);
            const double2 a_n = cmulD(g_n, make_double2(cs, sn));
            double2 F, Rmn;
            if (n > m) {
                const int p = m * N - m * (m - 1) / 2 + (n - m);
                F = conjD(gload<GT>(G, (int64_t)p * C + k));
                Rmn = R[(int64_t)k * P + p];
            } else if (n < m) {
                const int p = n * N - n * (n - 1) / 2 + (m - n);
                F = gload<GT>(G, (int64_t)p * C + k);
                Rmn = conjD(R[(int64_t)k * P + p]);
            } else {
                const int p = m * N - m * (m - 1) / 2;
                F = make_double2(2.0 * gload<GT>(G, (int64_t)p * C + k).x, 0.0);
                Rmn = R[(int64_t)k * P + p];
            }
            const double2 t = cmulD(F, cmulD(conjD(a_n), Rmn));
            B.x += t.x;
            B.y += t.y;
        }
        const double2 ga = conjD(B);                       // grad_a_m[k]
        double sn, cs;
        sincospi(2.0 * (double)k * tau_m / (double)K, &sn, &cs);   // conj(phi_m[k])
        const double2 t = cmulD(ga, make_double2(cs, sn));
        gg_re += t.x;
        gg_im += t.y;
        // a_m[k] and d a_m / d tau = (-2 pi i k / K) a_m
        const double2 a_m = cmulD(g_m, make_double2(cs, -sn));
        const double w = -2.0 * M_PI * (double)k / (double)K;
        const double2 da = make_double2(-w * a_m.y, w * a_m.x);
        gt += ga.x * da.x + ga.y * da.y;                  // Re(conj(ga) da)
    }
    __shared__ double red[3][kGradThreads];
    red[0][threadIdx.x] = gg_re;
    red[1][threadIdx.x] = gg_im;
    red[2][threadIdx.x] = gt;
    __syncthreads();
    for (int w = kGradThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        grad_g[m] = make_float2((float)red[0][0], (float)red[1][0]);
        grad_tau[m] = (float)red[2][0];
    }
}

}  // namespace

cudaError_t launch_grad(const double2* R, const void* G, int G_fp64, const float2* gains,
                        const float* delays, int N, int K, float2* grad_g, float* grad_tau,
                        cudaStream_t st) {
    if (G_fp64)
        grad_kernel<double2><<<N, kGradThreads, 0, st>>>(R, G, gains, delays, N, K, grad_g, grad_tau);
    else
        grad_kernel<float2><<<N, kGradThreads, 0, st>>>(R, G, gains, delays, N, K, grad_g, grad_tau);
    return cudaGetLastError();
}

}  // namespace gbcorr
