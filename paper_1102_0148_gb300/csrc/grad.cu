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
// FP64 throughout.  The factors a_n[k] are tabulated once (N x K/2
// sincospi); CTA (m, chunk) forms B_m[k] for 32 channels, 8 antenna groups
// per channel summed in a fixed order, and its share of the sums over k; a
// last kernel adds the chunks of each antenna in order, so the result is
// deterministic.
#include "corr_internal.h"

namespace gbcorr {
namespace {

constexpr int kGradCh = 32;       // channels per CTA
constexpr int kGradGroups = 8;    // antenna groups per channel
constexpr int kGradThreads = kGradCh * kGradGroups;

__device__ __forceinline__ double2 cmulD(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjD(double2 a) { return make_double2(a.x, -a.y); }

template <typename GT>
__device__ __forceinline__ double2 gload(const void* G, int64_t idx) {
    const GT v = static_cast<const GT*>(G)[idx];
    return make_double2((double)v.x, (double)v.y);
}

// a[n][k] = g_n exp(-2 pi i k tau_n / K)
__global__ void factor_kernel(const float2* gains, const float* delays, int N, int K, double2* a) {
    const int C = K / 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * C; e += gridDim.x * blockDim.x) {
        const int n = e / C;
        const int k = e - n * C;
        const double tau = delays ? (double)delays[n] : 0.0;
        const double2 g = gains ? make_double2(gains[n].x, gains[n].y) : make_double2(1.0, 0.0);
        double sn, cs;
        sincospi(-2.0 * (double)k * tau / (double)K, &sn, &cs);
        a[e] = cmulD(g, make_double2(cs, sn));
    }
}

template <typename GT>
__global__ void __launch_bounds__(kGradThreads) grad_partial_kernel(const double2* R, const void* G,
                                                                    const double2* a,
                                                                    const float* delays, int N,
                                                                    int K, double* part) {
    const int m = blockIdx.x;
    const int chunk = blockIdx.y;
    const int C = K / 2;
    const int P = N * (N + 1) / 2;
    const int kk = threadIdx.x % kGradCh;
    const int grp = threadIdx.x / kGradCh;
    const int k = chunk * kGradCh + kk;
    double2 B = make_double2(0.0, 0.0);
    if (k < C) {
        for (int n = grp; n < N; n += kGradGroups) {
            const double2 a_n = a[(int64_t)n * C + k];
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
    }
    __shared__ double2 sB[kGradGroups][kGradCh];
    sB[grp][kk] = B;
    __syncthreads();
    if (threadIdx.x >= kGradCh) return;
    double gg_re = 0.0, gg_im = 0.0, gt = 0.0;
    if (k < C) {
        double2 Bs = sB[0][kk];
        for (int g = 1; g < kGradGroups; ++g) {
            Bs.x += sB[g][kk].x;
            Bs.y += sB[g][kk].y;
        }
        const double2 ga = conjD(Bs);                      // grad_a_m[k]
        const double tau_m = delays ? (double)delays[m] : 0.0;
        double sn, cs;
        sincospi(2.0 * (double)k * tau_m / (double)K, &sn, &cs);   // conj(phi_m[k])
        const double2 t = cmulD(ga, make_double2(cs, sn));
        gg_re = t.x;
        gg_im = t.y;
        // a_m[k] and d a_m / d tau = (-2 pi i k / K) a_m
        const double2 a_m = a[(int64_t)m * C + k];
        const double w = -2.0 * M_PI * (double)k / (double)K;
        const double2 da = make_double2(-w * a_m.y, w * a_m.x);
        gt = ga.x * da.x + ga.y * da.y;                  // Re(conj(ga) da)
    }
    // sum over the 32 channels, a fixed shuffle tree
    for (int off = kGradCh / 2; off > 0; off >>= 1) {
        gg_re += __shfl_down_sync(0xffffffffu, gg_re, off);
        gg_im += __shfl_down_sync(0xffffffffu, gg_im, off);
        gt += __shfl_down_sync(0xffffffffu, gt, off);
    }
    if (kk == 0) {
        double* o = part + ((int64_t)m * gridDim.y + chunk) * 3;
        o[0] = gg_re;
        o[1] = gg_im;
        o[2] = gt;
    }
}

__global__ void grad_final_kernel(const double* part, int N, int nchunk, float2* grad_g,
                                  float* grad_tau) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < nchunk; ++c) {
        const double* o = part + ((int64_t)m * nchunk + c) * 3;
        s0 += o[0];
        s1 += o[1];
        s2 += o[2];
    }
    grad_g[m] = make_float2((float)s0, (float)s1);
    grad_tau[m] = (float)s2;
}

}  // namespace

size_t grad_scratch_bytes(int N, int K) {
    const int C = K / 2;
    const int nchunk = (C + kGradCh - 1) / kGradCh;
    return (size_t)N * C * sizeof(double2) + (size_t)N * nchunk * 3 * sizeof(double);
}

cudaError_t launch_grad(const double2* R, const void* G, int G_fp64, const float2* gains,
                        const float* delays, int N, int K, float2* grad_g, float* grad_tau,
                        void* scratch, cudaStream_t st) {
    const int C = K / 2;
    const int nchunk = (C + kGradCh - 1) / kGradCh;
    double2* a = static_cast<double2*>(scratch);
    double* part = reinterpret_cast<double*>(a + (size_t)N * C);
    const int fb = (N * C + 255) / 256;
    factor_kernel<<<fb < 1216 ? fb : 1216, 256, 0, st>>>(gains, delays, N, K, a);
    dim3 grid((unsigned)N, (unsigned)nchunk);
    if (G_fp64)
        grad_partial_kernel<double2><<<grid, kGradThreads, 0, st>>>(R, G, a, delays, N, K, part);
    else
        grad_partial_kernel<float2><<<grid, kGradThreads, 0, st>>>(R, G, a, delays, N, K, part);
    grad_final_kernel<<<(N + 127) / 128, 128, 0, st>>>(part, N, nchunk, grad_g, grad_tau);
    return cudaGetLastError();
}

}  // namespace gbcorr
