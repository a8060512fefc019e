// F-engine: 4-bit unpack -> optional gain/delay -> K-point real FFT -> the
// corner-turned spectra workspace the X-engine reads.
//
// Paper: Sec. 1 (split each stream into channels with an FFT), Sec. 4
// (forward, unnormalised float FFT; conversion of its output before the
// cross-multiply), Sec. 2.1 (a phase applied per stream before accumulation).
//
// A K-point real transform is done as one K/2-point complex transform of
// z[m] = x[2m] + i x[2m+1] -- exactly one packed input byte per complex
// point -- followed by the split into the transforms of the even and odd
// samples: X[k] = E[k] + W_K^k O[k], E[k] = (Z[k] + conj Z[L-k]) / 2,
// O[k] = (Z[k] - conj Z[L-k]) / 2i, L = K/2.
#include "corr_internal.h"

#include <cuda_fp8.h>

namespace gbcorr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// 4-bit two's complement: nibble v -> v for v < 8, v - 16 otherwise.
__device__ __forceinline__ float nib(unsigned v) { return (float)((int)((v ^ 8u) & 15u) - 8); }

__device__ __forceinline__ void store_spec(void* spec, int t, int64_t off, float v) {
    if (t == SPEC_F32) {
        static_cast<float*>(spec)[off] = v;
    } else if (t == SPEC_F16) {
        static_cast<__half*>(spec)[off] = __float2half_rn(v);
    } else {
        static_cast<__nv_fp8_storage_t*>(spec)[off] =
            __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

// Real transform of one frame, for k = tid, tid + kThreads, ...: the
// complex transform Z (natural order, length L) is in `Z`.
__device__ __forceinline__ float2 real_split(const float2* Z, int k, int L, const float2* tw) {
    const float2 zk = Z[k];
    const float2 zc = Z[(L - k) & (L - 1)];
    // E = (zk + conj zc)/2 ; O = (zk - conj zc)/(2i)
    const float2 E = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
    const float2 O = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
    const float2 t = cmul(O, tw[k]);
    return make_float2(E.x + t.x, E.y + t.y);
}

// Generic F-engine for any power-of-two K: one CTA transforms FT frames of one
// antenna, one frame at a time, with a radix-2 Stockham FFT in shared memory;
// the FT results of each channel are staged and written as one contiguous run
// of the workspace row (k, r).
template <bool DEBUG>
__global__ void __launch_bounds__(kThreads) fengine_generic(FengineArgs a, int FT) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.K >> 1;
    const int C = L;
    float2* bufA = reinterpret_cast<float2*>(smem_raw);
    float2* bufB = bufA + L;
    float* stg = reinterpret_cast<float*>(bufB + L);       // [2][C][FT]
    const int i = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * FT;
    const int tid = threadIdx.x;
    const int64_t s_end = DEBUG ? a.S : a.S_pad;

    for (int f = 0; f < FT; ++f) {
        const int64_t s = s0 + f;
        if (s >= s_end) break;                              // uniform in the CTA
        const bool valid = s < a.S;
        const uint8_t* src = a.in + (s * a.N + i) * (int64_t)L;
        for (int m = tid; m < L; m += kThreads) {
            float2 z = make_float2(0.f, 0.f);
            if (valid) {
                const unsigned b = src[m];
                z = make_float2(nib(b & 15u), nib(b >> 4));
            }
            bufA[m] = z;
        }
        __syncthreads();
        float2* x = bufA;
        float2* y = bufB;
        for (int Ns = 1; Ns < L; Ns <<= 1) {
            const int tstep = a.K / (2 * Ns);              // W_{2Ns}^j = W_K^{j K/(2Ns)}
            for (int j = tid; j < (L >> 1); j += kThreads) {
                const int kk = j & (Ns - 1);
                const float2 v0 = x[j];
                const float2 v1 = cmul(x[j + (L >> 1)], a.twiddle[kk * tstep]);
                const int d = ((j - kk) << 1) + kk;
                y[d] = make_float2(v0.x + v1.x, v0.y + v1.y);
                y[d + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
            }
            __syncthreads();
            float2* t = x;
            x = y;
            y = t;
        }
        for (int k = tid; k < C; k += kThreads) {
            float2 X = real_split(x, k, L, a.twiddle);
            if (a.corr) X = cmul(a.corr[(int64_t)i * C + k], X);
            if (DEBUG) {
                a.debug_out[((int64_t)i * a.S + s) * C + k] = X;
            } else {
                if (a.scale) {
                    const float sc = a.scale[(int64_t)i * C + k];
                    X.x *= sc;
                    X.y *= sc;
                }
                stg[k * FT + f] = X.x;
                stg[(C + k) * FT + f] = X.y;
            }
        }
        __syncthreads();
    }
    if (!DEBUG) {
        const int nfr = (int)min((int64_t)FT, a.S_pad - s0);
        for (int e = tid; e < 2 * C * FT; e += kThreads) {
            const int row = e / FT;
            const int f = e - row * FT;
            if (f >= nfr) continue;
            const int plane = row / C;
            const int k = row - plane * C;
            const int64_t off = ((int64_t)k * 2 * a.N + plane * a.N + i) * a.ld + s0 + f;
            store_spec(a.spec, a.spec_type, off, stg[row * FT + f]);
        }
    }
}

__global__ void correction_table_kernel(const float2* g, const float* tau, int N, int K,
                                        float2* out) {
    const int C = K / 2;
    const int64_t total = (int64_t)N * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / C);
        const int k = (int)(e - (int64_t)i * C);
        const double gr = g ? (double)g[i].x : 1.0;
        const double gi = g ? (double)g[i].y : 0.0;
        const double t = tau ? (double)tau[i] : 0.0;
        double sn, cs;
        sincospi(-2.0 * (double)k * t / (double)K, &sn, &cs);
        out[e] = make_float2((float)(gr * cs - gi * sn), (float)(gr * sn + gi * cs));
    }
}

}  // namespace

cudaError_t launch_fengine(const FengineArgs& a, cudaStream_t st) {
    const int L = a.K / 2;
    const int C = L;
    const bool dbg = a.debug_out != nullptr;
    int FT = 8192 / C;
    FT = FT < 1 ? 1 : (FT > 32 ? 32 : FT);
    const int64_t frames = dbg ? a.S : a.S_pad;
    if (frames <= 0) return cudaSuccess;
    const size_t smem = (size_t)16 * L + (dbg ? 0 : (size_t)8 * C * FT);
    dim3 grid((unsigned)((frames + FT - 1) / FT), (unsigned)a.N);
    cudaError_t e;
    if (dbg) {
        e = cudaFuncSetAttribute(fengine_generic<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        fengine_generic<true><<<grid, kThreads, smem, st>>>(a, FT);
    } else {
        e = cudaFuncSetAttribute(fengine_generic<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fengine_generic<false><<<grid, kThreads, smem, st>>>(a, FT);
    }
    return cudaGetLastError();
}

cudaError_t launch_correction_table(const float2* gains, const float* delays, int N, int K,
                                    float2* table, cudaStream_t st) {
    const int64_t total = (int64_t)N * (K / 2);
    const int blocks = (int)((total + 255) / 256);
    correction_table_kernel<<<blocks, 256, 0, st>>>(gains, delays, N, K, table);
    return cudaGetLastError();
}

}  // namespace gbcorr
