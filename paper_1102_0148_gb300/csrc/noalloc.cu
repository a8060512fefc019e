// corr_correlate_noalloc: a one-shot correlation that allocates no memory.
//
// Some callers cannot call cudaMalloc: a hard real-time acquisition loop,
// where cudaMalloc/cudaFree may synchronise the whole device and stall the
// stream that is draining the digitiser; or a host application whose device
// memory is entirely owned by another allocator (a framework's memory pool
// reserved up front), where a fresh cudaMalloc can fail or fragment it.  For
// them this entry point runs the FP32 CUDA-core path (the same F-engine and
// X-engine kernels as a CORR_FP32_SIMT handle) with every intermediate buffer
// carved out of one fixed array compiled into this library.
#include "corr_internal.h"

#include <cuda.h>

#include <cstdio>
#include <mutex>

namespace {

using namespace gbcorr;

// 32 MiB of scratch per device.  Every GPU on which the library's code is
// loaded holds this array until the process exits.
constexpr size_t kScratchBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress, looked up once per device and context: the context
// it was looked up in is kept beside it, and a different current context
// (the device was reset and its context re-created, which can load the
// module at another address) triggers a fresh lookup.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, reached through the runtime's entry-point
// query (the library links no driver import library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

constexpr int64_t kSplit = 256;     // fewest frames per X-engine split (sizes the partials)
constexpr int64_t kMaxPass = 2048;  // frames per pass at most

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch layout for one pass of S frames (S a multiple of kSpecPad):
// twiddles | FP64 accumulator [C][P] | partials [splits][C][P] | spectra (tile-major workspace, 32-frame tiles).
size_t scratch_bytes(int N, int K, int64_t S) {
    const size_t C = (size_t)K / 2, P = (size_t)N * (N + 1) / 2;
    const size_t splits = (size_t)((S + kSplit - 1) / kSplit);
    return al256((size_t)K * sizeof(float2)) + al256(C * P * sizeof(double2)) +
           al256(splits * C * P * sizeof(float2)) + al256(C * 2 * (size_t)N * (size_t)S * sizeof(float));
}

// W_K^m = exp(-2 pi i m / K) for m in [0, K), from an exact integer angle in FP64.
__global__ void noalloc_twiddles(float2* tw, int K) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < K; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)K, &s, &c);
        tw[m] = make_float2((float)c, (float)s);
    }
}

int fail(int code, const char* fmt, long long a = 0, long long b = 0, long long c = 0,
         long long d = 0) {
    char buf[320];
    snprintf(buf, sizeof buf, fmt, a, b, c, d);
    set_global_error(buf);
    return code;
}

int fail_cuda(cudaError_t e, const char* what) {
    char buf[320];
    snprintf(buf, sizeof buf, "corr_correlate_noalloc: %s: %s", what, cudaGetErrorString(e));
    set_global_error(buf);
    return CORR_ECUDA;
}

}  // namespace

extern "C" int corr_correlate_noalloc(const uint8_t* samples, int64_t n, int N, int K, float* vis,
                                      void* stream) {
    if (N < 1 || N > CORR_MAX_N)
        return fail(CORR_EINVAL, "corr_correlate_noalloc: N=%lld outside [1, %lld]", N, CORR_MAX_N);
    if (K < 16 || K > 4096 || (K & (K - 1)))
        return fail(CORR_EINVAL, "corr_correlate_noalloc: K=%lld is not a power of two in [16, 4096]",
                    K);
    if (n < 0 || n % K)
        return fail(CORR_EINVAL, "corr_correlate_noalloc: n=%lld is not a non-negative multiple of K=%lld",
                    n, K);
    const size_t need = scratch_bytes(N, K, kSpecPad);
    if (need > kScratchBytes)
        return fail(CORR_EINVAL,
                    "corr_correlate_noalloc: N=%lld, K=%lld needs %lld bytes of scratch, more than "
                    "the fixed %lld bytes this entry point has",
                    N, K, (long long)need, (long long)kScratchBytes);
    if (!samples || !vis) return fail(CORR_EINVAL, "corr_correlate_noalloc: NULL buffer");

    int64_t S_pass = kSpecPad;
    while (S_pass + kSpecPad <= kMaxPass && scratch_bytes(N, K, S_pass + kSpecPad) <= kScratchBytes)
        S_pass += kSpecPad;

    // Set-up, once per device, with that device current.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(CORR_EUNSUPPORTED, "corr_correlate_noalloc: device %lld", dev);
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        CUcontext ctx = nullptr;
        CtxGetCurrentFn cur = ctx_get_current();
        if (cur && cur(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        if (!g_scratch_addr[dev] || (ctx && ctx != g_scratch_ctx[dev])) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress");
            g_scratch_addr[dev] = p;
            if (!ctx && cur && cur(&ctx) != CUDA_SUCCESS) ctx = nullptr;   // created by the lookup
            g_scratch_ctx[dev] = ctx;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    }

    const int C = K / 2;
    const int P = N * (N + 1) / 2;
    const int max_split = (int)((S_pass + kSplit - 1) / kSplit);
    float2* tw = reinterpret_cast<float2*>(base);
    double2* acc = reinterpret_cast<double2*>(base + al256((size_t)K * sizeof(float2)));
    float2* part = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(acc) +
                                             al256((size_t)C * P * sizeof(double2)));
    float* spec = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(part) +
                                           al256((size_t)max_split * C * P * sizeof(float2)));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The array keeps the previous call's contents: clear the accumulator.
    e = cudaMemsetAsync(acc, 0, (size_t)C * P * sizeof(double2), st);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
    noalloc_twiddles<<<(K + 255) / 256, 256, 0, st>>>(tw, K);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "twiddle kernel");

    const int64_t frames = n / K;
    for (int64_t f0 = 0; f0 < frames; f0 += S_pass) {
        const int64_t S = frames - f0 < S_pass ? frames - f0 : S_pass;
        const int64_t S_pad = (S + kSpecPad - 1) / kSpecPad * kSpecPad;
        FengineArgs fa{};
        fa.in = samples + f0 * (int64_t)N * (K / 2);
        fa.N = N;
        fa.K = K;
        fa.S = S;
        fa.S_pad = S_pad;
        fa.twiddle = tw;
        fa.corr = nullptr;
        fa.spec = spec;
        fa.s_base = 0;
        fa.spec_type = SPEC_F32;
        fa.scale = nullptr;
        fa.debug_out = nullptr;
        if ((e = launch_fengine(fa, st)) != cudaSuccess) return fail_cuda(e, "F-engine");
        XengineArgs xa{};
        xa.spec = spec;
        xa.N = N;
        xa.C = C;
        xa.S_pad = S_pad;
        xa.spec_type = SPEC_F32;
        xa.max_split = max_split;
        xa.partial = part;
        if ((e = launch_xengine_simt(xa, st)) != cudaSuccess) return fail_cuda(e, "X-engine");
        if ((e = launch_reduce_partials(part, xa.n_split, (int64_t)C * P, acc, st)) != cudaSuccess)
            return fail_cuda(e, "reduction");
    }
    if ((e = launch_dump(acc, C, P, vis, 0, st)) != cudaSuccess) return fail_cuda(e, "dump");
    return CORR_OK;
}
