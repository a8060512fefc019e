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
#include "xengine_tc.h"
#include "fengine_k512.cuh"

#include <cuda_fp8.h>

#include <algorithm>

namespace gbcorr {
namespace {

using namespace fk;

constexpr int kThreads = 256;

// 4-bit two's complement: nibble v -> v for v < 8, v - 16 otherwise.
__device__ __forceinline__ float nib(unsigned v) { return (float)((int)((v ^ 8u) & 15u) - 8); }

__device__ __forceinline__ void store_spec(void* spec, int t, int64_t off, float v,
                                           int64_t plane_stride, float sigma) {
    if (t == SPEC_F32) {
        static_cast<float*>(spec)[off] = v;
    } else if (t == SPEC_F16X2) {
        const float xs = v * sigma;
        const __half hi = __float2half_rn(xs);
        const __half lo = __float2half_rn(xs - __half2float(hi));
        static_cast<__half*>(spec)[off] = hi;
        static_cast<__half*>(spec)[off + plane_stride] = lo;
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
// The body: FT frames from s0 of antenna i by kThreads threads (tid), `smem`
// 16 L + (DEBUG ? 0 : 8 C FT) bytes, `sync` a barrier of those threads.
template <bool DEBUG, class Sync>
__device__ __forceinline__ void fgeneric_block(const FengineArgs& a, int FT, int i, int64_t s0,
                                               unsigned char* smem, int tid, Sync sync) {
    const int L = a.K >> 1;
    const int C = L;
    float2* bufA = reinterpret_cast<float2*>(smem);
    float2* bufB = bufA + L;
    float* stg = reinterpret_cast<float*>(bufB + L);       // [2][C][FT]
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
        sync();
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
            sync();
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
        sync();
    }
    if (!DEBUG) {
        const float sigma = a.spec_type == SPEC_F16X2 ? __ldg(a.split + i) : 1.0f;
        const int nfr = (int)min((int64_t)FT, a.S_pad - s0);
        for (int e = tid; e < 2 * C * FT; e += kThreads) {
            const int row = e / FT;
            const int f = e - row * FT;
            if (f >= nfr) continue;
            const int plane = row / C;
            const int k = row - plane * C;
            const int64_t off = spec_off(k, spec_row(plane, i, a.N), a.s_base + s0 + f, a.N, C,
                                         spec_tile_shift(a.spec_type));
            store_spec(a.spec, a.spec_type, off, stg[row * FT + f], a.plane_stride, sigma);
        }
    }
}

template <bool DEBUG>
__global__ void __launch_bounds__(kThreads) fengine_generic(FengineArgs a, int FT) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fgeneric_block<DEBUG>(a, FT, blockIdx.y, (int64_t)blockIdx.x * FT, smem_raw, threadIdx.x,
                          []() { __syncthreads(); });
}

// K = 512 kernel: one 32-frame block of one antenna per CTA (the body is
// in fengine_k512.cuh).
template <int OUT, bool CORR>
__global__ void __launch_bounds__(kF512Threads, 3) fengine_k512(FengineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kScaled = OUT == SPEC_F16 || OUT == SPEC_F8;
    float* stg = reinterpret_cast<float*>(smem_raw);                        // [32][547]
    float2* tw_base = reinterpret_cast<float2*>(stg + kStgFloats);          // [2][4 m][16 t]
    // tables that exist only when used: scales (FP16/FP8), corrections
    float* sc_tab = reinterpret_cast<float*>(tw_base + 128);                // [256] if kScaled
    float2* corr_tab = reinterpret_cast<float2*>(sc_tab + (kScaled ? 256 : 0));   // [256] if a.corr
    // antenna fastest (a.ant_x): neighbouring CTAs read adjacent 256-byte
    // records of the same frames and write adjacent workspace rows
    const int i = a.ant_x ? blockIdx.x : blockIdx.y;
    const int64_t s0 = (int64_t)(a.ant_x ? blockIdx.y : blockIdx.x) * kF512Frames;
    F512Block b;
    b.in = a.in + (s0 * a.N + i) * 256;
    b.stride = (int64_t)a.N * 256;
    b.nvalid = (int)max((int64_t)0, min((int64_t)kF512Frames, a.S - s0));
    b.ant = i;
    b.post = OUT == SPEC_F16X2 ? __ldg(a.split + i) : 1.0f;
    b.spec = static_cast<char*>(a.spec);
    b.s = a.s_base + s0;
    b.N = a.N;
    b.plane_stride = a.plane_stride;
    b.debug = a.debug_out ? a.debug_out + ((int64_t)i * a.S + s0) * 256 : nullptr;
    f512_block<OUT, CORR>(b, a.twiddle, CORR ? a.corr + (int64_t)i * 256 : nullptr,
                          kScaled ? a.scale + (int64_t)i * 256 : nullptr, stg, tw_base, sc_tab,
                          corr_tab, threadIdx.x, []() { __syncthreads(); });
}


// ---------------------------------------------------------------------------
// K = 1024 F-engine: one warp per spectrum, 16 complex points per lane.
//
// The 512-point complex transform is split as n = t + 32 j (lane t < 32,
// register j < 16) and k = k1 + 16 k2:
//   Z[k1 + 16 k2] = sum_t W32^{t k2} [ W512^{t k1} sum_j z[t + 32 j] W16^{j k1} ].
// Stage 1 is an in-register 16-point DFT over j and the twiddle W512^{t k1};
// an exchange through shared memory gives lane l = k1 + 16 h the values of
// its k1 for t = 16 h .. 16 h + 15.  The 32-point transform over t is a
// radix-2 step across the two half-warps (one xor-16 shuffle per register):
//   Z[k1 + 16 h + 32 m] = sum_t' W16^{t' m} W32^{t' h} (B_t' + (-1)^h B_{t'+16})
// followed by an in-register 16-point DFT over t'.  Lane l ends with
// Z[k1 + 16 h + 32 m], m < 16; the partner Z[512 - k] of the real split is in
// lane (16 - k1) mod 16 + 16 (1 - h), register 15 - m (lanes 0 and 16 hold
// their own partners).
// ---------------------------------------------------------------------------

constexpr int kF1024Frames = 16;     // frames per CTA, two per warp
constexpr int kF1024Threads = 256;
constexpr int kX1024Stride = 33;     // exchange row stride (complex)
// Staging rows [frame][2 k + plane] (a channel's Re and Im side by side, one
// 8-byte store).  Row stride (floats): 1058 = 2 mod 32 puts the store phase's
// reads of (4 channels x Re/Im x 4 frame quads) on 32 distinct banks, and a
// row holds one warp's exchange area (16 x 33 complex = 1056 floats) at the
// 16-byte aligned offset 2 (f mod 2).  A warp exchanges through the row of
// its second frame, as in the K = 512 kernel, so three CTAs fit on an SM.
constexpr int kStg1024Row = 1058;
constexpr int kStg1024Floats = kF1024Frames * kStg1024Row;
static_assert(kStg1024Row % 8 == 2 && kStg1024Row >= 16 * kX1024Stride * 2 + 2, "staging row layout");

// The body: 16 frames from s0 of antenna i by kF1024Threads threads (tid),
// `smem` as the kernel's dynamic shared memory, `sync` a barrier of them.
template <int OUT, bool CORR, class Sync>
__device__ __forceinline__ void f1024_block(const FengineArgs& a, int i, int64_t s0,
                                            unsigned char* smem, int tid, Sync sync) {
    constexpr bool DEBUG = OUT == kOutDebug;
    float* stg = reinterpret_cast<float*>(smem);                            // [16][1058]
    float2* tw_base = reinterpret_cast<float2*>(stg + kStg1024Floats);      // [2][4 m][32 t]
    float2* tw32 = tw_base + 256;                                           // [2][16]
    constexpr bool kScaled = OUT == SPEC_F16 || OUT == SPEC_F8;
    float* sc_tab = reinterpret_cast<float*>(tw32 + 32);                    // [512] if kScaled

    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int k1 = lane & 15;
    const int hh = lane >> 4;
    const float post = OUT == SPEC_F16X2 ? __ldg(a.split + i) : 1.0f;
    const float chalf = 0.5f * post;
    // Twiddles as in the K = 512 kernel: the stage twiddle W512^{t q},
    // q = p + 4 r, is W512^{t p} W512^{4 t r} from a table of the six bases,
    // and the split's W1024^k, k = l + 32 q, is W1024^l W32^q.
    {
        const int j = tid >> 7, m = (tid >> 5) & 3, t = tid & 31;
        tw_base[tid] = a.twiddle[2 * t * m * (j ? 4 : 1)];   // W512^{t m 4^j}
    }
    // [2][16]: ones, then W32^{t'} = W1024^{32 t'}
    if (tid < 32) tw32[tid] = tid < 16 ? make_float2(1.0f, 0.0f) : a.twiddle[32 * (tid - 16)];
    // the antenna's pre-cast scales, read once per CTA instead of per output
    if (kScaled)
        for (int e = tid; e < 512; e += kF1024Threads) sc_tab[e] = __ldg(a.scale + (int64_t)i * 512 + e);
    const float2 wl = __ldg(a.twiddle + lane);
    const float2 u = make_float2(chalf * wl.x, chalf * wl.y);   // c W1024^l

    uint4 raw0 = make_uint4(0u, 0u, 0u, 0u), raw1 = raw0;
    {
        const int64_t sa = s0 + warp, sb = sa + 8;
        if (sa < a.S) raw0 = __ldg(reinterpret_cast<const uint4*>(a.in + (sa * a.N + i) * 512) + lane);
        if (sb < a.S) raw1 = __ldg(reinterpret_cast<const uint4*>(a.in + (sb * a.N + i) * 512) + lane);
    }
    sync();

    const int fx = warp + 8;                         // the warp's second frame
    float2* gx = reinterpret_cast<float2*>(stg + fx * kStg1024Row + 2 * (fx & 1));
    unsigned char* gbytes = reinterpret_cast<unsigned char*>(gx);

#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
        const int f = warp + 8 * r;
        const int64_t s = s0 + f;
        *reinterpret_cast<uint4*>(gbytes + 16 * lane) = r == 0 ? raw0 : raw1;
        __syncwarp();
        float2 x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const unsigned b = gbytes[lane + 32 * j];
            x[j] = make_float2(nib_lo(b), nib_hi(b));
        }
        __syncwarp();
        dft16(x);
        {
            float2 wp[4], wr[4];
#pragma unroll
            for (int m = 1; m < 4; ++m) {
                wp[m] = tw_base[m * 32 + lane];
                wr[m] = tw_base[128 + m * 32 + lane];
            }
#pragma unroll
            for (int q = 1; q < 16; ++q) {
                if (q & 3) x[q] = cmul(x[q], wp[q & 3]);
                if (q >> 2) x[q] = cmul(x[q], wr[q >> 2]);
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) gx[q * kX1024Stride + lane] = x[q];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = gx[k1 * kX1024Stride + 16 * hh + t];
        __syncwarp();
        // radix 2 across the half-warps: half 0 forms B_t' + B_t'+16, half 1
        // W32^{t'} (B_t' - B_t'+16).  Both halves run the same instructions,
        // y + sgn x (one packed FMA) times a twiddle row that is all ones for
        // half 0.
        const float sgn = hh ? -1.0f : 1.0f;
        const float2* twh = tw32 + 16 * hh;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            float2 y;
            y.x = __shfl_xor_sync(0xffffffffu, x[t].x, 16);
            y.y = __shfl_xor_sync(0xffffffffu, x[t].y, 16);
            const float2 v = __ffma2_rn(make_float2(sgn, sgn), x[t], y);
            x[t] = t > 0 ? cmul(v, twh[t]) : v;
        }
        dft16(x);
        // x[q] = Z[l + 32 q], l = k1 + 16 hh.  As in the K = 512 kernel, slot
        // q < 8 makes X[k] and X[512 - k] for k = l + 32 q from Z[k] and its
        // partner Z[512 - k], register 15 - q of lane 32 - l (lane 16 is its
        // own partner; lane 0 pairs its own registers q and 16 - q, and its
        // slot 0 makes X[0] and X[256]).
        const int src = (32 - lane) & 31;
        auto emit = [&](int k, float2 X) {
            if (CORR) X = cmul(__ldg(a.corr + (int64_t)i * 512 + k), X);
            if (DEBUG) {
                if (s < a.S) a.debug_out[((int64_t)i * a.S + s) * 512 + k] = X;
            } else {
                if (OUT == SPEC_F16 || OUT == SPEC_F8) {
                    const float sc = sc_tab[k];
                    X.x *= sc;
                    X.y *= sc;
                }
                *reinterpret_cast<float2*>(stg + f * kStg1024Row + 2 * k) = X;
            }
        };
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            float2 zc;
            zc.x = __shfl_sync(0xffffffffu, x[15 - q].x, src);
            zc.y = __shfl_sync(0xffffffffu, x[15 - q].y, src);
            if (lane == 0) zc = x[(16 - q) & 15];
            const float2 zk = x[q];
            const float2 S = add_conj(zk, zc);
            const float2 D = sub_conj(zk, zc);
            // B = w'_k D = -i c W1024^l W32^q D
            const float2 v = cmul(u, w32mul(D, q));
            const float2 B = make_float2(v.y, -v.x);
            emit(k, make_float2(fmaf(chalf, S.x, B.x), fmaf(chalf, S.y, B.y)));
            float2 Xp = make_float2(fmaf(chalf, S.x, -B.x), -fmaf(chalf, S.y, -B.y));
            int kp = 512 - k;
            if (q == 0 && lane == 0) {
                Xp = make_float2(post * x[8].x, -post * x[8].y);
                kp = 256;
            }
            emit(kp, Xp);
        }
    }
    if (DEBUG) return;
    sync();
    // 512 channels x (Re, Im) x 16 frames: lane = 8 c + 4 p + m writes frames
    // 4m .. 4m + 3 of plane p of channel 4 (warp + 8 j) + c.  The Re and Im
    // rows of a channel are adjacent in the workspace (rows 2i, 2i + 1), so
    // one warp store covers 4 channels' pairs of rows: 4 lines where the
    // (plane, channel)-major order touched 8.
    const int m = lane & 3, p = (lane >> 2) & 1, c = lane >> 3;
    for (int cg = warp; cg < 128; cg += kF1024Threads / 32) {
        const int k = 4 * cg + c;
        const float* src = stg + 4 * m * kStg1024Row + 2 * k + p;
        const int64_t off = spec_off(k, spec_row(p, i, a.N), a.s_base + s0 + 4 * m, a.N,
                                     a.K >> 1, spec_tile_shift(OUT));
        store4<OUT>(a.spec, off, a.plane_stride, src[0], src[kStg1024Row], src[2 * kStg1024Row],
                    src[3 * kStg1024Row]);
    }
}

template <int OUT, bool CORR>
__global__ void __launch_bounds__(kF1024Threads, 3) fengine_k1024(FengineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = a.ant_x ? blockIdx.x : blockIdx.y;
    const int64_t s0 = (int64_t)(a.ant_x ? blockIdx.y : blockIdx.x) * kF1024Frames;
    f1024_block<OUT, CORR>(a, i, s0, smem_raw, threadIdx.x, []() { __syncthreads(); });
}

// ---------------------------------------------------------------------------
// K = 512 R F-engine for R = 4, 8 (K = 2048, 4096): a group of B = 16 R
// threads per spectrum, 16 complex points per thread.
//
// With L = K/2 = 256 R, n = t + B j, t = r + R u (r < R, u < 16) and
// k = k1 + 16 k2 + 256 k3 (k1, k2 < 16, k3 < R):
//   X1[t][k1] = W_L^{t k1} sum_j z[t + B j] W16^{j k1}
//   Z[k]      = sum_r W_R^{r k3} W_B^{r k2} sum_u W16^{u k2} X1[r + R u][k1].
// Thread t does the first 16-point DFT; after an exchange through shared
// memory thread (k1 = t mod 16, r = t / 16) does the second over u, and after
// a second exchange the R-point DFTs over r for its Q = 16/R values of k2.  Z
// goes back to shared memory in natural order, where the real split reads
// Z[k] and Z[L-k].  Each group syncs on its own named barrier; the CTA
// stages 2 G frames (G groups, two rounds) and writes them as runs of the
// workspace rows like the kernels above.  The exchange strides (B + 1 and 17
// complex) keep every half-warp on distinct banks.
// ---------------------------------------------------------------------------

constexpr int kRadThreads = 512;

__device__ __forceinline__ void group_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// 8-point forward DFT in place (radix 2 x 4).
__device__ __forceinline__ void dft8(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4,
                                     float2& x5, float2& x6, float2& x7) {
    constexpr float r2 = 0.707106781186547524f;
    dft4(x0, x2, x4, x6);                         // E[0..3] in x0, x2, x4, x6
    dft4(x1, x3, x5, x7);                         // O[0..3] in x1, x3, x5, x7
    const float2 o1 = make_float2(r2 * (x3.x + x3.y), r2 * (x3.y - x3.x));    // W8^1 O1
    const float2 o2 = cmi(x5);                                                // W8^2 O2
    const float2 o3 = make_float2(r2 * (x7.y - x7.x), -r2 * (x7.x + x7.y));   // W8^3 O3
    const float2 e0 = x0, e1 = x2, e2 = x4, e3 = x6, o0 = x1;
    x0 = cadd(e0, o0);
    x4 = csub(e0, o0);
    x1 = cadd(e1, o1);
    x5 = csub(e1, o1);
    x2 = cadd(e2, o2);
    x6 = csub(e2, o2);
    x3 = cadd(e3, o3);
    x7 = csub(e3, o3);
}

template <int R>
__device__ __forceinline__ void dft_r(float2 (&v)[R]) {
    if constexpr (R == 4) {
        dft4(v[0], v[1], v[2], v[3]);
    } else {
        static_assert(R == 8, "radix");
        dft8(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    }
}

template <int R>
struct Rad16Shape {
    static constexpr int L = 256 * R;
    static constexpr int B = 16 * R;                  // threads per spectrum
    static constexpr int Q = 16 / R;
    static constexpr int G = kRadThreads / B;         // spectra in flight per CTA
    static constexpr int FT = 2 * G;                  // frames per CTA
    static constexpr int M = FT / 4;                  // lanes per row in the store
    // staging row [2 k + plane] (a channel's Re and Im side by side, one
    // 8-byte store); SR = 2 mod 32 (M = 4) or 4 mod 32 (M = 2) puts the store
    // phase's reads of (channels x Re/Im x frame groups) on 32 distinct banks
    static constexpr int SR = 2 * L + 32 + 8 / M;     // staging row stride (floats)
    static constexpr int STG = (FT * SR + 3) & ~3;    // staging floats
    static constexpr int XB = 272 * R;                // exchange complex per group
    static size_t smem(bool dbg) {
        return (size_t)(dbg ? 0 : STG) * sizeof(float) +
               ((size_t)G * XB + 16 * B + 16 * R) * sizeof(float2);
    }
};

// The body: FT frames from s0 of antenna i by kRadThreads threads (tid),
// `smem` as the kernel's dynamic shared memory; `sync` is a barrier of the
// kRadThreads threads and group g syncs on named barrier bar0 + g.
template <int R, int OUT, class Sync>
__device__ __forceinline__ void frad16_block(const FengineArgs& a, int i, int64_t s0,
                                             unsigned char* smem, int tid, int bar0, Sync sync) {
    constexpr bool DEBUG = OUT == kOutDebug;
    using Sh = Rad16Shape<R>;
    constexpr int L = Sh::L, B = Sh::B, Q = Sh::Q, G = Sh::G, M = Sh::M, SR = Sh::SR,
                  XB = Sh::XB;
    float* stg = reinterpret_cast<float*>(smem);                                // [FT][SR]
    float2* xbuf = reinterpret_cast<float2*>(stg + (DEBUG ? 0 : Sh::STG));      // [G][XB]
    float2* tw1 = xbuf + G * XB;                                                // [16 k1][B t]
    float2* tw2 = tw1 + 16 * B;                                                 // [R r][16 k2]

    const int g = tid / B;
    const int t = tid - g * B;
    const float post = OUT == SPEC_F16X2 ? __ldg(a.split + i) : 1.0f;
    const float chalf = 0.5f * post;

    // W_L^{t k1} = W_K^{2 t k1 mod K};  W_B^{r k2} = W_K^{32 r k2}
    for (int e = tid; e < 16 * B; e += kRadThreads) {
        const int kk = e / B, tt = e - kk * B;
        tw1[e] = a.twiddle[(2 * tt * kk) & (2 * L - 1)];
    }
    for (int e = tid; e < 16 * R; e += kRadThreads) tw2[e] = a.twiddle[32 * (e >> 4) * (e & 15)];
    // The split's W_K^k for k = t + B m is W_K^t (a register) times
    // W_K^{B m} = W32^m (an immediate), and the antenna's pre-cast scales of
    // the thread's 16 outputs are read once for both rounds: no global load
    // per output.
    const float2 wkt = __ldg(a.twiddle + t);
    float scl[16];
#pragma unroll
    for (int m = 0; m < 16; ++m)
        scl[m] = (OUT == SPEC_F16 || OUT == SPEC_F8) ? __ldg(a.scale + (int64_t)i * L + t + B * m) : 1.0f;

    uint4 raw0 = make_uint4(0u, 0u, 0u, 0u), raw1 = raw0;
    {
        const int64_t sa = s0 + g, sb = sa + G;
        if (sa < a.S) raw0 = __ldg(reinterpret_cast<const uint4*>(a.in + (sa * a.N + i) * L) + t);
        if (sb < a.S) raw1 = __ldg(reinterpret_cast<const uint4*>(a.in + (sb * a.N + i) * L) + t);
    }
    sync();

    float2* xb = xbuf + g * XB;
    const unsigned char* xbytes = reinterpret_cast<const unsigned char*>(xb);
    const int bar = bar0 + g;
    const int k1 = t & 15, r = t >> 4;

#pragma unroll 1
    for (int rd = 0; rd < 2; ++rd) {
        const int f = g + G * rd;
        const int64_t s = s0 + f;
        *reinterpret_cast<uint4*>(xb + 2 * t) = rd == 0 ? raw0 : raw1;
        group_bar(bar, B);
        float2 x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const unsigned b = xbytes[t + B * j];
            x[j] = make_float2(nib_lo(b), nib_hi(b));
        }
        group_bar(bar, B);
        dft16(x);
#pragma unroll
        for (int q = 1; q < 16; ++q) x[q] = cmul(x[q], tw1[q * B + t]);
#pragma unroll
        for (int q = 0; q < 16; ++q) xb[q * (B + 1) + t] = x[q];
        group_bar(bar, B);
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = xb[k1 * (B + 1) + r + R * u];
        group_bar(bar, B);
        dft16(x);
#pragma unroll
        for (int q = 1; q < 16; ++q) x[q] = cmul(x[q], tw2[r * 16 + q]);
#pragma unroll
        for (int q = 0; q < 16; ++q) xb[k1 + 17 * (q * R + r)] = x[q];
        group_bar(bar, B);
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) {
            float2 v[R];
#pragma unroll
            for (int rp = 0; rp < R; ++rp) v[rp] = xb[k1 + 17 * ((r * Q + qq) * R + rp)];
            dft_r<R>(v);
#pragma unroll
            for (int k3 = 0; k3 < R; ++k3) x[qq * R + k3] = v[k3];
        }
        group_bar(bar, B);
        // x[qq R + k3] = Z[k1 + 16 (r Q + qq) + 256 k3]
#pragma unroll
        for (int qq = 0; qq < Q; ++qq)
#pragma unroll
            for (int k3 = 0; k3 < R; ++k3) xb[k1 + 16 * (r * Q + qq) + 256 * k3] = x[qq * R + k3];
        group_bar(bar, B);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int k = t + B * m;
            const float2 zk = xb[k], zc = xb[(L - k) & (L - 1)];
            const float2 w = w32mul(wkt, m);                    // W_K^k
            const float2 wp = make_float2(0.5f * post * w.y, -0.5f * post * w.x);
            const float2 S = add_conj(zk, zc);
            const float2 D = sub_conj(zk, zc);
            const float2 wd = cmul(wp, D);
            float2 X = make_float2(fmaf(chalf, S.x, wd.x), fmaf(chalf, S.y, wd.y));
            if (a.corr) X = cmul(__ldg(a.corr + (int64_t)i * L + k), X);
            if (DEBUG) {
                if (s < a.S) a.debug_out[((int64_t)i * a.S + s) * L + k] = X;
            } else {
                if (OUT == SPEC_F16 || OUT == SPEC_F8) {
                    X.x *= scl[m];
                    X.y *= scl[m];
                }
                *reinterpret_cast<float2*>(stg + f * SR + 2 * k) = X;
            }
        }
        group_bar(bar, B);
    }
    if (DEBUG) return;
    sync();
    // L channels x (Re, Im) x FT frames: lane = (2 c + p) M + m writes frames
    // 4m .. 4m + 3 of plane p of channel CPW cg + c; a channel's Re and Im
    // rows are adjacent in the workspace, so a warp store covers CPW lines
    // where the (plane, channel)-major order touched 2 CPW
    const int l32 = tid & 31, warp = tid >> 5;
    const int m = l32 % M, p = (l32 / M) & 1, c = l32 / (2 * M);
    constexpr int CPW = 32 / (2 * M);
    if (s0 + 4 * m >= a.S_pad) return;
    for (int cg = warp; cg < L / CPW; cg += kRadThreads / 32) {
        const int k = CPW * cg + c;
        const int plane = p;
        const float* src = stg + 4 * m * SR + 2 * k + p;
        const int64_t off = spec_off(k, spec_row(plane, i, a.N), a.s_base + s0 + 4 * m, a.N,
                                     a.K >> 1, spec_tile_shift(OUT));
        store4<OUT>(a.spec, off, a.plane_stride, src[0], src[SR], src[2 * SR], src[3 * SR]);
    }
}

template <int R, int OUT>
__global__ void __launch_bounds__(kRadThreads, 1) fengine_rad16(FengineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    frad16_block<R, OUT>(a, blockIdx.y, (int64_t)blockIdx.x * Rad16Shape<R>::FT, smem_raw,
                         threadIdx.x, 1, []() { __syncthreads(); });
}

// ---------------------------------------------------------------------------
// Several modes' F-engines in one launch (the batching form): one persistent
// CTA of 768 threads per SM.  First every K = 2048 / 4096 block, each by the
// CTA's first 512 threads with the body of its standalone kernel (barriers
// 1 and 2 ..); after a CTA-wide barrier the three 256-thread sub-blocks each
// walk their own share of the K = 512, 1024 and generic-K blocks, with their
// own shared memory and named barrier (1 + sub-block).  The sub-blocks drift
// apart, so one's loads and FFT overlap another's stores as three separate
// CTAs of the standalone kernels do.  (Non-persistent CTAs of three
// sub-blocks started and ended their phases together: 20-30% slower.)
// ---------------------------------------------------------------------------

enum FKind { kFK512 = 0, kFK1024 = 1, kFKRad4 = 2, kFKRad8 = 3, kFKGeneric = 4 };
constexpr int kMultiThreads = 768;
constexpr int kMultiSubs = kMultiThreads / 256;

struct FModeDesc {
    FengineArgs a;
    int kind;
    int FT;              // frames per block of the body
    int64_t nblk;        // blocks: antennas x frame blocks (antenna fastest)
    int64_t blk0;        // first block of the mode in its phase's numbering
    uint32_t sub_bytes;  // shared memory of one 256-thread sub-block, or of the body
};

struct FMultiArgs {
    FModeDesc md[kMaxTcModes];
    int n;
    int64_t rad_blocks;  // phase 1: blocks of the K = 2048 / 4096 modes
    int64_t sub_blocks;  // phase 2: blocks of the other modes
    uint32_t sub_stride; // phase 2: shared memory per sub-block (the largest mode's),
                         // so sub-blocks on different modes never overlap
};

__device__ __forceinline__ bool fk_rad(int kind) { return kind == kFKRad4 || kind == kFKRad8; }

// Named-barrier sync of `n` threads.
struct BarSync {
    int id, n;
    __device__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
};

template <int OUT>
__global__ void __launch_bounds__(kMultiThreads, 1) fengine_multi(const __grid_constant__ FMultiArgs m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    if (tid < kRadThreads) {
        const BarSync sync{1, kRadThreads};
        for (int64_t g = blockIdx.x; g < m.rad_blocks; g += gridDim.x) {
            int mi = 0;
            while (!fk_rad(m.md[mi].kind) || g >= m.md[mi].blk0 + m.md[mi].nblk) ++mi;
            const FModeDesc& d = m.md[mi];
            const FengineArgs& a = d.a;
            const int64_t vb = g - d.blk0;
            const int i = (int)(vb % a.N);
            const int64_t s0 = (vb / a.N) * d.FT;
            if (d.kind == kFKRad4)
                frad16_block<4, OUT>(a, i, s0, smem_raw, tid, 2, sync);
            else
                frad16_block<8, OUT>(a, i, s0, smem_raw, tid, 2, sync);
            sync();                      // the staging is the next block's
        }
    }
    if (m.rad_blocks > 0) asm volatile("bar.sync 15, 768;" ::: "memory");
    const int sub = tid >> 8;
    const int t = tid & 255;
    const BarSync sync{1 + sub, 256};
    for (int64_t g = (int64_t)blockIdx.x * kMultiSubs + sub; g < m.sub_blocks;
         g += (int64_t)gridDim.x * kMultiSubs) {
        int mi = 0;
        while (fk_rad(m.md[mi].kind) || g >= m.md[mi].blk0 + m.md[mi].nblk) ++mi;
        const FModeDesc& d = m.md[mi];
        const FengineArgs& a = d.a;
        const int64_t vb = g - d.blk0;
        const int i = (int)(vb % a.N);
        const int64_t s0 = (vb / a.N) * d.FT;
        unsigned char* sm = smem_raw + (size_t)sub * m.sub_stride;
        if (d.kind == kFK512) {
            constexpr bool kScaled = OUT == SPEC_F16 || OUT == SPEC_F8;
            float* stg = reinterpret_cast<float*>(sm);
            float2* tw_base = reinterpret_cast<float2*>(stg + kStgFloats);
            float* sc_tab = reinterpret_cast<float*>(tw_base + 128);
            float2* corr_tab = reinterpret_cast<float2*>(sc_tab + (kScaled ? 256 : 0));
            F512Block b;
            b.in = a.in + (s0 * a.N + i) * 256;
            b.stride = (int64_t)a.N * 256;
            b.nvalid = (int)max((int64_t)0, min((int64_t)kF512Frames, a.S - s0));
            b.ant = i;
            b.post = OUT == SPEC_F16X2 ? __ldg(a.split + i) : 1.0f;
            b.spec = static_cast<char*>(a.spec);
            b.s = a.s_base + s0;
            b.N = a.N;
            b.plane_stride = a.plane_stride;
            b.debug = nullptr;
            const float* sc = kScaled ? a.scale + (int64_t)i * 256 : nullptr;
            if (a.corr)
                f512_block<OUT, true>(b, a.twiddle, a.corr + (int64_t)i * 256, sc, stg, tw_base,
                                      sc_tab, corr_tab, t, sync);
            else
                f512_block<OUT, false>(b, a.twiddle, nullptr, sc, stg, tw_base, sc_tab, corr_tab, t,
                                       sync);
        } else if (d.kind == kFK1024) {
            if (a.corr)
                f1024_block<OUT, true>(a, i, s0, sm, t, sync);
            else
                f1024_block<OUT, false>(a, i, s0, sm, t, sync);
        } else {
            fgeneric_block<false>(a, d.FT, i, s0, sm, t, sync);
        }
        sync();                          // the staging is the next block's
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
    // K = 512 with 16-byte aligned input (the fast kernel reads 16 B per lane).
    if (a.K == 512 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0) {
        const int64_t fr = dbg ? a.S : a.S_pad;
        if (fr <= 0) return cudaSuccess;
        const int64_t nfb = (fr + kF512Frames - 1) / kF512Frames;
        FengineArgs b = a;
        b.ant_x = nfb <= 65535;
        const dim3 grid = b.ant_x ? dim3((unsigned)a.N, (unsigned)nfb) : dim3((unsigned)nfb, (unsigned)a.N);
        // staging (also the exchange areas), the twiddle bases, and when used
        // the scales and the corrections, for the debug output too (at most
        // 72 KB: three CTAs per SM)
        const bool scaled = !dbg && (a.spec_type == SPEC_F16 || a.spec_type == SPEC_F8);
        const size_t smem = (size_t)kStgFloats * sizeof(float) + 128 * sizeof(float2) +
                            (scaled ? 256 * sizeof(float) : 0) +
                            (a.corr ? 256 * sizeof(float2) : 0);
        auto go = [&](auto kern) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<grid, kF512Threads, smem, st>>>(b);
            return cudaGetLastError();
        };
        auto go2 = [&](auto plain, auto corrected) { return a.corr ? go(corrected) : go(plain); };
        if (dbg) return go2(fengine_k512<kOutDebug, false>, fengine_k512<kOutDebug, true>);
        switch (a.spec_type) {
            case SPEC_F32: return go2(fengine_k512<SPEC_F32, false>, fengine_k512<SPEC_F32, true>);
            case SPEC_F16: return go2(fengine_k512<SPEC_F16, false>, fengine_k512<SPEC_F16, true>);
            case SPEC_F8: return go2(fengine_k512<SPEC_F8, false>, fengine_k512<SPEC_F8, true>);
            default: return go2(fengine_k512<SPEC_F16X2, false>, fengine_k512<SPEC_F16X2, true>);
        }
    }
    if (a.K == 1024 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0) {
        const int64_t fr = dbg ? a.S : a.S_pad;
        if (fr <= 0) return cudaSuccess;
        // frames fastest here (antenna fastest ran ~1% slower at K = 1024)
        const int64_t nfb = (fr + kF1024Frames - 1) / kF1024Frames;
        FengineArgs b = a;
        b.ant_x = 0;
        const dim3 grid((unsigned)nfb, (unsigned)a.N);
        // staging (also the exchange areas) and the twiddle tables, for the
        // debug output too
        // staging (also the exchange areas), the twiddle tables and for
        // FP16/FP8 the scales, for the debug output too (at most 71 KB: three
        // CTAs per SM)
        const bool scaled = !dbg && (a.spec_type == SPEC_F16 || a.spec_type == SPEC_F8);
        const size_t smem = (size_t)kStg1024Floats * sizeof(float) + (256 + 32) * sizeof(float2) +
                            (scaled ? 512 * sizeof(float) : 0);
        auto go = [&](auto kern) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<grid, kF1024Threads, smem, st>>>(b);
            return cudaGetLastError();
        };
        auto go2 = [&](auto plain, auto corrected) { return a.corr ? go(corrected) : go(plain); };
        if (dbg) return go2(fengine_k1024<kOutDebug, false>, fengine_k1024<kOutDebug, true>);
        switch (a.spec_type) {
            case SPEC_F32: return go2(fengine_k1024<SPEC_F32, false>, fengine_k1024<SPEC_F32, true>);
            case SPEC_F16: return go2(fengine_k1024<SPEC_F16, false>, fengine_k1024<SPEC_F16, true>);
            case SPEC_F8: return go2(fengine_k1024<SPEC_F8, false>, fengine_k1024<SPEC_F8, true>);
            default: return go2(fengine_k1024<SPEC_F16X2, false>, fengine_k1024<SPEC_F16X2, true>);
        }
    }
    if ((a.K == 2048 || a.K == 4096) && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0) {
        const int64_t fr = dbg ? a.S : a.S_pad;
        if (fr <= 0) return cudaSuccess;
        auto go = [&](auto kern, int FT, size_t smem) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            dim3 grid((unsigned)((fr + FT - 1) / FT), (unsigned)a.N);
            kern<<<grid, kRadThreads, smem, st>>>(a);
            return cudaGetLastError();
        };
        auto pick = [&](auto shape, auto k_dbg, auto k_f32, auto k_f16, auto k_f8, auto k_x2) {
            using Sh = decltype(shape);
            const size_t sm = Sh::smem(dbg);
            if (dbg) return go(k_dbg, Sh::FT, sm);
            switch (a.spec_type) {
                case SPEC_F32: return go(k_f32, Sh::FT, sm);
                case SPEC_F16: return go(k_f16, Sh::FT, sm);
                case SPEC_F8: return go(k_f8, Sh::FT, sm);
                default: return go(k_x2, Sh::FT, sm);
            }
        };
        if (a.K == 2048)
            return pick(Rad16Shape<4>{}, fengine_rad16<4, kOutDebug>, fengine_rad16<4, SPEC_F32>,
                        fengine_rad16<4, SPEC_F16>, fengine_rad16<4, SPEC_F8>,
                        fengine_rad16<4, SPEC_F16X2>);
        return pick(Rad16Shape<8>{}, fengine_rad16<8, kOutDebug>, fengine_rad16<8, SPEC_F32>,
                    fengine_rad16<8, SPEC_F16>, fengine_rad16<8, SPEC_F8>,
                    fengine_rad16<8, SPEC_F16X2>);
    }
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

cudaError_t launch_fengine_multi(const FengineArgs* modes, int n, cudaStream_t st) {
    if (n < 1 || n > kMaxTcModes) return cudaErrorInvalidValue;
    FMultiArgs m{};
    size_t smem = 0;
    const int out = modes[0].spec_type;
    for (int q = 0; q < n; ++q) {
        const FengineArgs& a = modes[q];
        if (a.debug_out || a.spec_type != out) return cudaErrorInvalidValue;
        if (a.S_pad <= 0) continue;
        FModeDesc& d = m.md[m.n];
        d.a = a;
        const bool al16 = (reinterpret_cast<uintptr_t>(a.in) & 15) == 0;
        const bool scaled = out == SPEC_F16 || out == SPEC_F8;
        size_t bytes;
        if (a.K == 512 && al16) {
            d.kind = kFK512;
            d.FT = kF512Frames;
            bytes = (size_t)kStgFloats * sizeof(float) + 128 * sizeof(float2) +
                    (scaled ? 256 * sizeof(float) : 0) + (a.corr ? 256 * sizeof(float2) : 0);
        } else if (a.K == 1024 && al16) {
            d.kind = kFK1024;
            d.FT = kF1024Frames;
            bytes = (size_t)kStg1024Floats * sizeof(float) + (256 + 32) * sizeof(float2) +
                    (scaled ? 512 * sizeof(float) : 0);
        } else if (a.K == 2048 && al16) {
            d.kind = kFKRad4;
            d.FT = Rad16Shape<4>::FT;
            bytes = Rad16Shape<4>::smem(false);
        } else if (a.K == 4096 && al16) {
            d.kind = kFKRad8;
            d.FT = Rad16Shape<8>::FT;
            bytes = Rad16Shape<8>::smem(false);
        } else {
            d.kind = kFKGeneric;
            const int C = a.K / 2;
            d.FT = std::max(1, std::min(32, 8192 / C));
            bytes = (size_t)16 * (a.K / 2) + (size_t)8 * C * d.FT;
        }
        bytes = (bytes + 127) & ~(size_t)127;
        const bool rad = d.kind == kFKRad4 || d.kind == kFKRad8;
        d.sub_bytes = (uint32_t)bytes;
        d.nblk = (int64_t)a.N * ((a.S_pad + d.FT - 1) / d.FT);
        int64_t& count = rad ? m.rad_blocks : m.sub_blocks;
        d.blk0 = count;
        count += d.nblk;
        if (!rad) m.sub_stride = std::max<uint32_t>(m.sub_stride, (uint32_t)bytes);
        smem = std::max(smem, rad ? bytes : bytes * kMultiSubs);
        ++m.n;
    }
    if (m.n == 0) return cudaSuccess;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t need = std::max(m.rad_blocks, (m.sub_blocks + kMultiSubs - 1) / kMultiSubs);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nsm, need));
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        kern<<<grid, kMultiThreads, smem, st>>>(m);
        return cudaGetLastError();
    };
    switch (out) {
        case SPEC_F32: return go(fengine_multi<SPEC_F32>);
        case SPEC_F16: return go(fengine_multi<SPEC_F16>);
        case SPEC_F8: return go(fengine_multi<SPEC_F8>);
        default: return go(fengine_multi<SPEC_F16X2>);
    }
}

// ---------------------------------------------------------------------------
// Coarse integer delays: y_i[t] = x_i[t - D_i], 0 <= D_i <= K, on the packed
// 4-bit stream before the F-engine.  A CTA takes frames s0 .. s0 + FB - 1 of
// one antenna plus the frame before them (from the previous chunk's last
// frame, `hist_in`, when s0 = 0; zeros without it) into shared memory and
// writes each output byte's two samples from their delayed positions.  The
// CTA holding the chunk's last frame copies it to `hist_out` for the next
// chunk.
// ---------------------------------------------------------------------------

constexpr int kDelayThreads = 256;
constexpr int kDelayLoads = 8;      // loads in flight per thread

template <int V>
struct DelayVec;
template <>
struct DelayVec<4> {
    using T = uint4;
};
template <>
struct DelayVec<2> {
    using T = uint2;
};

// V 32-bit words per thread and step (4 when a frame is a multiple of 16
// bytes, else 2): every frame of the CTA is copied in V-word chunks.
template <int V>
__global__ void __launch_bounds__(kDelayThreads) sample_delay_kernel(
    const uint8_t* __restrict__ in, int64_t S, int N, int K, const int* __restrict__ D,
    const uint8_t* __restrict__ hist_in, uint8_t* __restrict__ hist_out, uint8_t* __restrict__ out,
    int FB, int cshift, int aligned) {
    using Vec = typename DelayVec<V>::T;
    extern __shared__ __align__(16) uint8_t dbuf[];      // [FB + 1][K/2] (+ 16 bytes)
    const int L = K >> 1;
    const int wl = L >> 2;                               // 32-bit words per frame
    const int cl = 1 << cshift;                          // V-word chunks per frame
    const int i = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * FB;
    const int nf = (int)min((int64_t)FB, S - s0);
    const int d = __ldg(D + i);
    const int64_t NL = (int64_t)N * L;                   // bytes from one frame to the next
    uint32_t* b32 = reinterpret_cast<uint32_t*>(dbuf);
    // frames s0 - 1 .. s0 + nf - 1 of antenna i; the loads of a thread are
    // issued together (kDelayLoads at a time), then stored
    const uint8_t* first = in + (s0 * N + i) * (int64_t)L - NL;   // frame s0 - 1
    const int chunks = (nf + 1) << cshift;
    for (int c0 = threadIdx.x; c0 < chunks; c0 += kDelayThreads * kDelayLoads) {
        Vec v[kDelayLoads];
#pragma unroll
        for (int u = 0; u < kDelayLoads; ++u) {
            const int c = c0 + u * kDelayThreads;
            uint32_t* vw = reinterpret_cast<uint32_t*>(&v[u]);
#pragma unroll
            for (int k = 0; k < V; ++k) vw[k] = 0u;
            if (c < chunks) {
                const int f = c >> cshift;
                const int b = (c & (cl - 1)) * 4 * V;
                if (f > 0 || s0 > 0) {
                    const uint8_t* src = first + f * NL + b;
                    if (aligned) {
                        v[u] = __ldg(reinterpret_cast<const Vec*>(src));
                    } else {
                        for (int k = 0; k < 4 * V; ++k)
                            vw[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
                    }
                } else if (hist_in) {
                    v[u] = *reinterpret_cast<const Vec*>(hist_in + (int64_t)i * L + b);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kDelayLoads; ++u) {
            const int c = c0 + u * kDelayThreads;
            if (c < chunks) reinterpret_cast<Vec*>(b32)[c] = v[u];
        }
    }
    if (threadIdx.x < 4) b32[(nf + 1) * wl + threadIdx.x] = 0u;   // read past the end, never used
    __syncthreads();
    // Output sample u of the CTA's frames is buffer sample K + u - d: a shift
    // by the same Q0 bytes (+ a nibble when d is odd) for every output word.
    const int Q0 = L - ((d + 1) >> 1);
    const int wb = Q0 >> 2;
    const int sh = ((Q0 & 3) << 3) + ((d & 1) << 2);
    uint8_t* obase = out + (s0 * N + i) * (int64_t)L;
    for (int c = threadIdx.x; c < (nf << cshift); c += kDelayThreads) {
        const int f = c >> cshift;
        const int w = c * V;
        uint32_t a[V + 1];
#pragma unroll
        for (int k = 0; k <= V; ++k) a[k] = b32[wb + w + k];
        Vec o;
        uint32_t* ow = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
        for (int k = 0; k < V; ++k) ow[k] = __funnelshift_r(a[k], a[k + 1], sh);
        *reinterpret_cast<Vec*>(obase + f * NL + (c & (cl - 1)) * 4 * V) = o;
    }
    if (hist_out && s0 + nf == S)
        for (int w = threadIdx.x; w < wl; w += kDelayThreads)
            reinterpret_cast<uint32_t*>(hist_out + (int64_t)i * L)[w] = b32[nf * wl + w];
}

cudaError_t launch_correction_table(const float2* gains, const float* delays, int N, int K,
                                    float2* table, cudaStream_t st) {
    const int64_t total = (int64_t)N * (K / 2);
    const int blocks = (int)((total + 255) / 256);
    correction_table_kernel<<<blocks, 256, 0, st>>>(gains, delays, N, K, table);
    return cudaGetLastError();
}

cudaError_t launch_sample_delay(const uint8_t* in, int64_t S, int N, int K, const int* delays,
                                const uint8_t* hist_in, uint8_t* hist_out, uint8_t* out,
                                cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int L = K / 2;
    const int V = (L % 16 == 0) ? 4 : 2;
    int cshift = 0;
    while ((4 * V << cshift) < L) ++cshift;
    const int FB = std::max(1, 16384 / L);     // 64 frames at K = 512
    const size_t smem = (size_t)(FB + 1) * L + 16;
    const int aligned = (reinterpret_cast<uintptr_t>(in) & (4 * V - 1)) == 0 ? 1 : 0;
    dim3 grid((unsigned)((S + FB - 1) / FB), (unsigned)N);
    if (V == 4)
        sample_delay_kernel<4><<<grid, kDelayThreads, smem, st>>>(in, S, N, K, delays, hist_in,
                                                                  hist_out, out, FB, cshift, aligned);
    else
        sample_delay_kernel<2><<<grid, kDelayThreads, smem, st>>>(in, S, N, K, delays, hist_in,
                                                                  hist_out, out, FB, cshift, aligned);
    return cudaGetLastError();
}

}  // namespace gbcorr
