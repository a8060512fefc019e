// K = 512 F-engine body, shared by the standalone F-engine kernel
// (fengine.cu) and the fused F/X-engine kernel (fx_fused.cu): unpack ->
// optional gain/delay -> 512-point real FFT -> the corner-turned workspace.
//
// Paper: Sec. 1 (split each stream into channels with an FFT), Sec. 4
// (forward, unnormalised float FFT; conversion of its output before the
// cross-multiply), Sec. 2.1 (a phase applied per stream before accumulation).
#pragma once

#include "corr_internal.h"

#include <cuda_fp8.h>

namespace gbcorr {
namespace fk {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------------------
// K = 512 F-engine: 16 lanes per spectrum, 16 complex points per lane.
//
// The 256-point complex transform is split as n = t + 16 j (lane t, register
// j) and k = k1 + 16 k2:
//   Z[k1 + 16 k2] = sum_t W16^{t k2} [ W256^{t k1} sum_j z[t + 16 j] W16^{j k1} ]
// Stage 1 is an in-register 16-point DFT over j, then the twiddle
// W256^{t k1}, one exchange through shared memory (lane k1 gathers the 16
// values of its k1 from every t), and stage 2 is again an in-register
// 16-point DFT, leaving Z[k1 + 16 k2] in lane k1, register k2.  The
// real-to-complex split needs Z[256 - k], which lives in lane (16 - k1) mod
// 16, register 15 - k2 (register (16 - k2) mod 16 for k1 = 0): one shuffle per
// register.
// ---------------------------------------------------------------------------

constexpr int kF512Frames = 32;     // frames per CTA (one workspace tile)
constexpr int kF512Threads = 256;   // 16 groups of 16 lanes, 2 frames per group
constexpr int kXStride = 17;        // exchange row stride (complex), conflict-free

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// -i * a
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }
// The same add and subtract as one packed FP32x2 instruction each (a - b as
// b * -1 + a: one rounding, the scalar subtraction's result).  The packed
// forms issue to one of the two FP32 pipes: used in the 4-point DFTs they
// halve the adds' instructions (K = 512 F-engine 5-7% faster), used
// throughout the F-engine they made it slower.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// 4-point forward DFT in place: X[m] = sum_j x[j] (-i)^{jm}.  The two
// outputs that take -i (x1 - x3) are formed part by part.
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 t0 = padd(x0, x2), t1 = psub(x0, x2);
    const float2 t2 = padd(x1, x3), d = psub(x1, x3);
    x0 = padd(t0, t2);
    x2 = psub(t0, t2);
    x1 = make_float2(t1.x + d.y, t1.y - d.x);
    x3 = make_float2(t1.x - d.y, t1.y + d.x);
}

// W16^e = exp(-2 pi i e / 16) for the products e = j2 * m1 that occur.
__device__ __forceinline__ float2 w16mul(float2 a, int e) {
    constexpr float c8 = 0.923879532511286756f;   // cos(pi/8)
    constexpr float s8 = 0.382683432365089772f;   // sin(pi/8)
    constexpr float r2 = 0.707106781186547524f;   // 1/sqrt(2)
    switch (e) {
        case 0: return a;
        case 1: return cmul(a, make_float2(c8, -s8));
        case 2: return cmul(a, make_float2(r2, -r2));
        case 3: return cmul(a, make_float2(s8, -c8));
        case 4: return cmi(a);
        case 6: return cmul(a, make_float2(-r2, -r2));
        default: return cmul(a, make_float2(-c8, s8));   // e = 9
    }
}

// 16-point forward DFT in registers, natural order in and out (radix 4 x 4).
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) dft4(x[j2], x[4 + j2], x[8 + j2], x[12 + j2]);
    // x[4 m1 + j2] now holds the m1-th output of column j2; apply W16^{j2 m1}
#pragma unroll
    for (int j2 = 1; j2 < 4; ++j2)
#pragma unroll
        for (int m1 = 1; m1 < 4; ++m1) x[4 * m1 + j2] = w16mul(x[4 * m1 + j2], j2 * m1);
#pragma unroll
    for (int m1 = 0; m1 < 4; ++m1) dft4(x[4 * m1], x[4 * m1 + 1], x[4 * m1 + 2], x[4 * m1 + 3]);
    // x[4 m1 + m2] holds X[m1 + 4 m2]: transpose the 4 x 4 index map
    float2 y[16];
#pragma unroll
    for (int m1 = 0; m1 < 4; ++m1)
#pragma unroll
        for (int m2 = 0; m2 < 4; ++m2) y[m1 + 4 * m2] = x[4 * m1 + m2];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = y[q];
}

// Nibble v (0..15, 4-bit two's complement) to float without a conversion
// instruction: the bit pattern 0x4B000000 | u is the float 2^23 + u.  The
// high nibble is masked in place (u = 16 (v ^ 8)) and scaled back by the
// multiply-add, whose exact result needs no rounding.
__device__ __forceinline__ float nib_lo(unsigned b) {
    return __int_as_float((int)((b & 15u) ^ 0x4B000008u)) - 8388616.0f;
}
__device__ __forceinline__ float nib_hi(unsigned b) {
    return fmaf(__int_as_float((int)((b & 0xF0u) ^ 0x4B000080u)), 0.0625f, -524296.0f);
}

// zk + conj(zc) and zk - conj(zc) as one packed FMA each (zc times (1, -1)
// or (-1, 1), plus zk: one rounding per part, the scalar adds' results).
// In the K = 512 real split this saved ~1%; packing the split's outputs or
// the nibble conversion as well made the kernel slower.
__device__ __forceinline__ float2 add_conj(float2 zk, float2 zc) {
    return __ffma2_rn(zc, make_float2(1.0f, -1.0f), zk);
}
__device__ __forceinline__ float2 sub_conj(float2 zk, float2 zc) {
    return __ffma2_rn(zc, make_float2(-1.0f, 1.0f), zk);
}

// cos(q pi / 16) and sin(q pi / 16) for q in [0, 16].
__device__ __forceinline__ float cos_pi16(int q) {
    float r = 0.0f;
    switch (q < 9 ? q : 16 - q) {
        case 0: r = 1.0f; break;
        case 1: r = 0.980785280403230449f; break;
        case 2: r = 0.923879532511286756f; break;
        case 3: r = 0.831469612302545237f; break;
        case 4: r = 0.707106781186547524f; break;
        case 5: r = 0.555570233019602225f; break;
        case 6: r = 0.382683432365089772f; break;
        case 7: r = 0.195090322016128268f; break;
        default: r = 0.0f; break;
    }
    return q < 9 ? r : -r;
}
__device__ __forceinline__ float sin_pi16(int q) { return cos_pi16(q < 8 ? 8 - q : q - 8); }

// W32^q d = exp(-2 pi i q / 32) d for a compile-time q in [0, 16).
__device__ __forceinline__ float2 w32mul(float2 d, int q) {
    if (q == 0) return d;
    if (q == 8) return make_float2(d.y, -d.x);
    if (q == 4) {
        constexpr float r2 = 0.707106781186547524f;
        return make_float2(r2 * (d.x + d.y), r2 * (d.y - d.x));
    }
    const float c = cos_pi16(q), s = sin_pi16(q);
    return make_float2(fmaf(c, d.x, s * d.y), fmaf(c, d.y, -s * d.x));
}

constexpr int kOutDebug = -1;
// Staging row stride (floats): [frame][2 k + plane], the real and imaginary
// parts of a channel side by side like the workspace rows.  547 = 3 mod 32
// keeps both the staging writes and the store phase's column reads on
// distinct banks (the two half-warps of a warp hold consecutive frames, an
// odd bank shift apart), and leaves room in a row for one group's exchange
// area (16 x 17 complex = 544 floats) at the 16-byte aligned offset f mod 4
// within row f.  A group exchanges through the row of its second frame:
// during the first round no group writes that row, and in the second the
// group itself writes it only after its exchange.  With 4 KB of tables
// (twiddle bases, scales, corrections) that is all the shared memory
// (72 KB), so three CTAs fit on an SM.
constexpr int kStgRow = 547;
constexpr int kStgFloats = kF512Frames * kStgRow;
static_assert(kStgRow % 32 == 3 && kStgRow >= 16 * kXStride * 2 + 3, "staging row layout");
// Start of frame f's staging row: odd rows one float later, so every row
// starts on an 8-byte boundary and a channel's (Re, Im) is one 8-byte store
// (K = 512 FP32 mode 1.5% faster than two 4-byte stores).  The column reads
// of the store phase stay on distinct banks: the offset is the same for
// all lanes of a read.
__device__ __forceinline__ int stg_row(int f) { return f * kStgRow + (f & 1); }

// Four consecutive frames of one workspace row (channel k, row r) from the
// staging buffer, converted and stored with one vector store per plane.
template <int OUT>
__device__ __forceinline__ void store4(void* spec, int64_t off, int64_t plane_stride, float v0,
                                       float v1, float v2, float v3) {
    if (OUT == SPEC_F32) {
        *reinterpret_cast<float4*>(static_cast<float*>(spec) + off) = make_float4(v0, v1, v2, v3);
    } else if (OUT == SPEC_F16) {
        const __half2 a = __floats2half2_rn(v0, v1), b = __floats2half2_rn(v2, v3);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned*>(&a);
        u.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(static_cast<__half*>(spec) + off) = u;
    } else if (OUT == SPEC_F8) {
        const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t b = __nv_cvt_float2_to_fp8x2(make_float2(v2, v3), __NV_SATFINITE, __NV_E4M3);
        *reinterpret_cast<unsigned*>(static_cast<unsigned char*>(spec) + off) =
            (unsigned)a | ((unsigned)b << 16);
    } else {  // SPEC_F16X2: values already carry the pre-scale sigma_i
        const __half2 ha = __floats2half2_rn(v0, v1), hb = __floats2half2_rn(v2, v3);
        const float2 fa = __half22float2(ha), fb = __half22float2(hb);
        const __half2 la = __floats2half2_rn(v0 - fa.x, v1 - fa.y);
        const __half2 lb = __floats2half2_rn(v2 - fb.x, v3 - fb.y);
        uint2 uh, ul;
        uh.x = *reinterpret_cast<const unsigned*>(&ha);
        uh.y = *reinterpret_cast<const unsigned*>(&hb);
        ul.x = *reinterpret_cast<const unsigned*>(&la);
        ul.y = *reinterpret_cast<const unsigned*>(&lb);
        __half* base = static_cast<__half*>(spec);
        *reinterpret_cast<uint2*>(base + off) = uh;
        *reinterpret_cast<uint2*>(base + off + plane_stride) = ul;
    }
}

// store4 at a byte address; `lo` is the byte distance to the low plane.
template <int OUT>
__device__ __forceinline__ void store4p(char* p, int64_t lo, float v0, float v1, float v2,
                                        float v3) {
    if (OUT == SPEC_F32) {
        *reinterpret_cast<float4*>(p) = make_float4(v0, v1, v2, v3);
    } else if (OUT == SPEC_F16) {
        const __half2 a = __floats2half2_rn(v0, v1), b = __floats2half2_rn(v2, v3);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned*>(&a);
        u.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = u;
    } else if (OUT == SPEC_F8) {
        const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t b = __nv_cvt_float2_to_fp8x2(make_float2(v2, v3), __NV_SATFINITE, __NV_E4M3);
        *reinterpret_cast<unsigned*>(p) = (unsigned)a | ((unsigned)b << 16);
    } else {  // SPEC_F16X2: values already carry the pre-scale sigma_i
        const __half2 ha = __floats2half2_rn(v0, v1), hb = __floats2half2_rn(v2, v3);
        const float2 fa = __half22float2(ha), fb = __half22float2(hb);
        const __half2 la = __floats2half2_rn(v0 - fa.x, v1 - fa.y);
        const __half2 lb = __floats2half2_rn(v2 - fb.x, v3 - fb.y);
        uint2 uh, ul;
        uh.x = *reinterpret_cast<const unsigned*>(&ha);
        uh.y = *reinterpret_cast<const unsigned*>(&hb);
        ul.x = *reinterpret_cast<const unsigned*>(&la);
        ul.y = *reinterpret_cast<const unsigned*>(&lb);
        *reinterpret_cast<uint2*>(p) = uh;
        *reinterpret_cast<uint2*>(p + lo) = ul;
    }
}

template <int OUT>
__host__ __device__ constexpr int out_bytes() {
    return OUT == SPEC_F32 ? 4 : (OUT == SPEC_F8 ? 1 : 2);
}

// Eight consecutive frames of one workspace row converted and stored with
// one 16-byte store per plane (FP16 and the FP16 pair).
template <int OUT>
__device__ __forceinline__ void store8p(char* p, int64_t lo, const float (&v)[8]) {
    __half2 h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(h);
    if (OUT == SPEC_F16X2) {   // values already carry the pre-scale sigma_i
        __half2 l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 fh = __half22float2(h[e]);
            l[e] = __floats2half2_rn(v[2 * e] - fh.x, v[2 * e + 1] - fh.y);
        }
        *reinterpret_cast<uint4*>(p + lo) = *reinterpret_cast<const uint4*>(l);
    }
}

// Store phase of the K = 512 kernel: 256 channels x 2 rows (Re, Im) x 32
// frames of one antenna from the staging buffer [frame][2 k + plane].  The
// two rows of a channel are adjacent in the workspace (2 i, 2 i + 1), so each
// (channel, plane) is one contiguous run of whole lines, and the lanes are
// laid out to write runs whole:
// * 2-byte types (32-frame tiles, 64-byte rows): lane = 8 c + 4 p + m writes
//   frames 8 m .. 8 m + 7 of row p of channel 4 w + c + 32 j with 16-byte
//   stores -- 8 lanes cover the channel's 128 bytes, a warp 4 channels;
// * FP32 (32-frame tiles, 128-byte rows) and FP8 (128-frame tiles): lane =
//   16 c + 8 p + m writes frames 4 m .. 4 m + 3 of row p of channel
//   2 w + c + 16 j.
// Within a plane the workspace address steps by a constant number of
// channels; the loops stay rolled (unrolled copies, which hoist the staging
// loads of several rows, ran slower).  The staging column reads land on 32
// distinct banks (frame offsets 24 m or 12 m mod 32, plus 0..7 or 0..3).
template <int OUT>
__device__ __forceinline__ void store_rows(char* base, int N, int64_t plane_stride, const float* stg,
                                           int warp, int l32, int64_t s, int ant) {
    constexpr int eb = out_bytes<OUT>();
    constexpr int tsh = OUT == SPEC_F8 ? 7 : 5;
    const int64_t lo = plane_stride * eb;
    if (eb == 2) {
        const int m = l32 & 3, p = (l32 >> 2) & 1, c = l32 >> 3;
        const float* src = stg + 8 * m * kStgRow + 2 * (4 * warp + c) + p;
        char* dst = base + spec_off(4 * warp + c, spec_row(p, ant, N), s + 8 * m, N, 256, tsh) * eb;
        const int64_t step = ((int64_t)32 * 2 * N << tsh) * eb;     // 32 channels on
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = src[e * kStgRow + (e & 1)];
            store8p<OUT>(dst, lo, v);
            dst += step;
            src += 64;
        }
    } else {
        const int m = l32 & 7, p = (l32 >> 3) & 1, c = l32 >> 4;
        const float* src = stg + 4 * m * kStgRow + 2 * (2 * warp + c) + p;
        char* dst = base + spec_off(2 * warp + c, spec_row(p, ant, N), s + 4 * m, N, 256, tsh) * eb;
        const int64_t step = ((int64_t)16 * 2 * N << tsh) * eb;     // 16 channels on
#pragma unroll 1
        for (int j = 0; j < 16; ++j) {
            store4p<OUT>(dst, lo, src[0], src[kStgRow + 1], src[2 * kStgRow], src[3 * kStgRow + 1]);
            dst += step;
            src += 32;
        }
    }
}

// CORR: the per-antenna corrections are applied (a.corr set).  A run-time
// test in the split made the whole kernel 7% slower, so it is a template
// parameter.
// One 32-frame block of one antenna for the K = 512 body (the work of one
// 256-thread CTA of the standalone kernel).
struct F512Block {
    const uint8_t* in;       // 256-byte record of the block's first frame
    int64_t stride;          // bytes from one frame's record to the next (N * 256)
    int nvalid;              // frames 0 .. nvalid - 1 are read; later ones are zeros
    int ant;                 // antenna: workspace rows 2 ant, 2 ant + 1
    float post;              // two-plane pre-scale sigma_ant (SPEC_F16X2), else 1
    char* spec;              // workspace (spec_off layout) ...
    int64_t s;               // ... frame of the block's first frame in it
    int N;
    int64_t plane_stride;    // elements from the hi plane to the lo plane
    float2* debug;           // debug output of frame 0 ([frame][256] complex), or nullptr
};

// The K = 512 F-engine on one block by 256 threads (tid 0..255): tables,
// input prefetch, two rounds of 16 spectra, staging, and the store phase.
// `sync` synchronises the 256 threads (the CTA, or a named barrier of a
// sub-block); `stg` is the 32 x 547-float staging area, `tw_base` 128
// complex, `sc_tab` 256 floats (FP16 / FP8), `corr_tab` 256 complex (CORR).
template <int OUT, bool CORR, class Sync>
__device__ __forceinline__ void f512_block(const F512Block& b, const float2* __restrict__ twiddle,
                                           const float2* __restrict__ corr_i,
                                           const float* __restrict__ scale_i, float* stg,
                                           float2* tw_base, float* sc_tab, float2* corr_tab, int tid,
                                           Sync sync) {
    constexpr bool DEBUG = OUT == kOutDebug;
    constexpr bool kScaled = OUT == SPEC_F16 || OUT == SPEC_F8;
    const int lane = tid & 15;
    const int grp = tid >> 4;
    const int warp = tid >> 5;
    const int half = grp & 1;
    // The antenna's pre-scale sigma_i of the two-plane FP16 split is folded
    // into the real-split constants: X = c (zk + conj zc) + w'_k (zk - conj zc)
    // with c = 1/2 and w'_k = W512^k / (2i), both times the pre-scale.
    const float post = b.post;
    const float chalf = 0.5f * post;

    // Twiddles, kept off the shared-memory pipe where arithmetic can stand
    // in: the stage twiddle W256^{t k1}, k1 = p + 4 r, is W256^{t p} W256^{4 t r}
    // from a 1 KB table of the six bases, and the split's W512^k, k = t + 16 q,
    // is W512^t (a register) times W32^q (an immediate).
    if (tid < 128) {
        const int j = tid >> 6, m = (tid >> 4) & 3, t = tid & 15;
        tw_base[tid] = twiddle[2 * t * m * (j ? 4 : 1)];     // W256^{t m 4^j}
    }
    // the antenna's pre-cast scales and corrections, read once per CTA
    // instead of per output
    if (kScaled) sc_tab[tid] = __ldg(scale_i + tid);
    if (CORR) corr_tab[tid] = __ldg(corr_i + tid);
    const float2 wt = __ldg(twiddle + lane);
    const float2 u = make_float2(chalf * wt.x, chalf * wt.y);   // c W512^t

    // prefetch both rounds' 16 bytes per lane: group g = 2 warp + half takes
    // frames g and g + 16
    uint4 raw0 = make_uint4(0u, 0u, 0u, 0u), raw1 = raw0;
    {
        const int fa = 2 * warp + half, fb = fa + 16;
        if (fa < b.nvalid) raw0 = __ldg(reinterpret_cast<const uint4*>(b.in + fa * b.stride) + lane);
        if (fb < b.nvalid) raw1 = __ldg(reinterpret_cast<const uint4*>(b.in + fb * b.stride) + lane);
    }
    sync();

    const int fx = 2 * warp + half + 16;             // the group's second frame
    float2* gx = reinterpret_cast<float2*>(stg + stg_row(fx) + ((4 - (stg_row(fx) & 3)) & 3));
    unsigned char* gbytes = reinterpret_cast<unsigned char*>(gx);

#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
        const int f = 2 * warp + half + 16 * r;
        // byte transpose: lane t needs bytes t + 16 j
        *reinterpret_cast<uint4*>(gbytes + 16 * lane) = r == 0 ? raw0 : raw1;
        __syncwarp();
        float2 x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const unsigned b = gbytes[lane + 16 * j];
            x[j] = make_float2(nib_lo(b), nib_hi(b));
        }
        __syncwarp();
        dft16(x);
        // twiddle W256^{t k1}, then exchange: lane k1 collects register k1 of every t
        {
            float2 wp[4], wr[4];
#pragma unroll
            for (int m = 1; m < 4; ++m) {
                wp[m] = tw_base[m * 16 + lane];
                wr[m] = tw_base[64 + m * 16 + lane];
            }
#pragma unroll
            for (int k1 = 1; k1 < 16; ++k1) {
                if (k1 & 3) x[k1] = cmul(x[k1], wp[k1 & 3]);
                if (k1 >> 2) x[k1] = cmul(x[k1], wr[k1 >> 2]);
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) gx[k1 * kXStride + lane] = x[k1];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = gx[lane * kXStride + t];
        __syncwarp();
        dft16(x);
        // x[q] = Z[lane + 16 q].  Slot q < 8 of lane k1 makes both X[k] and
        // X[256 - k], k = k1 + 16 q, from Z[k] and its partner Z[256 - k]
        // (register 15 - q of lane 16 - k1; for lane 0 its own register
        // 16 - q): with S = Z[k] + conj Z[256-k] and D = Z[k] - conj Z[256-k],
        // X[k] = c S + w'_k D and, as w'_{256-k} = conj w'_k,
        // X[256 - k] = conj(c S - w'_k D).  Lane 0's slot 0 makes X[0] and,
        // in place of the dropped Nyquist term, X[128] = post conj Z[128].
        const int src = (16 - lane) & 15;
        auto emit = [&](int k, float2 X) {
            if (CORR) X = cmul(corr_tab[k], X);
            if (DEBUG) {
                if (f < b.nvalid) b.debug[(int64_t)f * 256 + k] = X;
            } else {
                if (OUT == SPEC_F16 || OUT == SPEC_F8) {
                    const float sc = sc_tab[k];
                    X.x *= sc;
                    X.y *= sc;
                }
                *reinterpret_cast<float2*>(stg + stg_row(f) + 2 * k) = X;
            }
        };
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 16 * q;
            float2 zc;
            zc.x = __shfl_sync(0xffffffffu, x[15 - q].x, src, 16);
            zc.y = __shfl_sync(0xffffffffu, x[15 - q].y, src, 16);
            if (lane == 0) zc = x[(16 - q) & 15];
            const float2 zk = x[q];
            const float2 S = add_conj(zk, zc);
            const float2 D = sub_conj(zk, zc);
            // B = w'_k D = -i c W512^t W32^q D
            const float2 v = cmul(u, w32mul(D, q));
            const float2 B = make_float2(v.y, -v.x);
            emit(k, make_float2(fmaf(chalf, S.x, B.x), fmaf(chalf, S.y, B.y)));
            float2 Xp = make_float2(fmaf(chalf, S.x, -B.x), -fmaf(chalf, S.y, -B.y));
            int kp = 256 - k;
            if (q == 0 && lane == 0) {
                Xp = make_float2(post * x[8].x, -post * x[8].y);
                kp = 128;
            }
            emit(kp, Xp);
        }
    }
    if (DEBUG) return;
    sync();
    store_rows<OUT>(b.spec, b.N, b.plane_stride, stg, warp, tid & 31, b.s, b.ant);
}



}  // namespace fk
}  // namespace gbcorr
