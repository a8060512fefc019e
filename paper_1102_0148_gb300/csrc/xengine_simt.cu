// X-engine on the FP32 CUDA cores, the FP64 partial reduction and the dump.
//
// Paper: Sec. 1 (cross-multiply the spectra of every pair of antennas per
// channel, accumulate to the required cadence), Sec. 4 ("complex cross
// multiply", one complex accumulator per channel per baseline).
//
// V_ij[k] += Y_i conj(Y_j) = (a_i a_j + b_i b_j) + i (b_i a_j - a_i b_j) with
// Y = a + i b.  One thread owns a 4 x 4 block of antenna pairs (block row
// bi <= block column bj) of one channel and one range of spectra.  The
// workspace tiles (per channel, rows 2 i + plane of 32 frames, 128 bytes) are
// copied unchanged into shared memory by cp.async, three tiles in flight, so
// the copies of later tiles overlap the arithmetic on this one (above 400
// antennas a stage holds half a tile, 16 frames).  Antenna block b's 8 rows
// (4 antennas x Re, Im) sit in rows 8 b .. 8 b + 7; a row's 16-byte groups
// (4 frames each) are XOR-swizzled by b mod 8, so the quarter-warp that reads
// one group of 8 different blocks hits 8 different bank groups.  A thread
// reads two frames of a row as one float2 and accumulates them with packed
// FP32 FMAs (FFMA2: even frames in .x, odd frames in .y, summed at the end),
// half the instructions of scalar FMAs for the same arithmetic.
#include "corr_internal.h"

#include <algorithm>

namespace gbcorr {
namespace {

constexpr int kTS = 32;          // frames per workspace tile
constexpr int kMaxStages = 3;    // stages in flight per CTA

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A CTA covers G consecutive channels (G > 1 when one channel's nt threads
// fill less than a CTA; their workspace tiles are adjacent) or, when G = 1,
// the nt threads of one channel over gridDim.z CTAs.  rows = 8 nb (2N rounded
// up to whole antenna blocks); stages: 2 or 3 in flight; tf: frames per stage
// (32, or 16 for the largest arrays).
__global__ void __launch_bounds__(256) xengine_simt_kernel(XengineArgs a, int nb, int nt, int G,
                                                           int rows, int stages, int tf) {
    extern __shared__ __align__(16) float smem_tiles[];  // [stage][G][rows][tf], swizzled groups
    const int N = a.N;
    const int g = G > 1 ? threadIdx.x / nt : 0;
    const int k0 = blockIdx.x * G;
    const int k = k0 + g;
    const int split = blockIdx.y;
    const int t = G > 1 ? threadIdx.x - g * nt : blockIdx.z * blockDim.x + threadIdx.x;
    const int Gc = min(G, a.C - k0);                 // channels this CTA holds
    const int tile_floats = rows * tf;
    const int gmask = tf / 4 - 1;                    // 16-byte groups of a row, minus one

    int bi = 0, bj = 0;
    const bool active = t < nt && g < Gc;
    if (active) {
        int rem = t;
        while (rem >= nb - bi) {
            rem -= nb - bi;
            ++bi;
        }
        bj = bi + rem;
    }
    // rows past 2N (the last block's padding antennas) stay zero: no copy
    // writes them
    if (rows > 2 * N)
        for (int st = 0; st < stages; ++st)
            for (int gg = 0; gg < G; ++gg) {
                float* tg = smem_tiles + (size_t)(st * G + gg) * tile_floats;
                for (int e = 2 * N * tf + threadIdx.x; e < tile_floats; e += blockDim.x) tg[e] = 0.f;
            }

    // packed pairs: .x sums the even frames, .y the odd ones (one FFMA2 does
    // both), added together at the end
    float2 ar[4][4], ai[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) ar[u][v] = ai[u][v] = make_float2(0.f, 0.f);

    const int64_t sb = (int64_t)split * a.s_per_split;
    const int64_t se = min(a.S_pad, sb + a.s_per_split);
    const int n_tiles = se > sb ? (int)((se - sb) / tf) : 0;
    const int gshift = tf == 32 ? 3 : 2;             // log2(tf / 4)

    // Copy stage j (frames sb + tf j ..) of channels k0 .. k0 + Gc - 1 (2N rows
    // of 32 frames each, adjacent in the workspace) into slot j mod stages.
    auto load_tile = [&](int j) {
        const float* src = static_cast<const float*>(a.spec) + spec_off(k0, 0, sb + (int64_t)j * tf, N, a.C, 5);
        float* dst = smem_tiles + (size_t)(j % stages) * G * tile_floats;
        for (int gg = 0; gg < Gc; ++gg) {
            const float* sg = src + (size_t)gg * 2 * N * kTS;
            float* dg = dst + (size_t)gg * tile_floats;
            for (int e = threadIdx.x; e < 2 * N * (tf / 4); e += blockDim.x) {
                const int r = e >> gshift;       // workspace row
                const int c = e & gmask;         // its frames 4c .. 4c + 3 of the stage
                cp_async16(dg + r * tf + ((c ^ ((r >> 3) & gmask)) << 2), sg + r * kTS + 4 * c);
            }
        }
    };
    for (int j = 0; j < stages - 1; ++j) {
        if (j < n_tiles) load_tile(j);
        cp_async_commit();
    }

    for (int j = 0; j < n_tiles; ++j) {
        // this thread's copies of tile j have landed (one younger group may
        // still be in flight with three stages) ...
        if (stages == 3)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        // ... and everyone's: the stage of tile j - 1 is free again
        __syncthreads();
        if (j + stages - 1 < n_tiles) load_tile(j + stages - 1);
        cp_async_commit();
        if (active) {
            const float* tile = smem_tiles + (size_t)((j % stages) * G + g) * tile_floats;
            const float* pi = tile + 8 * bi * tf;
            const float* pj = tile + 8 * bj * tf;
            const int swi = bi & gmask, swj = bj & gmask;
#pragma unroll 1
            for (int c = 0; c <= gmask; ++c) {
#pragma unroll
                for (int f2 = 0; f2 < 4; f2 += 2) {
                    // rows 2u (Re) and 2u + 1 (Im) of antennas 4 bi + u and
                    // 4 bj + u, frames 4c + f2 and 4c + f2 + 1
                    float2 X[8], Y[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        X[q] = *reinterpret_cast<const float2*>(pi + q * tf + ((c ^ swi) << 2) + f2);
                        Y[q] = *reinterpret_cast<const float2*>(pj + q * tf + ((c ^ swj) << 2) + f2);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 xr = X[2 * u], xi = X[2 * u + 1];
                        const float2 nxr = make_float2(-xr.x, -xr.y);
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float2 yr = Y[2 * v], yi = Y[2 * v + 1];
                            ar[u][v] = __ffma2_rn(xr, yr, ar[u][v]);
                            ar[u][v] = __ffma2_rn(xi, yi, ar[u][v]);
                            ai[u][v] = __ffma2_rn(xi, yr, ai[u][v]);
                            ai[u][v] = __ffma2_rn(nxr, yi, ai[u][v]);
                        }
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
    if (!active) return;
    const int P = N * (N + 1) / 2;
    float2* out = a.partial + ((int64_t)split * a.C + k) * P;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = 4 * bi + u;
            const int j = 4 * bj + v;
            if (i < N && j < N && i <= j) {
                const int p = i * N - i * (i - 1) / 2 + (j - i);
                out[p] = make_float2(ar[u][v].x + ar[u][v].y, ai[u][v].x + ai[u][v].y);
            }
        }
}

// The partials of one workspace pass are summed in FP32 (four independent
// running sums, so the loads overlap; a pass holds at most 131072 frames), and
// the pass total is added to the FP64 accumulator.  FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU, so one FP64 add per element
// and pass keeps the kernel bound by its loads.
__global__ void reduce_partials_kernel(const float2* part, int n_split, int64_t CP, double2* acc,
                                       int assign) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < CP;
         e += (int64_t)gridDim.x * blockDim.x) {
        float2 t[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                       make_float2(0.f, 0.f)};
        int s = 0;
        for (; s + 4 <= n_split; s += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = part[(int64_t)(s + q) * CP + e];
                t[q].x += v.x;
                t[q].y += v.y;
            }
        }
        for (; s < n_split; ++s) {
            const float2 v = part[(int64_t)s * CP + e];
            t[0].x += v.x;
            t[0].y += v.y;
        }
        // assign: acc is known to be zero (the first pass of an integration),
        // so its read is skipped
        double2 o = assign ? make_double2(0.0, 0.0) : acc[e];
        o.x += (double)((t[0].x + t[1].x) + (t[2].x + t[3].x));
        o.y += (double)((t[0].y + t[1].y) + (t[2].y + t[3].y));
        acc[e] = o;
    }
}

// acc [C][P] -> vis [P][C] through 32 x 32 shared-memory tiles, so both the
// reads (along p) and the writes (along k) are coalesced.  (acc is cleared by
// a memset after it: zero stores here, to the lines just loaded, held the
// kernel to a quarter of the HBM bandwidth.)  T = double2 for the FP64
// accumulator, float2 for a pass result still in partial slot 0 (its FP64
// reduction into a zero accumulator would give the same values); values
// change type only on the way out, as FP64 conversions are slow here.
constexpr int kDT = 32;

__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

template <typename T>
__global__ void __launch_bounds__(kDT * 8) dump_kernel(const T* __restrict__ acc, int C, int P,
                                                     void* __restrict__ vis, int fp64) {
    __shared__ T tile[kDT][kDT + 1];
    const int p0 = blockIdx.x * kDT;
    const int k0 = blockIdx.y * kDT;
    const int tx = threadIdx.x & (kDT - 1);
    const int ty = threadIdx.x / kDT;               // 0..7
    T v[kDT / 8];
    const int p = p0 + tx;
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) {
        const int k = k0 + ty + 8 * q;
        v[q] = (k < C && p < P) ? acc[(int64_t)k * P + p] : T{};
    }
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) tile[ty + 8 * q][tx] = v[q];
    __syncthreads();
    const int k = k0 + tx;
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) {
        const int pp = p0 + ty + 8 * q;
        if (k < C && pp < P) {
            const T w = tile[tx][ty + 8 * q];
            const int64_t e = (int64_t)pp * C + k;
            if (fp64)
                static_cast<double2*>(vis)[e] = to_d2(w);
            else
                static_cast<float2*>(vis)[e] = to_f2(w);
        }
    }
}

int grid_for(int64_t total) {
    int64_t b = (total + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_xengine_simt(XengineArgs& a, cudaStream_t st) {
    if (a.spec_type != SPEC_F32 || a.max_split < 1) return cudaErrorInvalidValue;
    const int nb = (a.N + 3) / 4;
    const int nt = nb * (nb + 1) / 2;
    const int rows = 8 * nb;
    // 32 frames per stage, or 16 where two stages of 32 would not fit
    const int tf = (size_t)2 * rows * kTS * sizeof(float) <= (200u << 10) ? kTS : kTS / 2;
    const size_t tile_bytes = (size_t)rows * tf * sizeof(float);
    // channels per CTA: up to 256 threads and 36 KB of tiles per stage
    int G = nt < 256 ? 256 / nt : 1;
    G = std::min<int>(G, (int)std::max<size_t>(1, (36u << 10) / tile_bytes));
    G = std::max(1, std::min(G, a.C));
    const int threads = G > 1 ? (G * nt + 31) / 32 * 32 : ((nt < 256 ? nt : 256) + 31) / 32 * 32;
    // three tiles in flight where they fit in 200 KB, else two
    const int stages = G * tile_bytes * kMaxStages <= (200u << 10) ? kMaxStages : 2;
    const size_t smem = (size_t)stages * G * tile_bytes;
    if (smem > (227u << 10)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(xengine_simt_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, xengine_simt_kernel, threads, smem)) !=
        cudaSuccess)
        return e;
    const int64_t groups = (int64_t)((a.C + G - 1) / G) * (G > 1 ? 1 : (nt + threads - 1) / threads);
    const int64_t slots = (int64_t)std::max(1, nsm) * std::max(1, occ);
    // Frames per split: the split count whose whole waves of CTAs cost least,
    // each CTA's cost its tiles plus ~3 tiles of pipeline fill and partial
    // store; at most max_split partials
    const int64_t tiles = a.S_pad / kTS;
    int64_t best_per = std::max<int64_t>(1, tiles), best_cost = -1;
    for (int64_t n = 1; n <= std::min<int64_t>(tiles, a.max_split); ++n) {
        const int64_t per = (tiles + n - 1) / n;
        const int64_t n_eff = (tiles + per - 1) / per;
        const int64_t waves = (groups * n_eff + slots - 1) / slots;
        const int64_t cost = waves * (per + 3);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_per = per;
        }
    }
    a.s_per_split = best_per * kTS;
    a.n_split = (int)((a.S_pad + a.s_per_split - 1) / a.s_per_split);
    dim3 grid((unsigned)((a.C + G - 1) / G), (unsigned)a.n_split,
              (unsigned)(G > 1 ? 1 : (nt + threads - 1) / threads));
    xengine_simt_kernel<<<grid, threads, smem, st>>>(a, nb, nt, G, rows, stages, tf);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const float2* partial, int n_split, int64_t CP, double2* acc,
                                   cudaStream_t st, bool assign) {
    reduce_partials_kernel<<<grid_for(CP), 256, 0, st>>>(partial, n_split, CP, acc, assign ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_dump(double2* acc, int C, int P, void* vis, int fp64, cudaStream_t st) {
    dim3 grid((unsigned)((P + kDT - 1) / kDT), (unsigned)((C + kDT - 1) / kDT));
    dump_kernel<double2><<<grid, kDT * 8, 0, st>>>(acc, C, P, vis, fp64);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(acc, 0, (size_t)C * P * sizeof(double2), st);
}

cudaError_t launch_dump_partial(const float2* part, int C, int P, void* vis, int fp64,
                                cudaStream_t st) {
    dim3 grid((unsigned)((P + kDT - 1) / kDT), (unsigned)((C + kDT - 1) / kDT));
    dump_kernel<float2><<<grid, kDT * 8, 0, st>>>(part, C, P, vis, fp64);
    return cudaGetLastError();
}

}  // namespace gbcorr
