// X-engine on the FP32 CUDA cores, the FP64 partial reduction and the dump.
//
// Paper: Sec. 1 (cross-multiply the spectra of every pair of antennas per
// channel, accumulate to the required cadence), Sec. 4 ("complex cross
// multiply", one complex accumulator per channel per baseline).
//
// V_ij[k] += Y_i conj(Y_j) = (a_i a_j + b_i b_j) + i (b_i a_j - a_i b_j) with
// Y = a + i b.  One thread owns a 4 x 4 block of antenna pairs (block row
// bi <= block column bj) of one channel and one range of spectra; the
// spectra of that channel are staged in shared memory 32 frames at a time,
// as [frame][plane][antenna] rows of NBP floats (a power of two >= 32) whose
// 16-byte groups are XOR-swizzled by the frame's group of four: the staging
// writes (8 lanes per workspace row, 4 frames each) then land on distinct
// banks, and a thread still reads 4 antennas of a frame as one float4.
#include "corr_internal.h"

#include <algorithm>

namespace gbcorr {
namespace {

constexpr int kTS = 32;  // frames per shared-memory tile

// A CTA covers G consecutive channels (G > 1 when one channel's nt threads
// fill less than a CTA; their workspace tiles are adjacent) or, when G = 1,
// the nt threads of one channel over gridDim.z CTAs.
template <int NBP>
__global__ void xengine_simt_kernel(XengineArgs a, int nb, int nt, int G) {
    constexpr int nbp = NBP;
    extern __shared__ __align__(16) float smem_tiles[];  // G x [kTS][2][nbp], swizzled columns
    const int N = a.N;
    const int g = G > 1 ? threadIdx.x / nt : 0;
    const int k0 = blockIdx.x * G;
    const int k = k0 + g;
    const int split = blockIdx.y;
    const int t = G > 1 ? threadIdx.x - g * nt : blockIdx.z * blockDim.x + threadIdx.x;
    const int Gc = min(G, a.C - k0);                 // channels this CTA holds
    float* tile = smem_tiles + (size_t)g * kTS * 2 * nbp;

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
    // antennas past N (the last block's padding) stay zero
    for (int e = threadIdx.x; e < G * kTS * 2 * nbp; e += blockDim.x) smem_tiles[e] = 0.f;

    float ar[4][4], ai[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) ar[u][v] = ai[u][v] = 0.f;

    const int64_t sb = (int64_t)split * a.s_per_split;
    const int64_t se = min(a.S_pad, sb + a.s_per_split);
    static_assert(kTS == 32, "one 32-frame FP32 workspace tile per step");

    for (int64_t s0 = sb; s0 < se; s0 += kTS) {
        __syncthreads();
        // the tiles' 2N rows x 32 frames of channels k0 .. k0 + Gc - 1 are
        // contiguous
        const float4* base = reinterpret_cast<const float4*>(
            static_cast<const float*>(a.spec) + spec_off(k0, 0, s0, N, a.C, 5));
        for (int gg = 0; gg < Gc; ++gg) {
            const float4* bg = base + gg * 2 * N * (kTS / 4);
            float* tg = smem_tiles + gg * kTS * 2 * nbp;
            for (int e = threadIdx.x; e < 2 * N * (kTS / 4); e += blockDim.x) {
                const int r = e >> 3;             // workspace row of channel k0 + gg
                const int c4 = (e & 7) << 2;      // its frames c4 .. c4 + 3
                const float4 v = bg[e];
                // row r = 2 antenna + plane
                const int plane = r & 1;
                float* d = tg + (c4 * 2 + plane) * nbp + ((r >> 1) ^ c4);
                d[0] = v.x;
                d[2 * nbp] = v.y;
                d[4 * nbp] = v.z;
                d[6 * nbp] = v.w;
            }
        }
        __syncthreads();
        if (active) {
            // frames c4 .. c4 + 3 share one swizzle, so their addresses are
            // two pointers plus constant offsets
#pragma unroll 1
            for (int c4 = 0; c4 < kTS; c4 += 4) {
                const float* pi = tile + (c4 * 2) * nbp + ((4 * bi) ^ c4);
                const float* pj = tile + (c4 * 2) * nbp + ((4 * bj) ^ c4);
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float4 ri = *reinterpret_cast<const float4*>(pi + (2 * f) * nbp);
                    const float4 ii = *reinterpret_cast<const float4*>(pi + (2 * f + 1) * nbp);
                    const float4 rj = *reinterpret_cast<const float4*>(pj + (2 * f) * nbp);
                    const float4 ij = *reinterpret_cast<const float4*>(pj + (2 * f + 1) * nbp);
                    const float xr[4] = {ri.x, ri.y, ri.z, ri.w};
                    const float xi[4] = {ii.x, ii.y, ii.z, ii.w};
                    const float yr[4] = {rj.x, rj.y, rj.z, rj.w};
                    const float yi[4] = {ij.x, ij.y, ij.z, ij.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            ar[u][v] = fmaf(xr[u], yr[v], ar[u][v]);
                            ar[u][v] = fmaf(xi[u], yi[v], ar[u][v]);
                            ai[u][v] = fmaf(xi[u], yr[v], ai[u][v]);
                            ai[u][v] = fmaf(-xr[u], yi[v], ai[u][v]);
                        }
                }
            }
        }
    }
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
                out[p] = make_float2(ar[u][v], ai[u][v]);
            }
        }
}

// The partials of one workspace pass are summed in FP32 (four independent
// running sums, so the loads overlap; a pass holds at most 131072 frames), and
// the pass total is added to the FP64 accumulator.  FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU, so one FP64 add per element
// and pass keeps the kernel bound by its loads.
__global__ void reduce_partials_kernel(const float2* part, int n_split, int64_t CP, double2* acc) {
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
        double2 o = acc[e];
        o.x += (double)((t[0].x + t[1].x) + (t[2].x + t[3].x));
        o.y += (double)((t[0].y + t[1].y) + (t[2].y + t[3].y));
        acc[e] = o;
    }
}

// acc [C][P] -> vis [P][C] through 32 x 32 shared-memory tiles, so both the
// reads (along p) and the writes (along k) are coalesced.  (acc is cleared by
// a memset after it: zero stores here, to the lines just loaded, held the
// kernel to a quarter of the HBM bandwidth.)
constexpr int kDT = 32;

__global__ void __launch_bounds__(kDT * 8) dump_kernel(const double2* __restrict__ acc, int C,
                                                     int P, void* __restrict__ vis, int fp64) {
    __shared__ double2 tile[kDT][kDT + 1];
    const int p0 = blockIdx.x * kDT;
    const int k0 = blockIdx.y * kDT;
    const int tx = threadIdx.x & (kDT - 1);
    const int ty = threadIdx.x / kDT;               // 0..7
    double2 v[kDT / 8];
    const int p = p0 + tx;
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) {
        const int k = k0 + ty + 8 * q;
        v[q] = (k < C && p < P) ? acc[(int64_t)k * P + p] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) tile[ty + 8 * q][tx] = v[q];
    __syncthreads();
    const int k = k0 + tx;
#pragma unroll
    for (int q = 0; q < kDT / 8; ++q) {
        const int pp = p0 + ty + 8 * q;
        if (k < C && pp < P) {
            const double2 w = tile[tx][ty + 8 * q];
            const int64_t e = (int64_t)pp * C + k;
            if (fp64)
                static_cast<double2*>(vis)[e] = w;
            else
                static_cast<float2*>(vis)[e] = make_float2((float)w.x, (float)w.y);
        }
    }
}

int grid_for(int64_t total) {
    int64_t b = (total + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_xengine_simt(const XengineArgs& a, cudaStream_t st) {
    if (a.spec_type != SPEC_F32) return cudaErrorInvalidValue;
    const int nb = (a.N + 3) / 4;
    const int nt = nb * (nb + 1) / 2;
    int nbp = 32;
    while (nbp < nb * 4) nbp *= 2;
    const size_t tile_bytes = (size_t)kTS * 2 * nbp * sizeof(float);
    // channels per CTA: up to 256 threads and 64 KB of tiles
    int G = nt < 256 ? 256 / nt : 1;
    G = std::min<int>(G, (int)((64 << 10) / tile_bytes));
    G = std::max(1, std::min(G, a.C));
    int threads = G > 1 ? (G * nt + 31) / 32 * 32 : ((nt < 256 ? nt : 256) + 31) / 32 * 32;
    dim3 grid((unsigned)((a.C + G - 1) / G), (unsigned)a.n_split,
              (unsigned)(G > 1 ? 1 : (nt + threads - 1) / threads));
    const size_t smem = G * tile_bytes;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, st>>>(a, nb, nt, G);
        return cudaGetLastError();
    };
    switch (nbp) {
        case 32: return go(xengine_simt_kernel<32>);
        case 64: return go(xengine_simt_kernel<64>);
        case 128: return go(xengine_simt_kernel<128>);
        case 256: return go(xengine_simt_kernel<256>);
        default: return go(xengine_simt_kernel<512>);
    }
}

cudaError_t launch_reduce_partials(const float2* partial, int n_split, int64_t CP, double2* acc,
                                   cudaStream_t st) {
    reduce_partials_kernel<<<grid_for(CP), 256, 0, st>>>(partial, n_split, CP, acc);
    return cudaGetLastError();
}

cudaError_t launch_dump(double2* acc, int C, int P, void* vis, int fp64, cudaStream_t st) {
    dim3 grid((unsigned)((P + kDT - 1) / kDT), (unsigned)((C + kDT - 1) / kDT));
    dump_kernel<<<grid, kDT * 8, 0, st>>>(acc, C, P, vis, fp64);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(acc, 0, (size_t)C * P * sizeof(double2), st);
}

}  // namespace gbcorr
