// X-engine on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Paper: Sec. 1 (cross-multiply every pair of antennas per channel and
// accumulate), Sec. 4 (the cross-multiply dominates the load; the paper
// converts the FFT output to a narrower type with prescaling before it).
//
// For one channel k the spectra of a pass form A = [Re Y_0..Re Y_{N-1};
// Im Y_0..Im Y_{N-1}] (2N rows, spectra along the contraction axis), and the
// real Gram matrix G = A A^T holds every product the visibilities need:
//   Re V_ij = G[i][j] + G[N+i][N+j],   Im V_ij = G[N+i][j] - G[i][N+j].
// G is a dense contraction: D[128 x Nn] += A_tile[128 x 16|32] * A_tile^T with
// both MMA operands read from the *same* TMA-loaded shared-memory tile (rows
// beyond 2N are zero-filled by TMA), FP32 accumulators in TMEM.
//
// Precisions (operands in shared memory, K-major, 128-byte swizzle):
//   mode 0 (FP32-accurate): two FP16 planes x/16 = hi + lo; two MMAs per
//           k-step, Dhh += hi hi^T and Dhl += hi lo^T; the epilogue forms
//           G = 256 (Dhh + Dhl + Dhl^T)  (the lo lo^T term is below 2^-22).
//   mode 1: one FP16 plane (pre-scaled per antenna and channel).
//   mode 2: one FP8-E4M3 plane (pre-scaled), kind::f8f6f4.
//
// CTA = 10 warps, persistent over work items (channel, range of spectra):
//   warp 0    TMA producer (one lane)     -> stage ring (full/empty mbarriers)
//   warp 1    TMEM allocator + MMA issuer (one lane) -> two TMEM accumulator sets
//   warps 2-9 epilogue: TMEM -> registers, summed over windows -> G in shared
//             memory -> V -> partials
// The tensor core's FP32 accumulation into TMEM is biased (it loses about one
// unit in the last place per accumulate, always toward zero), so TMEM only
// accumulates one window of kWindow spectra; the epilogue adds the windows
// with round-to-nearest FP32 arithmetic.  The two accumulator sets let the
// epilogue drain window n while the MMAs fill window n+1.
// Every mbarrier wait is bounded by a global-timer deadline; on expiry the
// kernel records a status code, drains its own copies and MMAs, frees TMEM
// and returns.
#include "xengine_tc.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <vector>

namespace gbcorr {
namespace {

constexpr int kTcThreads = 320;   // producer, MMA, 8 epilogue warps
constexpr int kWindow = 128;      // spectra per TMEM accumulation window
constexpr int kRows = 128;          // MMA M = TMA box rows
constexpr int kRowBytes = 128;      // one swizzle span per row
constexpr int kTileBytes = kRows * kRowBytes;
constexpr uint32_t kTmemCols = 512; // two accumulator sets of 256 columns
constexpr int kStatusTimeout = 2;

struct TcArgs {
    int N, C, R2, Nn, P;
    int mode;                 // 0 split FP16 (two planes), 1 FP16, 2 FP8
    int planes;
    int stages;
    int KT;                   // spectra per k-tile (one 128-byte row of operands)
    int W;                    // spectra per TMEM accumulation window (multiple of KT)
    int64_t S_pad;
    int64_t S_item;           // spectra per work item (multiple of KT)
    int n_items;              // C * n_split
    uint32_t idesc;
    float2* partial;          // [n_split][C][P]
    double2* acc;             // [C][P] FP64 accumulator, used directly when n_split == 1
    const float* scale;       // [N][C] (modes 1, 2)
    int* status;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity` of `bar`.  Returns false on timeout or when
// another role has already given up (the shared abort word is set).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_word,
                                         const TcArgs& a) {
    unsigned long long t0 = 0;
    for (uint32_t n = 0;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_word) return false;
        if ((n & 63) == 63) {
            const unsigned long long now = globaltimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > a.timeout_ns) {
                *abort_word = 1;
                atomicCAS(a.status, 0, kStatusTimeout);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart, descriptor version 1 (bits 46-47), layout type 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
    if (MODE == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// --------------------------------------------------------------------- kernel

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
    xengine_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int planes = MODE == 0 ? 2 : 1;
    constexpr uint32_t stage_bytes = planes * kTileBytes;
    unsigned char* stages = smem;
    const int ldg = a.R2 + 1;
    float* Gs = reinterpret_cast<float*>(smem + a.stages * stage_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(Gs + a.R2 * ldg) + 15) & ~(uintptr_t)15);
    uint64_t* full = bars;
    uint64_t* empty = full + a.stages;
    uint64_t* accf = empty + a.stages;
    uint64_t* acce = accf + 2;
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* epi_ok = abort_word + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf[b]), 1);
            mbar_init(smem_u32(&acce[b]), 256);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            int armed_phase[16];
            for (int s = 0; s < 16; ++s) armed_phase[s] = -1;
            bool ok = true;
            for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
                const int k = item % a.C;
                const int sp = item / a.C;
                const int64_t s_beg = (int64_t)sp * a.S_item;
                const int64_t s_end = min(a.S_pad, s_beg + a.S_item);
                for (int64_t s = s_beg; s < s_end; s += a.KT, ++it) {
                    const uint32_t st = it % a.stages;
                    const uint32_t ph = (it / a.stages) & 1u;
                    if (!wait_bar(smem_u32(&empty[st]), ph ^ 1u, abort_word, a)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full[st]);
                    mbar_expect_tx(fb, stage_bytes);
                    const uint32_t dst = smem_u32(stages + st * stage_bytes);
                    tma_load_3d(dst, &tmap, fb, (int)s, 0, k);
                    if (planes == 2) tma_load_3d(dst + kTileBytes, &tmap, fb, (int)s, 0, a.C + k);
                    armed_phase[st] = (int)ph;
                }
            }
            if (!ok) {
                // drain: every armed stage's copies must land before teardown
                const unsigned long long d2 = globaltimer() + a.timeout_ns;
                for (int s = 0; s < a.stages && s < 16; ++s) {
                    if (armed_phase[s] < 0) continue;
                    while (!mbar_try_wait(smem_u32(&full[s]), (uint32_t)armed_phase[s]))
                        if (globaltimer() > d2) break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        // One TMEM accumulation window = W spectra; windows alternate between
        // the two accumulator sets so the epilogue drains one while the next fills.
        if (lane == 0) {
            uint32_t it = 0;
            int wi = 0;
            bool ok = true;
            bool issued = false;
            for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
                const int sp = item / a.C;
                const int64_t s_beg = (int64_t)sp * a.S_item;
                const int64_t s_end = min(a.S_pad, s_beg + a.S_item);
                for (int64_t w0 = s_beg; ok && w0 < s_end; w0 += a.W, ++wi) {
                    const int b = wi & 1;
                    const uint32_t aph = (uint32_t)(wi >> 1) & 1u;
                    if (!wait_bar(smem_u32(&acce[b]), aph ^ 1u, abort_word, a)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_hh = tmem + (uint32_t)b * 256u;
                    const uint32_t d_hl = d_hh + 128u;
                    const int64_t w1 = min(s_end, w0 + a.W);
                    uint32_t acc = 0;
                    for (int64_t s = w0; s < w1; s += a.KT, ++it) {
                        const uint32_t st = it % a.stages;
                        const uint32_t ph = (it / a.stages) & 1u;
                        if (!wait_bar(smem_u32(&full[st]), ph, abort_word, a)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = smem_u32(stages + st * stage_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = sw128_desc(base + 32u * kk);
                            mma<MODE>(d_hh, ad, ad, a.idesc, acc);
                            if (planes == 2) {
                                const uint64_t bd = sw128_desc(base + kTileBytes + 32u * kk);
                                mma<MODE>(d_hl, ad, bd, a.idesc, acc);
                            }
                            acc = 1;
                        }
                        issued = true;
                        mma_commit(smem_u32(&empty[st]));
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&accf[b]));
                }
            }
            if (!ok && issued) {
                // drain: wait for every MMA this thread issued before TMEM is freed
                mma_commit(smem_u32(drain));
                const unsigned long long d2 = globaltimer() + a.timeout_ns;
                while (!mbar_try_wait(smem_u32(drain), 0u))
                    if (globaltimer() > d2) break;
            }
        }
    } else {
        // --------------------------------------------------------- epilogue
        // 8 warps: warp w reads TMEM lane quadrant w % 4 (rows 32q..32q+31) and
        // one half of the Nn accumulator columns.  Windows are summed in
        // registers with round-to-nearest FP32 adds (the tensor core's own
        // accumulation is only trusted over one short window).
        const int et = threadIdx.x - 64;            // 0..255
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int r = 32 * q + lane;
        const int NH = a.Nn >> 1;                   // columns per half, multiple of 8
        const int col0 = h * NH;
        const int N = a.N, R2 = a.R2, C = a.C, P = a.P;
        int wi = 0;
        bool ok = true;
        for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
            const int k = item % C;
            const int sp = item / C;
            const int64_t s_beg = (int64_t)sp * a.S_item;
            const int64_t s_end = min(a.S_pad, s_beg + a.S_item);
            float g[64], t[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                g[j] = 0.f;
                t[j] = 0.f;
            }
            for (int64_t w0 = s_beg; w0 < s_end; w0 += a.W, ++wi) {
                const int b = wi & 1;
                const uint32_t aph = (uint32_t)(wi >> 1) & 1u;
                if (et == 0) *epi_ok = wait_bar(smem_u32(&accf[b]), aph, abort_word, a) ? 1 : 0;
                epi_sync();
                if (!*epi_ok) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t trow =
                    tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * 256u + (uint32_t)col0;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (8 * c < NH) {
                        uint32_t v[8];
                        tmem_ld8(trow + 8u * c, v);
                        if (planes == 2) {
                            uint32_t w[8];
                            tmem_ld8(trow + 128u + 8u * c, w);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float wf = __uint_as_float(w[j]);
                                g[8 * c + j] += __uint_as_float(v[j]) + wf;
                                t[8 * c + j] += wf;
                            }
                        } else {
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 8; ++j) g[8 * c + j] += __uint_as_float(v[j]);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&acce[b]));   // this TMEM set may be refilled now
            }
            if (!ok) break;
            if (r < R2) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int col = col0 + 8 * c + j;
                        if (8 * c < NH && col < R2) Gs[r * ldg + col] = g[8 * c + j];
                    }
            }
            epi_sync();
            if (planes == 2) {
                // G[col][r] += Dhl[r][col]: each element is touched by one thread here
                if (r < R2) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = col0 + 8 * c + j;
                            if (8 * c < NH && col < R2) Gs[col * ldg + r] += t[8 * c + j];
                        }
                }
                epi_sync();
            }
            const float gs = MODE == 0 ? 1.0f / (kSplitScale * kSplitScale) : 1.0f;
            float2* out = a.partial + ((int64_t)sp * C + k) * P;
            int i = 0;
            int row_next = N;                       // first p of row i + 1
            for (int p = et; p < P; p += 256) {
                while (p >= row_next) {
                    ++i;
                    row_next += N - i;
                }
                const int j = i + (p - (row_next - (N - i)));
                const float re = Gs[i * ldg + j] + Gs[(N + i) * ldg + N + j];
                const float im = Gs[(N + i) * ldg + j] - Gs[i * ldg + N + j];
                float f = gs;
                if (MODE != 0)
                    f = 1.0f / (__ldg(a.scale + (int64_t)i * C + k) * __ldg(a.scale + (int64_t)j * C + k));
                if (a.acc) {
                    double2* d = a.acc + (int64_t)k * P + p;   // sole owner of (k, p) here
                    double2 v = *d;
                    v.x += (double)(re * f);
                    v.y += (double)(im * f);
                    *d = v;
                } else {
                    out[p] = make_float2(re * f, im * f);
                }
            }
            epi_sync();
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// ----------------------------------------------------------------- host side

constexpr uint32_t make_idesc(int M, int Nn) {
    // D = F32 (bits 4-5); A, B = F16 for kind::f16 and E4M3 for kind::f8f6f4
    // (format code 0 in both, bits 7-9 / 10-12); both K-major; N>>3 at
    // bits 17-22; M>>4 at bits 24-28.
    return (1u << 4) | ((uint32_t)(Nn >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

struct TcPlan {
    int N = 0, C = 0, R2 = 0, Nn = 0, P = 0;
    int mode = 0, planes = 1, stages = 4, KT = 64;
    int num_sms = 0;
    size_t smem_bytes = 0;
    CUtensorMap tmap;
    bool have_map = false;
    int64_t cap = 0;
    int max_split = 1;
    int last_split = 1;
    unsigned long long timeout_ns = 4000000000ull;
};

int tc_plan_create(TcPlan** out, int N, int C, int spec_type, std::string& err) {
    *out = nullptr;
    if (2 * N > kRows) {
        err = "tensor-core X-engine handles N <= 64 antennas; use CORR_FP32_SIMT for larger N";
        return CORR_EUNSUPPORTED;
    }
    if (!get_encoder()) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return CORR_ECUDA;
    }
    TcPlan* p = new TcPlan();
    p->N = N;
    p->C = C;
    p->R2 = 2 * N;
    p->Nn = (2 * N + 15) / 16 * 16;
    p->P = N * (N + 1) / 2;
    p->mode = spec_type == SPEC_F16X2 ? 0 : (spec_type == SPEC_F16 ? 1 : 2);
    p->planes = p->mode == 0 ? 2 : 1;
    p->KT = p->mode == 2 ? 128 : 64;
    const size_t stage_bytes = (size_t)p->planes * kTileBytes;
    const size_t gs_bytes = (size_t)p->R2 * (p->R2 + 1) * sizeof(float);
    const size_t budget = 227 * 1024 - 1024 - 256 - gs_bytes;
    p->stages = (int)(budget / stage_bytes);
    if (p->stages > 8) p->stages = 8;
    if (p->stages < 2) {
        delete p;
        err = "shared memory too small for the tensor-core X-engine";
        return CORR_EUNSUPPORTED;
    }
    p->smem_bytes = 1024 + p->stages * stage_bytes + gs_bytes + 16 + (2 * p->stages + 5) * 8 + 16;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete p;
        err = "cudaDeviceGetAttribute failed";
        return CORR_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    if (p->mode == 0)
        e = cudaFuncSetAttribute(xengine_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->smem_bytes);
    else if (p->mode == 1)
        e = cudaFuncSetAttribute(xengine_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->smem_bytes);
    else
        e = cudaFuncSetAttribute(xengine_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->smem_bytes);
    if (e != cudaSuccess) {
        delete p;
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return CORR_ECUDA;
    }
    *out = p;
    return CORR_OK;
}

int tc_plan_update(TcPlan* p, void* spec, int64_t cap, int N, int C, int spec_type,
                   std::string& err) {
    (void)N;
    (void)C;
    const int eb = spec_elem_bytes(spec_type);
    cuuint64_t dims[3] = {(cuuint64_t)cap, (cuuint64_t)p->R2, (cuuint64_t)p->planes * p->C};
    cuuint64_t strides[2] = {(cuuint64_t)cap * eb, (cuuint64_t)p->R2 * cap * eb};
    cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / eb), (cuuint32_t)kRows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = get_encoder()(&p->tmap, dt, 3, spec, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        err = buf;
        return CORR_ECUDA;
    }
    p->have_map = true;
    p->cap = cap;
    p->max_split = (int)((cap + 255) / 256);
    return CORR_OK;
}

// Split of the spectra range that balances whole k-tiles over the SMs.
static void choose_split(const TcPlan* p, int64_t S_pad, int& n_split, int64_t& S_item) {
    const int64_t tiles = S_pad / p->KT;
    double best = -1.0;
    n_split = 1;
    S_item = S_pad;
    for (int n = 1; n <= p->max_split && n <= tiles; ++n) {
        const int64_t per = (tiles + n - 1) / n;              // k-tiles per item
        const int nn = (int)((tiles + per - 1) / per);        // items per channel
        const int64_t items = (int64_t)p->C * nn;
        // round-robin over the SMs: the busiest SM does ceil(items/SMs) items
        const int64_t rounds = (items + p->num_sms - 1) / p->num_sms;
        const double work = (double)rounds * (double)(per + 2);   // +2: per-item overhead
        const double eff = (double)(tiles * p->C) / ((double)p->num_sms * work);
        const double bonus = nn == 1 ? 1.15 : 1.0;   // n = 1 needs no reduction launch
        if (eff * bonus > best + 1e-9) {
            best = eff * bonus;
            n_split = nn;
            S_item = per * p->KT;
        }
    }
}

int tc_num_partials(const TcPlan* p, int64_t S_pad) {
    int n;
    int64_t si;
    choose_split(p, S_pad, n, si);
    return n;
}

int tc_run(TcPlan* p, int64_t S_pad, float2* partial, double2* acc, const float* scale,
           int* status, cudaStream_t st, std::string& err, bool* direct) {
    *direct = false;
    if (!p->have_map) {
        err = "tensor-core plan has no workspace";
        return CORR_ESTATE;
    }
    if (S_pad <= 0) return CORR_OK;
    TcArgs a{};
    a.N = p->N;
    a.C = p->C;
    a.R2 = p->R2;
    a.Nn = p->Nn;
    a.P = p->P;
    a.mode = p->mode;
    a.planes = p->planes;
    a.stages = p->stages;
    a.KT = p->KT;
    a.W = kWindow;
    a.S_pad = S_pad;
    int n_split;
    choose_split(p, S_pad, n_split, a.S_item);
    a.n_items = p->C * n_split;
    a.idesc = make_idesc(kRows, p->Nn);
    a.partial = partial;
    a.acc = (n_split == 1) ? acc : nullptr;
    a.scale = scale;
    a.status = status;
    a.timeout_ns = p->timeout_ns;
    const int grid = a.n_items < p->num_sms ? a.n_items : p->num_sms;
    if (p->mode == 0)
        xengine_tc_kernel<0><<<grid, kTcThreads, p->smem_bytes, st>>>(p->tmap, a);
    else if (p->mode == 1)
        xengine_tc_kernel<1><<<grid, kTcThreads, p->smem_bytes, st>>>(p->tmap, a);
    else
        xengine_tc_kernel<2><<<grid, kTcThreads, p->smem_bytes, st>>>(p->tmap, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("tensor-core X-engine launch: ") + cudaGetErrorString(e);
        return CORR_ECUDA;
    }
    p->last_split = n_split;
    *direct = a.acc != nullptr;
    return CORR_OK;
}

void tc_plan_destroy(TcPlan* p) { delete p; }

}  // namespace gbcorr
