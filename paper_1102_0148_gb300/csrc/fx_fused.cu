// Fused F/X-engine: the K = 512, FP32-mode correlator for up to 44 antennas
// as ONE persistent kernel per run of device-resident input, with the
// spectra handed from the F-engine to the X-engine through a ring of
// workspace slots that stays in L2 instead of a workspace in HBM.
//
// Paper: Sec. 1 (FFT every stream into channels, cross-multiply every pair
// per channel, accumulate), Sec. 3-4 (the I/O core's FFT and the compute
// core's XMAC run side by side; the XMAC is I/O-bound once its data leave
// the near memory).  Here both run side by side on every SM: a CTA (one
// per SM, cooperative launch, so every CTA is resident) holds
//   warps 0-15   two F-engine sub-blocks of 8 warps (the K = 512 body of
//                fengine_k512.cuh, each with its own shared memory and
//                named barrier), taking (32-frame block, antenna) tasks from
//                a global counter in chunk order and writing them into ring
//                slot (chunk mod 3);
//   warp 16      TMA producer of the X-engine;
//   warp 17      TMEM allocator and tcgen05.mma issuer;
//   warps 18-21  epilogue: TMEM windows -> running sums in TMEM -> FP64.
// The CTA's X warps own channels blockIdx.x + 152 g.  A chunk (up to 8
// blocks of 32 frames of one push; every push starts a new chunk) is
// cross-multiplied once every F task of it has published its count
// (done[c]); the F tasks of chunk c + 3 wait until every CTA's X warps have
// released chunk c (freed[c]).  For channel k a window of W spectra is
// accumulated in TMEM: per 16 spectra one MMA of N = 2r (B = [hi; lo], r =
// 2N rounded up to 16) gives [hi hi^T | hi lo^T] and a second of N = r
// (A = lo, B = hi) adds lo hi^T = (hi lo^T)^T onto the first block, so
// G = D[:, 0:r] + D[:, r:2r] needs no transpose.  The epilogue adds G into
// a running FP32 sum, also in TMEM, which it turns into visibilities
// V_ij = (G[2i][2j] + G[2i+1][2j+1]) + i (G[2i+1][2j] - G[2i][2j+1]),
// descaled by 1/(sigma_i sigma_j), and adds to the FP64 accumulator at the
// end of every push (and every 64 chunks): a push is then summed the same
// way whether it shares a launch with others or not, so the result does not
// depend on how pushes are grouped into launches (checkpoints resume
// bit-identically).  TMEM accumulates only one window (its FP32
// accumulation truncates; windows are summed with round-to-nearest adds).
// Every wait -- mbarriers and the global chunk counters -- has a
// global-timer limit; on expiry the kernel records a status word, drains
// its own copies and MMAs, frees TMEM and returns.
#include "fx_fused.h"

#include "fengine_k512.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

namespace gbcorr {
namespace {

using namespace fk;
using namespace tc;

constexpr int kFxSub = 2;                       // F sub-blocks per CTA
constexpr int kFxWarps = 8 * kFxSub + 2 + 4;    // + producer, MMA, 4 epilogue warps
constexpr int kFxThreads = 32 * kFxWarps;       // 704
constexpr int kFxProducerWarp = 8 * kFxSub;
constexpr int kFxMmaWarp = kFxProducerWarp + 1;
constexpr int kFxEpiWarp = kFxProducerWarp + 2;
constexpr int kFxChunkBlocks = 8;               // 32-frame blocks per chunk
constexpr int kFxRing = 3;                      // ring slots (chunks)
constexpr int kFxStages = 2;                    // X operand stages
constexpr int kFxAtoms = 2;                     // 32-frame k-tiles per stage
constexpr int kFxRowBytes = 64;                 // 32 FP16 values per tile row
constexpr int kFxChannels = 256;
constexpr int kFxFlushChunks = 64;              // running sums -> FP64 every 64 chunks
constexpr size_t kFxSmemBudget = 227 * 1024;

struct FxBlock {
    const uint8_t* in;     // record of (first frame, antenna 0)
    int nvalid;            // frames of the block that are input (1..32)
    int chunk;             // its chunk ...
    int pos;               // ... and k-tile in it (0..15)
    int pad;
};

struct FxChunk {
    int nblk;              // blocks (k-tiles) of the chunk, 1..16
    int flush;             // the last chunk of a push: running sums -> FP64 after it
};

struct FxArgs {
    CUtensorMap tmap;              // ring: {32 frames, 2N rows, 256 channels, 2 x 3 x 16 tiles}
    const FxBlock* blocks;         // [n_blk]
    const FxChunk* chunks;         // [n_chunks]
    int n_blk, n_chunks, N, P;
    int sr;                        // operand tile rows: 2N rounded up to 16
    int W;                         // spectra per TMEM window (multiple of 64, divides 256)
    const float2* twiddle;
    const float* split;            // [N] two-plane pre-scales
    const float2* corr;            // [N][256] corrections (CORR)
    char* ring;
    int64_t plane_stride;          // elements from the ring's hi plane to its lo plane
    unsigned* next_task;           // zero before the launch
    unsigned* done;                // [n_chunks] F tasks finished per chunk, zero before
    unsigned* freed;               // [n_chunks] CTAs whose X part released the chunk, zero before
    double2* acc;                  // [256][P]
    int* status;
    unsigned long long timeout_ns;
    int withhold;                  // test hook: chunk 0 is never complete
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until *ctr >= need (another CTA's release).  False when the
// limit passes (status recorded) or another CTA or role has given up.
__device__ bool wait_count(const unsigned* ctr, unsigned need, volatile int* abort_word,
                           const FxArgs& a) {
    unsigned long long t0 = 0;
    for (uint32_t n = 0;; ++n) {
        if (ld_acquire(ctr) >= need) return true;
        if (*abort_word || ld_volatile(a.status)) {
            *abort_word = 1;
            return false;
        }
        if (n >= 4) __nanosleep(128);
        if ((n & 15) == 15) {
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

// mbarrier wait bounded like wait_count, also giving up when another CTA has
// recorded a status.
__device__ __forceinline__ bool wait_mbar(uint32_t bar, uint32_t parity, volatile int* abort_word,
                                          const FxArgs& a) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = 0;
    for (uint32_t n = 0;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_word) return false;
        if ((n & 63) == 63) {
            if (ld_volatile(a.status)) {
                *abort_word = 1;
                return false;
            }
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

__device__ __forceinline__ int chunk_tiles(const FxArgs& a, int c) { return a.chunks[c].nblk; }

// Shared-memory plan of one CTA (offsets from the 1024-byte aligned base).
struct FxSmem {
    uint32_t slot, atom, stage, ring, tscr, fsub, bars, total;
};

// sr: operand rows (2N rounded up to 16); r2: 2N, the rows of G.
__host__ __device__ inline FxSmem fx_smem(int sr, int r2, bool corr) {
    FxSmem m;
    m.slot = (uint32_t)sr * kFxRowBytes;
    m.atom = 2 * m.slot;                                     // hi slot, lo slot
    m.stage = kFxAtoms * m.atom;
    // rows an MMA reads past the ring: A (128 rows) from the last lo slot
    const int over = 128 - sr > 0 ? 128 - sr : 0;
    m.ring = kFxStages * m.stage + (uint32_t)over * kFxRowBytes;
    m.tscr = (uint32_t)r2 * (uint32_t)(r2 + 1) * 4;          // G of one channel at a flush
    m.fsub = (uint32_t)kStgFloats * 4 + 128 * 8 + (corr ? 256 * 8 : 0);
    m.bars = 256;
    m.total = m.ring + ((m.tscr + 15) & ~15u) + kFxSub * m.fsub + m.bars;
    return m;
}

template <bool CORR>
__global__ void __launch_bounds__(kFxThreads, 1) fx_fused_kernel(const __grid_constant__ FxArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int sr = a.sr;
    const int r2 = 2 * a.N;
    const FxSmem L = fx_smem(sr, r2, CORR);
    unsigned char* ring_s = smem;
    float* tscr = reinterpret_cast<float*>(smem + L.ring);
    unsigned char* fbase = smem + L.ring + ((L.tscr + 15) & ~15u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(fbase + kFxSub * L.fsub);
    uint64_t* full = bars;                     // [kFxStages]
    uint64_t* empty = full + kFxStages;        // [kFxStages]
    uint64_t* accf = empty + kFxStages;        // window full (MMA -> epilogue)
    uint64_t* acce = accf + 1;                 // window free (epilogue warps -> MMA)
    uint64_t* drain = acce + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* ep_flag = abort_word + 1;
    volatile unsigned* task_slot = reinterpret_cast<volatile unsigned*>(ep_flag + 1);   // [kFxSub]

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int N = a.N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFxStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accf), 1);
        mbar_init(smem_u32(acce), 4);          // one arrival per epilogue warp
        mbar_init(smem_u32(drain), 1);
        *abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == kFxMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kFxProducerWarp) {
        // ------------------------------------------------------ F-engine
        const int sb = warp >> 3;
        const int tsb = threadIdx.x - 256 * sb;
        unsigned char* fs = fbase + sb * L.fsub;
        float* stg = reinterpret_cast<float*>(fs);
        float2* tw_base = reinterpret_cast<float2*>(fs + (size_t)kStgFloats * 4);
        float2* corr_tab = tw_base + 128;
        auto sync = [sb]() { named_bar(1 + sb, 256); };
        const unsigned T = (unsigned)a.n_blk * (unsigned)N;
        for (;;) {
            if (tsb == 0) {
                unsigned t = atomicAdd(a.next_task, 1u);
                if (t < T) {
                    const int c = a.blocks[t / N].chunk;
                    if (*abort_word || ld_volatile(a.status)) t = T;
                    else if (c >= kFxRing && !wait_count(a.freed + (c - kFxRing), gridDim.x, abort_word, a))
                        t = T;
                }
                task_slot[sb] = t;
            }
            sync();
            const unsigned t = task_slot[sb];
            if (t >= T) break;
            const int blk = (int)(t / N);
            const int ant = (int)(t - (unsigned)blk * N);
            const FxBlock fb = a.blocks[blk];
            const int c = fb.chunk;
            F512Block b;
            b.in = fb.in + (int64_t)ant * 256;
            b.stride = (int64_t)N * 256;
            b.nvalid = fb.nvalid;
            b.ant = ant;
            b.post = __ldg(a.split + ant);
            b.spec = a.ring;
            b.s = (int64_t)(c % kFxRing) * (32 * kFxChunkBlocks) + (int64_t)fb.pos * 32;
            b.N = N;
            b.plane_stride = a.plane_stride;
            b.debug = nullptr;
            f512_block<SPEC_F16X2, CORR>(b, a.twiddle, CORR ? a.corr + (int64_t)ant * 256 : nullptr,
                                         nullptr, stg, tw_base, nullptr, corr_tab, tsb, sync);
            // publish the block to the X-engines of every CTA (their TMA reads
            // are async-proxy accesses)
            fence_proxy_async_global();
            __threadfence();
            sync();
            if (tsb == 0) atomicAdd(a.done + c, 1u);
        }
    } else if (warp == kFxProducerWarp) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0, st = 0, ph = 0, armed = 0, armed_ph = 0;
            bool ok = true;
            for (int c = 0; ok && c < a.n_chunks; ++c) {
                const int nkt = chunk_tiles(a, c);
                const unsigned need = (unsigned)nkt * N + ((a.withhold && c == 0) ? 1u : 0u);
                if (!wait_count(a.done + c, need, abort_word, a)) {
                    ok = false;
                    break;
                }
                fence_proxy_async_global();
                const int tile0 = (c % kFxRing) * kFxChunkBlocks;
                for (int ch = blockIdx.x; ok && ch < kFxChannels; ch += gridDim.x) {
                    for (int kt = 0; kt < nkt; kt += kFxAtoms, ++it) {
                        if (it > 0 && ++st == (uint32_t)kFxStages) {
                            st = 0;
                            ph ^= 1u;
                        }
                        if (!wait_mbar(smem_u32(&empty[st]), ph ^ 1u, abort_word, a)) {
                            ok = false;
                            break;
                        }
                        const int n_at = min(kFxAtoms, nkt - kt);
                        const uint32_t fb = smem_u32(&full[st]);
                        mbar_expect_tx(fb, (uint32_t)n_at * 2u * L.slot);
                        const uint32_t dst = smem_u32(ring_s + st * L.stage);
                        for (int at = 0; at < n_at; ++at) {
                            const int tile = tile0 + kt + at;
                            tma_load_4d(dst + at * L.atom, &a.tmap, fb, 0, ch, tile);
                            tma_load_4d(dst + at * L.atom + L.slot, &a.tmap, fb, 0, ch,
                                        kFxRing * kFxChunkBlocks + tile);
                        }
                        armed |= 1u << st;
                        armed_ph = (armed_ph & ~(1u << st)) | (ph << st);
                    }
                }
            }
            if (!ok) {
                // every armed stage's copies must land before teardown
                const unsigned long long d2 = globaltimer() + a.timeout_ns;
                for (int s2 = 0; s2 < kFxStages; ++s2) {
                    if (!((armed >> s2) & 1u)) continue;
                    while (!mbar_try_wait(smem_u32(&full[s2]), (armed_ph >> s2) & 1u))
                        if (globaltimer() > d2) break;
                }
            }
        }
    } else if (warp == kFxMmaWarp) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t it = 0, st = 0, ph = 0, wi = 0;
            bool ok = true, issued = false;
            // D = F32, A = B = F16, K-major, M = 128; N = 2 sr (B = [hi; lo]) and
            // N = sr (A = lo, B = hi, onto the first sr columns)
            const uint32_t idesc = (1u << 4) | ((uint32_t)((2 * sr) >> 3) << 17) | (8u << 24);
            const uint32_t idesc_lh = (1u << 4) | ((uint32_t)(sr >> 3) << 17) | (8u << 24);
            const int Wt = a.W / 32;                      // k-tiles per window
            for (int c = 0; ok && c < a.n_chunks; ++c) {
                const int nkt = chunk_tiles(a, c);
                for (int ch = blockIdx.x; ok && ch < kFxChannels; ch += gridDim.x) {
                    for (int w0 = 0; ok && w0 < nkt; w0 += Wt, ++wi) {
                        if (!wait_mbar(smem_u32(acce), (wi & 1u) ^ 1u, abort_word, a)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int w1 = min(nkt, w0 + Wt);
                        uint32_t accum = 0;
                        for (int kt = w0; kt < w1; kt += kFxAtoms, ++it) {
                            if (it > 0 && ++st == (uint32_t)kFxStages) {
                                st = 0;
                                ph ^= 1u;
                            }
                            if (!wait_mbar(smem_u32(&full[st]), ph, abort_word, a)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t base = smem_u32(ring_s + st * L.stage);
                            const int n_at = min(kFxAtoms, w1 - kt);
                            for (int at = 0; at < n_at; ++at) {
                                const uint32_t ab = base + (uint32_t)at * L.atom;
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk) {
                                    const uint64_t ah = sw64_desc(ab + 32u * kk);
                                    const uint64_t al = sw64_desc(ab + L.slot + 32u * kk);
                                    mma<0>(tmem, ah, ah, idesc, accum);
                                    mma<0>(tmem, al, ah, idesc_lh, 1u);
                                    accum = 1;
                                }
                            }
                            issued = true;
                            mma_commit(smem_u32(&empty[st]));
                        }
                        if (!ok) break;
                        mma_commit(smem_u32(accf));
                    }
                }
            }
            if (!ok && issued) {
                mma_commit(smem_u32(drain));
                const unsigned long long d2 = globaltimer() + a.timeout_ns;
                while (!mbar_try_wait(smem_u32(drain), 0u))
                    if (globaltimer() > d2) break;
            }
        }
    } else {
        // --------------------------------------------------------- epilogue
        // 4 warps; warp w reads TMEM lanes 32 (w mod 4) ..: thread r holds
        // row r of the window (columns 0 .. 2 sr - 1: [hi hi^T + lo hi^T |
        // hi lo^T]) and of the running sums G (columns 2 sr + g sr .. for
        // owned channel g).  Each warp waits for a window and frees it on
        // its own; the four meet once per chunk and around a flush.
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const int et = threadIdx.x - 32 * kFxEpiWarp;     // 0..127
        const bool live = 32 * q < r2;                   // the warp holds rows of G
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t run0 = 2u * (uint32_t)sr;
        auto esync = []() { named_bar(3, 128); };
        const int n_own = (kFxChannels - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        const int Wt = a.W / 32;
        // running sums start at zero
        if (live) {
            const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            for (int j = 0; j < n_own * sr; j += 8) tmem_st8(trow + run0 + (uint32_t)j, z);
            tmem_st_wait();
        }
        uint32_t wi = 0;
        for (int c = 0; c < a.n_chunks; ++c) {
            const int nkt = chunk_tiles(a, c);
            bool dead = false;
            for (int g = 0; g < n_own && !dead; ++g) {
                for (int w0 = 0; w0 < nkt; w0 += Wt, ++wi) {
                    int ok = 0;
                    if (lane == 0) ok = wait_mbar(smem_u32(accf), wi & 1u, abort_word, a) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        dead = true;
                        break;
                    }
                    tc_fence_after();
                    // G[r][col] += D[r][col] + D[r][sr + col]
                    if (live) {
                        const uint32_t rg = trow + run0 + (uint32_t)(g * sr);
                        for (int j = 0; j < sr; j += 8) {
                            uint32_t h[8], l[8], sm[8];
                            tmem_ld8(trow + (uint32_t)j, h);
                            tmem_ld8(trow + (uint32_t)(sr + j), l);
                            tmem_ld8(rg + (uint32_t)j, sm);
                            tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                sm[e] = __float_as_uint(__uint_as_float(sm[e]) +
                                                        (__uint_as_float(h[e]) + __uint_as_float(l[e])));
                            tmem_st8(rg + (uint32_t)j, sm);
                        }
                        tmem_st_wait();
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(acce));   // this warp's rows are free
                }
            }
            // every warp has drained chunk c (so its copies landed and its
            // MMAs ran): release the ring slot; flush the sums at a push's end
            if (dead) *abort_word = 1;
            esync();
            // one reading of the abort word for all four warps (other roles
            // may set it at any time)
            if (et == 0) *ep_flag = *abort_word;
            esync();
            if (*ep_flag) break;
            if (et == 0) {
                __threadfence();
                atomicAdd(a.freed + c, 1u);
            }
            const bool last = c == a.n_chunks - 1;
            if (last || a.chunks[c].flush || (c + 1) % kFxFlushChunks == 0) {
                // running sums -> visibilities -> the FP64 accumulator (this
                // CTA is the only one adding to its channels in this launch)
                const int P = a.P;
                for (int g = 0; g < n_own; ++g) {
                    const int ch = (int)blockIdx.x + g * (int)gridDim.x;
                    tc_fence_after();
                    if (live) {
                        const uint32_t rg = trow + run0 + (uint32_t)(g * sr);
                        const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                        for (int j = 0; j < sr; j += 8) {
                            uint32_t sm[8];
                            tmem_ld8(rg + (uint32_t)j, sm);
                            tmem_ld_wait();
                            if (r < r2)
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    if (j + e < r2) tscr[r * (r2 + 1) + j + e] = __uint_as_float(sm[e]);
                            tmem_st8(rg + (uint32_t)j, z);
                        }
                        tmem_st_wait();
                    }
                    esync();
                    int li = 0, row_next = N;
                    for (int p = et; p < P; p += 128) {
                        while (p >= row_next) {
                            ++li;
                            row_next += N - li;
                        }
                        const int lj = li + (p - (row_next - (N - li)));
                        const float* g0 = tscr + (2 * li) * (r2 + 1) + 2 * lj;
                        const float re = g0[0] + g0[r2 + 2];
                        const float im = g0[r2 + 1] - g0[1];
                        const double f = 1.0 / ((double)__ldg(a.split + li) * (double)__ldg(a.split + lj));
                        double2* dst = a.acc + (int64_t)ch * P + p;
                        double2 v = *dst;
                        v.x += (double)re * f;
                        v.y += (double)im * f;
                        *dst = v;
                    }
                    esync();
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kFxMmaWarp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

}  // namespace

struct FxPlan {
    int N = 0, sr = 0, num_sms = 0;
    char* ring = nullptr;            // [2 planes][3 x 16 tiles][256][2N][32] FP16
    int64_t plane_stride = 0;
    CUtensorMap tmap;
    unsigned* ctr = nullptr;         // next_task | done[max chunks] | freed[max chunks]
    FxBlock* blocks = nullptr;       // device block table, then the chunk table
    FxChunk* chunks = nullptr;
    FxBlock* host_blocks[2] = {};    // pinned, alternately: blocks, then chunks
    cudaEvent_t host_free[2] = {};
    int host_next = 0;
    int withhold = 0;
    unsigned long long timeout_ns = 4000000000ull, hook_timeout_ns = 0;
};

bool fx_supported(int N, int K, int spec_type) {
    if (K != 512 || spec_type != SPEC_F16X2 || N < 1 || N > kFxMaxN) return false;
    const int sr = (2 * N + 15) / 16 * 16;
    return fx_smem(sr, 2 * N, true).total + 1024 <= kFxSmemBudget;
}

int64_t fx_blocks(const FxSegment* segs, int nseg) {
    int64_t b = 0;
    for (int s = 0; s < nseg; ++s) b += (segs[s].frames + 31) / 32;
    return b;
}

namespace {
// Both tables in one buffer: kFxMaxBlocks blocks, then kFxMaxBlocks chunks.
constexpr size_t kFxTableBytes = (size_t)kFxMaxBlocks * (sizeof(FxBlock) + sizeof(FxChunk));
}  // namespace

int fx_plan_create(FxPlan** out, int N, std::string& err) {
    *out = nullptr;
    if (!fx_supported(N, 512, SPEC_F16X2)) {
        err = "fused F/X-engine: geometry not served";
        return CORR_EINVAL;
    }
    if (!get_encoder()) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return CORR_ECUDA;
    }
    FxPlan* p = new FxPlan();
    p->N = N;
    p->sr = (2 * N + 15) / 16 * 16;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    auto fail = [&](int code, const char* msg) {
        cudaGetLastError();
        fx_plan_destroy(p);
        err = msg;
        return code;
    };
    if (!coop) return fail(CORR_EUNSUPPORTED, "fused F/X-engine: no cooperative launch on this device");
    const int64_t tiles = (int64_t)kFxRing * kFxChunkBlocks;
    p->plane_stride = tiles * kFxChannels * 2 * N * 32;
    const size_t ring_bytes = (size_t)2 * p->plane_stride * 2;
    const int max_chunks = kFxMaxBlocks;
    if (dev_malloc((void**)&p->ring, ring_bytes) != cudaSuccess ||
        dev_malloc((void**)&p->ctr, (1 + 2 * (size_t)max_chunks) * sizeof(unsigned)) != cudaSuccess ||
        dev_malloc((void**)&p->blocks, kFxTableBytes) != cudaSuccess)
        return fail(CORR_ENOMEM, "fused F/X-engine: device allocation failed");
    for (int b = 0; b < 2; ++b) {
        if (cudaMallocHost((void**)&p->host_blocks[b], kFxTableBytes) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->host_free[b], cudaEventDisableTiming) != cudaSuccess)
            return fail(CORR_ENOMEM, "fused F/X-engine: host allocation failed");
    }
    // ring as a 4-D tensor: {32 frames, 2N rows, 256 channels, 2 planes x 48 tiles}
    cuuint64_t dims[4] = {32, (cuuint64_t)(2 * N), (cuuint64_t)kFxChannels, (cuuint64_t)(2 * tiles)};
    cuuint64_t strides[3] = {64, (cuuint64_t)2 * N * 64, (cuuint64_t)kFxChannels * 2 * N * 64};
    cuuint32_t box[4] = {32, (cuuint32_t)p->sr, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = get_encoder()(&p->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, p->ring, dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CORR_ECUDA, "fused F/X-engine: cuTensorMapEncodeTiled failed");
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = c ? cudaFuncSetAttribute(fx_fused_kernel<true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kFxSmemBudget)
                          : cudaFuncSetAttribute(fx_fused_kernel<false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kFxSmemBudget);
        if (e != cudaSuccess) return fail(CORR_ECUDA, "fused F/X-engine: kernel attribute");
    }
    *out = p;
    return CORR_OK;
}

void fx_plan_destroy(FxPlan* p) {
    if (!p) return;
    for (int b = 0; b < 2; ++b) {
        if (p->host_free[b]) {
            cudaEventSynchronize(p->host_free[b]);
            cudaEventDestroy(p->host_free[b]);
        }
        if (p->host_blocks[b]) cudaFreeHost(p->host_blocks[b]);
    }
    cudaFree(p->ring);
    cudaFree(p->ctr);
    cudaFree(p->blocks);
    delete p;
}

int fx_test_withhold(FxPlan* p, double wait_limit_s, std::string& err) {
    if (!(wait_limit_s >= 0.001 && wait_limit_s <= 10.0)) {
        err = "wait limit must be in [0.001, 10] s";
        return CORR_EINVAL;
    }
    p->withhold = 1;
    p->hook_timeout_ns = (unsigned long long)(wait_limit_s * 1e9);
    return CORR_OK;
}

int fx_launch(FxPlan* p, const FxSegment* segs, int nseg, const float2* twiddle,
              const float* split, const float2* corr, double2* acc, int* status, cudaStream_t st,
              std::string& err) {
    const int64_t nb = fx_blocks(segs, nseg);
    if (nb == 0) return CORR_OK;
    if (nb > kFxMaxBlocks) {
        err = "fused F/X-engine: too many blocks in one launch";
        return CORR_EINVAL;
    }
    // block table, built in the pinned buffer not in flight and copied on st
    const int hb = p->host_next;
    p->host_next ^= 1;
    if (cudaEventSynchronize(p->host_free[hb]) != cudaSuccess) {
        err = "fused F/X-engine: event wait failed";
        return CORR_ECUDA;
    }
    // every push (segment) starts a chunk; its last chunk flushes the sums
    FxBlock* tb = p->host_blocks[hb];
    FxChunk* tc = reinterpret_cast<FxChunk*>(tb + kFxMaxBlocks);
    int64_t k = 0;
    int n_chunks = 0;
    const int64_t rec = (int64_t)p->N * 256;
    for (int s = 0; s < nseg; ++s) {
        int pos = kFxChunkBlocks;
        for (int64_t f0 = 0; f0 < segs[s].frames; f0 += 32, ++k) {
            if (pos == kFxChunkBlocks) {
                tc[n_chunks].nblk = 0;
                tc[n_chunks].flush = 0;
                ++n_chunks;
                pos = 0;
            }
            tb[k].in = segs[s].in + f0 * rec;
            tb[k].nvalid = (int)std::min<int64_t>(32, segs[s].frames - f0);
            tb[k].chunk = n_chunks - 1;
            tb[k].pos = pos++;
            tb[k].pad = 0;
            tc[n_chunks - 1].nblk += 1;
        }
        if (n_chunks > 0) tc[n_chunks - 1].flush = 1;
    }
    p->chunks = reinterpret_cast<FxChunk*>(p->blocks + kFxMaxBlocks);
    cudaError_t e = cudaMemcpyAsync(p->blocks, tb, (size_t)nb * sizeof(FxBlock),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->chunks, tc, (size_t)n_chunks * sizeof(FxChunk),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->host_free[hb], st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p->ctr, 0, (1 + 2 * (size_t)n_chunks) * sizeof(unsigned), st);
    if (e != cudaSuccess) {
        err = std::string("fused F/X-engine: ") + cudaGetErrorString(e);
        return CORR_ECUDA;
    }
    FxArgs a;
    memset(&a, 0, sizeof a);
    a.tmap = p->tmap;
    a.blocks = p->blocks;
    a.chunks = p->chunks;
    a.n_blk = (int)nb;
    a.n_chunks = n_chunks;
    a.N = p->N;
    a.P = p->N * (p->N + 1) / 2;
    a.sr = p->sr;
    a.W = 256;
    a.twiddle = twiddle;
    a.split = split;
    a.corr = corr;
    a.ring = p->ring;
    a.plane_stride = p->plane_stride;
    a.next_task = p->ctr;
    a.done = p->ctr + 1;
    a.freed = p->ctr + 1 + n_chunks;
    a.acc = acc;
    a.status = status;
    a.timeout_ns = p->timeout_ns;
    if (p->withhold) {
        a.withhold = 1;
        a.timeout_ns = p->hook_timeout_ns;
        p->withhold = 0;
    }
    const FxSmem L = fx_smem(p->sr, 2 * p->N, corr != nullptr);
    const size_t smem = L.total + 1024;
    void* args[] = {&a};
    e = corr ? cudaLaunchCooperativeKernel((const void*)fx_fused_kernel<true>, p->num_sms,
                                           kFxThreads, args, smem, st)
             : cudaLaunchCooperativeKernel((const void*)fx_fused_kernel<false>, p->num_sms,
                                           kFxThreads, args, smem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("fused F/X-engine launch: ") + cudaGetErrorString(e);
        return CORR_ECUDA;
    }
    return CORR_OK;
}

}  // namespace gbcorr
