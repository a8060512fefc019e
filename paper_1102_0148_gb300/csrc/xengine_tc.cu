// X-engine on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Paper: Sec. 1 (cross-multiply every pair of antennas per channel and
// accumulate), Sec. 4 (the cross-multiply dominates the load; the paper
// converts the FFT output to a narrower type with prescaling before it).
//
// For one channel k the spectra of a pass form the real matrix A whose rows
// are the real and imaginary parts of every antenna (spectra along the
// contraction axis); the Gram matrix G = A A^T holds every product the
// visibilities need.  Antennas come in blocks of 64 (128 rows at most); for
// a pair of blocks (b1 <= b2) with local antennas i' < nb1 and j' < nb2
// (block rows 2 i' = Re, 2 i' + 1 = Im:
//   Re V_ij = G[2i'][2j'] + G[2i'+1][2j'+1],  Im V_ij = G[2i'+1][2j'] - G[2i'][2j'+1].)
// Each block pair is a dense contraction D[128 x Nn] += A_b1[128 x 16|32] *
// A_b2^T on the tensor cores, operands loaded by TMA (rows past the antenna
// count are zero-filled), FP32 accumulators in TMEM.  For a diagonal pair
// both operands are the same shared-memory tile.
//
// Precisions (operands in shared memory, K-major; FP16 tiles of 32 spectra in
// 64-byte rows with the 64-byte swizzle, FP8 tiles of 128 in 128-byte rows
// with the 128-byte swizzle; rows 2 i' and 2 i' + 1 of a block are the real
// and imaginary parts of its antenna i'):
//   mode 0 (FP32-accurate): two FP16 planes sigma_i x = hi + lo, sigma_i a
//           power of two per antenna.  Diagonal pairs issue Dhh += hi hi^T
//           and Dhl += hi lo^T and form G = Dhh + Dhl + Dhl^T; off-diagonal
//           pairs issue hi hi^T, hi lo^T and lo hi^T into one accumulator
//           (lo lo^T is below 2^-22); V_ij is descaled by 1/(sigma_i sigma_j).
//   mode 1: one FP16 plane (pre-scaled per antenna and channel).
//   mode 2: one FP8-E4M3 plane (pre-scaled), kind::f8f6f4.
//
// One launch may serve several correlators ("modes") of different N and K
// that share the precision: work items (mode, channel, block pair, range of
// spectra) are enumerated mode by mode and dealt round-robin to persistent
// CTAs of 10 warps:
//   warp 0    TMA producer (one lane)     -> stage ring (full/empty mbarriers)
//   warp 1    TMEM allocator + MMA issuer (one lane) -> two TMEM accumulator sets
//   warps 2-9 epilogue: TMEM -> registers, summed over windows -> G in shared
//             memory -> V -> FP64 accumulator (or FP32 partials)
// The tensor core's FP32 accumulation into TMEM is biased (it loses about one
// unit in the last place per accumulate, always toward zero), so TMEM only
// accumulates one window of W spectra; the epilogue adds the windows with
// round-to-nearest FP32 arithmetic.  The two accumulator sets let the
// epilogue drain window n while the MMAs fill window n+1.
// Every mbarrier wait is bounded by a global-timer deadline; on expiry the
// kernel records a status code, drains its own copies and MMAs, frees TMEM
// and returns.
#include "xengine_tc.h"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <vector>

namespace gbcorr {
namespace {

using namespace tc;

constexpr int kTcThreads = 320;     // producer, MMA, 8 epilogue warps
constexpr int kRows = 128;          // MMA M = TMA box rows = one antenna block
constexpr uint32_t kTmemCols = 512; // two accumulator sets of 256 columns
constexpr int kVB = 2;              // accumulator loads in flight per epilogue thread
constexpr int kVCols = 16;          // baselines per antenna in one staging round
constexpr int kVRow = kVCols + 1;   // float2 per staging row (+1: bank offset)

struct TcModeArgs {
    int N, C, P;
    int nblk, npairs;         // antenna blocks of 64 and the work groups of a channel
    int n_split;
    int item_base, n_items;   // items: block pair fastest, then channel, then split
    int64_t S_pad, S_item;
    int64_t tiles;            // k-tiles of the pass (balanced deal)
    int cap_tiles;            // k-tiles of a workspace plane (the lo plane's first tile)
    uint32_t box_bytes;       // bytes one TMA box of this mode lands in shared memory
    int64_t unit_base;        // first work unit of this mode (balanced deal)
    float2* partial;          // [n_split][C][P] FP32 partials (n_split > 1)
    double2* acc;             // [C][P] FP64 accumulator
    int* ticket;              // [C][npairs] arrival counters (n_split > 1), zero between launches
    const float* scale;       // [N][C] pre-cast scales (modes 1, 2)
    const float* split;       // [N] two-plane pre-scales sigma_i (mode 0)
};

struct TcArgs {
    CUtensorMap tmap[kMaxTcModes];
    TcModeArgs md[kMaxTcModes];
    int n_modes, total_items;
    int stages, KT, W;
    int kt_shift;             // log2(KT): the single-lane roles avoid 64-bit division
    int atoms;                // k-tiles of KT spectra per pipeline stage
    int row_bytes;            // bytes of one tile row: 64 (FP16 modes) or 128 (FP8)
    int wide;                 // a mode has several antenna blocks: atoms hold A, B0, B1 slots
    int gs_floats;            // epilogue G buffer (largest 2nb x (2nb + 1) of the modes)
    int slot_rows;            // rows of one operand tile slot in shared memory (<= 128)
    int* status;
    unsigned long long timeout_ns;
    int withhold;             // test hook: CTA 0 does not load its first k-tile
    int balanced;             // 1: contiguous deal of weighted k-tiles; 0: round-robin items
    int64_t units;            // total work units of the balanced deal
};

struct Item {
    int m, k, b1, b2, nbB, sp, pr;
};

// One CTA's share of an item: k-tiles [s_beg, s_end) of the pass, the
// item's slot among the CTAs sharing it and their number.
struct Piece {
    Item itm;
    int64_t s_beg, s_end;
    int slot, nslots;
};

// Work groups of a channel.  One antenna block (N <= 64): the single
// diagonal block pair.  Several blocks: block b1 against the blocks
// b2 .. b2 + nbB - 1 (b2 = b1, b1 + 2, ...; nbB = 2, or 1 for the last one of
// a row), so one A tile feeds an MMA of N = 256 and a channel's 4 blocks
// (N = 256 antennas) take 6 groups instead of 10 pairs.
__host__ __device__ __forceinline__ int groups_of(int nblk) {
    if (nblk == 1) return 1;
    int g = 0;
    for (int b1 = 0; b1 < nblk; ++b1) g += (nblk - b1 + 1) >> 1;
    return g;
}

__host__ __device__ __forceinline__ void group_decode(int gi, int nblk, int& b1, int& b2, int& nbB) {
    b1 = 0;
    if (nblk > 1)
        while (gi >= ((nblk - b1 + 1) >> 1)) {
            gi -= (nblk - b1 + 1) >> 1;
            ++b1;
        }
    b2 = b1 + 2 * gi;
    nbB = nblk == 1 ? 1 : (nblk - b2 < 2 ? nblk - b2 : 2);
}

// Work units per k-tile: 2 for the single diagonal pair (one tile loaded,
// two MMAs in FP32 mode); for a group, one per tile loaded (an A tile that
// is the group's first B block is not loaded again) plus one.  Each item
// (with k-tiles) starts with kEndUnits more, standing for the cost of an
// item's end (~4 k-tiles); they hold no k-tile.
constexpr int kEndUnits = 8;

__host__ __device__ __forceinline__ int64_t item_units(int64_t tiles, int w) {
    return tiles > 0 ? kEndUnits + tiles * w : 0;
}
__host__ __device__ __forceinline__ int pair_units(int gi, int nblk) {
    if (nblk == 1) return 2;
    int b1, b2, nbB;
    group_decode(gi, nblk, b1, b2, nbB);
    return nbB + (b2 != b1 ? 1 : 0) + 1;
}

__device__ __forceinline__ Item decode_item(const TcArgs& a, int g) {
    int m = 0;
    while (m + 1 < a.n_modes && g >= a.md[m + 1].item_base) ++m;
    const TcModeArgs& d = a.md[m];
    int l = g - d.item_base;
    Item it;
    it.m = m;
    // group fastest: the CTAs that take one channel's groups at the same
    // time share its block tiles through L2
    const int pr = l % d.npairs;
    l /= d.npairs;
    it.pr = pr;
    it.k = l % d.C;
    it.sp = l / d.C;
    group_decode(pr, d.nblk, it.b1, it.b2, it.nbB);
    return it;
}

__device__ __forceinline__ int block_ants(int N, int b) { return min(64, N - 64 * b); }

// The pieces of one CTA, in the same order for every role.
//
// Balanced deal: every mode's items (block pair major, channel fastest) are
// laid end to end as k-tiles of pair_units() units each, U units in all; CTA
// c owns the k-tiles whose first unit u has floor(u G / U) = c, so every CTA
// gets the same work to within one k-tile, whatever the channel count.  An
// item cut between CTAs is combined by the last of them (ticket).
// Round-robin deal (tile choices fixed by the caller): item g goes to CTA
// g mod G, its range is split number sp of n_split equal ranges.
struct PieceCursor {
    int m, pr, k, g;
    int64_t ibase, lo, hi;
};

__device__ __forceinline__ int64_t ceil_div64(int64_t x, int64_t y) { return (x + y - 1) / y; }

__device__ __forceinline__ void cursor_init(const TcArgs& a, PieceCursor& c) {
    c.g = blockIdx.x;
    c.m = a.n_modes;
    if (!a.balanced) return;
    const int64_t G = gridDim.x;
    c.lo = ceil_div64((int64_t)blockIdx.x * a.units, G);
    c.hi = ceil_div64((int64_t)(blockIdx.x + 1) * a.units, G);
    for (int m = 0; m < a.n_modes; ++m) {
        const TcModeArgs& d = a.md[m];
        int64_t base = d.unit_base;
        for (int pr = 0; pr < d.npairs; ++pr) {
            const int64_t iu = item_units(d.tiles, pair_units(pr, d.nblk));
            const int64_t pu = iu * d.C;
            if (c.lo < base + pu) {
                c.m = m;
                c.pr = pr;
                c.k = (int)((c.lo - base) / iu);
                c.ibase = base + (int64_t)c.k * iu;
                return;
            }
            base += pu;
        }
    }
}

__device__ __forceinline__ bool next_piece(const TcArgs& a, PieceCursor& c, Piece& p) {
    if (!a.balanced) {
        if (c.g >= a.total_items) return false;
        p.itm = decode_item(a, c.g);
        const TcModeArgs& d = a.md[p.itm.m];
        p.s_beg = (int64_t)p.itm.sp * d.S_item;
        p.s_end = min(d.S_pad, p.s_beg + d.S_item);
        p.slot = p.itm.sp;
        p.nslots = d.n_split;
        c.g += gridDim.x;
        return true;
    }
    const int64_t G = gridDim.x;
    while (c.m < a.n_modes && c.ibase < c.hi) {
        const TcModeArgs& d = a.md[c.m];
        const int w = pair_units(c.pr, d.nblk);
        const int64_t t0 = c.ibase + kEndUnits;          // first unit of k-tile 0
        const int64_t j0 = c.lo > t0 ? ceil_div64(c.lo - t0, w) : 0;
        const int64_t j1 = c.hi > t0 ? min(d.tiles, ceil_div64(c.hi - t0, w)) : 0;
        const bool mine = j0 < j1;
        if (mine) {
            p.itm.m = c.m;
            p.itm.k = c.k;
            p.itm.pr = c.pr;
            group_decode(c.pr, d.nblk, p.itm.b1, p.itm.b2, p.itm.nbB);
            p.itm.sp = 0;
            const int64_t KT = a.KT;
            p.s_beg = j0 * KT;
            p.s_end = j1 * KT;
            const int first = (int)(t0 * G / a.units);
            const int last = (int)((t0 + (d.tiles - 1) * w) * G / a.units);
            p.slot = (int)blockIdx.x - first;
            p.nslots = last - first + 1;
        }
        c.ibase += item_units(d.tiles, w);
        if (++c.k == d.C) {
            c.k = 0;
            if (++c.pr == d.npairs) {
                c.pr = 0;
                ++c.m;
            }
        }
        if (mine) return true;
    }
    return false;
}

// Bounded wait with this launch's limit and status word.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_word,
                                         const TcArgs& a) {
    return wait_bar_t(bar, parity, abort_word, a.timeout_ns, a.status);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }


// --------------------------------------------------------------------- kernel

// Stage layout of one item.  A group (several antenna blocks) fills each
// k-tile's atom of the launch's layout.  A single-block item packs its tiles
// densely: atom = [hi | lo] tiles of its own box (2N rows rounded up to 8),
// as many per stage as fit and divide a window, so a single-block mode in a
// launch with a multi-block one still moves up to a window of spectra per
// stage handshake.  (In a launch of single-block modes only this is the
// launch's own layout for the largest mode and denser for smaller ones.)
struct ItemLayout {
    uint32_t atom;      // bytes per k-tile
    uint32_t plo;       // hi -> lo plane within a k-tile
    int at;             // k-tiles per stage
};

__device__ __forceinline__ ItemLayout item_layout(const TcArgs& a, const TcModeArgs& d, bool single,
                                                  int planes, uint32_t stage_bytes,
                                                  uint32_t atom_bytes, uint32_t plane_off) {
    ItemLayout L;
    if (!single) {
        L.atom = atom_bytes;
        L.plo = plane_off;
        L.at = a.atoms;
        return L;
    }
    L.atom = (uint32_t)planes * d.box_bytes;
    L.plo = d.box_bytes;
    const int wk = a.W >> a.kt_shift;                 // k-tiles per window
    int at = (int)min((uint32_t)wk, stage_bytes / L.atom);
    while (at > 1 && wk % at) --at;
    L.at = max(at, 1);
    return L;
}

// WIDE: some mode of the launch has several antenna blocks (work groups of
// one A block and two B blocks); launches of single-block modes only take
// the narrow instance, which has none of the group code.
template <int MODE, bool WIDE>
__global__ void __launch_bounds__(kTcThreads, 1) xengine_tc_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int planes = MODE == 0 ? 2 : 1;
    // Stage layout of a group (several antenna blocks, WIDE): per k-tile
    // ("atom") the A slot of each plane [hi | lo], then the B slots
    // [B0 hi | B1 hi | B0 lo | B1 lo] (one plane: [B0 | B1]), so a group's
    // two B blocks form one operand of 256 rows; a slot has slot_rows = 128
    // rows.  A single-block item packs its k-tiles densely instead
    // ([hi | lo] of its own 2N-rounded-up-to-8 rows each, item_layout).  The
    // MMA reads 128 rows from a tile (and a single block's concatenated
    // [hi; lo] B operand 2 box rows); rows past the antennas only feed
    // outputs the epilogue ignores, and the ring is followed by enough shared
    // memory for the reads past its last tile.
    const uint32_t slot = (uint32_t)a.slot_rows * (uint32_t)a.row_bytes;
    constexpr int KK = MODE == 2 ? 4 : 2;       // MMA k-steps (32 bytes of a row) per k-tile
    const uint32_t plane_off = slot;                                // A: hi -> lo plane
    const uint32_t bh_off = planes * slot;                          // B0 hi (B1 hi follows)
    const uint32_t bl_off = bh_off + 2 * slot;                      // B0 lo (planes == 2)
    const uint32_t atom_bytes = planes * slot * (WIDE ? 3u : 1u);
    const uint32_t stage_bytes = atom_bytes * (uint32_t)a.atoms;
    unsigned char* stages = smem;
    float* Gs = reinterpret_cast<float*>(smem + a.stages * stage_bytes);   // <= 128 x 129
    // WIDE: each epilogue warp's staging rows for V, [16][kVRow] float2
    float2* vstage = reinterpret_cast<float2*>(Gs + a.gs_floats);
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(vstage + (WIDE ? 8 * 16 * kVRow : 0)) + 15) & ~(uintptr_t)15);
    uint64_t* full = bars;
    uint64_t* empty = full + a.stages;
    uint64_t* accf = empty + a.stages;
    uint64_t* acce = accf + 2;
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* epi_last = abort_word + 2;
    PieceCursor* epi_cur = reinterpret_cast<PieceCursor*>(
        (reinterpret_cast<uintptr_t>(epi_last + 2) + 15) & ~(uintptr_t)15);
    Piece* epi_pc = reinterpret_cast<Piece*>(epi_cur + 1);
    volatile int* epi_more = reinterpret_cast<volatile int*>(epi_pc + 1);
    volatile int* epi_abort = epi_more + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf[b]), 1);
            mbar_init(smem_u32(&acce[b]), 8);      // one arrival per epilogue warp
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
            uint32_t it = 0, st = 0, ph = 0;       // stage slot and its phase parity
            uint32_t armed = 0, armed_ph = 0;     // slots with copies in flight, their parity
            bool ok = true;
            PieceCursor cur;
            cursor_init(a, cur);
            Piece pc;
            while (ok && next_piece(a, cur, pc)) {
                const Item& itm = pc.itm;
                const TcModeArgs& d = a.md[itm.m];
                const CUtensorMap* map = &a.tmap[itm.m];
                const bool single = !WIDE || d.nblk == 1;  // one block: A = B, one tile
                const bool alias = !single && itm.b2 == itm.b1;   // A is the group's first B block
                const int ra = kRows * itm.b1;
                const int rb = kRows * itm.b2;
                const uint32_t ntile = single ? 1u : (uint32_t)itm.nbB + (alias ? 0u : 1u);
                const ItemLayout lay = item_layout(a, d, single, planes, stage_bytes, atom_bytes, plane_off);
                const int step_i = a.KT * lay.at;
                const int64_t s_beg = pc.s_beg;
                const int64_t s_end = pc.s_end;
                for (int64_t s = s_beg; s < s_end; s += step_i, ++it) {
                    if (it > 0 && ++st == (uint32_t)a.stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (!wait_bar(smem_u32(&empty[st]), ph ^ 1u, abort_word, a)) {
                        ok = false;
                        break;
                    }
                    if (a.withhold && blockIdx.x == 0 && it == 0) continue;   // test hook
                    const int n_at = (int)min((int64_t)lay.at, (s_end - s) >> a.kt_shift);
                    const uint32_t bytes = (uint32_t)n_at * planes * d.box_bytes * ntile;
                    const uint32_t fb = smem_u32(&full[st]);
                    mbar_expect_tx(fb, bytes);
                    const uint32_t dst = smem_u32(stages + st * stage_bytes);
                    for (int at = 0; at < n_at; ++at) {
                        const int st4 = (int)(s >> a.kt_shift) + at;   // k-tile of the pass
                        const uint32_t o = (uint32_t)at * lay.atom;
                        if (!alias) {
                            tma_load_4d(dst + o, map, fb, ra, itm.k, st4);
                            if (planes == 2)
                                tma_load_4d(dst + lay.plo + o, map, fb, ra, itm.k, d.cap_tiles + st4);
                        }
                        if (!single)
                            for (int bb = 0; bb < itm.nbB; ++bb) {
                                tma_load_4d(dst + bh_off + bb * slot + o, map, fb, rb + kRows * bb,
                                            itm.k, st4);
                                if (planes == 2)
                                    tma_load_4d(dst + bl_off + bb * slot + o, map, fb, rb + kRows * bb,
                                                itm.k, d.cap_tiles + st4);
                            }
                    }
                    armed |= 1u << st;
                    armed_ph = (armed_ph & ~(1u << st)) | (ph << st);
                }
            }
            if (!ok) {
                // drain: every armed stage's copies must land before teardown
                const unsigned long long d2 = globaltimer() + a.timeout_ns;
                for (int s2 = 0; s2 < a.stages && s2 < 16; ++s2) {
                    if (!((armed >> s2) & 1u)) continue;
                    while (!mbar_try_wait(smem_u32(&full[s2]), (armed_ph >> s2) & 1u))
                        if (globaltimer() > d2) break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t it = 0, st = 0, ph = 0;
            int wi = 0;
            bool ok = true;
            bool issued = false;
            PieceCursor cur;
            cursor_init(a, cur);
            Piece pc;
            while (ok && next_piece(a, cur, pc)) {
                const Item& itm = pc.itm;
                const TcModeArgs& d = a.md[itm.m];
                const bool single = !WIDE || d.nblk == 1;
                const bool alias = !single && itm.b2 == itm.b1;
                // single block: N = 2N rounded up to 16; group: N = 128 per B block
                const int Nn = single ? (2 * block_ants(d.N, 0) + 15) & ~15 : kRows * itm.nbB;
                // D = F32, A/B = F16 (kind::f16) or E4M3 (kind::f8f6f4), K-major,
                // N>>3 at bits 17-22, M>>4 at bits 24-28
                const uint32_t idesc =
                    (1u << 4) | ((uint32_t)(Nn >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
                // group: A from its own slots, or the first B block's
                const uint32_t a_hi = alias ? bh_off : 0u;
                const uint32_t a_lo = alias ? bl_off : plane_off;
                const ItemLayout lay = item_layout(a, d, single, planes, stage_bytes, atom_bytes, plane_off);
                const int step_i = a.KT * lay.at;
                // FP32 mode, single block: B = [hi; lo], the k-tile's two tiles
                // of box_rows rows each, N = 2 box_rows, so one MMA forms
                // [Dhh | Dhl] (Dhl from column box_rows)
                const int box_rows = (int)(d.box_bytes / (uint32_t)a.row_bytes);
                const uint32_t idesc_cat = (1u << 4) | ((uint32_t)((2 * box_rows) >> 3) << 17) |
                                           ((uint32_t)(kRows >> 4) << 24);
                const int64_t s_beg = pc.s_beg;
                const int64_t s_end = pc.s_end;
                for (int64_t w0 = s_beg; ok && w0 < s_end; w0 += a.W, ++wi) {
                    const int b = wi & 1;
                    const uint32_t aph = (uint32_t)(wi >> 1) & 1u;
                    if (!wait_bar(smem_u32(&acce[b]), aph ^ 1u, abort_word, a)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = tmem + (uint32_t)b * 256u;
                    const int64_t w1 = min(s_end, w0 + a.W);
                    uint32_t acc = 0;
                    for (int64_t s = w0; s < w1; s += step_i, ++it) {
                        if (it > 0 && ++st == (uint32_t)a.stages) {
                            st = 0;
                            ph ^= 1u;
                        }
                        if (!wait_bar(smem_u32(&full[st]), ph, abort_word, a)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = smem_u32(stages + st * stage_bytes);
                        const int n_at = (int)min((int64_t)lay.at, (w1 - s) >> a.kt_shift);
                        for (int at = 0; at < n_at; ++at) {
                            const uint32_t ab = base + (uint32_t)at * lay.atom;
#pragma unroll
                            for (int kk = 0; kk < KK; ++kk) {
                                if (single) {
                                    const uint64_t ah = op_desc<MODE>(ab + 32u * kk);
                                    // FP32 mode: B = [hi; lo] forms [Dhh | Dhl]
                                    mma<MODE>(d0, ah, ah, MODE == 0 ? idesc_cat : idesc, acc);
                                } else {
                                    const uint64_t ah = op_desc<MODE>(ab + a_hi + 32u * kk);
                                    const uint64_t bh = op_desc<MODE>(ab + bh_off + 32u * kk);
                                    mma<MODE>(d0, ah, bh, idesc, acc);
                                    if (MODE == 0) {
                                        const uint64_t al = op_desc<MODE>(ab + a_lo + 32u * kk);
                                        const uint64_t bl = op_desc<MODE>(ab + bl_off + 32u * kk);
                                        mma<MODE>(d0, ah, bl, idesc, 1u);
                                        mma<MODE>(d0, al, bh, idesc, 1u);
                                    }
                                }
                                acc = 1;
                            }
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
        // 8 warps: warp w reads TMEM lane quadrant w % 4 (rows 32q..32q+31)
        // and one half of the Nn accumulator columns.  Each warp waits for a
        // window on its own (lane 0 polls, the warp then loads its slice) and
        // frees the accumulator set by one arrival per warp; the 8 warps meet
        // only at the end of an item.  A warp whose wait fails stops loading
        // but still joins the item-end barriers, after which every warp sees
        // the shared abort word and leaves together.
        const int et = threadIdx.x - 64;            // 0..255
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int r = 32 * q + lane;
        int wi = 0;
        // one cursor for the 8 warps, in shared memory (registers are scarce here)
        if (et == 0) cursor_init(a, *epi_cur);
        for (;;) {
            if (et == 0) *epi_more = next_piece(a, *epi_cur, *epi_pc) ? 1 : 0;
            epi_sync();
            if (!*epi_more) break;
            const Piece pc = *epi_pc;
            const Item& itm = pc.itm;
            const TcModeArgs& d = a.md[itm.m];
            const bool single = !WIDE || d.nblk == 1;
            const bool diag = single;                // the single block's pair (b1 = b2 = 0)
            const bool use_t = MODE == 0 && single;
            const int nb1 = block_ants(d.N, itm.b1);
            const int nb2 = single ? nb1 : block_ants(d.N, itm.b2);
            const int R2a = 2 * nb1;
            const int R2b = 2 * nb2;
            // columns per half: one block 2N rounded up to 16, halved (<= 64);
            // a group 128 per B block, halved (<= 128)
            const int NH = single ? ((R2b + 15) & ~15) >> 1 : (kRows * itm.nbB) >> 1;
            const int col0 = h * NH;
            const int64_t s_beg = pc.s_beg;
            const int64_t s_end = pc.s_end;
            // window sums: acc[0 .. NH) (single block, FP32 mode: [0, 64) from
            // hi hi^T and [64, 64 + NH) from hi lo^T)
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            bool dead = false;
            for (int64_t w0 = s_beg; w0 < s_end; w0 += a.W, ++wi) {
                if (dead) continue;
                const int b = wi & 1;
                const uint32_t aph = (uint32_t)(wi >> 1) & 1u;
                int ok = 0;
                if (lane == 0) ok = wait_bar(smem_u32(&accf[b]), aph, abort_word, a) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    dead = true;
                    continue;
                }
                tc_fence_after();
                const uint32_t trow =
                    tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * 256u + (uint32_t)col0;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (8 * c < NH) {
                        uint32_t v[8];
                        tmem_ld8(trow + 8u * c, v);
                        if (c < 8 && use_t) {
                            uint32_t w[8];
                            tmem_ld8(trow + d.box_bytes / (uint32_t)a.row_bytes + 8u * c, w);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                acc[8 * c + j] += __uint_as_float(v[j]);
                                acc[(64 + 8 * c + j) & 127] += __uint_as_float(w[j]);
                            }
                        } else {
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[8 * c + j] += __uint_as_float(v[j]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acce[b]));   // this warp's slice is free
            }
            epi_sync();
            // one reading of the abort word for the 8 warps (the producer and
            // the MMA thread may set it at any time)
            if (et == 0) *epi_abort = *abort_word;
            epi_sync();
            if (*epi_abort) break;
            const int N = d.N, C = d.C, P = d.P;
            const bool direct = pc.nslots == 1;
            if (!single) {
                // Group: rows 2 i' and 2 i' + 1 (Re and Im of antenna i') are
                // adjacent lanes, so V comes from one exchange with the partner
                // lane: for B columns 2 j'' and 2 j'' + 1 the even lane holds
                // G[2i'][..], the odd lane G[2i'+1][..];
                //   Re V = G[2i'][2j''] + G[2i'+1][2j''+1], Im V = G[2i'+1][2j''] - G[2i'][2j''+1].
                // The even lane takes the even column pairs, the odd lane the
                // odd ones, into the warp's staging rows (16 antennas x kVCols
                // baselines per round); the warp then writes each antenna's
                // kVCols baselines, consecutive in the accumulator layout, as
                // one coalesced run of FP32 stores into the item's partial
                // slot.  (FP64 reductions straight into the accumulator, one
                // per word, cost a group pass at N = 256 ~70% more time.)
                const int odd = r & 1;
                float2* vst = vstage + (warp - 2) * 16 * kVRow;
                const int jg0 = col0 >> 1;                  // the warp's first baseline of the group
                float2* pout = d.partial + ((int64_t)pc.slot * C + itm.k) * P;
#pragma unroll
                for (int rho = 0; rho < 64 / kVCols; ++rho) {
                    if (2 * kVCols * rho < NH) {
#pragma unroll
                        for (int kk = 0; kk < kVCols; ++kk) {
                            const int k2 = kVCols * rho + kk;
                            const float v0 = acc[2 * k2], v1 = acc[2 * k2 + 1];
                            const float x0 = __shfl_xor_sync(0xffffffffu, v0, 1);
                            const float x1 = __shfl_xor_sync(0xffffffffu, v1, 1);
                            if ((kk & 1) == odd) {
                                const float av = odd ? x0 : v0, bv = odd ? x1 : v1;
                                const float cv = odd ? v0 : x0, dv = odd ? v1 : x1;
                                vst[(lane >> 1) * kVRow + kk] = make_float2(av + dv, cv - bv);
                            }
                        }
                        __syncwarp();
                        // lane -> baseline jj of the round and one of 32 / kVCols
                        // antennas of each step over the warp's 16
                        constexpr int kRowsPerStep = 32 / kVCols;
                        const int jj = lane % kVCols;
                        const int jg = jg0 + kVCols * rho + jj;
                        const int b2 = itm.b2 + (jg >> 6);
                        const int j_loc = jg & 63;
                        const bool jv = j_loc < block_ants(N, b2);
                        const int j = 64 * b2 + j_loc;
                        const float sj = !jv ? 1.f
                                             : (MODE == 0 ? __ldg(d.split + j)
                                                          : __ldg(d.scale + (int64_t)j * C + itm.k));
#pragma unroll 1
                        for (int i0 = 0; i0 < 16; i0 += kRowsPerStep) {
                            const int i16 = i0 + lane / kVCols;
                            const int i_loc = 16 * q + i16;
                            if (16 * q + i0 >= nb1) break;
                            if (i_loc < nb1 && jv && !(b2 == itm.b1 && j_loc < i_loc)) {
                                const int i = 64 * itm.b1 + i_loc;
                                const float si = MODE == 0 ? __ldg(d.split + i)
                                                           : __ldg(d.scale + (int64_t)i * C + itm.k);
                                const float f = 1.0f / (si * sj);
                                const float2 v = vst[i16 * kVRow + jj];
                                const int p = i * N - i * (i - 1) / 2 + (j - i);
                                pout[p] = make_float2(v.x * f, v.y * f);
                            }
                        }
                        __syncwarp();
                    }
                }
            } else {
            const int ldg = R2b + 1;
            if (r < R2a) {
#pragma unroll
                for (int c = 0; c < 64; ++c) {
                    const int col = col0 + c;
                    if (c < NH && col < R2b) Gs[r * ldg + col] = acc[c] + (use_t ? acc[64 + c] : 0.f);
                }
            }
            epi_sync();
            if (use_t) {
                // G[col][r] += Dhl[r][col]: each element is touched by one thread here
                if (r < R2a) {
#pragma unroll
                    for (int c = 0; c < 64; ++c) {
                        const int col = col0 + c;
                        if (c < NH && col < R2b) Gs[col * ldg + r] += acc[64 + c];
                    }
                }
                epi_sync();
            }
            const int npl = nb1 * (nb1 + 1) / 2;
            {
                // kVB pairs per thread at a time: their accumulator loads are
                // issued together, so their latencies overlap
                int li = 0;
                int row_next = nb1;                 // triangle: first index of row li + 1
                for (int base = et; base < npl; base += kVB * 256) {
                    int pp[kVB];
                    float vre[kVB], vim[kVB];
#pragma unroll
                    for (int u = 0; u < kVB; ++u) {
                        const int pl = base + 256 * u;
                        pp[u] = -1;
                        vre[u] = vim[u] = 0.f;
                        if (pl < npl) {
                            int lj;
                            if (diag) {
                                while (pl >= row_next) {
                                    ++li;
                                    row_next += nb1 - li;
                                }
                                lj = li + (pl - (row_next - (nb1 - li)));
                            } else {
                                li = pl / nb2;
                                lj = pl - li * nb2;
                            }
                            // block rows 2 i' (Re) and 2 i' + 1 (Im)
                            const float* g0 = Gs + (2 * li) * ldg + 2 * lj;
                            const float re = g0[0] + g0[ldg + 1];
                            const float im = g0[ldg] - g0[1];
                            const int i = 64 * itm.b1 + li;
                            const int j = 64 * itm.b2 + lj;
                            float f;
                            if (MODE == 0)
                                f = 1.0f / (__ldg(d.split + i) * __ldg(d.split + j));
                            else
                                f = 1.0f / (__ldg(d.scale + (int64_t)i * C + itm.k) *
                                            __ldg(d.scale + (int64_t)j * C + itm.k));
                            pp[u] = i * N - i * (i - 1) / 2 + (j - i);
                            vre[u] = re * f;
                            vim[u] = im * f;
                        }
                    }
                    if (direct) {
                        double2 old[kVB];
#pragma unroll
                        for (int u = 0; u < kVB; ++u)
                            if (pp[u] >= 0) old[u] = __ldcg(d.acc + (int64_t)itm.k * P + pp[u]);
#pragma unroll
                        for (int u = 0; u < kVB; ++u)
                            if (pp[u] >= 0)       // sole owner of (k, p) in this launch
                                d.acc[(int64_t)itm.k * P + pp[u]] =
                                    make_double2(old[u].x + (double)vre[u], old[u].y + (double)vim[u]);
                    } else {
#pragma unroll
                        for (int u = 0; u < kVB; ++u)
                            if (pp[u] >= 0)
                                d.partial[((int64_t)pc.slot * C + itm.k) * P + pp[u]] =
                                    make_float2(vre[u], vim[u]);
                    }
                }
            }
            }
            if (!direct) {
                // The last of the CTAs sharing this (channel, block pair) to
                // finish adds every partial, in slot order, into the FP64
                // accumulator (a group: into slot 0, see the run's reduction):
                // deterministic.
                __threadfence();
                epi_sync();
                if (et == 0) {
                    const int old = atomicAdd(d.ticket + itm.k * d.npairs + itm.pr, 1);
                    *epi_last = old == pc.nslots - 1 ? 1 : 0;
                }
                epi_sync();
                if (*epi_last) {
                    __threadfence();
                    // every pair of the item: the single block's upper
                    // triangle, or a group's nb1 x (64 per B block) rows and
                    // columns (the diagonal block's upper triangle)
                    int li = 0;
                    int row_next = nb1;
                    const int npl_all = single ? nb1 * (nb1 + 1) / 2 : nb1 * 64 * itm.nbB;
                    for (int pl = et; pl < npl_all; pl += 256) {
                        int i, j;
                        if (single) {
                            while (pl >= row_next) {
                                ++li;
                                row_next += nb1 - li;
                            }
                            i = li;
                            j = li + (pl - (row_next - (nb1 - li)));
                        } else {
                            const int i_loc = pl / (64 * itm.nbB);
                            const int rest = pl - i_loc * 64 * itm.nbB;
                            const int b2 = itm.b2 + (rest >> 6);
                            const int j_loc = rest & 63;
                            if (j_loc >= block_ants(N, b2) || (b2 == itm.b1 && j_loc < i_loc)) continue;
                            i = 64 * itm.b1 + i_loc;
                            j = 64 * b2 + j_loc;
                        }
                        const int p = i * N - i * (i - 1) / 2 + (j - i);
                        double re = 0.0, im = 0.0;
                        for (int sp = 0; sp < pc.nslots; ++sp) {
                            const float2 v = __ldcg(d.partial + ((int64_t)sp * C + itm.k) * P + p);
                            re += (double)v.x;
                            im += (double)v.y;
                        }
                        if (single) {
                            double2* dst = d.acc + (int64_t)itm.k * P + p;
                            double2 v = *dst;
                            v.x += re;
                            v.y += im;
                            *dst = v;
                        } else {
                            // a group's pass result lives in slot 0 until the
                            // reduction launch adds it to the accumulator
                            d.partial[(int64_t)itm.k * P + p] = make_float2((float)re, (float)im);
                        }
                    }
                    if (et == 0) d.ticket[itm.k * d.npairs + itm.pr] = 0;
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

constexpr size_t kSmemBudget = 227 * 1024;

}  // namespace

// How a launch deals its work to the CTAs (see next_piece).
struct DealPlan {
    std::vector<int> sp;      // round-robin deal: ranges per item of each mode
    bool balanced = false;    // contiguous deal of weighted k-tiles instead
    int grid = 0;             // CTAs of the balanced deal
    int64_t units = 0;        // its total work units
};

struct TcPlan {
    int N = 0, C = 0, P = 0, nblk = 1, npairs = 1;
    int mode = 0, planes = 1, KT = 32;
    int row_bytes = 64;       // tile row: 32 FP16 values, or 128 FP8
    int num_sms = 0;
    int box_rows = 128;       // TMA box rows: 2N rounded up to 8 for one block, else 128
    CUtensorMap tmap;
    bool have_map = false;
    int64_t cap = 0;
    int max_split = 1;
    int window = 0;           // 0 = per-mode default
    int stages = 0;           // 0 = as many as shared memory allows
    int split = 0;            // 0 = planner's choice
    int atoms = 0;            // k-tiles per stage, 0 = automatic
    unsigned long long timeout_ns = 4000000000ull;
    int withhold = 0;                    // test hook for the next launch
    unsigned long long hook_timeout_ns = 0;
    int* ticket = nullptr;               // [C][npairs] arrival counters
    // split decisions already made, keyed by the S_pad of every mode in the launch
    std::vector<std::pair<std::vector<int64_t>, DealPlan>> split_cache;
};

int tc_plan_create(TcPlan** out, int N, int C, int spec_type, std::string& err) {
    *out = nullptr;
    if (!get_encoder()) {
        err = "cuTensorMapEncodeTiled is not available from the driver";
        return CORR_ECUDA;
    }
    TcPlan* p = new TcPlan();
    p->N = N;
    p->C = C;
    p->P = N * (N + 1) / 2;
    p->nblk = (N + 63) / 64;
    p->npairs = groups_of(p->nblk);
    p->mode = spec_type == SPEC_F16X2 ? 0 : (spec_type == SPEC_F16 ? 1 : 2);
    p->planes = p->mode == 0 ? 2 : 1;
    p->KT = p->mode == 2 ? 128 : 32;
    p->row_bytes = p->mode == 2 ? 128 : 64;
    p->box_rows = p->nblk == 1 ? (2 * N + 7) / 8 * 8 : kRows;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete p;
        err = "cudaDeviceGetAttribute failed";
        return CORR_ECUDA;
    }
    const size_t tb = (size_t)p->C * p->npairs * sizeof(int);
    if (dev_malloc((void**)&p->ticket, tb) != cudaSuccess || cudaMemset(p->ticket, 0, tb) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p->ticket);
        delete p;
        err = "device allocation failed";
        return CORR_ENOMEM;
    }
    *out = p;
    return CORR_OK;
}

int tc_reset(TcPlan* p) {
    // after an aborted launch some arrival counters may be left non-zero
    return cudaMemset(p->ticket, 0, (size_t)p->C * p->npairs * sizeof(int)) == cudaSuccess
               ? CORR_OK
               : CORR_ECUDA;
}

int tc_plan_update(TcPlan* p, void* spec, int64_t cap, int N, int C, int spec_type,
                   std::string& err) {
    (void)N;
    (void)C;
    const int eb = spec_elem_bytes(spec_type);
    const int R2 = 2 * p->N;
    // tile-major workspace: [plane][cap/T tiles][C][2N rows][T frames], T = KT
    const int T = p->row_bytes / eb;
    cuuint64_t dims[4] = {(cuuint64_t)T, (cuuint64_t)R2, (cuuint64_t)p->C,
                          (cuuint64_t)p->planes * (cap / T)};
    cuuint64_t strides[3] = {(cuuint64_t)T * eb, (cuuint64_t)R2 * T * eb,
                             (cuuint64_t)p->C * R2 * T * eb};
    cuuint32_t box[4] = {(cuuint32_t)T, (cuuint32_t)p->box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = get_encoder()(&p->tmap, dt, 4, spec, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE,
                               p->row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        err = buf;
        return CORR_ECUDA;
    }
    p->have_map = true;
    p->cap = cap;
    p->max_split = (int)std::min<int64_t>(8, (cap + 255) / 256);
    p->split_cache.clear();
    return CORR_OK;
}

int tc_set_tiles(TcPlan* p, int window, int stages, int split, int atoms, std::string& err) {
    if (atoms < 0 || atoms > 8) {
        err = "atoms must be in [0, 8]";
        return CORR_EINVAL;
    }
    if (split < 0 || split > 64) {
        err = "split must be in [0, 64]";
        return CORR_EINVAL;
    }
    if (window != 0 && (window < p->KT || window % p->KT || window > 4096)) {
        err = "window must be a multiple of the k-tile (32 spectra, 128 for FP8) up to 4096";
        return CORR_EINVAL;
    }
    if (stages != 0 && (stages < 2 || stages > 16)) {
        err = "stages must be in [2, 16]";
        return CORR_EINVAL;
    }
    p->window = window;
    p->stages = stages;
    p->split = split;
    p->atoms = atoms;
    p->split_cache.clear();
    return CORR_OK;
}

namespace {

// Work units per k-tile of work group pr (pair_units()).
int host_pair_units(int pr, int nblk) { return pair_units(pr, nblk); }

struct LaunchShape {
    int wide, gs_floats, stages, W, atoms, slot_rows;
    size_t smem;
};

LaunchShape launch_shape(TcPlan* const* plans, int n) {
    LaunchShape L{};
    int r2max = 0;     // the G buffer serves the single-block modes only
    for (int m = 0; m < n; ++m) {
        L.wide |= plans[m]->nblk > 1;
        if (plans[m]->nblk == 1) r2max = std::max(r2max, 2 * plans[m]->N);
    }
    L.gs_floats = r2max * (r2max + 1);
    L.slot_rows = 8;
    int min_box = kRows;      // the MMA reads 128 rows from a tile: reserve the excess past the ring
    for (int m = 0; m < n; ++m) {
        L.slot_rows = std::max(L.slot_rows, plans[m]->box_rows);
        min_box = std::min(min_box, plans[m]->box_rows);
    }
    const size_t slot = (size_t)L.slot_rows * plans[0]->row_bytes;
    // + the rows an MMA reads past the ring's last slot
    const size_t vstage = L.wide ? (size_t)8 * 16 * kVRow * sizeof(float2) : 0;
    const size_t fixed = 1024 + (size_t)L.gs_floats * 4 + vstage + 16 + 16 + 8 * (2 * 16 + 5) + 256 +
                         (size_t)(kRows - min_box) * plans[0]->row_bytes;
    auto fit = [&](int atoms) {
        const size_t sb = (size_t)plans[0]->planes * atoms * slot * (L.wide ? 3 : 1);
        return std::min<int>(16, (int)((kSmemBudget - fixed) / sb));
    };
    // k-tiles per stage, unless set: as many (up to 256 spectra: 8 k-tiles of
    // 32, or 4 of the FP8 mode's 128) as still leave 3 stages; with two tiles
    // per k-tile (several antenna blocks) 2 stages suffice -- each stage
    // handshake costs a fixed latency, measured at N = 256: 2 stages of 128
    // spectra 1.10 ms against 4 of 64 1.24 ms per pass
    L.atoms = plans[0]->atoms;
    if (!L.atoms) {
        L.atoms = 1;
        const int min_stages = L.wide ? 2 : 3;
        for (int at = plans[0]->KT == 32 ? 8 : 4; at > 1; at /= 2)
            if (fit(at) >= min_stages) {
                L.atoms = at;
                break;
            }
    }
    while (L.atoms > 1 && fit(L.atoms) < 2) L.atoms /= 2;
    const size_t stage_bytes =
        (size_t)plans[0]->planes * L.atoms * slot * (L.wide ? 3 : 1);
    const int smax = fit(L.atoms);
    // default depth: as many stages as fit, up to 8; FP32 mode with one
    // antenna block, which streams its workspace from HBM at the copy rate,
    // takes 3 (at N = 44 a 1 s integration's pass: 0.92 ms against 0.95 with
    // the 4 that fit, 1.03 with 2)
    const int sdef = plans[0]->mode == 0 && !L.wide ? 3 : 8;
    L.stages = plans[0]->stages ? std::min(plans[0]->stages, smax) : std::min(smax, sdef);
    const int step = plans[0]->KT * L.atoms;
    // default window: 256 spectra in FP32 mode (TMEM accumulation bias ~1e-6
    // at full size); 512 for FP16 (its input rounding dominates), 1024 when
    // a mode has several antenna blocks (~10% less time per pass at N = 256;
    // at N = 44 it raised the 1 s FP16 error from 5.7e-6 to 8.1e-6 for no
    // gain); 2048 for FP8 (16 k-tiles of 128 spectra, the MMA steps of a
    // 1024-spectrum FP16 window: 30% less time per pass than 1024 at
    // N = 256, 13% at N = 44, against an input rounding error near 1e-2)
    const int W0 = plans[0]->mode == 0 ? 256 : plans[0]->mode == 2 ? 2048 : (L.wide ? 1024 : 512);
    int W = plans[0]->window ? plans[0]->window : std::max(W0, plans[0]->KT);
    L.W = (W + step - 1) / step * step;   // windows hold whole stages
    L.smem = fixed + (size_t)L.stages * stage_bytes;
    return L;
}

// Work deal of one launch.  Round-robin: every mode's pass of S_pad frames
// is cut into n_split ranges of whole k-tiles per item and items go to CTAs
// in turn; the range count minimises the busiest CTA's work in a simulation
// of that deal.  Balanced (single-mode launches): contiguous shares of the
// weighted k-tiles (see next_piece).  The cheaper of the two in the same
// cost model is taken (per item or piece: its k-tiles x 1 on a diagonal
// block pair, x 1.5 off it, plus ~4 k-tiles for its end, measured on GB300,
// and 2 more when its partial is combined with others).  At N = 44, K = 512
// and 8192 frames per pass the round-robin deal leaves 104 CTAs with two
// channels and 48 with one; the balanced deal gives each 1.7 channels.
DealPlan choose_deal(TcPlan* const* plans, int n, const int64_t* S_pad) {
    std::vector<int64_t> key(S_pad, S_pad + n);
    DealPlan out;
    if (plans[0]->split > 0) {
        // fixed by corr_set_tiles: round-robin, ranges per channel, at most one per k-tile
        out.sp.resize(n);
        for (int m = 0; m < n; ++m) {
            const int64_t tiles = std::max<int64_t>(1, S_pad[m] / plans[m]->KT);
            out.sp[m] = (int)std::min<int64_t>(std::min(plans[0]->split, plans[m]->max_split), tiles);
        }
        return out;
    }
    auto& cache = plans[0]->split_cache;
    for (auto& e : cache)
        if (e.first == key) return e.second;
    const int sms = plans[0]->num_sms;
    int64_t max_tiles = 1;
    for (int m = 0; m < n; ++m) max_tiles = std::max<int64_t>(max_tiles, S_pad[m] / plans[m]->KT);
    std::vector<int> best(n, 1);
    double best_score = 1e300;
    std::vector<double> load(sms);
    for (int64_t T = 1; T <= max_tiles * 2; T *= 2) {
        std::vector<int> sp(n);
        for (int m = 0; m < n; ++m) {
            const int64_t tiles = std::max<int64_t>(1, S_pad[m] / plans[m]->KT);
            int64_t ns = (tiles + T - 1) / T;
            ns = std::min<int64_t>(ns, plans[m]->max_split);
            const int64_t per = (tiles + ns - 1) / ns;
            sp[m] = (int)((tiles + per - 1) / per);
        }
        std::fill(load.begin(), load.end(), 0.0);
        int64_t g = 0;
        for (int m = 0; m < n; ++m) {
            const TcPlan* p = plans[m];
            const int64_t tiles = std::max<int64_t>(1, S_pad[m] / p->KT);
            const int64_t per = (tiles + sp[m] - 1) / sp[m];
            for (int s = 0; s < sp[m]; ++s) {
                const int64_t t = std::min<int64_t>(per, tiles - (int64_t)s * per);
                for (int k = 0; k < p->C; ++k)
                    for (int pr = 0; pr < p->npairs; ++pr, ++g)
                        load[g % sms] += (double)t * 0.5 * host_pair_units(pr, p->nblk) + 4.0 +
                                         (sp[m] > 1 ? 2.0 : 0.0);
            }
        }
        const double score = *std::max_element(load.begin(), load.end());
        if (score < best_score - 1e-9) {
            best_score = score;
            best = sp;
        }
    }
    out.sp = best;
    // balanced deal: every CTA gets U/G units; an item then spans at most
    // (tiles - 1) w G / U + 2 CTAs, which must fit the partial slots, and a
    // CTA holds at least 3 units (the heaviest k-tile), so it owns a k-tile of
    // every item it overlaps and an item's CTAs are consecutive
    int64_t units = 0, max_span = 0;
    int cap_slots = 1 << 30;
    for (int m = 0; m < n; ++m) {
        const TcPlan* p = plans[m];
        const int64_t tiles = S_pad[m] / p->KT;
        for (int pr = 0; pr < p->npairs; ++pr) {
            const int w = host_pair_units(pr, p->nblk);
            units += item_units(tiles, w) * p->C;
            if (tiles > 0) max_span = std::max<int64_t>(max_span, (tiles - 1) * w);
        }
        cap_slots = std::min(cap_slots, p->max_split);
    }
    // (one mode only: with several, the round-robin deal spreads every mode's
    // items, whose ends differ in cost, evenly over the CTAs -- measured
    // faster on the four-mode batch)
    // (single antenna block only: with several, the round-robin deal hands one
    // channel's block pairs to neighbouring CTAs at once, which then share its
    // tiles through L2; contiguous shares would read them from HBM per pair)
    if (n == 1 && plans[0]->nblk == 1 && units > 0 && cap_slots >= 3) {
        int64_t G = sms;
        if (max_span > 0)
            G = std::min<int64_t>(G, std::max<int64_t>(1, (int64_t)(cap_slots - 2) * units / max_span));
        G = std::min<int64_t>(G, std::max<int64_t>(1, units / 3));
        std::vector<double> bl(G, 0.0);
        int64_t ibase = 0;
        for (int m = 0; m < n; ++m) {
            const TcPlan* p = plans[m];
            const int64_t tiles = S_pad[m] / p->KT;
            if (tiles == 0) continue;
            for (int pr = 0; pr < p->npairs; ++pr) {
                const int w = host_pair_units(pr, p->nblk);
                for (int k = 0; k < p->C; ++k, ibase += item_units(tiles, w)) {
                    const int64_t t0 = ibase + kEndUnits;
                    const int64_t first = t0 * G / units;
                    const int64_t last = (t0 + (tiles - 1) * w) * G / units;
                    for (int64_t j = 0; j < tiles; ++j) bl[(t0 + j * w) * G / units] += 0.5 * w;
                    for (int64_t c = first; c <= last; ++c) bl[c] += 4.0 + (last > first ? 2.0 : 0.0);
                }
            }
        }
        const double score = *std::max_element(bl.begin(), bl.end());
        if (score < best_score - 1e-9) {
            out.balanced = true;
            out.grid = (int)G;
            out.units = units;
        }
    }
    cache.emplace_back(key, out);
    if (cache.size() > 16) cache.erase(cache.begin());
    return out;
}

}  // namespace

int tc_launch(TcPlan* const* plans, int n, TcRun* runs, cudaStream_t st, std::string& err) {
    if (n < 1 || n > kMaxTcModes) {
        err = "between 1 and 4 modes per tensor-core launch";
        return CORR_EINVAL;
    }
    for (int m = 0; m < n; ++m) {
        if (!plans[m]->have_map) {
            err = "tensor-core plan has no workspace";
            return CORR_ESTATE;
        }
        if (plans[m]->mode != plans[0]->mode) {
            err = "modes of one tensor-core launch must share the X-engine precision";
            return CORR_EINVAL;
        }
    }
    std::vector<int64_t> S(n);
    for (int m = 0; m < n; ++m) S[m] = runs[m].S_pad;
    const DealPlan deal = choose_deal(plans, n, S.data());
    const std::vector<int>& sp = deal.sp;
    const LaunchShape L = launch_shape(plans, n);
    TcArgs a;
    memset(&a, 0, sizeof a);
    a.n_modes = n;
    a.stages = L.stages;
    a.KT = plans[0]->KT;
    a.kt_shift = a.KT == 128 ? 7 : 5;
    a.row_bytes = plans[0]->row_bytes;
    a.W = L.W;
    a.atoms = L.atoms;
    a.wide = L.wide;
    a.gs_floats = L.gs_floats;
    a.slot_rows = L.slot_rows;
    a.status = runs[0].status;
    a.timeout_ns = plans[0]->timeout_ns;
    if (plans[0]->withhold) {
        a.withhold = 1;
        a.timeout_ns = plans[0]->hook_timeout_ns;
        plans[0]->withhold = 0;
    }
    int base = 0;
    int64_t units = 0;
    for (int m = 0; m < n; ++m) {
        const TcPlan* p = plans[m];
        a.tmap[m] = p->tmap;
        TcModeArgs& d = a.md[m];
        d.N = p->N;
        d.C = p->C;
        d.P = p->P;
        d.nblk = p->nblk;
        d.npairs = p->npairs;
        d.S_pad = runs[m].S_pad;
        const int64_t tiles = std::max<int64_t>(1, d.S_pad / p->KT);
        const int64_t per = (tiles + sp[m] - 1) / sp[m];
        d.S_item = per * p->KT;
        d.n_split = d.S_pad > 0 ? (int)((d.S_pad + d.S_item - 1) / d.S_item) : 0;
        d.item_base = base;
        d.n_items = d.n_split * p->npairs * p->C;
        base += d.n_items;
        d.partial = runs[m].partial;
        d.acc = runs[m].acc;
        d.ticket = plans[m]->ticket;
        d.scale = runs[m].scale;
        d.split = runs[m].split;
        d.tiles = d.S_pad / p->KT;
        d.cap_tiles = (int)(p->cap / p->KT);
        d.box_bytes = (uint32_t)p->box_rows * p->row_bytes;
        d.unit_base = units;
        for (int pr = 0; pr < p->npairs; ++pr)
            units += item_units(d.tiles, host_pair_units(pr, p->nblk)) * p->C;
        // single block: splits are combined inside the kernel, into acc;
        // several blocks: every pass result lands in partial slot 0 (coalesced
        // FP32 stores), which one reduction launch adds to acc
        runs[m].direct = p->nblk == 1;
        runs[m].n_split = runs[m].direct ? d.n_split : 1;
    }
    a.total_items = base;
    if (base == 0) return CORR_OK;
    int grid = std::min(base, plans[0]->num_sms);
    if (deal.balanced) {
        a.balanced = 1;
        a.units = units;
        grid = deal.grid;
    }
    cudaError_t e;
    auto go = [&](auto kern) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L.smem);
        if (r == cudaSuccess) kern<<<grid, kTcThreads, L.smem, st>>>(a);
        return r;
    };
    if (plans[0]->mode == 0)
        e = L.wide ? go(xengine_tc_kernel<0, true>) : go(xengine_tc_kernel<0, false>);
    else if (plans[0]->mode == 1)
        e = L.wide ? go(xengine_tc_kernel<1, true>) : go(xengine_tc_kernel<1, false>);
    else
        e = L.wide ? go(xengine_tc_kernel<2, true>) : go(xengine_tc_kernel<2, false>);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("tensor-core X-engine launch: ") + cudaGetErrorString(e);
        return CORR_ECUDA;
    }
    return CORR_OK;
}

int tc_test_withhold(TcPlan* p, double wait_limit_s, std::string& err) {
    if (!(wait_limit_s >= 0.001 && wait_limit_s <= 10.0)) {
        err = "wait limit must be in [0.001, 10] s";
        return CORR_EINVAL;
    }
    p->withhold = 1;
    p->hook_timeout_ns = (unsigned long long)(wait_limit_s * 1e9);
    return CORR_OK;
}

void tc_plan_destroy(TcPlan* p) {
    if (!p) return;
    cudaFree(p->ticket);
    delete p;
}

}  // namespace gbcorr
