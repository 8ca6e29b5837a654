// replay_tp.cu - time-parallel batched replay of the MAGUS control step (jump mode).
//
// The per-round recurrence (Sec. 3.1 Alg. 1, Sec. 3.2 Alg. 2, Sec. 6.1) splits into
//   * stencils over the trace: the prediction of round t needs delta_t and delta_{t-W};
//     the high-frequency state of round t needs the flags of rounds t-L+1 .. t;
//   * a two-valued latch: after round t the level is the top of the ladder if the round
//     is high-frequency or predicts +1, the bottom if it predicts -1 (and is not
//     high-frequency), and unchanged otherwise; "last event wins" is associative.
// So a trace is cut into 32-round rows: lane j of a warp owns rows of 32 consecutive
// rounds, builds bit masks of its rounds' predictions, and resolves the latch of its row
// with one 33-bit addition (carries run from a set-to-top bit until the next
// set-to-bottom bit).  Rows are chained by a ballot scan inside the warp, warps of a
// chunk by a short exchange through shared memory, chunks by a carried level.
//
// Data path: the CTA streams one trace through a two-stage shared-memory ring with 2-D TMA
// tensor copies (cp.async.bulk.tensor + mbarrier complete_tx) of time_groups x 32 rows of
// 32 deltas, 128-byte swizzled so that every lane reads its own row with conflict-free
// 128-bit loads; each stage keeps the 2 rows (64 deltas) that precede it so the window
// W <= 64 never reaches outside shared memory.  One staged chunk feeds every policy the
// CTA holds (policy_slots groups of time_groups warps).  With one policy slot (and in the
// 4-slot tile of single warps) the 8 rows before a chunk arrive with its copy and the last
// warp done with a stage refills it with the chunk two ahead; otherwise a CTA barrier per
// chunk orders the copies.  A trace's last chunk is copied only up to the trace's end.  One-member
// groups stage their change-log entries per warp and write them 32 at a time.
//
// Policies that share Alg. 1's parameters (W, inc, dec) make identical predictions and
// flags; they differ only in Alg. 2 (L, threshold).  A slot therefore holds a policy group
// of up to GP such policies: the row predictions are made once and Alg. 2, the latch, the
// energy charge and the log run per member.
//
// Energy: per level the kernel counts unstretched intervals and sums the deltas of
// stretched ones (integers, exact); the FP64 totals are formed once per pair.
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"
#include "replay_core.cuh"
#include "tma.cuh"

namespace magus {
namespace {

using tma::mbar_init;
using tma::fence_mbar_init;
using tma::mbar_expect_tx;
using tma::mbar_wait_bounded;
using tma::tma_rows;

constexpr int HALO = 64;            // deltas kept before each stage (>= max W)
constexpr int SB = 1024;            // rounds per warp sub-block: 32 rows x 32
using core::FULL;

using core::smem_u32;

__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
struct MemberCarry {
    uint64_t count;     // change-log entries emitted so far for the pair
    uint32_t level;     // level (0 bottom / 1 top) governing the chunk's first round
    uint32_t pad;
};

template <int TG, int CW, int GP>
struct Shared {
    uint64_t bar[2];                  // stage s holds its chunk (copy complete)
    uint32_t rel[2];                  // one slot: warps done with stage s's chunk
    int issued[2];                    // one slot: sequence number of the last copy into stage s, -1 none
    uint64_t xf[CW][TG];              // flags of the last 64 rounds of each sub-block
    uint64_t hist[CW][2];             // flags of the 64 rounds before the chunk (by parity)
    uint32_t xs[CW][GP][TG];          // sub-block summary: has | exit<<1 | first<<2 | nch<<3
    MemberCarry carry[CW][GP][2];     // per member, double-buffered by chunk parity
    // grouped tiles: each member's count4_ge constants for its kmin (A0..A3, and all-ones
    // when kmin <= 0), formed once per item
    uint32_t kmask[GP > 1 ? CW : 1][GP > 1 ? GP : 1][7];
    unsigned long long red_s0[TG * CW][GP], red_sm[TG * CW][GP], red_hash[TG * CW][GP];
    uint32_t red_n0[TG * CW][GP], red_nm[TG * CW][GP], red_hf[TG * CW][GP];
    // per warp, one-member groups only: change-log entries waiting for a full warp's worth
    core::Staged stage[GP == 1 ? TG * CW : 1][GP == 1 ? core::kStageCap : 1];
    int item;
    int abort;
};

// Stage: a 1024-byte block whose last two rows hold the preceding 64 deltas (one slot: the
// block holds the 8 rows before the chunk, copied with it), then the chunk's TG * 32 rows;
// both 1024-byte aligned (the 128-byte swizzle repeats every 8 rows).
template <int TG>
__host__ __device__ constexpr size_t stage_bytes() {
    return 1024 + (size_t)TG * SB * sizeof(uint32_t);
}
template <int TG, int CW, int GP>
__host__ __device__ constexpr size_t stage_offset() {
    return (sizeof(Shared<TG, CW, GP>) + 1023) / 1024 * 1024;
}
// Shared memory of one CTA from a 1024-byte aligned base (the stages need that alignment for
// the 128-byte swizzle).
template <int TG, int CW, int GP>
__host__ __device__ constexpr size_t smem_bytes() {
    return stage_offset<TG, CW, GP>() + 2 * stage_bytes<TG>();
}

// Register budgets per tile: 80 for the one-slot tiles of one-member groups (three CTAs of 256
// threads or six of 128 per SM: the 4-warp tile's shared memory is sized to fit six, which
// measured 4.5 % faster than five at 88 registers), 96 for the other one-member tiles and for
// the 4-slot grouped tile of 4 warps (five CTAs of 128 threads: 3 % faster on the policy sweep
// than four at 128, despite 8 bytes of spill), 128 for the other grouped tiles.  The kernel's
// allocation is sensitive: left alone the compiler has taken from 74 to 224 registers for
// these shapes as the source changed.
// WK > 0: an instance for policy groups whose window length W is WK (the predictor inline for
// that W alone: with all the common W behind a switch per row, instruction fetch cost the
// batched replay 2.4 %); WK = 0: any W.
template <int TG, int CW, int GP, int WK = 0>
__global__ void __launch_bounds__(TG * CW * 32)
    __maxnreg__(GP == 1 ? (CW == 1 ? 80 : 96) : (TG == 1 && CW == 4 ? 96 : 128)) replay_tp_kernel(const TpParams p,
                                                                   const __grid_constant__ CUtensorMap tmap,
                                                                   const __grid_constant__ CUtensorMap tmap_tail) {
    constexpr int CH = TG * SB;              // rounds per chunk
    constexpr int CH_ROWS = TG * 32;         // 32-delta rows per chunk
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // The launch adds no alignment slack where the dynamic window starts on a 1024-byte
    // boundary (tp_smem_slack); a window that does not, or is too small, is reported, never used.
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    {
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if (pad + (uint32_t)smem_bytes<TG, CW, GP>() > dyn) {
            if (threadIdx.x == 0) atomicCAS(p.status, 0, MAGUS_ECUDA);
            return;
        }
    }
    unsigned char *smem_al = smem_raw + pad;
    Shared<TG, CW, GP> &sh = *reinterpret_cast<Shared<TG, CW, GP> *>(smem_al);
    // data row 0 of stage s (shared-window byte address)
    const uint32_t stage0 = smem_u32(smem_al + stage_offset<TG, CW, GP>()) + 1024;
    auto stage_base = [&](int s_) { return stage0 + (uint32_t)s_ * (uint32_t)stage_bytes<TG>(); };

    // every warp waits for its own stage and the last reader refills it: the one-slot tiles
    // and 1 x 4 x 4 (policy sweep 1.9 % faster than with two CTA barriers per chunk; the
    // other grouped tiles measured slower this way)
    constexpr bool kPipe = CW == 1 || (TG == 1 && CW == 4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cw = warp / TG, g = warp % TG;
    const DevModel &M = p.model;
    const uint32_t topK = (uint32_t)(M.K - 1);
    const uint32_t lanemask_lt = (1u << lane) - 1u;

    if (tid == 0) {
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        fence_mbar_init();
        sh.abort = 0;
        sh.rel[0] = sh.rel[1] = 0;
        sh.issued[0] = sh.issued[1] = -1;
    }
    __syncthreads();

    // per-chunk wait limit (the tiles whose warps wait for their stages themselves; the
    // others keep the default, which also keeps their register allocation where it was
    // measured)
    const unsigned long long wlim = (kPipe && p.chunk_wait_ns) ? p.chunk_wait_ns : tma::kWaitNs;
    uint32_t seq = 0;         // chunks loaded by this CTA so far (selects stage and parity)
    int pend[2] = {-1, -1};   // thread 0: parity of an outstanding bulk copy per stage

    while (true) {
        if (tid == 0) sh.item = (int)atomicAdd(p.queue, 1u);
        __syncthreads();
        const int item = sh.item;
        if (item >= p.n_items || sh.abort) break;
        const WorkItem wi = p.items[item];
        const int grp = (int)wi.cfg0 + cw;
        const bool active = grp < p.n_groups;
        const PolicyGroup G = p.groups[active ? grp : (int)wi.cfg0];
        const int cnt = G.count;
        const uint64_t n = p.lengths[wi.trace];
        const int64_t pbase = (int64_t)wi.trace * p.n_pols;
        const int64_t pair0 = pbase + p.groups[wi.cfg0].member[0];   // the block's first pair

        const DevPolicy P = p.pols[G.member[0]];     // Alg. 1 parameters of the group
        int Lm[GP], Km[GP];
#pragma unroll
        for (int m = 0; m < GP; m++) {
            const int id = G.member[m < cnt ? m : 0];
            // bit 8 marks a static baseline (no control), bit 9 one pinned at the top; L
            // itself is at most 64
            Lm[m] = p.pols[id].L | (p.pols[id].pin ? 0x100 : 0) | (p.pols[id].pin > 1 ? 0x200 : 0);
            Km[m] = p.pols[id].kmin;
        }
        uint64_t n_seen0 = 0;
        if (p.state) n_seen0 = p.state[pbase + G.member[0]].n_seen;

        // Carried state per member: level and log count; per group: the flag history.
        if (g == 0 && lane == 0) {
            sh.hist[cw][0] = (p.state && active) ? p.state[pbase + G.member[0]].flags : 0ull;
#pragma unroll
            for (int m = 0; m < GP; m++) {
                uint32_t lv = 0;
                if (Lm[m] & 0x100) {
                    lv = (Lm[m] & 0x200) ? topK : 0u;   // a static baseline ignores the carried level
                } else if (p.state && active && m < cnt) {
                    lv = p.state[pbase + G.member[m]].level;
                    if (lv != 0 && lv != topK) {
                        atomicCAS(p.status, 0, MAGUS_EINVAL);
                        lv = 0;
                    }
                }
                MemberCarry c0;
                c0.count = 0;
                c0.level = lv ? 1u : 0u;
                c0.pad = 0;
                sh.carry[cw][m][0] = c0;
                if constexpr (GP > 1) {
                    const int km = Km[m];
                    const uint32_t a = (km > 0 && km <= 10) ? 16u - (uint32_t)km : 0u;
                    sh.kmask[cw][m][0] = 0u - (a & 1u);
                    sh.kmask[cw][m][1] = 0u - ((a >> 1) & 1u);
                    sh.kmask[cw][m][2] = 0u - ((a >> 2) & 1u);
                    sh.kmask[cw][m][3] = 0u - ((a >> 3) & 1u);
                    sh.kmask[cw][m][4] = km <= 0 ? FULL : 0u;
                    sh.kmask[cw][m][5] = (Lm[m] & 0x100) ? 0u : FULL;   // controlled (not a pin)
                    sh.kmask[cw][m][6] = (uint32_t)G.member[m];         // its policy index
                }
            }
        }
        // Deltas before the first chunk (the first pair's carried history), rows -2, -1.
        if (warp == 0) {
            const uint32_t b0 = stage_base(seq & 1);
            for (int k = lane; k < HALO; k += 32)
                core::sts32(core::swz_elem(b0, k - HALO), p.state ? p.state[pair0].hist[k] : 0u);
        }
        __syncthreads();

        const uint32_t nchunks = (uint32_t)((n + CH - 1) / CH);
        const int row0 = (int)(p.offsets[wi.trace] / 32);   // first tensor row of the trace
        const uint32_t rows = (uint32_t)((n + 31) / 32);    // rows holding the trace
        auto issue = [&](uint32_t c, uint32_t sq) {
            const uint32_t left_rows = rows - c * (uint32_t)CH_ROWS;
            // one slot: the 8 rows before a later chunk (its 64-delta halo in rows -2, -1)
            // come with the copy, so a stage can be refilled before the chunk ahead of it
            // has been read (same swizzle phase: CH_ROWS is a multiple of 8)
            const uint32_t halo = (kPipe && c > 0) ? (uint32_t)kTailRows * 128u : 0u;
            if (GP > 1 || left_rows >= (uint32_t)CH_ROWS) {
                mbar_expect_tx(&sh.bar[sq & 1], (uint32_t)CH_ROWS * 128u + halo);
                tma_rows(stage_base(sq & 1), &tmap, row0 + (int)c * CH_ROWS, &sh.bar[sq & 1]);
            } else {
                // the trace's last, partial chunk: boxes of kTailRows rows up to its end only
                // (rows past it in the stage keep stale deltas; they lie past the trace's
                // end, where every mask is zero).  One-member tiles only: the grouped tiles
                // are bound by arithmetic, not by the bytes they read, and the extra branch
                // doubles their register demand.
                const uint32_t nb = (left_rows + kTailRows - 1) / kTailRows;
                mbar_expect_tx(&sh.bar[sq & 1], nb * (uint32_t)kTailRows * 128u + halo);
                for (uint32_t b = 0; b < nb; b++)
                    tma_rows(stage_base(sq & 1) + b * (uint32_t)kTailRows * 128u, &tmap_tail,
                             row0 + (int)c * CH_ROWS + (int)(b * kTailRows), &sh.bar[sq & 1]);
            }
            if (halo)   // after the expect-tx above, which counts its bytes
                tma_rows(stage_base(sq & 1) - halo, &tmap_tail, row0 + (int)c * CH_ROWS - kTailRows, &sh.bar[sq & 1]);
            if (kPipe) sh.issued[sq & 1] = (int)sq;
            else pend[sq & 1] = (int)((sq >> 1) & 1);
        };
        if (tid == 0 && nchunks > 0) issue(0, seq);
        // one slot: the second stage is free as well (every warp finished the last item)
        if (kPipe && tid == 0 && nchunks > 1) issue(1, seq + 1);

        core::Acc acc[GP];
#pragma unroll
        for (int m = 0; m < GP; m++) core::acc_zero(acc[m]);
        // one-member groups stage their change-log entries while interval indices fit 31
        // bits (grouped tiles write them directly: staging per member raised their register
        // demand past two CTAs per SM, which cost more than it saved)
        const bool can_stage = GP == 1 && n_seen0 + n < (1ull << 31);
        uint32_t pending = 0;   // entries waiting in this warp's table
        // one-member groups: the constants of count4_ge for this item's kmin, formed once
        uint32_t kA0 = 0, kA1 = 0, kA2 = 0, kA3 = 0, kAll = 0;
        if (GP == 1) {
            const int km = Km[0];
            if (km <= 0) {
                kAll = FULL;
            } else if (km <= 10) {
                const uint32_t a = 16u - (uint32_t)km;
                kA0 = 0u - (a & 1u);
                kA1 = 0u - ((a >> 1) & 1u);
                kA2 = 0u - ((a >> 2) & 1u);
                kA3 = 0u - ((a >> 3) & 1u);
            }
        }

        for (uint32_t c = 0; c < nchunks; c++) {
            const uint32_t sq = seq + c;
            const int s = (int)(sq & 1);
            const uint32_t sbase = stage_base(s);
            if constexpr (kPipe) {
                // No CTA barrier per chunk.  Every warp waits for its stage
                // itself; the last warp to finish a chunk refills its stage with the chunk
                // two ahead (see the end of the loop), so copies run up to two chunks ahead
                // and a warp that finishes a chunk early starts the next one.  A bounded wait
                // that gives up marks the CTA aborted; later waits are skipped and the chunk
                // loop runs to the end of the item, where the CTA stops.
                if (!*(volatile int *)&sh.abort) {
                    if (!mbar_wait_bounded(&sh.bar[s], (sq >> 1) & 1, wlim)) {
                        atomicCAS(p.status, 0, MAGUS_ETIMEDOUT);
                        sh.abort = 1;
                    }
                }
            } else {
                if (tid == 0) {
                    if (!mbar_wait_bounded(&sh.bar[s], (sq >> 1) & 1, wlim)) {
                        atomicCAS(p.status, 0, MAGUS_ETIMEDOUT);
                        sh.abort = 1;
                    } else {
                        pend[s] = -1;
                    }
                }
                __syncthreads();
                if (sh.abort) break;
                // every thread observes the completed phase (acquire of the bulk-copy data)
                if (tid != 0) (void)mbar_wait_bounded(&sh.bar[s], (sq >> 1) & 1, wlim);
                if (c > 0 && warp == 0) {
                    // the previous chunk's last two rows become rows -2, -1 (same swizzle
                    // phase: CH_ROWS is a multiple of 8)
                    const uint32_t prev = stage_base(s ^ 1) + (uint32_t)(CH_ROWS - 2) * 128u;
                    for (int k = lane; k < HALO; k += 32)
                        core::sts32(sbase - 256u + 4u * k, core::lds32(prev + 4u * k));
                }
                __syncthreads();   // the first warp of every policy slot reads the halo
                if (tid == 0 && c + 1 < nchunks) issue(c + 1, sq + 1);
            }
            if constexpr (kPipe && CW > 1) {
                if (!active) {
                    // an empty slot still releases the stage
                    __syncwarp();
                    if (lane == 0 && atomicAdd(&sh.rel[s], 1u) == (uint32_t)(TG * CW - 1)) {
                        sh.rel[s] = 0;
                        if (c + 2 < nchunks && !*(volatile int *)&sh.abort) {
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            issue(c + 2, sq + 2);
                        }
                    }
                    continue;
                }
            }
            if (!active) continue;

            // ---------------------------------------------------------------- phase A
            // Alg. 1 predictions and stretch bits of this lane's row (shared by the group)
            const uint32_t sub = sbase + (uint32_t)g * (SB * 4u);   // data row 0 of the sub-block
            // a chunk between the first and the last: every row full and past the first W rounds
            const bool interior = c > 0 && c + 1 < nchunks;
            const int64_t r0 = (int64_t)c * CH + g * SB + 32 * lane;  // row start (local)
            const int64_t left = interior ? (int64_t)CH : (int64_t)n - r0;
            const uint32_t vmask = interior ? FULL : core::valid_mask(left);
            const uint32_t pmask = interior ? FULL : core::predict_mask(vmask, n_seen0 + (uint64_t)r0, P.W);
            const core::RowPred rp = core::row_predict<(WK > 0 ? WK : -1), GP == 1, GP == 1>(sub, lane, P, M, vmask, pmask);
            const uint32_t UP = rp.UP, DN = rp.DN;
            const uint32_t FL = UP | DN;   // uncore_tune_ls entries of the row
            {
                // (one-member tiles: lanes 30 and 31 store their own words, 0.8 % faster on the
                // batched replay; the grouped tiles measured 0.4 .. 0.8 % slower that way)
                if constexpr (GP == 1) {
                    if (lane >= 30) core::sts32(smem_u32(&sh.xf[cw][g]) + 4u * (uint32_t)(lane - 30), FL);
                } else {
                    const uint32_t f30 = __shfl_sync(FULL, FL, 30), f31 = __shfl_sync(FULL, FL, 31);
                    if (lane == 0) sh.xf[cw][g] = (uint64_t)f30 | ((uint64_t)f31 << 32);
                }
            }
            if (TG > 1) group_sync(1 + cw, TG * 32); else __syncwarp();
            const uint64_t tailH = (g == 0) ? sh.hist[cw][c & 1] : sh.xf[cw][g > 0 ? g - 1 : 0];
            const uint64_t H = core::row_history(FL, tailH, lane);

            // Algorithm 2's sliding counts once for a group whose members share L
            uint32_t hw[GP > 1 ? 8 : 1];
            const bool shared_counts = GP > 1 && cnt > 1 && G.same_L;
            // a shared 10-round window: the bit-sliced counts (four words) take hw[0..3]
            const bool sliced10 = shared_counts && (Lm[0] & 0xff) == 10;
            if constexpr (GP > 1) {
                if (sliced10) {
                    const core::Count4 c10 = core::window10_counts(H, FL);
                    hw[0] = c10.c0;
                    hw[1] = c10.c1;
                    hw[2] = c10.c2;
                    hw[3] = c10.c3;
                } else if (shared_counts) {
                    core::hf_counts(H, FL, Lm[0] & 0xff, hw);
                }
            }
            // members one after another (not unrolled: unrolling four members doubles the
            // registers and halves the resident CTAs, measured slower)
#pragma unroll 1
            for (int m = 0; m < (GP == 1 ? 1 : cnt); m++) {
                // ------------------------------------------------------------ phase B
                const uint32_t act = GP > 1 ? sh.kmask[GP > 1 ? cw : 0][GP > 1 ? m : 0][5] : ((Lm[m] & 0x100) ? 0u : FULL);
                uint32_t HFr;
                if constexpr (GP > 1) {
                    if (sliced10) {
                        const uint32_t *km = sh.kmask[GP > 1 ? cw : 0][GP > 1 ? m : 0];
                        uint32_t cy = hw[0] & km[0];
                        cy = core::maj3(hw[1], cy, km[1]);
                        cy = core::maj3(hw[2], cy, km[2]);
                        HFr = core::maj3(hw[3], cy, km[3]) | km[4];
                    } else {
                        HFr = shared_counts ? core::hf_from_counts(hw, Km[m]) : core::hf_row(H, FL, Lm[m] & 0xff, Km[m]);
                    }
                } else {
                    // the 10-round tune window bit-sliced (measured 1.5 % faster on the batched
                    // replay than the byte-parallel counts, which serve every other length)
                    if ((Lm[m] & 0xff) == 10) {
                        const core::Count4 c4 = core::window10_counts(H, FL);
                        uint32_t cy = c4.c0 & kA0;
                        cy = core::maj3(c4.c1, cy, kA1);
                        cy = core::maj3(c4.c2, cy, kA2);
                        HFr = core::maj3(c4.c3, cy, kA3) | kAll;
                    } else {
                        HFr = core::hf_row(H, FL, Lm[m] & 0xff, Km[m]);
                    }
                }
                const uint32_t HF = HFr & vmask & act;
                const uint32_t SETM = (HF | UP) & act;
                const uint32_t SET0 = DN & ~HF & act;
                const uint32_t EV = SETM | SET0;
                const bool has = EV != 0;
                // SETM and SET0 are disjoint: the row's last event sets the top exactly when
                // SETM's highest bit lies above SET0's (SETM > SET0), its first event exactly
                // when SETM holds the lowest bit of EV; the same holds for lane masks
                const uint32_t exitv = SETM > SET0 ? 1u : 0u;
                const uint32_t firstv = (SETM & (0u - EV)) != 0u ? 1u : 0u;
                const uint32_t bev = __ballot_sync(FULL, has), bex = __ballot_sync(FULL, exitv);
                const uint32_t prior = bev & lanemask_lt;
                const uint32_t pex = bex & lanemask_lt;   // earlier event rows that exit at the top
                const uint32_t cin_prior = pex > (prior ^ pex) ? 1u : 0u;
                {
                    // changes that do not depend on the level entering the sub-block: rows
                    // after the first event row are fixed; the first event row is counted as
                    // if it entered at its own first event's level (no change at that event)
                    uint32_t det = 0;
                    if (GP == 1 || prior || has) {
                        // (branch-free in one-member tiles, -0.2 %: a row with no event so far
                        // latches its entering level, so it counts no change either way)
                        const uint32_t ca = prior ? cin_prior : firstv;
                        const uint32_t lm = core::latch_row(SETM, SET0, ca);
                        det = __popc((lm ^ ((lm << 1) | ca)) & vmask);
                    }
                    const uint32_t wdet = __reduce_add_sync(FULL, det);
                    const uint32_t bfi = __ballot_sync(FULL, firstv);
                    if (lane == 0) {
                        const uint32_t whas = bev != 0;
                        const uint32_t wfirst = (bfi & (0u - bev)) != 0u ? 1u : 0u;
                        const uint32_t wexit = bex > (bev ^ bex) ? 1u : 0u;
                        sh.xs[cw][m][g] = whas | (wexit << 1) | (wfirst << 2) | (wdet << 3);
                    }
                }
                if (TG > 1) group_sync(1 + cw, TG * 32); else __syncwarp();

                // ------------------------------------------------------------ phase C
                const MemberCarry cr = sh.carry[cw][m][c & 1];
                // level entering this sub-block and the chunk's changes before it
                uint32_t wcin = cr.level;
                uint64_t before = 0;
                if constexpr (TG >= 4) {
                    // lane i holds sub-block i's summary: the last earlier sub-block with an
                    // event sets the level (a ballot); each earlier sub-block adds its own
                    // changes plus one if its first event flips the level it entered with.
                    // Branch-free, so the warps of a chunk reach the next barrier together.
                    const uint32_t sv_i = lane < TG ? sh.xs[cw][m][lane] : 0u;
                    const uint32_t hasb = __ballot_sync(FULL, sv_i & 1u), exb = __ballot_sync(FULL, (sv_i >> 1) & 1u);
                    const uint32_t prior_i = hasb & lanemask_lt;
                    const uint32_t pex_i = exb & lanemask_lt;
                    const uint32_t lin_i = prior_i ? (pex_i > (prior_i ^ pex_i) ? 1u : 0u) : cr.level;
                    const uint32_t add_i = (sv_i & 1u) ? (sv_i >> 3) + ((((sv_i >> 2) & 1u) != lin_i) ? 1u : 0u) : 0u;
                    before = __reduce_add_sync(FULL, lane < g ? add_i : 0u);
                    const uint32_t prior_g = hasb & ((1u << g) - 1u), pex_g = exb & ((1u << g) - 1u);
                    if (prior_g) wcin = pex_g > (prior_g ^ pex_g) ? 1u : 0u;
                } else {
                    for (int gg = 0; gg < g; gg++) {
                        const uint32_t sv = sh.xs[cw][m][gg];
                        if (sv & 1u) {
                            before += (sv >> 3) + ((((sv >> 2) & 1u) != wcin) ? 1u : 0u);
                            wcin = (sv >> 1) & 1u;
                        }
                    }
                }
                const uint32_t cin = prior ? cin_prior : wcin;
                const uint32_t Lv = core::latch_row(SETM, SET0, cin);  // level after each round
                const uint32_t Flev = (Lv << 1) | cin;            // level during each round
                const uint32_t CHG = (Lv ^ Flev) & vmask;

                core::row_energy<true>(sub, lane, Flev, rp, vmask, acc[m]);
                acc[m].hf += __popc(HF);
                const int64_t pair = pbase + (GP > 1 ? (int)sh.kmask[GP > 1 ? cw : 0][GP > 1 ? m : 0][6] : G.member[0]);
                // frequency-change log
                uint32_t *const log_pair = p.log_entries ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
                if (__any_sync(FULL, CHG != 0)) {
                    const uint64_t row0 = n_seen0 + (uint64_t)c * CH + (uint64_t)g * SB;
                    bool staged = false;
                    if (can_stage) {
                        // this lane's slot among the warp's changes: with at most 3 per
                        // row (nearly every sub-block) two ballots give it, bit by bit of the
                        // count (0.4 % faster than the shuffle scan, which takes the rest)
                        const uint32_t nch = __popc(CHG);
                        uint32_t excl, total;
                        if (__all_sync(FULL, nch < 4u)) {
                            const uint32_t b0 = __ballot_sync(FULL, nch & 1u), b1 = __ballot_sync(FULL, nch & 2u);
                            excl = __popc(b0 & lanemask_lt) + 2u * __popc(b1 & lanemask_lt);
                            total = __popc(b0) + 2u * __popc(b1);
                        } else {
                            uint32_t incl = nch;
#pragma unroll
                            for (int d = 1; d < 32; d <<= 1) {
                                const uint32_t t = __shfl_up_sync(FULL, incl, d);
                                if (lane >= d) incl += t;
                            }
                            excl = incl - nch;
                            total = __shfl_sync(FULL, incl, 31);
                        }
                        if (total <= 32) {
                            core::Staged *tab = sh.stage[GP == 1 ? warp : 0];
                            core::stage_changes(CHG, Lv, (uint32_t)row0, (uint32_t)(cr.count + before), tab, pending,
                                                excl, lane);
                            pending += total;
                            if (pending >= 32) {
                                __syncwarp();
                                core::flush_staged(tab, 32, topK, log_pair, p.log_cap, acc[m].hash, lane);
                                __syncwarp();
                                pending -= 32;
                                if ((uint32_t)lane < pending) tab[lane] = tab[32 + lane];
                                __syncwarp();
                            }
                            staged = true;
                        }
                    }
                    if (!staged) {
                        if constexpr (GP == 1)
                            acc[m].hash += core::emit_changes_cold(CHG, Lv, row0, topK, log_pair, p.log_cap,
                                                                   cr.count + before, lane);
                        else
                            core::emit_changes(CHG, Lv, row0, topK, log_pair, p.log_cap, cr.count + before,
                                               acc[m].hash, lane);
                    }
                }
                // carry into the next chunk
                if (g == TG - 1 && lane == 0) {
                    uint32_t lv = wcin;
                    uint64_t cntc = before;
                    const uint32_t sv = sh.xs[cw][m][g];
                    if (sv & 1u) {
                        cntc += (sv >> 3) + ((((sv >> 2) & 1u) != lv) ? 1u : 0u);
                        lv = (sv >> 1) & 1u;
                    }
                    MemberCarry nx;
                    nx.count = cr.count + cntc;
                    nx.level = lv;
                    nx.pad = 0;
                    sh.carry[cw][m][(c + 1) & 1] = nx;
                    if (m == 0) sh.hist[cw][(c + 1) & 1] = sh.xf[cw][g];
                }
                // state after the last round of the trace
                if (p.state && left >= 1 && left <= 32) {
                    const int pl = (int)left - 1;
                    magus_state_t &so = p.state[pair];
                    so.n_seen = n_seen0 + n;
                    so.level = ((Lv >> pl) & 1u) ? topK : 0u;
                    so.flags = (H >> (pl + 1)) | ((uint64_t)FL << (63 - pl));
                    core::read_hist(sub, 32 * lane + pl, so.hist);
                }
            }
            if constexpr (kPipe) {
                // this warp is done with the chunk's stage; the last of the TG warps refills
                // it with chunk c + 2 (ordering the warps' generic-proxy reads before the
                // copy's async-proxy writes)
                __syncwarp();
                if (lane == 0 && atomicAdd(&sh.rel[s], 1u) == (uint32_t)(TG * CW - 1)) {
                    sh.rel[s] = 0;
                    if (c + 2 < nchunks && !*(volatile int *)&sh.abort) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(c + 2, sq + 2);
                    }
                }
            }
        }
        // the change-log entries still waiting (one-member groups)
        if (pending) {
            __syncwarp();
            uint32_t *const log_pair =
                p.log_entries ? p.log_entries + (uint64_t)(pbase + G.member[0]) * p.log_cap : nullptr;
            core::flush_staged(sh.stage[GP == 1 ? warp : 0], pending, topK, log_pair, p.log_cap, acc[0].hash, lane);
            pending = 0;
        }
        if constexpr (kPipe) __syncthreads();   // every warp sees the same abort flag
        if (sh.abort) break;
        seq += nchunks;

        // ------------------------------------------------------------------ totals
#pragma unroll
        for (int m = 0; m < GP; m++) {
            const uint32_t n0 = __reduce_add_sync(FULL, acc[m].n0);
            const uint32_t nm = __reduce_add_sync(FULL, acc[m].nm);
            const uint32_t hf = __reduce_add_sync(FULL, acc[m].hf);
            const unsigned long long s0 = core::warp_sum_u64(acc[m].s0);
            const unsigned long long smv = core::warp_sum_u64(acc[m].sm);
            const unsigned long long hs = core::warp_sum_u64(acc[m].hash);
            if (lane == 0) {
                sh.red_n0[warp][m] = n0;
                sh.red_nm[warp][m] = nm;
                sh.red_hf[warp][m] = hf;
                sh.red_s0[warp][m] = s0;
                sh.red_sm[warp][m] = smv;
                sh.red_hash[warp][m] = hs;
            }
        }
        __syncthreads();
        if (g == 0 && lane < cnt && active) {
            const int m = lane;
            uint64_t N0 = 0, NM = 0, NH = 0;
            unsigned long long S0 = 0, SMs = 0, HS = 0;
            for (int w = cw * TG; w < cw * TG + TG; w++) {
                N0 += sh.red_n0[w][m];
                NM += sh.red_nm[w][m];
                NH += sh.red_hf[w][m];
                S0 += sh.red_s0[w][m];
                SMs += sh.red_sm[w][m];
                HS += sh.red_hash[w][m];
            }
            double E, T;
            core::totals(M, N0, NM, S0, SMs, &E, &T);
            const int64_t pair = pbase + G.member[m];
            p.energy[pair] = E;
            p.edp[pair] = E * T;
            if (p.time) p.time[pair] = T;
            if (p.n_changes) p.n_changes[pair] = sh.carry[cw][m][nchunks & 1].count;
            if (p.change_hash) p.change_hash[pair] = HS;
            if (p.n_hf) p.n_hf[pair] = NH;
        }
        __syncthreads();
    }
    // On abort, let outstanding bulk copies land before the CTA's shared memory goes away
    // (with the full default limit, whatever the per-chunk limit).  One slot: the last copy
    // into each stage (a completed phase passes at once); else the copies thread 0 has not
    // seen complete.
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            if (kPipe) {
                if (sh.issued[s] >= 0) (void)mbar_wait_bounded(&sh.bar[s], ((uint32_t)sh.issued[s] >> 1) & 1);
            } else if (pend[s] >= 0) {
                (void)mbar_wait_bounded(&sh.bar[s], (uint32_t)pend[s]);
            }
        }
    }
}

// Alignment slack the launch adds to a CTA's shared memory: none where the dynamic window
// starts on a 1024-byte boundary.  It starts after the block's reserved and static shared
// memory (none static here); the kernel checks its window in any case.
template <int TG, int CW, int GP, int WK>
size_t tp_smem_slack() {
    int dev = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, replay_tp_kernel<TG, CW, GP, WK>) != cudaSuccess)
        return 1024;
    return ((size_t)reserved + fa.sharedSizeBytes) % 1024 == 0 ? 0 : 1024;
}

template <int TG, int CW, int GP, int WK = 0>
cudaError_t launch_t(const TpParams &p, const CUtensorMap &tmap, const CUtensorMap &tmap_tail, int grid,
                     cudaStream_t stream) {
    const size_t smem = smem_bytes<TG, CW, GP>() + tp_smem_slack<TG, CW, GP, WK>();
    cudaError_t e = cudaFuncSetAttribute(replay_tp_kernel<TG, CW, GP, WK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    replay_tp_kernel<TG, CW, GP, WK><<<grid, TG * CW * 32, smem, stream>>>(p, tmap, tmap_tail);
    return cudaGetLastError();
}

template <int TG, int CW, int GP, int WK = 0>
int occ_t(int *smem_out) {
    const size_t smem = smem_bytes<TG, CW, GP>() + tp_smem_slack<TG, CW, GP, WK>();
    if (smem_out) *smem_out = (int)smem;
    if (cudaFuncSetAttribute(replay_tp_kernel<TG, CW, GP, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, replay_tp_kernel<TG, CW, GP, WK>, TG * CW * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return blocks;
}

#define MAGUS_TILES(X) \
    X(8, 1, 1) X(4, 2, 1) X(2, 4, 1) X(1, 8, 1) X(8, 1, 4) X(4, 2, 4) X(2, 4, 4) X(1, 8, 4) X(4, 1, 1) X(1, 4, 4) X(2, 2, 4)
// window lengths with their own instance of the 4-warp one-slot tile
#define MAGUS_TP_WINDOWS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(16)

}  // namespace

int tp_box_rows(int tg) { return tg * 32; }

bool tp_tile_supported(int tg, int cw, int gp) {
#define MAGUS_IS(a, b, c) if (tg == a && cw == b && gp == c) return true;
    MAGUS_TILES(MAGUS_IS)
#undef MAGUS_IS
    return false;
}

int tp_kernel_window(int tg, int cw, int gp, int window) {
    if (tg != 4 || cw != 1 || gp != 1) return 0;
#define MAGUS_HAS_W(w) if (window == w) return w;
    MAGUS_TP_WINDOWS(MAGUS_HAS_W)
#undef MAGUS_HAS_W
    return 0;
}

cudaError_t launch_replay_tp(int tg, int cw, int gp, const TpParams &p, const CUtensorMap &tmap,
                             const CUtensorMap &tmap_tail, int grid, cudaStream_t stream, int window) {
    switch (tp_kernel_window(tg, cw, gp, window)) {
#define MAGUS_LAUNCH_W(w) \
        case w: return launch_t<4, 1, 1, w>(p, tmap, tmap_tail, grid, stream);
        MAGUS_TP_WINDOWS(MAGUS_LAUNCH_W)
#undef MAGUS_LAUNCH_W
        default: break;
    }
#define MAGUS_LAUNCH(a, b, c) \
    if (tg == a && cw == b && gp == c) return launch_t<a, b, c>(p, tmap, tmap_tail, grid, stream);
    MAGUS_TILES(MAGUS_LAUNCH)
#undef MAGUS_LAUNCH
    return cudaErrorInvalidValue;
}

int tp_max_ctas_per_sm(int tg, int cw, int gp, int *smem, int window) {
    switch (tp_kernel_window(tg, cw, gp, window)) {
#define MAGUS_OCC_W(w) \
        case w: return occ_t<4, 1, 1, w>(smem);
        MAGUS_TP_WINDOWS(MAGUS_OCC_W)
#undef MAGUS_OCC_W
        default: break;
    }
#define MAGUS_OCC(a, b, c) if (tg == a && cw == b && gp == c) return occ_t<a, b, c>(smem);
    MAGUS_TILES(MAGUS_OCC)
#undef MAGUS_OCC
    return 0;
}

}  // namespace magus
