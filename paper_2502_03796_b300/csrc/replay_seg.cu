// replay_seg.cu - warp-autonomous, segment-parallel batched replay (jump mode).
//
// Every warp works alone: it takes a work item (one trace, one policy group, one time
// segment of seg_len rounds) from the device queue and streams the segment's 1024-round
// sub-blocks through its own two-stage shared-memory ring with 2-D TMA tensor copies (32
// rows of 32 deltas, 128-byte swizzle), so no barrier ever couples warps, and segments of
// equal length keep all warps busy to the end of the launch.
//
// A segment does not know the level it starts at: the latch of the replay (Sec. 3.2,
// Sec. 6.1: high-frequency or +1 -> top, -1 -> bottom, else hold) forgets it at the first
// event.  So the rounds before the segment's first event are charged for both possible
// levels, the possible change at the first event is left open, and everything after it is
// exact.  Its flag history (the 64 flags before the segment, needed by Algorithm 2) depends
// on deltas only and is recomputed from the 128 deltas before the segment.
//
// A combine kernel then walks each pair's segments in order, fixes each entering level,
// adds the right prefix charge, decides the first-event change, and compacts the change
// log from the per-segment scratch into the caller's log.
#include <cuda.h>
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

using core::FULL;
using core::smem_u32;

constexpr int SB = 1024;            // rounds per sub-block: 32 rows x 32
constexpr int SEG_WARPS = 4;        // warps per CTA (independent)
constexpr uint32_t kNone = 0xffffffffu;

// per-warp ring: 2 stages of [1024-byte block whose last 2 rows hold the 64 preceding
// deltas | 32 rows]; 1024-byte aligned for the 128-byte swizzle
constexpr uint32_t kStageBytes = 1024 + SB * 4;
constexpr uint32_t kWarpBytes = 2 * kStageBytes;
constexpr size_t kSmemBytes = 1024 + SEG_WARPS * (size_t)kWarpBytes + 64;


// Per member of the warp's policy group, kept across the sub-blocks of a segment.
struct MemberRun {
    uint32_t known;         // the level entering the next sub-block is known
    uint32_t level;         // that level (0 bottom / 1 top) when known
    uint32_t first_pos;     // segment round of the first event (kNone before it)
    uint32_t first_val;     // level set by the first event
    uint32_t n_det;         // change entries after the first event
};

// WK > 0: an instance for one-member groups whose window length W is WK (the compile-time-W
// predictor: the segment kernel 11 % faster on 16 x 4,000,000 intervals); WK = 0: any W.
template <int GP, int WK = 0>
__global__ void __launch_bounds__(SEG_WARPS * 32) replay_seg_kernel(const SegParams p,
                                                                      const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem_al = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_al + SEG_WARPS * (size_t)kWarpBytes) + 2 * wib;
    // data row 0 of stage s of this warp
    const uint32_t ring = smem_u32(smem_al) + (uint32_t)wib * kWarpBytes;
    auto stage_base = [&](uint32_t s_) { return ring + s_ * kStageBytes + 1024u; };
    const DevModel &M = p.model;
    const uint32_t topK = (uint32_t)(M.K - 1);
    const uint32_t lanemask_lt = (1u << lane) - 1u;

    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    uint32_t seq = 0;            // sub-blocks this warp has loaded (stage and parity)
    int pend[2] = {-1, -1};      // lane 0: parity of an outstanding copy per stage
    bool abort = false;

    while (!abort) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= (uint32_t)p.n_items) break;
        const SegItem wi = p.items[item];
        const PolicyGroup G = p.groups[wi.grp];
        const int cnt = G.count;
        const uint64_t n = p.lengths[wi.trace];
        const uint64_t s0 = (uint64_t)wi.seg * p.seg_len;
        const uint64_t len = n - s0 < (uint64_t)p.seg_len ? n - s0 : (uint64_t)p.seg_len;
        const uint32_t nsub = (uint32_t)((len + SB - 1) / SB);
        const int64_t pbase = (int64_t)wi.trace * p.n_pols;
        const int64_t pair0 = pbase + G.member[0];
        const uint64_t sidx = p.seg_base[wi.trace] + wi.seg;   // global segment index
        const bool last_seg = s0 + len == n;
        const DevPolicy P = p.pols[G.member[0]];
        const uint64_t n_seen_base = p.state ? p.state[pair0].n_seen : 0;
        const uint32_t *tr = p.traces + p.offsets[wi.trace];

        // ---- the 64 deltas and 64 flags before the segment
        uint64_t tailH;
        uint32_t h0, h1;
        if (wi.seg == 0) {
            tailH = p.state ? p.state[pair0].flags : 0ull;
            h0 = p.state ? p.state[pair0].hist[lane] : 0u;
            h1 = p.state ? p.state[pair0].hist[32 + lane] : 0u;
        } else {
            // rounds s0-64 .. s0-1 (s0 >= 1024, so every window reaches inside the trace)
            const uint64_t t0 = s0 - 64 + lane, t1 = s0 - 32 + lane;
            h0 = tr[t0];
            h1 = tr[t1];
            bool u0, d0, u1, d1;
            core::predict_exact(h0, tr[t0 - P.W], P, M, u0, d0);
            core::predict_exact(h1, tr[t1 - P.W], P, M, u1, d1);
            const uint32_t f0 = __ballot_sync(FULL, u0 || d0), f1 = __ballot_sync(FULL, u1 || d1);
            tailH = (uint64_t)f0 | ((uint64_t)f1 << 32);
        }
        {
            const uint32_t b0 = stage_base(seq & 1);
            core::sts32(core::swz_elem(b0, lane - 64), h0);
            core::sts32(core::swz_elem(b0, lane - 32), h1);
        }
        __syncwarp();
        const int row_y = (int)((p.offsets[wi.trace] + s0) / 32);
        auto issue = [&](uint32_t j, uint32_t sq) {
            mbar_expect_tx(&bars[sq & 1], 32u * 128u);
            tma_rows(stage_base(sq & 1), &tmap, row_y + (int)j * 32, &bars[sq & 1]);
            pend[sq & 1] = (int)((sq >> 1) & 1);
        };
        if (lane == 0 && nsub > 0) issue(0, seq);

        int Lm[GP], Km[GP];
        MemberRun run[GP];
        core::Acc acc[GP];
        core::PAcc pacc[GP];
#pragma unroll
        for (int m = 0; m < GP; m++) {
            const int id = G.member[m < cnt ? m : 0];
            // bit 8 marks a static baseline (no control), bit 9 one pinned at the top; L
            // itself is at most 64
            Lm[m] = p.pols[id].L | (p.pols[id].pin ? 0x100 : 0) | (p.pols[id].pin > 1 ? 0x200 : 0);
            Km[m] = p.pols[id].kmin;
            core::acc_zero(acc[m]);
            core::pacc_zero(pacc[m]);
            // a static baseline knows its level in every segment
            run[m].known = (wi.seg == 0 || (Lm[m] & 0x100)) ? 1u : 0u;
            uint32_t lv = 0;
            if (Lm[m] & 0x100) {
                lv = (Lm[m] & 0x200) ? topK : 0u;
            } else if (wi.seg == 0 && p.state && m < cnt) {
                lv = p.state[pbase + G.member[m]].level;
                if (lv != 0 && lv != topK) {
                    if (lane == 0) atomicCAS(p.status, 0, MAGUS_EINVAL);
                    lv = 0;
                }
            }
            run[m].level = lv ? 1u : 0u;
            run[m].first_pos = kNone;
            run[m].first_val = 0;
            run[m].n_det = 0;
        }

        for (uint32_t j = 0; j < nsub; j++) {
            const uint32_t sq = seq + j;
            const uint32_t s = sq & 1;
            const uint32_t base = stage_base(s);
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait_bounded(&bars[s], (sq >> 1) & 1) ? 1 : 0;
                if (ok) pend[s] = -1;
                else atomicCAS(p.status, 0, MAGUS_ETIMEDOUT);
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) { abort = true; break; }
            if (lane != 0) (void)mbar_wait_bounded(&bars[s], (sq >> 1) & 1);
            if (j > 0) {
                // rows 30, 31 of the previous sub-block become rows -2, -1 (same swizzle phase)
                const uint32_t prev = stage_base(s ^ 1) + 30u * 128u;
                const uint32_t v0 = core::lds32(prev + 4u * lane), v1 = core::lds32(prev + 128u + 4u * lane);
                core::sts32(base - 256u + 4u * lane, v0);
                core::sts32(base - 128u + 4u * lane, v1);
            }
            __syncwarp();
            if (lane == 0 && j + 1 < nsub) issue(j + 1, sq + 1);

            const uint64_t r0 = s0 + (uint64_t)j * SB + 32u * lane;      // row start (trace round)
            const int64_t left = (int64_t)n - (int64_t)r0;
            const uint32_t vmask = core::valid_mask(left);
            const uint32_t pmask = core::predict_mask(vmask, n_seen_base + r0, P.W);
            const core::RowPred rp = core::row_predict<(WK > 0 ? WK : -1)>(base, lane, P, M, vmask, pmask);
            const uint32_t UP = rp.UP, DN = rp.DN;
            const uint32_t FL = UP | DN;
            const uint64_t H = core::row_history(FL, tailH, lane);

#pragma unroll 1
            for (int m = 0; m < (GP == 1 ? 1 : cnt); m++) {
                const uint32_t act = (Lm[m] & 0x100) ? 0u : FULL;
                const uint32_t HF = core::hf_row_any(H, FL, Lm[m] & 0xff, Km[m]) & vmask & act;
                const uint32_t SETM = (HF | UP) & act;
                const uint32_t SET0 = DN & ~HF & act;
                const uint32_t EV = SETM | SET0;
                const bool has = EV != 0;
                // disjoint masks: the last event sets the top exactly when SETM > SET0, the
                // first exactly when SETM holds EV's lowest bit (no bit scans)
                const uint32_t exitv = SETM > SET0 ? 1u : 0u;
                const uint32_t firstv = (SETM & (0u - EV)) != 0u ? 1u : 0u;
                const uint32_t bev = __ballot_sync(FULL, has), bex = __ballot_sync(FULL, exitv);
                const uint32_t prior = bev & lanemask_lt;
                const uint32_t pex = bex & lanemask_lt;
                const uint32_t cin_prior = pex > (prior ^ pex) ? 1u : 0u;
                acc[m].hf += __popc(HF);
                uint32_t cin, PM = 0;                // PM: rounds at the unknown entering level
                if (run[m].known) {
                    cin = prior ? cin_prior : run[m].level;
                } else if (!bev) {
                    cin = 0;
                    PM = vmask;                      // no event yet: the whole row waits
                } else {
                    const int fl = __ffs(bev) - 1;
                    if (lane < fl) {
                        cin = 0;
                        PM = vmask;
                    } else if (lane == fl) {
                        const int q1 = __ffs(EV) - 1;
                        cin = firstv;                // no change at the first event itself
                        PM = vmask & (0xffffffffu >> (31 - q1));
                    } else {
                        cin = cin_prior;
                    }
                    const uint32_t q1 = __shfl_sync(FULL, (uint32_t)(__ffs(EV) - 1), fl);
                    run[m].first_pos = j * SB + 32u * (uint32_t)fl + q1;
                    run[m].first_val = __shfl_sync(FULL, firstv, fl);
                }
                const uint32_t Lv = core::latch_row(SETM, SET0, cin);
                const uint32_t Flev = (Lv << 1) | cin;
                const uint32_t DM = vmask & ~PM;
                const uint32_t CHG = (Lv ^ Flev) & DM;
                core::row_energy(base, lane, Flev, rp, DM, acc[m]);
                if (__any_sync(FULL, PM != 0)) core::row_energy_prefix(base, lane, PM, rp, pacc[m]);
                if (__any_sync(FULL, CHG != 0)) {
                    const uint32_t pol = G.member[m];
                    uint32_t *slog = nullptr;
                    uint64_t scap = 0;
                    if (p.scratch_base) {
                        const uint64_t sb = p.scratch_base[wi.trace];
                        if (sb == kInPlace) {
                            slog = p.log + (uint64_t)(pbase + pol) * p.log_cap + s0;
                            scap = p.seg_len;
                        } else {
                            slog = p.scratch_log + sb + ((uint64_t)wi.seg * p.n_pols + pol) * p.seg_cap;
                            scap = p.seg_cap;
                        }
                    }
                    core::emit_changes(CHG, Lv, n_seen_base + s0 + (uint64_t)j * SB, topK, slog, scap,
                                       run[m].n_det, acc[m].hash, lane);
                    run[m].n_det += __reduce_add_sync(FULL, __popc(CHG));
                }
                if (bev) {
                    run[m].known = 1u;
                    run[m].level = bex > (bev ^ bex) ? 1u : 0u;
                }
                // flags and deltas after the trace's last round (the combine kernel stores
                // them with the final level)
                if (last_seg && left >= 1 && left <= 32) {
                    const int pl = (int)left - 1;
                    SegTail &tl = p.tails[pbase + G.member[m]];
                    tl.flags = (H >> (pl + 1)) | ((uint64_t)FL << (63 - pl));
                    core::read_hist(base, 32 * lane + pl, tl.hist);
                }
            }
            const uint32_t f30 = __shfl_sync(FULL, FL, 30), f31 = __shfl_sync(FULL, FL, 31);
            tailH = (uint64_t)f30 | ((uint64_t)f31 << 32);
        }
        if (abort) break;
        seq += nsub;

        // ---- segment summary per member
#pragma unroll 1
        for (int m = 0; m < (GP == 1 ? 1 : cnt); m++) {
            const uint32_t n0 = __reduce_add_sync(FULL, acc[m].n0), nm = __reduce_add_sync(FULL, acc[m].nm);
            const uint32_t hf = __reduce_add_sync(FULL, acc[m].hf);
            const uint32_t pn0 = __reduce_add_sync(FULL, pacc[m].n0), pnm = __reduce_add_sync(FULL, pacc[m].nm);
            const unsigned long long s0v = core::warp_sum_u64(acc[m].s0), smv = core::warp_sum_u64(acc[m].sm);
            const unsigned long long ps0 = core::warp_sum_u64(pacc[m].s0), psm = core::warp_sum_u64(pacc[m].sm);
            const unsigned long long hs = core::warp_sum_u64(acc[m].hash);
            if (lane == 0) {
                SegSummary o;
                o.s0 = s0v;
                o.sm = smv;
                o.p_s0 = ps0;
                o.p_sm = psm;
                o.hash = hs;
                o.n0 = n0;
                o.nm = nm;
                o.p_n0 = pn0;
                o.p_nm = pnm;
                o.nhf = hf;
                o.n_det = run[m].n_det;
                o.first_pos = run[m].first_pos;
                o.vals = run[m].first_val | ((run[m].known ? run[m].level : 0u) << 1) | (run[m].known << 2);
                p.summ[(uint64_t)sidx * p.n_pols + G.member[m]] = o;
            }
        }
    }
    // let outstanding copies land before the warp's shared memory goes away
    if (lane == 0) {
        for (int s = 0; s < 2; s++)
            if (pend[s] >= 0) (void)mbar_wait_bounded(&bars[s], (uint32_t)pend[s]);
    }
}

// One warp per pair; lane i takes segment 32c + i of chunk c.  The level entering a
// segment is the end level of the last earlier segment that saw an event (a ballot over the
// chunk plus the level carried from the previous chunk), which fixes its prefix charge and
// whether its first event is a change.  Log slots follow from an exclusive scan of the
// segments' entry counts; the entries are then moved in segment order, which keeps every
// in-place move from overwriting a source not moved yet.
__global__ void __launch_bounds__(256) combine_kernel(const SegParams p, int64_t n_pairs, double *energy,
                                                       double *edp, double *time, uint64_t *n_changes,
                                                       uint64_t *change_hash, uint64_t *n_hf) {
    const int lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (pair >= n_pairs) return;
    const int64_t trace = pair / p.n_pols, pol = pair % p.n_pols;
    if (!tp_policy(p.pols[pol], p.model.K)) return;   // replayed by another kernel
    const uint64_t n = p.lengths[trace];
    const uint64_t nseg = (n + p.seg_len - 1) / p.seg_len;
    const uint32_t topK = (uint32_t)(p.model.K - 1);
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    uint32_t level = 0;
    uint64_t n_seen_base = 0;
    if (p.state) {
        n_seen_base = p.state[pair].n_seen;
        level = (p.state[pair].level == topK) ? 1u : 0u;
    }
    if (p.pols[pol].pin) level = p.pols[pol].pin > 1 ? 1u : 0u;
    uint32_t *const plog = p.log ? p.log + (uint64_t)pair * p.log_cap : nullptr;
    const uint64_t log_cap = p.log_cap;
    const uint64_t sbase = p.scratch_base ? p.scratch_base[trace] : 0;
    unsigned long long N0 = 0, NM = 0, NH = 0, S0 = 0, SMs = 0, HS = 0;
    uint64_t cnt = 0;                       // entries of the segments before this chunk
    for (uint64_t c0 = 0; c0 < nseg; c0 += 32) {
        const uint64_t k = c0 + lane;
        const bool act = k < nseg;
        SegSummary sm;
        if (act) {
            sm = p.summ[(p.seg_base[trace] + k) * p.n_pols + pol];
        } else {
            memset(&sm, 0, sizeof(sm));
            sm.first_pos = kNone;
        }
        const bool known = (sm.vals & 4u) != 0;
        const uint32_t bk = __ballot_sync(FULL, known);
        const uint32_t bx = __ballot_sync(FULL, known && ((sm.vals >> 1) & 1u));
        const uint32_t prior = bk & lanemask_lt;
        const uint32_t enter = prior ? (bx >> (31 - __clz(prior))) & 1u : level;
        if (enter == 0) { N0 += sm.p_n0; S0 += sm.p_s0; }
        else { NM += sm.p_nm; SMs += sm.p_sm; }
        N0 += sm.n0;
        NM += sm.nm;
        S0 += sm.s0;
        SMs += sm.sm;
        NH += sm.nhf;
        HS += sm.hash;
        // a change at the segment's first event when it flips the entering level
        const uint32_t f = (act && sm.first_pos != kNone && (sm.vals & 1u) != enter) ? 1u : 0u;
        uint32_t first_entry = 0;
        if (f) {
            const uint64_t when = n_seen_base + k * p.seg_len + sm.first_pos + 1;
            const uint32_t lv = (sm.vals & 1u) ? topK : 0u;
            first_entry = (uint32_t)(when << 5) | lv;
            HS += core::mix64((when << 8) | lv);
        }
        // exclusive scan of the segments' entry counts
        const uint64_t mine = f + (uint64_t)sm.n_det;
        uint64_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += t;
        }
        const uint64_t slot = cnt + incl - mine;              // this segment's first slot
        if (plog && p.scratch_base) {
            uint32_t todo = __ballot_sync(FULL, sm.n_det != 0);
            while (todo) {
                const int src_lane = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint64_t dst = __shfl_sync(FULL, slot + f, src_lane);
                const uint64_t nd = __shfl_sync(FULL, (uint64_t)sm.n_det, src_lane);
                const uint64_t take = dst < log_cap ? (nd < log_cap - dst ? nd : log_cap - dst) : 0;
                const uint64_t kk = c0 + src_lane;
                if (sbase == kInPlace) {
                    // the source starts at slot kk * seg_len >= dst - 1 (one change per round at
                    // most); a destination one slot to the right is copied from the end
                    const uint64_t src = kk * p.seg_len;
                    if (src != dst) {
                        const uint64_t nchunk = (take + 31) / 32;
                        for (uint64_t q = 0; q < nchunk; q++) {
                            const uint64_t qq = dst > src ? nchunk - 1 - q : q;
                            const uint64_t e = qq * 32 + lane;
                            const uint32_t v = e < take ? plog[src + e] : 0u;
                            __syncwarp();
                            if (e < take) plog[dst + e] = v;
                            __syncwarp();
                        }
                    }
                } else {
                    const uint32_t *srcp = p.scratch_log + sbase + (kk * p.n_pols + pol) * p.seg_cap;
                    for (uint64_t e = lane; e < take; e += 32) plog[dst + e] = srcp[e];
                }
            }
            __syncwarp();
        }
        if (plog && f && slot < log_cap) plog[slot] = first_entry;
        __syncwarp();
        cnt += __shfl_sync(FULL, incl, 31);
        const uint32_t last_known = bk ? (31 - __clz(bk)) : 32u;
        if (bk) level = (bx >> last_known) & 1u;
    }
    N0 = core::warp_sum_u64(N0);
    NM = core::warp_sum_u64(NM);
    S0 = core::warp_sum_u64(S0);
    SMs = core::warp_sum_u64(SMs);
    NH = core::warp_sum_u64(NH);
    HS = core::warp_sum_u64(HS);
    if (lane != 0) return;
    double E, T;
    core::totals(p.model, N0, NM, S0, SMs, &E, &T);
    energy[pair] = E;
    edp[pair] = E * T;
    if (time) time[pair] = T;
    if (n_changes) n_changes[pair] = cnt;
    if (change_hash) change_hash[pair] = HS;
    if (n_hf) n_hf[pair] = NH;
    if (p.state && n > 0) {
        magus_state_t &st = p.state[pair];
        st.n_seen = n_seen_base + n;
        st.level = level ? topK : 0u;
        st.flags = p.tails[pair].flags;
        for (int q = 0; q < 64; q++) st.hist[q] = p.tails[pair].hist[q];
    }
}

template <int GP, int WK = 0>
cudaError_t launch_seg_t(const SegParams &p, const CUtensorMap &tmap, int grid, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(replay_seg_kernel<GP, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    replay_seg_kernel<GP, WK><<<grid, SEG_WARPS * 32, kSmemBytes, stream>>>(p, tmap);
    return cudaGetLastError();
}

template <int GP, int WK = 0>
int occ_seg_t() {
    if (cudaFuncSetAttribute(replay_seg_kernel<GP, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
        cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, replay_seg_kernel<GP, WK>, SEG_WARPS * 32, kSmemBytes) !=
        cudaSuccess)
        return 0;
    return blocks;
}

}  // namespace

int seg_warps_per_cta() { return SEG_WARPS; }

// window lengths with their own instance (one-member groups)
#define MAGUS_SEG_WINDOWS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(16)
static int seg_window(int gp, int window) {
    if (gp != 1) return 0;
#define MAGUS_HAS_W(w) if (window == w) return w;
    MAGUS_SEG_WINDOWS(MAGUS_HAS_W)
#undef MAGUS_HAS_W
    return 0;
}

cudaError_t launch_replay_seg(int gp, const SegParams &p, const CUtensorMap &tmap, int grid, cudaStream_t stream,
                              int window) {
    switch (seg_window(gp, window)) {
#define MAGUS_LAUNCH_W(w) \
        case w: return launch_seg_t<1, w>(p, tmap, grid, stream);
        MAGUS_SEG_WINDOWS(MAGUS_LAUNCH_W)
#undef MAGUS_LAUNCH_W
        default: break;
    }
    if (gp == 1) return launch_seg_t<1>(p, tmap, grid, stream);
    if (gp == 4) return launch_seg_t<4>(p, tmap, grid, stream);
    return cudaErrorInvalidValue;
}

int seg_max_ctas_per_sm(int gp, int window) {
    switch (seg_window(gp, window)) {
#define MAGUS_OCC_W(w) \
        case w: return occ_seg_t<1, w>();
        MAGUS_SEG_WINDOWS(MAGUS_OCC_W)
#undef MAGUS_OCC_W
        default: break;
    }
    if (gp == 1) return occ_seg_t<1>();
    if (gp == 4) return occ_seg_t<4>();
    return 0;
}

cudaError_t launch_combine(const SegParams &p, int64_t n_pairs, double *energy, double *edp, double *time,
                           uint64_t *n_changes, uint64_t *change_hash, uint64_t *n_hf, cudaStream_t stream) {
    if (n_pairs <= 0) return cudaSuccess;
    const int64_t blocks = (n_pairs + 7) / 8;
    combine_kernel<<<(unsigned)blocks, 256, 0, stream>>>(p, n_pairs, energy, edp, time, n_changes, change_hash,
                                                         n_hf);
    return cudaGetLastError();
}

}  // namespace magus
