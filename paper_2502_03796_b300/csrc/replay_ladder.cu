// replay_ladder.cu - time-parallel replay in the one-rung mode (step_mode 1, open loop).
//
// Predictions, flags and the high-frequency state depend on the deltas only, exactly as in
// the jump mode (Sec. 3.1 Alg. 1, Sec. 3.2 Alg. 2), so they come from the same row
// machinery.  Only the decision differs: a high-frequency round sets the top rung, +1 moves
// one rung up, -1 one rung down (clamped to the ladder), 0 holds.  Every such step is a
// clamped shift x -> min(max(x + s, lo), hi), and clamped shifts compose into clamped
// shifts, so a row's 32 decisions fold into one (s, lo, hi), a warp scan of those gives
// every row the function from the sub-block's entering level to its own, and sub-blocks
// chain through the carried level.
//
// Each warp replays one (trace, policy) pair at a time (items from the device queue,
// longest traces first), streaming the trace through its own two-stage ring of 32-row TMA
// boxes.  Energy: per rung, integer counts of unstretched intervals and sums of stretched
// deltas (32-bit shared-memory atomics per run of constant rung, folded into 64-bit totals
// per sub-block), FP64 totals once per pair.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"
#include "replay_core.cuh"
#include "tma.cuh"

namespace magus {
namespace {

using core::FULL;
using core::smem_u32;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait_bounded;
using tma::tma_rows;

constexpr int SB = 1024;            // rounds per sub-block: 32 rows x 32
constexpr int LW = 4;               // warps per CTA (independent)
constexpr uint32_t kStageBytes = 1024 + SB * 4;   // [block whose last 2 rows are the halo | 32 rows]
constexpr uint32_t kWarpBytes = 2 * kStageBytes;
constexpr int kLevels = MAGUS_MAX_LEVELS;

// Per rung, over one sub-block (then folded into 64-bit totals that lane k keeps for rung
// k): unstretched intervals, and the stretched delta sums of the runs split into their low
// 16 bits and the rest (at most 1,056 runs of under 2^37 each: both halves stay below 2^32,
// so 32-bit shared atomics suffice)
struct WarpAcc {
    uint32_t n[kLevels];
    uint32_t slo[kLevels];
    uint32_t shi[kLevels];
};
struct LadderShared {
    uint64_t bar[LW][2];
    uint32_t thr[kLevels];
    WarpAcc acc[LW];
};
constexpr size_t kSmemBytes = 1024 + LW * (size_t)kWarpBytes + ((sizeof(LadderShared) + 127) / 128) * 128;

// x -> min(max(x + s, lo), hi) on the rungs 0 .. km1; |s| <= km1 loses nothing.
struct Clamp {
    int s, lo, hi;
};
__device__ __forceinline__ Clamp identity(int km1) { return Clamp{0, 0, km1}; }
// g after f
__device__ __forceinline__ Clamp then(const Clamp &f, const Clamp &g, int km1) {
    Clamp r;
    r.s = max(-km1, min(km1, f.s + g.s));
    r.lo = min(max(f.lo + g.s, g.lo), g.hi);
    r.hi = min(max(f.hi + g.s, g.lo), g.hi);
    return r;
}
__device__ __forceinline__ int apply(const Clamp &f, int x) { return min(max(x + f.s, f.lo), f.hi); }
__device__ __forceinline__ Clamp shfl_up(const Clamp &f, int d) {
    return Clamp{__shfl_up_sync(FULL, f.s, d), __shfl_up_sync(FULL, f.lo, d), __shfl_up_sync(FULL, f.hi, d)};
}
__device__ __forceinline__ Clamp shfl(const Clamp &f, int src) {
    return Clamp{__shfl_sync(FULL, f.s, src), __shfl_sync(FULL, f.lo, src), __shfl_sync(FULL, f.hi, src)};
}
// one decision: high-frequency -> top, +1 -> up one rung, -1 -> down one rung
__device__ __forceinline__ int step(int cur, uint32_t hf, uint32_t up, int km1) {
    return hf ? km1 : (up ? min(cur + 1, km1) : max(cur - 1, 0));
}

// WK > 0: an instance for calls whose one-rung policies all have window length W = WK (the
// compile-time-W predictor: 9 % faster on 4,096 x 100,000); WK = 0: any W.
template <int WK = 0>
__global__ void __launch_bounds__(LW * 32) replay_ladder_kernel(const LadderParams p,
                                                                  const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem_al = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    LadderShared &sh = *reinterpret_cast<LadderShared *>(smem_al + LW * (size_t)kWarpBytes);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t ring = smem_u32(smem_al) + (uint32_t)wib * kWarpBytes;
    auto stage_base = [&](uint32_t s_) { return ring + s_ * kStageBytes + 1024u; };
    const DevModel &M = p.model;
    const int km1 = M.K - 1;
    uint64_t *bars = sh.bar[wib];
    WarpAcc &wa = sh.acc[wib];

    for (int k = threadIdx.x; k < kLevels; k += blockDim.x) sh.thr[k] = k < M.K ? M.thr[k] : 0xffffffffu;
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        tma::fence_mbar_init();
    }
    __syncthreads();

    uint32_t seq = 0;            // sub-blocks this warp has loaded (stage and parity)
    int pend[2] = {-1, -1};      // lane 0: parity of an outstanding copy per stage
    bool abort = false;

    while (!abort) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(p.queue, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= (uint32_t)p.n_items) break;
        const LadderItem wi = p.items[item];
        const uint64_t n = p.lengths[wi.trace];
        const int64_t pair = (int64_t)wi.trace * p.n_pols + wi.pol;
        const DevPolicy P = p.pols[wi.pol];
        uint64_t n_seen0 = 0, tailH = 0;
        int level = 0;
        uint32_t h0 = 0, h1 = 0;
        if (p.state) {
            const magus_state_t &st = p.state[pair];
            n_seen0 = st.n_seen;
            tailH = st.flags;
            level = (int)st.level;
            if (level > km1) {
                if (lane == 0) atomicCAS(p.status, 0, MAGUS_EINVAL);
                level = 0;
            }
            h0 = st.hist[lane];
            h1 = st.hist[32 + lane];
        }
        for (int k = lane; k < kLevels; k += 32) {
            wa.n[k] = 0;
            wa.slo[k] = 0;
            wa.shi[k] = 0;
        }
        unsigned long long tot_n = 0, tot_s = 0;   // rung `lane`
        {
            const uint32_t b0 = stage_base(seq & 1);
            core::sts32(core::swz_elem(b0, lane - 64), h0);
            core::sts32(core::swz_elem(b0, lane - 32), h1);
        }
        __syncwarp();
        const uint32_t nsub = (uint32_t)((n + SB - 1) / SB);
        const int row_y = (int)(p.offsets[wi.trace] / 32);
        auto issue = [&](uint32_t j, uint32_t sq) {
            mbar_expect_tx(&bars[sq & 1], 32u * 128u);
            tma_rows(stage_base(sq & 1), &tmap, row_y + (int)j * 32, &bars[sq & 1]);
            pend[sq & 1] = (int)((sq >> 1) & 1);
        };
        if (lane == 0 && nsub > 0) issue(0, seq);

        uint64_t cnt = 0;                     // change entries of the pair so far
        unsigned long long hash = 0;
        uint32_t nhf = 0;
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

            // ---- predictions, flags, high-frequency state (shared with the jump mode)
            const uint64_t r0 = (uint64_t)j * SB + 32u * lane;
            const int64_t left = (int64_t)n - (int64_t)r0;
            const uint32_t vmask = core::valid_mask(left);
            const uint32_t pmask = core::predict_mask(vmask, n_seen0 + r0, P.W);
            const core::RowPred rp = core::row_predict<(WK > 0 ? WK : -1), false, true>(base, lane, P, M, vmask, pmask);
            const uint32_t FL = rp.UP | rp.DN;
            const uint64_t H = core::row_history(FL, tailH, lane);
            const uint32_t HF = core::hf_row_any(H, FL, P.L, P.kmin) & vmask;
            // Decisions that can move the rung: +1 / -1 outside the high-frequency state, and
            // the first round of every high-frequency run (it sets the top; the rest of the
            // run keeps it there, so they are no-ops and are left out)
            const uint32_t UPm = rp.UP & ~HF;
            const uint32_t EV = ((rp.UP | rp.DN) & ~HF) | (HF & ~(HF << 1));
            nhf += __popc(HF);

            // ---- this row's decisions folded into one clamped shift; warp scan
            Clamp F = identity(km1);
            for (uint32_t bits = EV; bits; bits &= bits - 1) {
                const int q = __ffs(bits) - 1;
                if ((HF >> q) & 1u) F = Clamp{0, km1, km1};
                else if ((UPm >> q) & 1u) F = Clamp{min(F.s + 1, km1), min(F.lo + 1, km1), min(F.hi + 1, km1)};
                else F = Clamp{max(F.s - 1, -km1), max(F.lo - 1, 0), max(F.hi - 1, 0)};
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Clamp prev = shfl_up(F, d);
                if (lane >= d) F = then(prev, F, km1);
            }
            Clamp Fx = shfl_up(F, 1);
            if (lane == 0) Fx = identity(km1);
            const int enter = apply(Fx, level);             // rung entering this lane's row
            const int exit_level = apply(shfl(F, 31), level);

            // ---- energy: runs of constant rung
            {
                uint32_t v[32];
                core::load_row(base, lane, v);
                int cur = enter;
                uint32_t thr = sh.thr[cur];
                uint32_t run_n = 0;
                unsigned long long run_s = 0;
                uint32_t nch = 0, CH = 0;
                // the decision taken branch-free (a round without an event holds; events lie
                // inside vmask): only the flush of a finished run branches (0.9 % faster)
#pragma unroll
                for (int k = 0; k < 32; k++) {
                    const bool valid = (vmask >> k) & 1u;
                    const bool stretched = v[k] > thr;
                    run_n += (valid && !stretched) ? 1u : 0u;
                    run_s += (valid && stretched) ? v[k] : 0u;
                    const int nxt = ((EV >> k) & 1u) ? step(cur, (HF >> k) & 1u, (UPm >> k) & 1u, km1) : cur;
                    if (nxt != cur) {
                        atomicAdd(&wa.n[cur], run_n);
                        atomicAdd(&wa.slo[cur], (uint32_t)run_s & 0xffffu);
                        atomicAdd(&wa.shi[cur], (uint32_t)(run_s >> 16));
                        run_n = 0;
                        run_s = 0;
                        cur = nxt;
                        thr = sh.thr[cur];
                        CH |= 1u << k;
                        nch++;
                    }
                }
                if (run_n) atomicAdd(&wa.n[cur], run_n);
                if (run_s) {
                    atomicAdd(&wa.slo[cur], (uint32_t)run_s & 0xffffu);
                    atomicAdd(&wa.shi[cur], (uint32_t)(run_s >> 16));
                }

                // ---- change log: slots from a warp scan of the rows' counts
                uint32_t incl = nch;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(FULL, incl, d);
                    if (lane >= d) incl += t;
                }
                if (nch) {
                    uint64_t off = cnt + incl - nch;
                    uint32_t *log = p.log_entries ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
                    int c2 = enter;
                    // only the rounds where the rung changed (CH): the other events are
                    // clamped no-ops
                    for (uint32_t bits = CH; bits; bits &= bits - 1) {
                        const int q = __ffs(bits) - 1;
                        const int nxt = step(c2, (HF >> q) & 1u, (UPm >> q) & 1u, km1);
                        const uint64_t when = n_seen0 + r0 + (uint64_t)q + 1u;
                        if (log && off < p.log_cap) log[off] = (uint32_t)(when << 5) | (uint32_t)nxt;
                        hash += core::mix64((when << 8) | (uint64_t)nxt);
                        off++;
                        c2 = nxt;
                    }
                }
                cnt += __shfl_sync(FULL, incl, 31);
            }
            // state after the trace's last round
            if (p.state && left >= 1 && left <= 32) {
                const int pl = (int)left - 1;
                magus_state_t &so = p.state[pair];
                so.flags = (H >> (pl + 1)) | ((uint64_t)FL << (63 - pl));
                core::read_hist(base, 32 * lane + pl, so.hist);
            }
            // this sub-block's rung totals into lane k's 64-bit totals
            __syncwarp();
            if (lane < M.K) {
                tot_n += wa.n[lane];
                tot_s += (unsigned long long)wa.slo[lane] + ((unsigned long long)wa.shi[lane] << 16);
                wa.n[lane] = 0;
                wa.slo[lane] = 0;
                wa.shi[lane] = 0;
            }
            __syncwarp();
            level = exit_level;
            const uint32_t f30 = __shfl_sync(FULL, FL, 30), f31 = __shfl_sync(FULL, FL, 31);
            tailH = (uint64_t)f30 | ((uint64_t)f31 << 32);
        }
        if (abort) break;
        seq += nsub;
        __syncwarp();

        // ---- totals: lane k sums rung k, FP64 reduction in a fixed order
        double t_k = 0.0, e_k = 0.0;
        if (lane < M.K) {
            t_k = M.dt * (double)tot_n + M.ak[lane] * (double)tot_s;
            e_k = M.pw[lane] * t_k;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            t_k += __shfl_xor_sync(FULL, t_k, d);
            e_k += __shfl_xor_sync(FULL, e_k, d);
        }
        const unsigned long long hs = core::warp_sum_u64(hash);
        const uint32_t hf_total = __reduce_add_sync(FULL, nhf);
        if (lane == 0) {
            p.energy[pair] = e_k;
            p.edp[pair] = e_k * t_k;
            if (p.time) p.time[pair] = t_k;
            if (p.n_changes) p.n_changes[pair] = cnt;
            if (p.change_hash) p.change_hash[pair] = hs;
            if (p.n_hf) p.n_hf[pair] = hf_total;
            if (p.state && n > 0) {
                p.state[pair].n_seen = n_seen0 + n;
                p.state[pair].level = (uint32_t)level;
            }
        }
        __syncwarp();
    }
    // let outstanding copies land before the warp's shared memory goes away
    if (lane == 0) {
        for (int s = 0; s < 2; s++)
            if (pend[s] >= 0) (void)mbar_wait_bounded(&bars[s], (uint32_t)pend[s]);
    }
}

}  // namespace

int ladder_warps_per_cta() { return LW; }

namespace {
template <int WK>
int ladder_occ_t() {
    if (cudaFuncSetAttribute(replay_ladder_kernel<WK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, replay_ladder_kernel<WK>, LW * 32, kSmemBytes) !=
        cudaSuccess)
        return 0;
    return blocks;
}
template <int WK>
cudaError_t ladder_launch_t(const LadderParams &p, const CUtensorMap &tmap, int grid, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(replay_ladder_kernel<WK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    replay_ladder_kernel<WK><<<grid, LW * 32, kSmemBytes, stream>>>(p, tmap);
    return cudaGetLastError();
}
}  // namespace

// window lengths with their own instance
#define MAGUS_LADDER_WINDOWS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(16)

int ladder_max_ctas_per_sm(int window) {
    switch (window) {
#define MAGUS_OCC_W(w) \
        case w: return ladder_occ_t<w>();
        MAGUS_LADDER_WINDOWS(MAGUS_OCC_W)
#undef MAGUS_OCC_W
        default: return ladder_occ_t<0>();
    }
}

cudaError_t launch_replay_ladder(const LadderParams &p, const CUtensorMap &tmap, int grid, cudaStream_t stream,
                                 int window) {
    switch (window) {
#define MAGUS_LAUNCH_W(w) \
        case w: return ladder_launch_t<w>(p, tmap, grid, stream);
        MAGUS_LADDER_WINDOWS(MAGUS_LAUNCH_W)
#undef MAGUS_LAUNCH_W
        default: return ladder_launch_t<0>(p, tmap, grid, stream);
    }
}

}  // namespace magus
