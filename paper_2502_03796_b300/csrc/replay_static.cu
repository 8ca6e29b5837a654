// replay_static.cu - static baselines (Sec. 5.3 default setting, Sec. 6.3 minimum) at any
// rung, in any mode, without carried state.
//
// A policy pinned to rung k runs no control: no change, no high-frequency round, every
// interval at rung k.  What remains of a replay is the energy model over the trace: an
// interval lasts dt when its demand fits C(k), else dt * x / C(k) -- a count of unstretched
// intervals and an integer sum of stretched deltas (delta > thr[k]), whatever the step mode
// or loop (the closed loop changes what the predictor sees, and a pinned policy ignores the
// predictor).  Only the carried state would need the predictions (its flag history): with
// io_state these policies take the literal kernel.
//
// One CTA per trace charges every rung in one pass.  The stretch thresholds increase with
// the rung, so a delta a is stretched exactly at the rungs below r(a) = #{k : thr[k] < a};
// each delta adds a to a sum and 1 to a count kept per r in shared-memory columns (one per
// thread, so no two lanes touch one word), and the rung totals are prefix / suffix sums of
// those at the end.  Consecutive deltas change r about every other interval on noisy
// traces, so the columns take every delta (no run kept in registers).
//
// The columns pack a sum and a count into one 64-bit word per r (one load and one store per
// delta); every 4,096 deltas per thread, and at the end, a warp sums each r's words into
// totals that lane r keeps in registers.
//
// r(a) comes from a table of cells of 2^shift counter units: a cell's word holds the number
// of thresholds below its start (top 6 bits) and the offset of the one threshold inside it,
// if any (low 26 bits), so r(a) = lo + (a - start > offset) after one shared-memory load;
// deltas above the last cell (the one holding the top threshold) take that cell.  The host
// picks the coarsest cells that still give each threshold its own (few distinct cells per
// warp: few bank conflicts), of at most 2^26 units and kMaxCells cells; if no such cells
// exist, the kernel searches the thresholds instead (a branch-free binary search, five
// dependent loads).
//
// Pins at a ladder bound in jump mode join this kernel when it runs for another pin (no
// state): the tile kernel would replay each of them separately; else they stay there.
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"
#include "replay_core.cuh"

namespace magus {
namespace {

constexpr int kWarps = 4;   // per CTA (one trace)
constexpr int kThreads = kWarps * 32;
constexpr int kMaxCells = 512;
constexpr int kSumBits = 44;    // 2^12 deltas below 2^32 sum below 2^44; their count fits 20 bits
constexpr unsigned long long kSumMask = (1ull << kSumBits) - 1ull;
constexpr int kFlush = 4096;    // deltas per thread between flushes of the packed columns

template <bool kCells>
__global__ void __launch_bounds__(kThreads) replay_static_kernel(const StaticParams p, const uint32_t shift,
                                                                  const uint32_t n_cells) {
    // per thread and r = 0 .. K: sum and count of the deltas with r thresholds below them
    extern __shared__ unsigned long long st_s[];
    __shared__ uint32_t thr_s[MAGUS_MAX_LEVELS];   // padded with never-exceeded thresholds
    __shared__ uint32_t cell_s[kCells ? kMaxCells : 1];
    __shared__ unsigned long long red_n[kWarps][MAGUS_MAX_LEVELS + 1], red_s[kWarps][MAGUS_MAX_LEVELS + 1];
    __shared__ unsigned long long rung_n[MAGUS_MAX_LEVELS], rung_s[MAGUS_MAX_LEVELS];
    const DevModel &M = p.model;
    const int K = M.K;
    const int64_t trace = blockIdx.x;
    const uint32_t *tr = p.traces + p.offsets[trace];
    const uint64_t n = p.lengths[trace];
    // thread i takes deltas 4i .. 4i+3 of every 512 (the packed layout pads each trace to a
    // multiple of 32 deltas, so whole 16-byte loads stay inside it): the first 2048 deltas'
    // loads are issued before the tables are set up, each next 2048's before a block is charged
    const uint32_t lo4 = 4u * threadIdx.x;
    uint4 v[4];
    if (n >= 2048) {
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldg(reinterpret_cast<const uint4 *>(tr + 512u * u + lo4));
    }
    if (threadIdx.x < MAGUS_MAX_LEVELS) thr_s[threadIdx.x] = threadIdx.x < (unsigned)K ? M.thr[threadIdx.x] : 0xffffffffu;
    if (kCells) {
        // cell c covers [c << shift, (c + 1) << shift): thresholds below it, the one inside
        // (none: an offset no delta of the cell exceeds)
        for (uint32_t c = threadIdx.x; c < n_cells; c += kThreads) {
            const uint64_t lo = (uint64_t)c << shift, hi = lo + (1ull << shift);
            uint32_t below = 0, off = (1u << 26) - 1u;
            for (int k = 0; k < K; k++) {
                const uint32_t t = M.thr[k];
                if (t == 0xffffffffu) continue;   // never exceeded
                if (t < lo) below++;
                else if (t < hi) off = (uint32_t)(t - lo);
            }
            cell_s[c] = below << 26 | off;
        }
    }
    // packed per-thread columns, one word per r: bits 0..43 the sum of the deltas, 44..63
    // their count; at most kFlush deltas per thread between two flushes keep both exact
    unsigned long long *pk = st_s + threadIdx.x;
    for (int r = 0; r <= K; r++) pk[r * kThreads] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the warp's totals of r = lane (and r = 32 in lane 0), in registers
    unsigned long long tot_s = 0, tot_n = 0, tot_s2 = 0, tot_n2 = 0;
    auto flush = [&]() {
        for (int r = 0; r <= K; r++) {
            const unsigned long long w = pk[r * kThreads];
            pk[r * kThreads] = 0;
            const unsigned long long ws = core::warp_sum_u64(w & kSumMask);
            uint32_t wn = (uint32_t)(w >> kSumBits);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, d);
            if (r == lane) {
                tot_s += ws;
                tot_n += wn;
            } else if (r == lane + 32) {
                tot_s2 += ws;
                tot_n2 += wn;
            }
        }
    };
    auto charge = [&](uint32_t a) {
        int r;
        if (kCells) {
            const uint32_t c = min(a >> shift, n_cells - 1);
            const uint32_t e = cell_s[c];
            r = (int)(e >> 26) + (a - (c << shift) > (e & ((1u << 26) - 1u)) ? 1 : 0);
        } else {
            r = 0;
#pragma unroll
            for (int step = MAGUS_MAX_LEVELS / 2; step > 0; step >>= 1) r += thr_s[r + step - 1] < a ? step : 0;
        }
        pk[r * kThreads] += (1ull << kSumBits) | a;
    };
    uint64_t base = 0;
    if (n >= 2048) {
        for (uint32_t blk = 1;; blk++) {
            const bool more = base + 4096 <= n;
            uint4 w[4];
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; u++) w[u] = __ldg(reinterpret_cast<const uint4 *>(tr + base + 2048 + 512u * u + lo4));
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                charge(v[u].x);
                charge(v[u].y);
                charge(v[u].z);
                charge(v[u].w);
            }
            base += 2048;
            if (blk % (kFlush / 16) == 0) flush();   // 16 deltas per thread and block
            if (!more) break;
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = w[u];
        }
    }
    flush();
    for (; base < n; base += 512) {   // at most 12 deltas per thread
        const uint64_t e = base + lo4;
        if (e >= n) continue;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tr + e));
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (e + (uint64_t)j < n) charge(vv[j]);
    }
    flush();
    // rung k: unstretched deltas have r <= k, stretched ones r > k
    red_n[warp][lane] = tot_n;
    red_s[warp][lane] = tot_s;
    if (lane == 0) {
        red_n[warp][32] = tot_n2;
        red_s[warp][32] = tot_s2;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)K) {
        const int k = threadIdx.x;
        unsigned long long N = 0, S = 0;
        for (int w = 0; w < kWarps; w++)
            for (int r = 0; r <= K; r++) {
                if (r <= k) N += red_n[w][r];
                else S += red_s[w][r];
            }
        rung_n[k] = N;
        rung_s[k] = S;
    }
    __syncthreads();
    // every listed policy pinned at some rung k
    for (int i = threadIdx.x; i < p.n_lit; i += kThreads) {
        const int pol = p.lit[i];
        const DevPolicy &P = p.pols[pol];
        if (!static_policy(P, K)) continue;
        const int k = P.pin - 1;
        const int64_t pair = trace * p.n_pols + pol;
        const double T = M.dt * (double)rung_n[k] + M.ak[k] * (double)rung_s[k];
        const double E = M.pw[k] * T;
        p.energy[pair] = E;
        p.edp[pair] = E * T;
        if (p.time) p.time[pair] = T;
        if (p.n_changes) p.n_changes[pair] = 0;
        if (p.change_hash) p.change_hash[pair] = 0;
        if (p.n_hf) p.n_hf[pair] = 0;
    }
}

// The coarsest cells of 2^shift units (shift <= 26), at most kMaxCells of them up to the
// top finite threshold, with at most one threshold in each; false if there are none such.
// Without finite thresholds: 64 cells of 2^26 cover every delta, none stretched.
bool choose_cells(const DevModel &m, uint32_t *shift, uint32_t *n_cells) {
    uint32_t top = 0;
    bool any = false;
    for (int k = 0; k < m.K; k++)
        if (m.thr[k] != 0xffffffffu) {
            top = m.thr[k];
            any = true;
        }
    if (!any) {
        *shift = 26;
        *n_cells = 64;
        return true;
    }
    for (int s = 26; s >= 0; s--) {
        bool distinct = true;
        for (int k = 0; k + 1 < m.K; k++)
            if (m.thr[k + 1] != 0xffffffffu && (m.thr[k] >> s) == (m.thr[k + 1] >> s)) distinct = false;
        if (!distinct) continue;
        const uint32_t cells = (top >> s) + 1;
        if (cells > (uint32_t)kMaxCells) return false;
        *shift = (uint32_t)s;
        *n_cells = cells;
        return true;
    }
    return false;
}

}  // namespace

cudaError_t launch_replay_static(const StaticParams &p, cudaStream_t stream) {
    if (p.n_traces <= 0) return cudaSuccess;
    const size_t smem = (size_t)(p.model.K + 1) * kThreads * sizeof(unsigned long long);
    uint32_t shift = 0, n_cells = 0;
    const bool cells = choose_cells(p.model, &shift, &n_cells);
    cudaError_t e = cells ? cudaFuncSetAttribute(replay_static_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(replay_static_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cells)
        replay_static_kernel<true><<<(unsigned)p.n_traces, kThreads, smem, stream>>>(p, shift, n_cells);
    else
        replay_static_kernel<false><<<(unsigned)p.n_traces, kThreads, smem, stream>>>(p, 0, 1);
    return cudaGetLastError();
}

}  // namespace magus
