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
// One pass over each trace charges every rung.  The stretch thresholds increase with
// the rung, so a delta a is stretched exactly at the rungs below r(a) = #{k : thr[k] < a};
// each delta adds a to a sum and 1 to a count kept per r in shared-memory columns (one per
// thread, so no two lanes touch one word), and the rung totals are prefix / suffix sums of
// those at the end.  Consecutive deltas change r about every other interval on noisy
// traces, so the columns take every delta (no run kept in registers).
//
// The columns pack a sum and a count into one 64-bit word per r (one load and one store per
// delta), exact for up to 4,096 deltas per thread: a CTA charges a part of a trace of at most
// 256 blocks of 2048 deltas.  Parts are whole blocks, about four waves of CTAs, longest
// first; a trace in several parts adds each part's totals to its accumulators in global
// memory, and the part that arrives last charges the rungs.
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

#include <algorithm>
#include <atomic>
#include <vector>

#include "replay_core.cuh"
#include "replay_static.h"

namespace magus {
namespace {

constexpr int kWarps = 4;   // per CTA (one trace)
constexpr int kThreads = kWarps * 32;
constexpr int kMaxCells = 512;
constexpr int kSumBits = 44;    // 2^12 deltas below 2^32 sum below 2^44; their count fits 20 bits
constexpr unsigned long long kSumMask = (1ull << kSumBits) - 1ull;
constexpr uint32_t kMaxPartBlocks = 256;   // 2048-delta blocks per CTA: 4096 deltas per thread

template <bool kCells>
__global__ void __launch_bounds__(kThreads, 10) replay_static_kernel(const StaticParams p, const uint32_t shift,
                                                                  const uint32_t n_cells) {
    // per thread and r = 0 .. K: sum and count of the deltas with r thresholds below them
    extern __shared__ unsigned long long st_s[];
    __shared__ uint32_t thr_s[MAGUS_MAX_LEVELS];   // padded with never-exceeded thresholds
    __shared__ uint32_t cell_s[kCells ? kMaxCells : 1];
    __shared__ unsigned long long red_n[MAGUS_MAX_LEVELS + 1], red_s[MAGUS_MAX_LEVELS + 1];   // per r
    __shared__ unsigned long long rung_n[MAGUS_MAX_LEVELS], rung_s[MAGUS_MAX_LEVELS];
    __shared__ int last_s;
    const DevModel &M = p.model;
    const int K = M.K;
    // this CTA's part of a trace: blocks of 2048 deltas [first, first + count)
    const StaticItem it = p.items[blockIdx.x];
    const int64_t trace = it.trace;
    const uint32_t *tr = p.traces + p.offsets[trace];
    const uint64_t len = p.lengths[trace];
    const uint64_t start = (uint64_t)it.first * 2048;
    const uint64_t n = min(len, start + (uint64_t)it.count * 2048);   // end of the part
    // thread i takes deltas 4i .. 4i+3 of every 512 (the packed layout pads each trace to a
    // multiple of 32 deltas, so whole 16-byte loads stay inside it): the first 2048 deltas'
    // loads are issued before the tables are set up, each next 2048's before a block is charged
    const uint32_t lo4 = 4u * threadIdx.x;
    uint4 v[4];
    if (start + 2048 <= n) {
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldg(reinterpret_cast<const uint4 *>(tr + start + 512u * u + lo4));
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
    // their count (at most kMaxPartBlocks * 16 deltas per thread keep both exact)
    unsigned long long *pk = st_s + threadIdx.x;
    for (int r = 0; r <= K; r++) pk[r * kThreads] = 0;
    __syncthreads();
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
    uint64_t base = start;
    if (start + 2048 <= n) {
        for (;;) {
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
            if (!more) break;
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = w[u];
        }
    }
    for (; base < n; base += 512) {   // at most 12 deltas per thread
        const uint64_t e = base + lo4;
        if (e >= n) continue;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tr + e));
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (e + (uint64_t)j < n) charge(vv[j]);
    }
    __syncthreads();
    // the columns' totals: four threads per r, 32 columns each (rotated: few bank conflicts)
    for (int t0 = 0; t0 < 4 * (K + 1); t0 += kThreads) {
        const int t = t0 + (int)threadIdx.x;
        const int r = t >> 2, q = t & 3;
        unsigned long long cs = 0, cn = 0;
        if (t < 4 * (K + 1)) {
            const unsigned long long *col = st_s + (size_t)r * kThreads + 32 * q;
            for (int i = 0; i < 32; i++) {
                const unsigned long long w = col[(i + r + 8 * q) & 31];
                cs += w & kSumMask;
                cn += w >> kSumBits;
            }
        }
        cs += __shfl_xor_sync(0xffffffffu, cs, 1);
        cs += __shfl_xor_sync(0xffffffffu, cs, 2);
        cn += __shfl_xor_sync(0xffffffffu, cn, 1);
        cn += __shfl_xor_sync(0xffffffffu, cn, 2);
        if (t < 4 * (K + 1) && q == 0) {
            red_n[r] = cn;
            red_s[r] = cs;
        }
    }
    __syncthreads();
    // the CTA's totals per r; a trace in several parts adds them to its accumulators, and
    // the part that arrives last charges the rungs from those
    if (it.parts > 1 && threadIdx.x <= (unsigned)K) {
        const int r = threadIdx.x;
        unsigned long long *acc = p.acc + (size_t)trace * 2 * (MAGUS_MAX_LEVELS + 1);
        atomicAdd(acc + r, red_n[r]);
        atomicAdd(acc + MAGUS_MAX_LEVELS + 1 + r, red_s[r]);
    }
    if (it.parts > 1) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last_s = atomicAdd(p.arrived + trace, 1u) == it.parts - 1u;
        __syncthreads();
        if (!last_s) return;
        __threadfence();
        if (threadIdx.x <= (unsigned)K) {
            const unsigned long long *acc = p.acc + (size_t)trace * 2 * (MAGUS_MAX_LEVELS + 1);
            red_n[threadIdx.x] = __ldcg(acc + threadIdx.x);
            red_s[threadIdx.x] = __ldcg(acc + MAGUS_MAX_LEVELS + 1 + threadIdx.x);
        }
    }
    __syncthreads();
    // rung k: unstretched deltas have r <= k, stretched ones r > k
    if (threadIdx.x < (unsigned)K) {
        const int k = threadIdx.x;
        unsigned long long N = 0, S = 0;
        for (int r = 0; r <= K; r++) {
            if (r <= k) N += red_n[r];
            else S += red_s[r];
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

size_t static_smem(int K) { return (size_t)(K + 1) * kThreads * sizeof(unsigned long long); }

}  // namespace

void static_items(const std::vector<uint64_t> &lengths, int sms, int K, std::vector<StaticItem> *out) {
    // resident CTAs per SM, per ladder size (the columns grow with K); asked once
    static std::atomic<int> resident[MAGUS_MAX_LEVELS + 1];
    int per_sm = K >= 1 && K <= MAGUS_MAX_LEVELS ? resident[K].load(std::memory_order_relaxed) : 0;
    if (per_sm < 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, replay_static_kernel<true>, kThreads,
                                                          static_smem(K)) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        } else if (K >= 1 && K <= MAGUS_MAX_LEVELS) {
            resident[K].store(per_sm, std::memory_order_relaxed);
        }
    }
    uint64_t total = 0;
    for (uint64_t n : lengths) total += n;
    // deltas per part: about four waves of CTAs, no part under 16 blocks
    const uint64_t waves = 4ull * (uint64_t)std::max(sms, 1) * (uint64_t)per_sm;
    const uint64_t target = std::min<uint64_t>(kMaxPartBlocks, std::max<uint64_t>(16, (total / waves + 2047) / 2048));
    // longest parts first (the last wave holds the short ones): a counting sort on the
    // block count, trace order within a count
    std::vector<uint32_t> at(kMaxPartBlocks + 2, 0);
    size_t n_items = 0;
    auto split = [&](uint64_t blocks, uint64_t *parts, uint64_t *per) {
        *parts = std::max<uint64_t>(1, (blocks + target - 1) / target);
        *per = (blocks + *parts - 1) / *parts;
        *parts = *per ? (blocks + *per - 1) / *per : 1;
    };
    for (uint64_t n : lengths) {
        const uint64_t blocks = (n + 2047) / 2048;
        uint64_t parts, per;
        split(blocks, &parts, &per);
        for (uint64_t j = 0; j < parts; j++) at[kMaxPartBlocks - std::min(per, blocks - j * per)]++;
        n_items += parts;
    }
    for (uint32_t c = 0, sum = 0; c < at.size(); c++) {   // slot of the first item per count
        const uint32_t k = at[c];
        at[c] = sum;
        sum += k;
    }
    out->resize(n_items);
    for (size_t t = 0; t < lengths.size(); t++) {
        const uint64_t blocks = (lengths[t] + 2047) / 2048;
        uint64_t parts, per;
        split(blocks, &parts, &per);
        for (uint64_t j = 0; j < parts; j++) {
            const uint64_t c = std::min(per, blocks - j * per);
            (*out)[at[kMaxPartBlocks - c]++] = StaticItem{(uint32_t)t, (uint32_t)(j * per), (uint32_t)c, (uint32_t)parts};
        }
    }
}

cudaError_t launch_replay_static(const StaticParams &p, cudaStream_t stream) {
    if (p.n_traces <= 0) return cudaSuccess;
    const size_t smem = static_smem(p.model.K);
    uint32_t shift = 0, n_cells = 0;
    const bool cells = choose_cells(p.model, &shift, &n_cells);
    cudaError_t e = cells ? cudaFuncSetAttribute(replay_static_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(replay_static_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!p.items) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)p.n_items;
    if (grid == 0) return cudaSuccess;
    if (cells)
        replay_static_kernel<true><<<grid, kThreads, smem, stream>>>(p, shift, n_cells);
    else
        replay_static_kernel<false><<<grid, kThreads, smem, stream>>>(p, 0, 1);
    return cudaGetLastError();
}

}  // namespace magus
