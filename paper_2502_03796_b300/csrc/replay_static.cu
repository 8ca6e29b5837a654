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
// the rung, so a delta a is stretched exactly at the rungs below r(a) = #{k : thr[k] < a}
// (a branch-free binary search over the thresholds in shared memory): each delta adds a to
// a sum and 1 to a count kept per r -- in registers while r repeats, else in shared-memory
// columns per thread -- and the rung totals are suffix / prefix sums of those at the end.
// Pins at a ladder bound in jump mode stay on the tile and segment kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"
#include "replay_core.cuh"

namespace magus {
namespace {

constexpr int kWarps = 4;   // per CTA (one trace)
constexpr int kThreads = kWarps * 32;

__global__ void __launch_bounds__(kThreads, 8) replay_static_kernel(const StaticParams p) {
    // per thread and r = 0 .. K: sums, then counts of the deltas with r thresholds below them
    extern __shared__ unsigned long long st_s[];
    __shared__ uint32_t thr_s[MAGUS_MAX_LEVELS];   // padded with never-exceeded thresholds
    __shared__ unsigned long long red_n[kWarps], red_s[kWarps];
    const DevModel &M = p.model;
    const int K = M.K;
    const int64_t trace = blockIdx.x;
    if (threadIdx.x < MAGUS_MAX_LEVELS) thr_s[threadIdx.x] = threadIdx.x < (unsigned)K ? M.thr[threadIdx.x] : 0xffffffffu;
    unsigned long long *ds = st_s + threadIdx.x;
    unsigned long long *dn = st_s + (size_t)(K + 1) * kThreads + threadIdx.x;
    for (int r = 0; r <= K; r++) {
        ds[r * kThreads] = 0;
        dn[r * kThreads] = 0;
    }
    __syncthreads();
    const uint32_t *tr = p.traces + p.offsets[trace];
    const uint64_t n = p.lengths[trace];
    // run of deltas in the same bucket, kept in registers
    int rc = 0;
    unsigned long long cs = 0, cn = 0;
    auto charge = [&](uint32_t a) {
        int r = 0;
#pragma unroll
        for (int step = MAGUS_MAX_LEVELS / 2; step > 0; step >>= 1) r += thr_s[r + step - 1] < a ? step : 0;
        if (r != rc) {
            ds[rc * kThreads] += cs;
            dn[rc * kThreads] += cn;
            rc = r;
            cs = 0;
            cn = 0;
        }
        cs += a;
        cn += 1;
    };
    // thread i takes deltas 4i .. 4i+3 of every 512 (the packed layout pads each trace to a
    // multiple of 32 deltas, so whole 16-byte loads stay inside it); four loads in flight
    const uint32_t lo4 = 4u * threadIdx.x;
    uint64_t base = 0;
    for (; base + 2048 <= n; base += 2048) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldg(reinterpret_cast<const uint4 *>(tr + base + 512u * u + lo4));
#pragma unroll
        for (int u = 0; u < 4; u++) {
            charge(v[u].x);
            charge(v[u].y);
            charge(v[u].z);
            charge(v[u].w);
        }
    }
    for (; base < n; base += 512) {
        const uint64_t e = base + lo4;
        if (e >= n) continue;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tr + e));
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (e + (uint64_t)j < n) charge(vv[j]);
    }
    ds[rc * kThreads] += cs;
    dn[rc * kThreads] += cn;
    // rung k: stretched deltas have r > k, unstretched ones r <= k
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long s_above = 0;
    for (int r = 1; r <= K; r++) s_above += ds[r * kThreads];
    unsigned long long n_upto = 0;
    for (int k = 0; k < K; k++) {
        n_upto += dn[k * kThreads];
        if (k > 0) s_above -= ds[k * kThreads];
        const unsigned long long wn = core::warp_sum_u64(n_upto), ws = core::warp_sum_u64(s_above);
        if (lane == 0) {
            red_n[warp] = wn;
            red_s[warp] = ws;
        }
        __syncthreads();
        unsigned long long N = 0, S = 0;
        for (int w = 0; w < kWarps; w++) {
            N += red_n[w];
            S += red_s[w];
        }
        __syncthreads();
        // every listed policy pinned at rung k
        for (int i = threadIdx.x; i < p.n_lit; i += kThreads) {
            const int pol = p.lit[i];
            const DevPolicy &P = p.pols[pol];
            if (!static_policy(P, K) || P.pin - 1 != k) continue;
            const int64_t pair = trace * p.n_pols + pol;
            const double T = M.dt * (double)N + M.ak[k] * (double)S;
            const double E = M.pw[k] * T;
            p.energy[pair] = E;
            p.edp[pair] = E * T;
            if (p.time) p.time[pair] = T;
            if (p.n_changes) p.n_changes[pair] = 0;
            if (p.change_hash) p.change_hash[pair] = 0;
            if (p.n_hf) p.n_hf[pair] = 0;
        }
    }
}

}  // namespace

cudaError_t launch_replay_static(const StaticParams &p, cudaStream_t stream) {
    if (p.n_traces <= 0) return cudaSuccess;
    const size_t smem = (size_t)(p.model.K + 1) * kThreads * 2 * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(replay_static_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    replay_static_kernel<<<(unsigned)p.n_traces, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace magus
