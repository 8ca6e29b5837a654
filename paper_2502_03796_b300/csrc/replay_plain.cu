// replay_plain.cu - the plain form of the MAGUS replay: one launch per trace, one thread
// per policy, every round evaluated literally in FP64 straight from global memory.
//
// Round t (Sec. 3 monitor, Sec. 3.1 Alg. 1, Sec. 3.2 Alg. 2, Sec. 6.1 actuation):
//   x = bpc * delta_t / q;  charge interval t at the current level;
//   FIFO of W+1 throughputs -> derivative = (newest - oldest) / W -> +1 / -1 / 0;
//   FIFO of L flags (prediction != 0) -> high-frequency iff sum / L >= threshold;
//   high-frequency -> top; +1 -> top (or one rung up); -1 -> bottom (or one rung down).
// This kernel is the baseline the time-parallel kernel is measured against and the
// source of per-interval detail (level and derivative logs).
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"

namespace magus {
namespace {

__device__ __forceinline__ uint64_t mix64_plain(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void replay_plain_kernel(const PlainParams p) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_pols) return;
    const DevPolicy P = p.pols[c];
    const DevModel &M = p.model;
    const int W = P.W, L = P.L, K = M.K;
    const int64_t pair = p.pair_base + c;
    double ls[MAGUS_MAX_WINDOW + 1];   // mem_throughput_ls ring
    int ls_len = 0, ls_head = 0;       // head = index of the oldest entry
    uint64_t tune = 0;                 // uncore_tune_ls, bit 0 = newest
    const uint64_t tmask = L == 64 ? ~0ull : ((1ull << L) - 1ull);
    // a static baseline (Sec. 5.3, Sec. 6.3) holds its ladder index and runs no control
    const bool pinned = P.pin > 0;
    const bool ladder = (P.step_mode & 1) != 0, closed = (P.step_mode & 2) != 0;
    int level = pinned ? P.pin - 1 : 0;
    double E = 0.0, T = 0.0;
    uint64_t nch = 0, hash = 0, nhf = 0;
    for (uint64_t t = 0; t < p.n; t++) {
        const double x = __ddiv_rn(__dmul_rn(M.bpc, (double)p.trace[t]), M.q);
        // energy model: interval t at `level`
        double s = __ddiv_rn(x, M.cap[level]);
        if (s < 1.0) s = 1.0;
        const double tau = __dmul_rn(M.dt, s);
        T = __dadd_rn(T, tau);
        E = __dadd_rn(E, __dmul_rn(M.pw[level], tau));
        if (p.level_log) p.level_log[t] = (uint8_t)level;
        // Alg. 1: FIFO of W+1 throughputs
        if (ls_len == W + 1) {
            ls_head = ls_head == W ? 0 : ls_head + 1;
            ls_len = W;
        }
        int tail = ls_head + ls_len;
        if (tail > W) tail -= W + 1;
        // closed loop: the monitor reads what the uncore at `level` delivered
        ls[tail] = (closed && x > M.cap[level]) ? M.cap[level] : x;
        ls_len++;
        int pred = 0;
        double der = __longlong_as_double(0x7ff8000000000000ll);
        if (ls_len == W + 1) {
            const int newest = ls_head == 0 ? W : ls_head - 1;
            der = __ddiv_rn(__dsub_rn(ls[newest], ls[ls_head]), (double)W);
            pred = der > P.inc ? 1 : (der < P.dec ? -1 : 0);
        }
        if (p.deriv_log) p.deriv_log[t] = der;
        // Alg. 2: FIFO of L flags, zero-filled
        tune = ((tune << 1) | (pred != 0 ? 1ull : 0ull)) & tmask;
        const double freq = __ddiv_rn((double)__popcll(tune), (double)L);
        const bool hf = !pinned && freq >= P.th;
        nhf += hf ? 1 : 0;
        int next;
        if (pinned) next = level;
        else if (hf) next = K - 1;
        else if (pred == 1) next = !ladder ? K - 1 : (level + 1 < K ? level + 1 : K - 1);
        else if (pred == -1) next = !ladder ? 0 : (level > 0 ? level - 1 : 0);
        else next = level;
        if (next != level) {
            const uint64_t when = t + 1;
            if (p.log_entries && nch < p.log_cap)
                p.log_entries[(uint64_t)pair * p.log_cap + nch] = (uint32_t)(when << 5) | (uint32_t)next;
            nch++;
            hash += mix64_plain((when << 8) | (uint64_t)next);
        }
        level = next;
    }
    p.energy[pair] = E;
    p.edp[pair] = __dmul_rn(E, T);
    if (p.time) p.time[pair] = T;
    if (p.n_changes) p.n_changes[pair] = nch;
    if (p.change_hash) p.change_hash[pair] = hash;
    if (p.n_hf) p.n_hf[pair] = nhf;
}

}  // namespace

cudaError_t launch_replay_plain(const PlainParams &p, cudaStream_t stream) {
    const int block = p.n_pols < 128 ? ((p.n_pols + 31) / 32) * 32 : 128;
    const int grid = (p.n_pols + block - 1) / block;
    replay_plain_kernel<<<grid, block, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace magus
