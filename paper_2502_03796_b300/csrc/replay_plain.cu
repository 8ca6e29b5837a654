// replay_plain.cu - the literal form of the MAGUS replay: one thread per (trace, policy)
// pair, every round evaluated literally in FP64 straight from global memory.
//
// Round t (Sec. 3 monitor, Sec. 3.1 Alg. 1, Sec. 3.2 Alg. 2, Sec. 6.1 actuation):
//   x = bpc * delta_t / q;  charge interval t at the current level;
//   FIFO of W+1 throughputs -> derivative = (newest - oldest) / W -> +1 / -1 / 0;
//   FIFO of L flags (prediction != 0) -> high-frequency iff sum / L >= threshold;
//   high-frequency -> top; +1 -> top (or one rung up); -1 -> bottom (or one rung down).
// Two kernels share the per-pair routine:
//   * replay_plain_kernel: one launch per trace, one thread per policy -- the baseline the
//     time-parallel kernel is measured against and the source of per-interval detail
//     (level and derivative logs);
//   * replay_literal_kernel: one launch over all traces for the policies the time-parallel
//     kernels do not replay (pins inside the ladder in jump mode, pins in the other modes;
//     the closed loop when its segmented replay is switched off or over budget), with
//     carried state.
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

struct LitOut {
    double *energy, *edp, *time;
    uint32_t *log;           // this pair's log, or NULL
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    uint8_t *level_log;
    double *deriv_log;
    int *status;
};

// One pair, rounds in order.  st (optional): carried state, read at the start and written
// at the end (the FIFO of throughputs is rebuilt from the last deltas; a closed loop would
// also need the levels of those intervals, so it only starts from a fresh state).
// kDirect: the plain form -- every expression evaluated as written (divisions included).
// Otherwise the same decisions without divisions on the round-to-round chain: Alg. 1
// compares the FP64 difference with thresholds equivalent to RN(d / W) > inc and < dec,
// Alg. 2 compares the flag count with kmin, and the energy is charged as integer counts and
// stretched-delta sums per level (E and T formed once, within 1e-15 relative of the
// sequential FP64 sums).
template <bool kDirect>
__device__ void replay_pair_literal(const uint32_t *trace, uint64_t n, const DevPolicy &P, const DevModel &M,
                                    int64_t pair, const LitOut &o, magus_state_t *st) {
    const int W = P.W, L = P.L, K = M.K;
    const bool pinned = P.pin > 0;
    const bool ladder = (P.step_mode & 1) != 0, closed = (P.step_mode & 2) != 0;
    double ls[MAGUS_MAX_WINDOW + 1];   // mem_throughput_ls ring
    int ls_len = 0, ls_head = 0;       // head = index of the oldest entry
    uint64_t tune = 0;                 // flag history, bit 0 = newest
    const uint64_t tmask = L == 64 ? ~0ull : ((1ull << L) - 1ull);
    int level = 0;
    uint64_t n_seen0 = 0;
    if (st) {
        n_seen0 = st->n_seen;
        if (closed && n_seen0 > 0) {
            atomicCAS(o.status, 0, MAGUS_EINVAL);
            return;
        }
        level = (int)st->level;
        if (level >= K && !pinned) {
            atomicCAS(o.status, 0, MAGUS_EINVAL);
            level = 0;
        }
        tune = __brevll(st->flags);
        // the last min(n_seen, W) throughputs (a full FIFO drops its oldest before the
        // next push, so W of them decide the next round)
        const int k0 = (int)(n_seen0 < (uint64_t)W ? n_seen0 : (uint64_t)W);
        for (int j = 0; j < k0; j++) ls[j] = __ddiv_rn(__dmul_rn(M.bpc, (double)st->hist[64 - k0 + j]), M.q);
        ls_len = k0;
    }
    // a static baseline (Sec. 5.3, Sec. 6.3) holds its ladder index and runs no control
    if (pinned) level = P.pin - 1;
    double E = 0.0, T = 0.0;
    uint64_t nch = 0, hash = 0, nhf = 0;
    // integer energy per level (kDirect == false): counts of unstretched intervals and sums
    // of stretched deltas, flushed per run of constant level
    uint64_t lv_n[kDirect ? 1 : MAGUS_MAX_LEVELS], lv_s[kDirect ? 1 : MAGUS_MAX_LEVELS];
    uint64_t run_n = 0, run_s = 0;
    uint32_t thr_cur = 0;
    if (!kDirect) {
        for (int k = 0; k < K; k++) lv_n[k] = lv_s[k] = 0;
        thr_cur = M.thr[level];
    }
    double x_next = n ? __ddiv_rn(__dmul_rn(M.bpc, (double)trace[0]), M.q) : 0.0;
    for (uint64_t t = 0; t < n; t++) {
        const uint32_t delta = trace[t];
        const double x = kDirect ? __ddiv_rn(__dmul_rn(M.bpc, (double)delta), M.q) : x_next;
        // the next round's throughput does not depend on this round's decision
        if (!kDirect && t + 1 < n) x_next = __ddiv_rn(__dmul_rn(M.bpc, (double)trace[t + 1]), M.q);
        // energy model: interval t at `level`
        if (kDirect) {
            double s = __ddiv_rn(x, M.cap[level]);
            if (s < 1.0) s = 1.0;
            const double tau = __dmul_rn(M.dt, s);
            T = __dadd_rn(T, tau);
            E = __dadd_rn(E, __dmul_rn(M.pw[level], tau));
        } else {
            const bool stretched = delta > thr_cur;
            run_n += stretched ? 0u : 1u;
            run_s += stretched ? delta : 0u;
        }
        if (o.level_log) o.level_log[t] = (uint8_t)level;
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
            const double d = __dsub_rn(ls[newest], ls[ls_head]);
            if (kDirect) {
                der = __ddiv_rn(d, (double)W);
                pred = der > P.inc ? 1 : (der < P.dec ? -1 : 0);
            } else {
                pred = d > P.up_last ? 1 : (d <= P.dn_last ? -1 : 0);
            }
        }
        if (o.deriv_log) o.deriv_log[t] = der;
        // Alg. 2: FIFO of L flags, zero-filled
        tune = (tune << 1) | (pred != 0 ? 1ull : 0ull);
        bool hf;
        if (kDirect) hf = !pinned && __ddiv_rn((double)__popcll(tune & tmask), (double)L) >= P.th;
        else hf = !pinned && __popcll(tune & tmask) >= P.kmin;
        nhf += hf ? 1 : 0;
        int next;
        if (pinned) next = level;
        else if (hf) next = K - 1;
        else if (pred == 1) next = !ladder ? K - 1 : (level + 1 < K ? level + 1 : K - 1);
        else if (pred == -1) next = !ladder ? 0 : (level > 0 ? level - 1 : 0);
        else next = level;
        if (next != level) {
            const uint64_t when = n_seen0 + t + 1;
            if (o.log && nch < o.log_cap) o.log[nch] = (uint32_t)(when << 5) | (uint32_t)next;
            nch++;
            hash += mix64_plain((when << 8) | (uint64_t)next);
            if (!kDirect) {
                lv_n[level] += run_n;
                lv_s[level] += run_s;
                run_n = run_s = 0;
                thr_cur = M.thr[next];
            }
        }
        level = next;
    }
    if (!kDirect) {
        lv_n[level] += run_n;
        lv_s[level] += run_s;
        for (int k = 0; k < K; k++) {
            const double tk = M.dt * (double)lv_n[k] + M.ak[k] * (double)lv_s[k];
            T += tk;
            E += M.pw[k] * tk;
        }
    }
    o.energy[pair] = E;
    o.edp[pair] = __dmul_rn(E, T);
    if (o.time) o.time[pair] = T;
    if (o.n_changes) o.n_changes[pair] = nch;
    if (o.change_hash) o.change_hash[pair] = hash;
    if (o.n_hf) o.n_hf[pair] = nhf;
    if (st && n > 0) {
        st->n_seen = n_seen0 + n;
        st->level = (uint32_t)level;
        st->flags = __brevll(tune);
        // last 64 deltas of (previous ones, this trace); hist[n + k] is read before it could
        // be overwritten (n >= 1)
        for (int k = 0; k < 64; k++) {
            const int64_t idx = (int64_t)n - 64 + k;
            st->hist[k] = idx >= 0 ? trace[idx] : st->hist[64 + idx];
        }
    }
}

__global__ void replay_plain_kernel(const PlainParams p) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_pols) return;
    const DevPolicy P = p.pols[c];
    const int64_t pair = p.pair_base + c;
    LitOut o;
    o.energy = p.energy;
    o.edp = p.edp;
    o.time = p.time;
    o.log = p.log_entries ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
    o.log_cap = p.log_cap;
    o.n_changes = p.n_changes;
    o.change_hash = p.change_hash;
    o.n_hf = p.n_hf;
    o.level_log = p.level_log;
    o.deriv_log = p.deriv_log;
    o.status = nullptr;
    replay_pair_literal<true>(p.trace, p.n, P, p.model, pair, o, nullptr);
}

__global__ void replay_literal_kernel(const LiteralParams p) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)p.n_traces * p.n_lit) return;
    const int64_t trace = k / p.n_lit;
    const int pol = p.lit[k % p.n_lit];
    const DevPolicy P = p.pols[pol];
    if (p.skip_pinned && P.pin > 0) return;   // replayed by the static kernel
    const int64_t pair = trace * p.n_pols + pol;
    LitOut o;
    o.energy = p.energy;
    o.edp = p.edp;
    o.time = p.time;
    o.log = p.log_entries ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
    o.log_cap = p.log_cap;
    o.n_changes = p.n_changes;
    o.change_hash = p.change_hash;
    o.n_hf = p.n_hf;
    o.level_log = nullptr;
    o.deriv_log = nullptr;
    o.status = p.status;
    replay_pair_literal<false>(p.traces + p.offsets[trace], p.lengths[trace], P, p.model, pair, o,
                               p.state ? p.state + pair : nullptr);
}

}  // namespace

cudaError_t launch_replay_plain(const PlainParams &p, cudaStream_t stream) {
    const int block = p.n_pols < 128 ? ((p.n_pols + 31) / 32) * 32 : 128;
    const int grid = (p.n_pols + block - 1) / block;
    replay_plain_kernel<<<grid, block, 0, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_replay_literal(const LiteralParams &p, cudaStream_t stream) {
    const int64_t threads = (int64_t)p.n_traces * p.n_lit;
    if (threads <= 0) return cudaSuccess;
    // one latency-bound chain per thread: one warp per block spreads the pairs over all SMs
    const int block = 32;
    replay_literal_kernel<<<(unsigned)((threads + block - 1) / block), block, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace magus
