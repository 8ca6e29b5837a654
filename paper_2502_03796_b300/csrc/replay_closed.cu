// replay_closed.cu - time-parallel replay of the closed loop in jump mode.
//
// In the closed loop the monitor reads what the uncore at the level in effect delivers,
// min(demand, capacity) (Sec. 3 monitor, Sec. 6.3 on the throttled minimum frequency), so a
// round's prediction (Sec. 3.1, Alg. 1) depends on past levels and the open-loop latch
// decomposition does not apply.  What a round needs from the past is small, though: the
// level, the levels of the last W rounds (which of the throughputs in Alg. 1's window were
// capped) and the last L flags (Sec. 3.2, Alg. 2).  Two replays that agree on that state at
// one round agree from then on.
//
// Every (pair, time segment) is therefore replayed on its own thread:
//   pass 1  from a guessed state `burn` rounds before the segment (bottom level, no flags;
//           the true initial state when that reaches round 0), recording the state reached
//           at the segment's start, its charges, change entries and end state;
//   pass 2  a segment whose recorded start state differs from the end state of the segment
//           before it (pass 1) is replayed again from that end state;
//   final   one thread per pair walks its segments in order from the true initial state,
//           takes a replay whose start state equals the state reached so far, replays the
//           segment once more where neither does, and adds up charges and change entries.
// The final walk makes the result exact whatever the guesses; the guesses only decide how
// much is replayed twice.
//
// Alg. 1 runs on integers: a throughput is capped exactly when its delta exceeds a
// per-level threshold, each case with one capped throughput is a threshold on the other
// delta and both capped is a constant (host-derived with the oracle's FP64 expressions,
// plan.cu); two uncapped throughputs take the open-loop test with its FP64 evaluation
// inside the rounding band.  Energy is charged as integer counts and sums per level.
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"
#include "replay_core.cuh"

namespace magus {
namespace {

constexpr int kThreads = 128;

struct CState {
    uint32_t lv;     // 0 bottom, 1 top
    uint64_t lvh;    // bit j: level bit of round t-1-j
    uint64_t fl;     // bit j: flag of round t-1-j
};

struct CAcc {
    uint32_t n0, nm, nhf, nch;
    unsigned long long s0, sm, hash;
};

__device__ __forceinline__ bool same_state(const CState &x, const CState &y, uint64_t wmask, uint64_t lmask) {
    return x.lv == y.lv && ((x.lvh ^ y.lvh) & wmask) == 0 && ((x.fl ^ y.fl) & lmask) == 0;
}
__device__ __forceinline__ uint64_t low_mask(int k) { return k >= 64 ? ~0ull : ((1ull << k) - 1ull); }

// The pair's state before round 0: fresh, or the carried one (which must not have seen a
// round: the throughput FIFO would need the levels behind it).  A carried level other than
// the bottom or the top is invalid in jump mode.
__device__ CState initial_state(const ClosedParams &p, int64_t pair) {
    CState s{0u, 0ull, 0ull};
    if (p.state) {
        const magus_state_t &st = p.state[pair];
        if (st.n_seen > 0) atomicCAS(p.status, 0, MAGUS_EINVAL);
        const uint32_t top = (uint32_t)(p.model.K - 1);
        if (st.level != 0 && st.level != top) atomicCAS(p.status, 0, MAGUS_EINVAL);
        s.lv = st.level == top ? 1u : 0u;
        s.fl = __brevll(st.flags);
    }
    return s;
}

// Per-thread ring of the last R deltas in shared memory, slot-major ([slot][thread]): the
// lanes of a warp always touch distinct banks.
struct Ring {
    uint32_t *col;     // this thread's column
    uint32_t mask;     // R - 1
    __device__ __forceinline__ uint32_t &at(uint64_t t) const { return col[((uint32_t)t & mask) * kThreads]; }
};

__device__ __forceinline__ void prefill(const uint32_t *tr, uint64_t t0, const Ring &ring) {
    const uint64_t h0 = t0 > ring.mask ? t0 - ring.mask - 1 : 0;
    for (uint64_t t = h0; t < t0; t++) ring.at(t) = __ldg(tr + t);
}

// Rounds [t0, t1) of one pair's trace from state s (t0 a multiple of 4; the packed layout
// pads every trace to a multiple of 32 deltas, so the 16-byte loads stay inside it).
// kCount: charge the rounds, count flags and changes, emit change entries.
template <bool kCount, class Emit>
__device__ __forceinline__ void run_rounds(const uint32_t *tr, uint64_t t0, uint64_t t1, CState &s, CAcc &acc,
                                           const DevPolicy &P, const ClosedThr &C, const DevModel &M,
                                           const Ring &ring, Emit emit) {
    const int W = P.W;
    const uint64_t lmask = low_mask(P.L);
    const uint32_t topK = (uint32_t)(M.K - 1);
#pragma unroll 1
    for (uint64_t tq = t0; tq < t1; tq += 4) {
        const uint4 v4 = __ldg(reinterpret_cast<const uint4 *>(tr + tq));
        const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint64_t t = tq + (uint64_t)j;
            if (t >= t1) break;
            const uint32_t a = vv[j];
            const uint32_t b = ring.at(t - (uint64_t)W);   // read before round t's slot is reused
            ring.at(t) = a;
            const uint32_t lv = s.lv;
            const uint32_t lb = (uint32_t)(s.lvh >> (W - 1)) & 1u;   // level of round t - W
            // Alg. 1 on obs_t = min(x_t, C(lv)) and obs_{t-W} = min(x_{t-W}, C(lb))
            bool up = false, dn = false;
            if (t >= (uint64_t)W) {
                const bool ca = a > (lv ? C.cthr[1] : C.cthr[0]);
                const bool cb = b > (lb ? C.cthr[1] : C.cthr[0]);
                if (!ca && !cb) {
                    core::predict_exact(a, b, P, M, up, dn);
                } else if (ca && cb) {
                    const uint32_t k = 2u * lv + lb;
                    up = (C.cc >> k) & 1u;
                    dn = (C.cc >> (4u + k)) & 1u;
                } else if (ca) {
                    up = (int64_t)b < (lv ? C.bu[1] : C.bu[0]);
                    dn = (int64_t)b >= (lv ? C.bd[1] : C.bd[0]);
                } else {
                    up = (int64_t)a >= (lb ? C.au[1] : C.au[0]);
                    dn = (int64_t)a < (lb ? C.ad[1] : C.ad[0]);
                }
                dn = dn && !up;   // Alg. 1 tests +1 first
            }
            // Alg. 2: the flag enters the list, then the share of flagged rounds is tested
            s.fl = (s.fl << 1) | ((up || dn) ? 1ull : 0ull);
            const bool hf = __popcll(s.fl & lmask) >= P.kmin;
            const uint32_t next = (hf || up) ? 1u : (dn ? 0u : lv);
            if (kCount) {
                // energy model: round t at level lv, stretched when the demand exceeds C(lv)
                const bool se = a > (lv ? M.thrM : M.thr0);
                if (lv) {
                    acc.nm += se ? 0u : 1u;
                    acc.sm += se ? a : 0u;
                } else {
                    acc.n0 += se ? 0u : 1u;
                    acc.s0 += se ? a : 0u;
                }
                acc.nhf += hf ? 1u : 0u;
                if (next != lv) {
                    const uint64_t when = t + 1;   // the new level governs the next round
                    const uint32_t lvl = next ? topK : 0u;
                    emit((uint32_t)(when << 5) | lvl, acc.nch);
                    acc.nch++;
                    acc.hash += core::mix64((when << 8) | lvl);
                }
            }
            s.lvh = (s.lvh << 1) | lv;
            s.lv = next;
        }
    }
}

struct NoEmit {
    __device__ __forceinline__ void operator()(uint32_t, uint32_t) const {}
};
struct BufEmit {
    uint32_t *buf;
    uint64_t cap;
    __device__ __forceinline__ void operator()(uint32_t e, uint32_t i) const {
        if (buf && i < cap) buf[i] = e;
    }
};

struct ItemPos {
    int trace, ci;
    uint64_t k, nseg;
};
__device__ ItemPos locate(const ClosedParams &p, uint64_t item) {
    int lo = 0, hi = p.n_traces;   // ibase[lo] <= item < ibase[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (p.ibase[mid] <= item) lo = mid;
        else hi = mid;
    }
    ItemPos q;
    q.trace = lo;
    q.nseg = (p.lengths[lo] + p.seg_len - 1) / p.seg_len;
    const uint64_t r = item - p.ibase[lo];
    q.ci = (int)(r / q.nseg);
    q.k = r % q.nseg;
    return q;
}

__device__ __forceinline__ void store_slot(ClosedSlot &o, const CState &in, const CState &out, const CAcc &acc,
                                           uint32_t ok) {
    o.s0 = acc.s0;
    o.sm = acc.sm;
    o.hash = acc.hash;
    o.lvh_in = in.lvh;
    o.fl_in = in.fl;
    o.lvh_out = out.lvh;
    o.fl_out = out.fl;
    o.n0 = acc.n0;
    o.nm = acc.nm;
    o.nhf = acc.nhf;
    o.nch = acc.nch;
    o.lv_in = in.lv;
    o.lv_out = out.lv;
    o.pad = 0;
    o.ok = ok;
}

// pass 1 (first replay of every segment) and pass 2 (second replay where pass 1 started
// from a state other than its predecessor's end state)
__global__ void __launch_bounds__(kThreads, 5) closed_pass_kernel(const ClosedParams p, int pass) {
    extern __shared__ uint32_t ring_s[];
    const uint64_t item = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (item >= p.n_items) return;
    const ItemPos q = locate(p, item);
    const int pol = p.cls[q.ci];
    const DevPolicy P = p.pols[pol];
    const ClosedThr C = p.thr[q.ci];
    const DevModel &M = p.model;
    const int64_t pair = (int64_t)q.trace * p.n_pols + pol;
    const uint32_t *tr = p.traces + p.offsets[q.trace];
    const uint64_t n = p.lengths[q.trace];
    const uint64_t s0 = q.k * p.seg_len, s1 = min(n, s0 + p.seg_len);
    ClosedSlot &out = p.slots[(uint64_t)(pass - 1) * p.n_items + item];
    const Ring ring{ring_s + threadIdx.x, p.ring - 1u};
    CState st;
    uint32_t ok = 1u;
    if (pass == 1) {
        const uint64_t t0 = s0 > p.burn ? s0 - p.burn : 0;
        if (t0 == 0) {
            st = initial_state(p, pair);
            ok |= 2u;   // started from the true state
        } else {
            st = CState{0u, 0ull, 0ull};
        }
        prefill(tr, t0, ring);
        CAcc none{};
        run_rounds<false>(tr, t0, s0, st, none, P, C, M, ring, NoEmit{});
    } else {
        if (q.k == 0) {
            out.ok = 0;
            return;
        }
        const ClosedSlot &prev = p.slots[item - 1];   // segment k - 1, pass 1
        const ClosedSlot &mine = p.slots[item];
        const CState e{prev.lv_out, prev.lvh_out, prev.fl_out};
        const CState u{mine.lv_in, mine.lvh_in, mine.fl_in};
        if ((mine.ok & 2u) || same_state(e, u, low_mask(P.W), low_mask(P.L))) {
            out.ok = 0;
            return;
        }
        st = e;
        prefill(tr, s0, ring);
        atomicAdd(&p.stats[0], 1ull);
    }
    const CState in = st;
    CAcc acc{};
    BufEmit em{p.scratch ? p.scratch + ((uint64_t)(pass - 1) * p.n_items + item) * p.scr_cap : nullptr, p.scr_cap};
    run_rounds<true>(tr, s0, s1, st, acc, P, C, M, ring, em);
    if (p.scratch && acc.nch > p.scr_cap) ok |= 4u;   // entries lost: the final pass replays it
    store_slot(out, in, st, acc, ok);
}

// Final pass: one thread per (trace, closed-loop policy) pair.
__global__ void __launch_bounds__(kThreads) closed_final_kernel(const ClosedParams p) {
    extern __shared__ uint32_t ring_s[];
    const int64_t id = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (id >= (int64_t)p.n_traces * p.n_cls) return;
    const int trace = (int)(id / p.n_cls), ci = (int)(id % p.n_cls);
    const int pol = p.cls[ci];
    const int64_t pair = (int64_t)trace * p.n_pols + pol;
    if (p.state && p.state[pair].n_seen > 0) {
        atomicCAS(p.status, 0, MAGUS_EINVAL);
        return;
    }
    const DevPolicy P = p.pols[pol];
    const ClosedThr C = p.thr[ci];
    const DevModel &M = p.model;
    const uint32_t *tr = p.traces + p.offsets[trace];
    const uint64_t n = p.lengths[trace];
    const uint64_t nseg = (n + p.seg_len - 1) / p.seg_len;
    const uint64_t item0 = p.ibase[trace] + (uint64_t)ci * nseg;
    const uint64_t wmask = low_mask(P.W), lmask = low_mask(P.L);
    const bool logging = p.log_entries && p.log_cap > 0;
    uint32_t *lg = logging ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
    const Ring ring{ring_s + threadIdx.x, p.ring - 1u};
    CState E = initial_state(p, pair);
    uint64_t N0 = 0, NM = 0, NHF = 0, NCH = 0;
    unsigned long long S0 = 0, SM = 0, HS = 0;
    for (uint64_t k = 0; k < nseg; k++) {
        const uint64_t item = item0 + k;
        const ClosedSlot *pick = nullptr;
        uint64_t which = 0;
        for (uint64_t w = 0; w < 2 && !pick; w++) {
            const ClosedSlot &c = p.slots[w * p.n_items + item];
            if (!(c.ok & 1u) || (logging && (c.ok & 4u))) continue;
            const CState u{c.lv_in, c.lvh_in, c.fl_in};
            if ((c.ok & 2u) || same_state(E, u, wmask, lmask)) {
                pick = &c;
                which = w;
            }
        }
        if (pick) {
            if (logging) {
                const uint32_t *src = p.scratch + (which * p.n_items + item) * p.scr_cap;
                for (uint32_t j = 0; j < pick->nch && NCH + j < p.log_cap; j++) lg[NCH + j] = src[j];
            }
            N0 += pick->n0;
            NM += pick->nm;
            NHF += pick->nhf;
            NCH += pick->nch;
            S0 += pick->s0;
            SM += pick->sm;
            HS += pick->hash;
            E = CState{pick->lv_out, pick->lvh_out, pick->fl_out};
        } else {
            // neither replay started from the state reached here: replay the segment now
            const uint64_t s0 = k * p.seg_len, s1 = min(n, s0 + p.seg_len);
            prefill(tr, s0, ring);
            CAcc acc{};
            BufEmit em{lg ? lg + NCH : nullptr, NCH < p.log_cap ? p.log_cap - NCH : 0};
            run_rounds<true>(tr, s0, s1, E, acc, P, C, M, ring, em);
            N0 += acc.n0;
            NM += acc.nm;
            NHF += acc.nhf;
            NCH += acc.nch;
            S0 += acc.s0;
            SM += acc.sm;
            HS += acc.hash;
            atomicAdd(&p.stats[1], 1ull);
        }
    }
    double En, T;
    core::totals(M, N0, NM, S0, SM, &En, &T);
    p.energy[pair] = En;
    p.edp[pair] = En * T;
    if (p.time) p.time[pair] = T;
    if (p.n_changes) p.n_changes[pair] = NCH;
    if (p.change_hash) p.change_hash[pair] = HS;
    if (p.n_hf) p.n_hf[pair] = NHF;
    if (p.state && n > 0) {
        magus_state_t &so = p.state[pair];
        so.n_seen = n;
        so.level = E.lv ? (uint32_t)(M.K - 1) : 0u;
        so.flags = __brevll(E.fl);
        // last 64 deltas (earlier carried ones first when the trace is shorter); hist[n + k]
        // is read before it could be overwritten (n >= 1)
        for (int k = 0; k < 64; k++) {
            const int64_t idx = (int64_t)n - 64 + k;
            so.hist[k] = idx >= 0 ? tr[idx] : so.hist[64 + idx];
        }
    }
}

}  // namespace

int closed_threads_per_cta() { return kThreads; }

cudaError_t launch_replay_closed(const ClosedParams &p, cudaStream_t stream) {
    const size_t smem = (size_t)p.ring * kThreads * sizeof(uint32_t);
    if (p.n_items) {
        const uint64_t grid = (p.n_items + kThreads - 1) / kThreads;
        closed_pass_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(p, 1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        closed_pass_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(p, 2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t pairs = (int64_t)p.n_traces * p.n_cls;
    if (pairs > 0) {
        closed_final_kernel<<<(unsigned)((pairs + kThreads - 1) / kThreads), kThreads, smem, stream>>>(p);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace magus
