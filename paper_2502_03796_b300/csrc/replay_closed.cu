// replay_closed.cu - time-parallel replay of the closed loop, jump and one-rung modes.
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
//   log     with a change log, segments whose entries overflowed their replay's scratch are
//           replayed once more from their true start state, writing straight to the log.
// The final walk makes the result exact whatever the guesses; the guesses only decide how
// much is replayed twice.  A second replay runs in lockstep with a repeat of the first one
// and stops once their states agree: from there on the first replay's charges and entries
// stand, so a wrong guess costs the rounds until the two trajectories meet, not a segment.
//
// Alg. 1 runs on integers: a throughput is capped exactly when its delta exceeds a
// per-level threshold, each case with one capped throughput is a threshold on the other
// delta and both capped is a constant (host-derived with the oracle's FP64 expressions,
// plan.cu); two uncapped throughputs take the open-loop test with its FP64 evaluation
// inside the rounding band.  Jump mode (kL = false) keeps the level as a bit and the levels
// of the last 64 rounds in a word, and charges energy as integer counts and sums at the two
// levels; one rung per decision (kL = true) keeps the rung and a shared-memory ring of past
// rungs, and charges energy as integer counts and sums per rung in shared memory (FP64 once
// per segment: B300's FP64 pipe is too narrow for a charge at every rung change).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "replay_closed.h"
#include "replay_core.cuh"

namespace magus {
namespace {

constexpr int kThreads = 128;

struct CState {
    uint32_t lv;     // jump: 0 bottom / 1 top; one-rung: the rung
    uint64_t lvh;    // jump: bit j = level bit of round t-1-j (one-rung: in the ring)
    uint64_t fl;     // bit j: flag of round t-1-j
};

struct CAcc {
    uint32_t n0, nm, nhf, nch;
    unsigned long long s0, sm, hash;
    double e, t;     // one-rung mode: energy and time
};

__device__ __forceinline__ uint64_t low_mask(int k) { return k >= 64 ? ~0ull : ((1ull << k) - 1ull); }
__device__ __forceinline__ bool same_state(const CState &x, const CState &y, uint64_t wmask, uint64_t lmask) {
    return x.lv == y.lv && ((x.lvh ^ y.lvh) & wmask) == 0 && ((x.fl ^ y.fl) & lmask) == 0;
}
__device__ __forceinline__ bool same_hist(const uint8_t *a, const uint8_t *b, int W) {
    for (int j = 0; j < W; j++)
        if (a[j] != b[j]) return false;
    return true;
}

// The pair's state before round 0: fresh, or the carried one (which must not have seen a
// round: the throughput FIFO would need the levels behind it).  Jump mode: a carried level
// other than the bottom or the top is invalid; one-rung mode: any rung of the ladder.
template <bool kL>
__device__ CState initial_state(const ClosedParams &p, int64_t pair) {
    CState s{0u, 0ull, 0ull};
    if (p.state) {
        const magus_state_t &st = p.state[pair];
        if (st.n_seen > 0) atomicCAS(p.status, 0, MAGUS_EINVAL);
        const uint32_t top = (uint32_t)(p.model.K - 1);
        if (kL) {
            if (st.level > top) atomicCAS(p.status, 0, MAGUS_EINVAL);
            s.lv = st.level > top ? 0u : st.level;
        } else {
            if (st.level != 0 && st.level != top) atomicCAS(p.status, 0, MAGUS_EINVAL);
            s.lv = st.level == top ? 1u : 0u;
        }
        s.fl = __brevll(st.flags);
    }
    return s;
}

// Per-thread rings in shared memory, slot-major ([slot][thread]) so that the lanes of a warp
// always touch distinct banks (bytes of a word for the rung rings): the last R deltas, and
// in one-rung mode the rungs of the last R rounds of one or two replays.
struct Ring {
    uint32_t *col;     // this thread's delta column
    uint32_t mask;     // R - 1
    __device__ __forceinline__ uint32_t &at(uint64_t t) const { return col[((uint32_t)t & mask) * kThreads]; }
};
struct LRing {
    uint8_t *col;      // this thread's rung column (NULL in jump mode)
    uint32_t mask;
    __device__ __forceinline__ uint8_t &at(uint64_t t) const { return col[((uint32_t)t & mask) * kThreads]; }
};
// Shared memory of the one-rung kernels: delta ring [R][threads] u32 | per replay: sums of
// stretched deltas per rung [K][threads] u64 | counts of unstretched rounds [K][threads]
// u32 | rung ring [R][threads] u8 (8-byte multiples throughout).
__device__ __forceinline__ Ring delta_ring(uint32_t *smem, uint32_t R) { return Ring{smem + threadIdx.x, R - 1u}; }
__host__ __device__ constexpr size_t rung_block_bytes(uint32_t R, int K) {
    return (size_t)K * kThreads * (sizeof(uint64_t) + sizeof(uint32_t)) + (size_t)R * kThreads;
}
__device__ __forceinline__ unsigned char *rung_block(uint32_t *smem, uint32_t R, int K, int which) {
    return reinterpret_cast<unsigned char *>(smem + (size_t)R * kThreads) + (size_t)which * rung_block_bytes(R, K);
}

__device__ __forceinline__ void prefill(const uint32_t *tr, uint64_t t0, const Ring &ring) {
    const uint64_t h0 = t0 > ring.mask ? t0 - ring.mask - 1 : 0;
    for (uint64_t t = h0; t < t0; t++) ring.at(t) = __ldg(tr + t);
}
// rungs of the W rounds before t0 (newest first) into / out of a ring (NULL: all bottom)
__device__ __forceinline__ void hist_to_ring(const LRing &r, uint64_t t0, const uint8_t *h, int W) {
    for (int j = 0; j < W; j++) r.at(t0 - 1 - (uint64_t)j) = h ? h[j] : (uint8_t)0;
}
__device__ __forceinline__ void ring_to_hist(const LRing &r, uint64_t t1, uint8_t *h, int W) {
    for (int j = 0; j < W; j++) h[j] = r.at(t1 - 1 - (uint64_t)j);
}

// Alg. 1 for two uncapped throughputs inside the rounding band around a threshold: the FP64
// evaluation in the oracle's order (rare; kept out of the round loop).  Bit 0: +1, bit 1: -1.
static __device__ __noinline__ uint32_t predict_band(uint32_t a, uint32_t b, const DevPolicy *Pg, double bpc,
                                                      double q) {
    const double xa = __ddiv_rn(__dmul_rn(bpc, (double)a), q);
    const double xb = __ddiv_rn(__dmul_rn(bpc, (double)b), q);
    const double der = __ddiv_rn(__dsub_rn(xa, xb), (double)Pg->W);
    return (der > Pg->inc ? 1u : 0u) | (der < Pg->dec ? 2u : 0u);
}

struct NoEmit {
    __device__ __forceinline__ void operator()(uint32_t, uint32_t) const {}
};
struct BufEmit {
    uint32_t *buf;
    uint32_t cap;
    __device__ __forceinline__ void operator()(uint32_t e, uint32_t i) const {
        if (buf && i < cap) buf[i] = e;
    }
};

// One replay of a pair over consecutive rounds: its state, its charges (energy per run of
// constant level: count of unstretched rounds, sum of stretched deltas) and change entries.
// The thresholds of the level in effect (lv) and of the level W rounds back (lb) are kept
// in registers and reloaded when that level changes; the flag count of Alg. 2's window is
// kept up to date instead of recounted.
template <bool kL>
struct Replay {
    CState s;
    CAcc acc;
    uint32_t run_n;
    unsigned long long run_s;
    uint32_t capa, ccu, ccd, thr;   // level lv: capped above capa; both capped: bit lb +1 / -1
    int64_t bu, bd;                 // a capped, b not: +1 iff b < bu, -1 iff b >= bd
    uint32_t lbp, capb;             // level lb (as last loaded): capped above capb
    int64_t au, ad;                 // b capped, a not: +1 iff a >= au, -1 iff a < ad
    uint32_t cnt;                   // flags among the last L rounds
    LRing lr;                       // one-rung mode: this replay's rungs
    unsigned long long *rs;         // one-rung mode: stretched-delta sum per rung (stride kThreads)
    uint32_t *rn;                   //                unstretched rounds per rung

    // one-rung mode: rings and accumulators of replay `which` of this thread
    __device__ __forceinline__ void bind(uint32_t *smem, uint32_t R, int K, int which) {
        if (kL) {
            unsigned char *b = rung_block(smem, R, K, which);
            rs = reinterpret_cast<unsigned long long *>(b) + threadIdx.x;
            rn = reinterpret_cast<uint32_t *>(b + (size_t)K * kThreads * 8) + threadIdx.x;
            lr = LRing{b + (size_t)K * kThreads * 12 + threadIdx.x, R - 1u};
        } else {
            rs = nullptr;
            rn = nullptr;
            lr = LRing{nullptr, 0u};
        }
    }

    __device__ __forceinline__ void load_a(const ClosedThr *Cg, const DevModel &M) {
        capa = __ldg(&Cg->cthr[s.lv]);
        bu = __ldg(&Cg->bu[s.lv]);
        bd = __ldg(&Cg->bd[s.lv]);
        ccu = __ldg(&Cg->ccu[s.lv]);
        ccd = __ldg(&Cg->ccd[s.lv]);
        thr = kL ? M.thr[s.lv] : (s.lv ? M.thrM : M.thr0);
    }
    __device__ __forceinline__ void load_b(const ClosedThr *Cg) {
        capb = __ldg(&Cg->cthr[lbp]);
        au = __ldg(&Cg->au[lbp]);
        ad = __ldg(&Cg->ad[lbp]);
    }
    __device__ __forceinline__ uint32_t level_back(uint64_t t, uint32_t W) const {
        return kL ? (uint32_t)lr.at(t - W) : ((uint32_t)(s.lvh >> (W - 1u)) & 1u);
    }
    // state at round t0 (one-rung mode: its rungs already in lr)
    __device__ __forceinline__ void start(const CState &st, uint64_t t0, const DevPolicy &P, const ClosedThr *Cg,
                                          const DevModel &M) {
        s = st;
        acc = CAcc{};
        run_n = 0;
        run_s = 0;
        load_a(Cg, M);
        lbp = level_back(t0, (uint32_t)P.W);
        load_b(Cg);
        cnt = (uint32_t)__popcll(s.fl & low_mask(P.L));
        if (kL)
            for (int k = 0; k < M.K; k++) {
                rs[k * kThreads] = 0;
                rn[k * kThreads] = 0;
            }
    }
    __device__ __forceinline__ void flush(const DevModel &M) {
        if (kL) {
            rn[s.lv * kThreads] += run_n;
            rs[s.lv * kThreads] += run_s;
        } else if (s.lv) {
            acc.nm += run_n;
            acc.sm += run_s;
        } else {
            acc.n0 += run_n;
            acc.s0 += run_s;
        }
        run_n = 0;
        run_s = 0;
    }
    // one-rung mode: energy and time from the per-rung counts (after the last flush)
    __device__ __forceinline__ void finish(const DevModel &M) {
        if (!kL) return;
        double e = 0.0, t = 0.0;
        for (int k = 0; k < M.K; k++) {
            const double tk = M.dt * (double)rn[k * kThreads] + M.ak[k] * (double)rs[k * kThreads];
            t += tk;
            e += M.pw[k] * tk;
        }
        acc.e = e;
        acc.t = t;
    }
    // Round t = t0 + j with a = delta_t, b = delta_{t-W} and lb the level of round t - W.
    // kCount: charge it, count its flag and change, emit its entry.  kWarm: rounds j < warm
    // come before the FIFO holds W + 1.
    template <bool kCount, bool kWarm, class Emit>
    __device__ __forceinline__ void step(uint32_t a, uint32_t b, uint32_t lb, uint32_t j, uint64_t t0, uint32_t warm,
                                         const DevPolicy &P, const DevPolicy *Pg, const ClosedThr *Cg,
                                         const DevModel &M, Emit emit) {
        const uint64_t t = t0 + j;
        const uint32_t lv = s.lv;
        if (lb != lbp) {
            lbp = lb;
            load_b(Cg);
        }
        // Alg. 1 on obs_t = min(x_t, C(lv)) and obs_{t-W} = min(x_{t-W}, C(lb)); every case
        // evaluated, one selected
        const bool ca = a > capa, cb = b > capb;
        const int64_t m = (int64_t)a - (int64_t)b;
        const bool up_b = ca ? ((ccu >> lb) & 1u) != 0 : (int64_t)a >= au;
        const bool dn_b = ca ? ((ccd >> lb) & 1u) != 0 : (int64_t)a < ad;
        const bool up_n = ca ? (int64_t)b < bu : m > P.up_mid;
        const bool dn_n = ca ? (int64_t)b >= bd : m < P.dn_mid;
        bool up = cb ? up_b : up_n, dn = cb ? dn_b : dn_n;
        const uint32_t m32 = a - b;
        if (!(ca | cb) && ((m32 - P.up_lo) <= P.up_w || (m32 - P.dn_lo) <= P.dn_w)) {
            const uint32_t r = predict_band(a, b, Pg, M.bpc, M.q);
            up = (r & 1u) != 0;
            dn = (r & 2u) != 0;
        }
        if (kWarm && j < warm) up = dn = false;
        dn = dn && !up;   // Alg. 1 tests +1 first
        // Alg. 2: the flag enters the list (the one L rounds back leaves it), then the share
        // of flagged rounds is tested
        const uint32_t f = (up || dn) ? 1u : 0u;
        const uint32_t gone = (uint32_t)(s.fl >> (P.L - 1)) & 1u;
        s.fl = (s.fl << 1) | f;
        cnt = cnt + f - gone;
        const bool hf = (int)cnt >= P.kmin;
        uint32_t next;
        if (kL) {
            // one rung per decision; the high-frequency state goes to the top (Sec. 3.2)
            const uint32_t top = (uint32_t)(M.K - 1);
            next = hf ? top : (up ? (lv < top ? lv + 1u : top) : (dn ? (lv > 0 ? lv - 1u : 0u) : lv));
        } else {
            next = (hf || up) ? 1u : (dn ? 0u : lv);
        }
        if (kCount) {
            // energy model: the round at level lv, stretched when the demand exceeds C(lv)
            const bool se = a > thr;
            run_n += se ? 0u : 1u;
            run_s += se ? a : 0u;
            acc.nhf += hf ? 1u : 0u;
        }
        if (kL) lr.at(t) = (uint8_t)lv;
        else s.lvh = (s.lvh << 1) | lv;
        if (next != lv) {
            if (kCount) {
                flush(M);
                const uint64_t when = t + 1;   // the new level governs the next round
                const uint32_t lvl = kL ? next : (next ? (uint32_t)(M.K - 1) : 0u);
                emit((uint32_t)(when << 5) | lvl, acc.nch);
                acc.nch++;
                acc.hash += core::mix64((when << 8) | lvl);
            }
            s.lv = next;
            load_a(Cg, M);
        }
    }
};

// Rounds [t0, t1) of one pair's trace (t0 a multiple of 4, t1 - t0 < 2^32; the packed layout
// pads every trace to a multiple of 32 deltas, so the 16-byte loads stay inside it).  The
// delta ring holds the deltas before t0; x has been started.
template <bool kL, bool kCount, class Emit>
__device__ __forceinline__ void run_rounds(const uint32_t *tr, uint64_t t0, uint64_t t1, Replay<kL> &x,
                                           const DevPolicy *Pg, const ClosedThr *Cg, const DevModel &M,
                                           const Ring &ring, Emit emit) {
    const DevPolicy P = *Pg;
    const uint32_t W = (uint32_t)P.W;
    const uint32_t nr = (uint32_t)(t1 - t0);
    const uint32_t warm = t0 < W ? (uint32_t)(W - t0) : 0u;   // rounds before the FIFO holds W + 1
    uint32_t j = 0;
    // one-rung mode: the rung of round t - W is fetched a round ahead (for W = 1 it is the
    // rung in effect now; otherwise its ring slot was written rounds before and is not the
    // one this round writes), off the round's dependency chain
    uint32_t lbn = kL ? x.level_back(t0, W) : 0u;
    auto lb_of = [&](uint32_t jj) -> uint32_t {
        if (!kL) return x.level_back(t0 + jj, W);
        const uint32_t lb = lbn;
        lbn = W == 1u ? x.s.lv : (uint32_t)x.lr.at(t0 + jj + 1u - W);
        return lb;
    };
    // the rounds before the FIFO fills (a trace's first W), to a multiple of 4
    const uint32_t jw = min(nr, (warm + 3u) & ~3u);
#pragma unroll 1
    for (; j < jw; j++) {
        const uint32_t a = __ldg(tr + t0 + j);
        const uint32_t b = ring.at(t0 + j - W);
        ring.at(t0 + j) = a;
        const uint32_t lb = lb_of(j);
        x.template step<kCount, true>(a, b, lb, j, t0, warm, P, Pg, Cg, M, emit);
    }
    auto round = [&](uint32_t a, uint32_t jj) {
        const uint32_t b = ring.at(t0 + jj - W);   // read before round t's slot is reused (W may equal R)
        ring.at(t0 + jj) = a;
        const uint32_t lb = lb_of(jj);
        x.template step<kCount, false>(a, b, lb, jj, t0, 0u, P, Pg, Cg, M, emit);
    };
#pragma unroll 1
    for (; j + 4u <= nr; j += 4u) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tr + t0 + j));
        round(v.x, j);
        round(v.y, j + 1u);
        round(v.z, j + 2u);
        round(v.w, j + 3u);
    }
#pragma unroll 1
    for (; j < nr; j++) round(__ldg(tr + t0 + j), j);
    if (kCount) {
        x.flush(M);
        x.finish(M);
    }
}

// Rounds [t0, t1) with W = WK known at compile time: the deltas W rounds back come from a
// register window of the last WK + 4 deltas instead of the shared-memory ring (no ring
// stores, no slot addresses).  The level W rounds back: jump mode, a fixed bit of the level
// history; one rung per decision, the rung ring as in run_rounds.  Same alignment as
// run_rounds; x has been started.
template <bool kL, int WK, bool kCount, class Emit>
__device__ __forceinline__ void run_rounds_w(const uint32_t *tr, uint64_t t0, uint64_t t1, Replay<kL> &x,
                                             const DevPolicy *Pg, const ClosedThr *Cg, const DevModel &M,
                                             Emit emit) {
    const DevPolicy P = *Pg;
    const uint32_t nr = (uint32_t)(t1 - t0);
    const uint32_t warm = t0 < (uint64_t)WK ? (uint32_t)(WK - t0) : 0u;   // rounds before the FIFO holds W + 1
    // w[i]: the delta of round t - WK + i, t the first round of the group of four in hand
    uint32_t w[WK + 4];
#pragma unroll
    for (int i = 0; i < WK; i++) w[i] = t0 + i >= (uint64_t)WK ? __ldg(tr + t0 + i - WK) : 0u;
    // one-rung mode: the rung of round t - W fetched a round ahead, as in run_rounds
    uint32_t lbn = kL ? x.level_back(t0, WK) : 0u;
    auto lb_of = [&](uint32_t jj) -> uint32_t {
        if (!kL) return (uint32_t)(x.s.lvh >> (WK - 1)) & 1u;
        const uint32_t lb = lbn;
        lbn = WK == 1 ? x.s.lv : (uint32_t)x.lr.at(t0 + jj + 1u - WK);
        return lb;
    };
    // a group of four rounds; kEdge: the trace's first rounds (FIFO filling) or the last,
    // partial group (rounds past t1 are left out; the packed layout pads every trace to a
    // multiple of 32 deltas, so the 16-byte load stays inside it)
    auto group = [&](uint32_t j, auto edge) {
        constexpr bool kEdge = decltype(edge)::value;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tr + t0 + j));
        w[WK] = v.x;
        w[WK + 1] = v.y;
        w[WK + 2] = v.z;
        w[WK + 3] = v.w;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (kEdge && j + k >= nr) break;
            const uint32_t lb = lb_of(j + (uint32_t)k);
            x.template step<kCount, kEdge>(w[WK + k], w[k], lb, j + (uint32_t)k, t0, warm, P, Pg, Cg, M, emit);
        }
#pragma unroll
        for (int i = 0; i < WK; i++) w[i] = w[i + 4];
    };
    uint32_t j = 0;
#pragma unroll 1
    for (; j < nr && j < warm; j += 4u) group(j, std::true_type{});
#pragma unroll 1
    for (; j + 4u <= nr; j += 4u) group(j, std::false_type{});
    if (j < nr) group(j, std::true_type{});
    if (kCount) {
        x.flush(M);
        x.finish(M);
    }
}

// Rounds [t0, t1) replayed twice in lockstep: x (charged, entries emitted) and y (charged,
// no entries: it repeats an earlier replay) until their states agree, checked every 8
// rounds -- the level, the levels of the last W rounds and all 64 flags (the carried state
// written at a trace's end holds 64).  Returns the rounds run (both replays then hold the
// state after them, runs flushed); t1 - t0 when they never agreed.  Both have been started.
template <bool kL, class Emit>
__device__ __forceinline__ uint32_t run_until_same(const uint32_t *tr, uint64_t t0, uint64_t t1, Replay<kL> &x,
                                                   Replay<kL> &y, const DevPolicy *Pg, const ClosedThr *Cg,
                                                   const DevModel &M, const Ring &ring, Emit emit) {
    const DevPolicy P = *Pg;
    const uint64_t wmask = low_mask(P.W);
    const uint32_t W = (uint32_t)P.W;
    const uint32_t nr = (uint32_t)(t1 - t0);
    const uint32_t warm = t0 < W ? (uint32_t)(W - t0) : 0u;
    // one-rung mode: rungs that differ among the last W rounds of the two replays
    int diff = 0;
    if (kL)
        for (uint32_t i = 1; i <= W; i++) diff += x.lr.at(t0 - i) != y.lr.at(t0 - i) ? 1 : 0;
    uint32_t j = 0;
#pragma unroll 1
    while (j < nr) {
        const uint32_t je = min(nr, j + 8u);
#pragma unroll 1
        for (; j < je; j++) {
            const uint32_t a = __ldg(tr + t0 + j);
            const uint32_t b = ring.at(t0 + j - W);
            ring.at(t0 + j) = a;
            const uint32_t xl = x.s.lv, yl = y.s.lv;
            const uint32_t xb = x.level_back(t0 + j, W), yb = y.level_back(t0 + j, W);
            x.template step<true, true>(a, b, xb, j, t0, warm, P, Pg, Cg, M, emit);
            y.template step<true, true>(a, b, yb, j, t0, warm, P, Pg, Cg, M, NoEmit{});
            if (kL) diff += (xl != yl ? 1 : 0) - (xb != yb ? 1 : 0);
        }
        if (kL ? (x.s.lv == y.s.lv && x.s.fl == y.s.fl && diff == 0) : same_state(x.s, y.s, wmask, ~0ull)) break;
    }
    x.flush(M);
    y.flush(M);
    x.finish(M);
    y.finish(M);
    return j;
}

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

// rung histories of a slot (one-rung mode): io 0 at its start, 1 at its end
__device__ __forceinline__ uint8_t *slot_hist(const ClosedParams &p, uint64_t which, uint64_t item, int io) {
    return p.lhist + ((which * p.n_items + item) * 2 + (uint64_t)io) * MAGUS_MAX_WINDOW;
}

__device__ __forceinline__ void store_counts(ClosedSlot &o, const CAcc &acc) {
    o.s0 = acc.s0;
    o.sm = acc.sm;
    o.hash = acc.hash;
    o.e = acc.e;
    o.t = acc.t;
    o.n0 = acc.n0;
    o.nm = acc.nm;
    o.nhf = acc.nhf;
    o.nch = acc.nch;
}
__device__ __forceinline__ void store_in(ClosedSlot &o, const CState &in) {
    o.lv_in = in.lv;
    o.lvh_in = in.lvh;
    o.fl_in = in.fl;
}
__device__ __forceinline__ void store_out(ClosedSlot &o, const CState &out, uint32_t ok) {
    o.lv_out = out.lv;
    o.lvh_out = out.lvh;
    o.fl_out = out.fl;
    o.pad = 0;
    o.ok = ok;
}
__device__ __forceinline__ CAcc slot_acc(const ClosedSlot &r) {
    CAcc a;
    a.n0 = r.n0;
    a.nm = r.nm;
    a.nhf = r.nhf;
    a.nch = r.nch;
    a.s0 = r.s0;
    a.sm = r.sm;
    a.hash = r.hash;
    a.e = r.e;
    a.t = r.t;
    return a;
}
__device__ __forceinline__ CAcc acc_add_diff(const CAcc &x, const ClosedSlot &r, const CAcc &y) {
    CAcc o;
    o.n0 = x.n0 + (r.n0 - y.n0);
    o.nm = x.nm + (r.nm - y.nm);
    o.nhf = x.nhf + (r.nhf - y.nhf);
    o.nch = x.nch + (r.nch - y.nch);
    o.s0 = x.s0 + (r.s0 - y.s0);
    o.sm = x.sm + (r.sm - y.sm);
    o.hash = x.hash + (r.hash - y.hash);
    o.e = x.e + (r.e - y.e);
    o.t = x.t + (r.t - y.t);
    return o;
}

// Pass 1: the first replay of every segment.  Pass 2: a second replay where pass 1 started
// from a state other than its predecessor's end state.  Separate kernels, so that the
// lockstep replay of pass 2 does not raise the register count of pass 1.
// WK > 0 (first pass): every policy of the call has W = WK, and the rounds run from a register
// window of deltas (run_rounds_w) without the shared-memory delta ring.
template <bool kL, int kPass, int WK = 0>
__device__ __forceinline__ void closed_pass(const ClosedParams &p) {
    extern __shared__ uint32_t ring_s[];
    const uint64_t item = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (item >= p.n_items) return;
    const ItemPos q = locate(p, item);
    const int pol = p.cls[q.ci];
    const DevPolicy *Pg = p.pols + pol;
    const ClosedThr *C = p.thr + q.ci;
    const DevModel &M = p.model;
    const int W = Pg->W;
    const int64_t pair = (int64_t)q.trace * p.n_pols + pol;
    const uint32_t *tr = p.traces + p.offsets[q.trace];
    const uint64_t n = p.lengths[q.trace];
    const uint64_t s0 = q.k * p.seg_len, s1 = min(n, s0 + p.seg_len);
    ClosedSlot &out = p.slots[(uint64_t)(kPass - 1) * p.n_items + item];
    const Ring ring = delta_ring(ring_s, p.ring);
    const bool logging = p.log_entries && p.log_cap > 0;
    uint32_t *scr = p.scratch ? p.scratch + ((uint64_t)(kPass - 1) * p.n_items + item) * p.scr_cap : nullptr;
    const BufEmit em{scr, (uint32_t)p.scr_cap};   // scr_cap <= segment rounds < 2^32
    Replay<kL> x;
    x.bind(ring_s, p.ring, p.model.K, 0);
    if constexpr (kPass == 1) {
        uint32_t ok = 1u;
        const uint64_t t0 = s0 > p.burn ? s0 - p.burn : 0;
        CState st{0u, 0ull, 0ull};
        if (t0 == 0) {
            st = initial_state<kL>(p, pair);
            ok |= 2u;   // started from the true state
        }
        if constexpr (WK > 0) {
            if (kL) hist_to_ring(x.lr, t0, nullptr, W);
            x.start(st, t0, *Pg, C, M);
            run_rounds_w<kL, WK, false>(tr, t0, s0, x, Pg, C, M, NoEmit{});
            store_in(out, x.s);
            if (kL) ring_to_hist(x.lr, s0, slot_hist(p, 0, item, 0), W);
            x.start(x.s, s0, *Pg, C, M);
            run_rounds_w<kL, WK, true>(tr, s0, s1, x, Pg, C, M, em);
        } else {
            prefill(tr, t0, ring);
            if (kL) hist_to_ring(x.lr, t0, nullptr, W);
            x.start(st, t0, *Pg, C, M);
            run_rounds<kL, false>(tr, t0, s0, x, Pg, C, M, ring, NoEmit{});
            // the start state goes out now (fewer live registers through the segment)
            store_in(out, x.s);
            if (kL) ring_to_hist(x.lr, s0, slot_hist(p, 0, item, 0), W);
            x.start(x.s, s0, *Pg, C, M);
            run_rounds<kL, true>(tr, s0, s1, x, Pg, C, M, ring, em);
        }
        if (logging && x.acc.nch > p.scr_cap) ok |= 4u;   // entries lost: the log pass writes them
        store_counts(out, x.acc);
        if (kL) ring_to_hist(x.lr, s1, slot_hist(p, 0, item, 1), W);
        store_out(out, x.s, ok);
    } else {
        if (q.k == 0) {
            out.ok = 0;
            return;
        }
        const ClosedSlot &prev = p.slots[item - 1];   // segment k - 1, pass 1
        const ClosedSlot &mine = p.slots[item];
        const CState e{prev.lv_out, prev.lvh_out, prev.fl_out};
        const CState u{mine.lv_in, mine.lvh_in, mine.fl_in};
        const uint8_t *eh = kL ? slot_hist(p, 0, item - 1, 1) : nullptr;
        const uint8_t *uh = kL ? slot_hist(p, 0, item, 0) : nullptr;
        if ((mine.ok & 2u) ||
            (same_state(e, u, low_mask(W), low_mask(Pg->L)) && (!kL || same_hist(eh, uh, W)))) {
            out.ok = 0;
            return;
        }
        atomicAdd(&p.stats[0], 1ull);
        prefill(tr, s0, ring);
        Replay<kL> y;
        y.bind(ring_s, p.ring, p.model.K, 1);
        if (kL) {
            hist_to_ring(x.lr, s0, eh, W);
            hist_to_ring(y.lr, s0, uh, W);
        }
        x.start(e, s0, *Pg, C, M);
        y.start(u, s0, *Pg, C, M);
        CAcc acc;
        CState end;
        bool lost = false;   // entries incomplete
        const uint32_t r = run_until_same(tr, s0, s1, x, y, Pg, C, M, ring, em);
        const bool met = r < (uint32_t)(s1 - s0);
        if (met) {
            // from round s0 + r on the first replay stands: its charges, entries, end state
            acc = acc_add_diff(x.acc, mine, y.acc);
            end = CState{mine.lv_out, mine.lvh_out, mine.fl_out};
            lost = (mine.ok & 4u) != 0;
            if (scr && !lost) {
                const uint32_t *src = p.scratch + item * p.scr_cap;
                for (uint32_t i = y.acc.nch; i < mine.nch; i++) {
                    const uint64_t d = (uint64_t)x.acc.nch + (i - y.acc.nch);
                    if (d < p.scr_cap) scr[d] = src[i];
                }
            }
        } else {
            acc = x.acc;
            end = x.s;
        }
        lost = lost || acc.nch > p.scr_cap;
        store_in(out, e);
        store_counts(out, acc);
        if (kL) {
            uint8_t *ih = slot_hist(p, 1, item, 0), *oh = slot_hist(p, 1, item, 1);
            for (int i = 0; i < W; i++) ih[i] = eh[i];
            if (met) {
                const uint8_t *mh = slot_hist(p, 0, item, 1);
                for (int i = 0; i < W; i++) oh[i] = mh[i];
            } else {
                ring_to_hist(x.lr, s1, oh, W);
            }
        }
        store_out(out, end, 1u | ((logging && lost) ? 4u : 0u));
    }
}
template <bool kL, int WK = 0>
__global__ void __launch_bounds__(kThreads, 5) closed_first_kernel(const ClosedParams p) {
    closed_pass<kL, 1, WK>(p);
}
template <bool kL>
__global__ void __launch_bounds__(kThreads) closed_second_kernel(const ClosedParams p) {
    closed_pass<kL, 2>(p);
}

// Final pass: one thread per (trace, closed-loop policy) pair.
template <bool kL>
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
    const DevPolicy *Pg = p.pols + pol;
    const ClosedThr *C = p.thr + ci;
    const DevModel &M = p.model;
    const int W = Pg->W;
    const uint32_t *tr = p.traces + p.offsets[trace];
    const uint64_t n = p.lengths[trace];
    const uint64_t nseg = (n + p.seg_len - 1) / p.seg_len;
    const uint64_t item0 = p.ibase[trace] + (uint64_t)ci * nseg;
    const uint64_t wmask = low_mask(W), lmask = low_mask(Pg->L);
    const bool logging = p.log_entries && p.log_cap > 0;
    uint32_t *lg = logging ? p.log_entries + (uint64_t)pair * p.log_cap : nullptr;
    const Ring ring = delta_ring(ring_s, p.ring);
    CState E = initial_state<kL>(p, pair);
    uint8_t Eh[kL ? MAGUS_MAX_WINDOW : 1];   // one-rung mode: rungs of the W rounds before
    if (kL)
        for (int i = 0; i < W; i++) Eh[i] = 0;
    uint64_t N0 = 0, NM = 0, NHF = 0, NCH = 0;
    unsigned long long S0 = 0, SM = 0, HS = 0;
    double ET = 0.0, TT = 0.0;
    auto add = [&](const CAcc &a) {
        N0 += a.n0;
        NM += a.nm;
        NHF += a.nhf;
        NCH += a.nch;
        S0 += a.s0;
        SM += a.sm;
        HS += a.hash;
        ET += a.e;
        TT += a.t;
    };
    // copy entries [i0, i1) of a replay's scratch to the log at entry `at`
    auto copy = [&](uint64_t which, uint64_t item, uint32_t i0, uint32_t i1, uint64_t at) {
        const uint32_t *src = p.scratch + (which * p.n_items + item) * p.scr_cap;
        for (uint32_t i = i0; i < i1 && at + (i - i0) < p.log_cap; i++) lg[at + (i - i0)] = src[i];
    };
    auto take_hist = [&](const uint8_t *h) {
        for (int i = 0; i < W; i++) Eh[i] = h[i];
    };
    for (uint64_t k = 0; k < nseg; k++) {
        const uint64_t item = item0 + k;
        const uint64_t s0 = k * p.seg_len, s1 = min(n, s0 + p.seg_len);
        // a replay's end state holds 64 flags of its own: after fewer rounds than that, the
        // last segment must have started with all 64 flags right for the written state
        const uint64_t fmask = (k + 1 == nseg && s1 - s0 < 64 && p.state) ? ~0ull : lmask;
        const ClosedSlot *pick = nullptr;
        uint64_t which = 0;
        for (uint64_t w = 0; w < 2 && !pick; w++) {
            const ClosedSlot &c = p.slots[w * p.n_items + item];
            if (!(c.ok & 1u)) continue;
            const CState u{c.lv_in, c.lvh_in, c.fl_in};
            if ((c.ok & 2u) ||
                (same_state(E, u, wmask, fmask) && (!kL || same_hist(Eh, slot_hist(p, w, item, 0), W)))) {
                pick = &c;
                which = w;
            }
        }
        // with a log: the segment's entries come from a replay's scratch, else (it overflowed)
        // from the log pass, replaying the segment from the state reached here
        if (logging) {
            ClosedJob &jb = p.jobs[item];
            jb.on = 0;
            if (pick ? (pick->ok & 4u) != 0 : (p.slots[item].ok & 4u) != 0) {
                jb.lvh = E.lvh;
                jb.fl = E.fl;
                jb.lv = E.lv;
                jb.off = NCH;
                if (kL)
                    for (int i = 0; i < W; i++) jb.hist[i] = Eh[i];
                jb.on = 1;
            }
        }
        if (pick) {
            if (logging && !(pick->ok & 4u)) copy(which, item, 0, pick->nch, NCH);
            add(slot_acc(*pick));
            E = CState{pick->lv_out, pick->lvh_out, pick->fl_out};
            if (kL) take_hist(slot_hist(p, which, item, 1));
            continue;
        }
        // neither replay started from the state reached here: replay the segment now,
        // alongside a repeat of the first replay until the two agree
        atomicAdd(&p.stats[1], 1ull);
        const ClosedSlot &first = p.slots[item];
        prefill(tr, s0, ring);
        const BufEmit em{lg ? lg + NCH : nullptr,
                         NCH < p.log_cap ? (uint32_t)min(p.log_cap - NCH, (uint64_t)0xffffffffull) : 0u};
        Replay<kL> x, y;
        x.bind(ring_s, p.ring, p.model.K, 0);
        y.bind(ring_s, p.ring, p.model.K, 1);
        if (kL) {
            hist_to_ring(x.lr, s0, Eh, W);
            hist_to_ring(y.lr, s0, slot_hist(p, 0, item, 0), W);
        }
        x.start(E, s0, *Pg, C, M);
        y.start(CState{first.lv_in, first.lvh_in, first.fl_in}, s0, *Pg, C, M);
        const uint32_t r = run_until_same(tr, s0, s1, x, y, Pg, C, M, ring, em);
        if (r < (uint32_t)(s1 - s0)) {
            // (entries of an overflowed first replay: the log pass writes the segment)
            if (logging && !(first.ok & 4u)) copy(0, item, y.acc.nch, first.nch, NCH + x.acc.nch);
            add(acc_add_diff(x.acc, first, y.acc));
            E = CState{first.lv_out, first.lvh_out, first.fl_out};
            if (kL) take_hist(slot_hist(p, 0, item, 1));
        } else {
            if (logging) p.jobs[item].on = 0;   // every entry went straight to the log
            add(x.acc);
            E = x.s;
            if (kL) ring_to_hist(x.lr, s1, Eh, W);
        }
    }
    double En, T;
    if (kL) {
        En = ET;
        T = TT;
    } else {
        core::totals(M, N0, NM, S0, SM, &En, &T);
    }
    p.energy[pair] = En;
    p.edp[pair] = En * T;
    if (p.time) p.time[pair] = T;
    if (p.n_changes) p.n_changes[pair] = NCH;
    if (p.change_hash) p.change_hash[pair] = HS;
    if (p.n_hf) p.n_hf[pair] = NHF;
    if (p.state && n > 0) {
        magus_state_t &so = p.state[pair];
        so.n_seen = n;
        so.level = kL ? E.lv : (E.lv ? (uint32_t)(M.K - 1) : 0u);
        so.flags = __brevll(E.fl);
        // last 64 deltas (earlier carried ones first when the trace is shorter); hist[n + k]
        // is read before it could be overwritten (n >= 1)
        for (int k = 0; k < 64; k++) {
            const int64_t idx = (int64_t)n - 64 + k;
            so.hist[k] = idx >= 0 ? tr[idx] : so.hist[64 + idx];
        }
    }
}

// Log pass: the segments the final pass marked, replayed from their true start state with
// their entries written straight to the pair's log.
template <bool kL>
__global__ void __launch_bounds__(kThreads) closed_log_kernel(const ClosedParams p) {
    extern __shared__ uint32_t ring_s[];
    const uint64_t item = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (item >= p.n_items || !p.jobs[item].on) return;
    const ClosedJob &jb = p.jobs[item];
    const ItemPos q = locate(p, item);
    const int pol = p.cls[q.ci];
    const DevPolicy *Pg = p.pols + pol;
    const ClosedThr *C = p.thr + q.ci;
    const int64_t pair = (int64_t)q.trace * p.n_pols + pol;
    const uint32_t *tr = p.traces + p.offsets[q.trace];
    const uint64_t n = p.lengths[q.trace];
    const uint64_t s0 = q.k * p.seg_len, s1 = min(n, s0 + p.seg_len);
    if (jb.off >= p.log_cap) return;
    atomicAdd(&p.stats[2], 1ull);
    const Ring ring = delta_ring(ring_s, p.ring);
    prefill(tr, s0, ring);
    Replay<kL> x;
    x.bind(ring_s, p.ring, p.model.K, 0);
    if (kL) hist_to_ring(x.lr, s0, jb.hist, Pg->W);
    x.start(CState{jb.lv, jb.lvh, jb.fl}, s0, *Pg, C, p.model);
    const BufEmit em{p.log_entries + (uint64_t)pair * p.log_cap + jb.off,
                     (uint32_t)min(p.log_cap - jb.off, (uint64_t)0xffffffffull)};
    run_rounds<kL, true>(tr, s0, s1, x, Pg, C, p.model, ring, em);
}

// shared memory: the delta ring, and in one-rung mode the rung block of each replay a
// thread runs (one in the first and log kernels, two in the lockstep kernels)
template <bool kL>
size_t smem_of(uint32_t ring, int replays, int K) {
    return (size_t)ring * kThreads * sizeof(uint32_t) + (kL ? (size_t)replays * rung_block_bytes(ring, K) : 0);
}

// window lengths with their own first-replay kernel (jump mode)
#define MAGUS_CLOSED_WINDOWS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(16)

// the first-replay kernel for ClosedParams::window: its W instance (no shared memory) or the
// any-W kernel with the delta ring (smem bytes)
template <bool kL, int WK>
cudaError_t launch_first_t(const ClosedParams &p, size_t smem, unsigned grid, cudaStream_t stream) {
    const size_t sm = (WK > 0 && !kL) ? 0 : smem;   // one rung per decision keeps its rung block
    cudaError_t e = cudaFuncSetAttribute(closed_first_kernel<kL, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    closed_first_kernel<kL, WK><<<grid, kThreads, sm, stream>>>(p);
    return cudaGetLastError();
}
template <bool kL>
cudaError_t launch_first(const ClosedParams &p, size_t smem, unsigned grid, cudaStream_t stream) {
    switch (p.window) {
#define MAGUS_CLOSED_LAUNCH_W(w) \
        case w: return launch_first_t<kL, w>(p, smem, grid, stream);
        MAGUS_CLOSED_WINDOWS(MAGUS_CLOSED_LAUNCH_W)
#undef MAGUS_CLOSED_LAUNCH_W
        default: return launch_first_t<kL, 0>(p, smem, grid, stream);
    }
}

template <bool kL>
cudaError_t launch_t(const ClosedParams &p, cudaStream_t stream) {
    const size_t sm1 = smem_of<kL>(p.ring, 1, p.model.K), sm2 = smem_of<kL>(p.ring, 2, p.model.K);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(closed_second_kernel<kL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) ||
        (e = cudaFuncSetAttribute(closed_final_kernel<kL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) ||
        (e = cudaFuncSetAttribute(closed_log_kernel<kL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)))
        return e;
    if (p.n_items) {
        const uint64_t grid = (p.n_items + kThreads - 1) / kThreads;
        if ((e = launch_first<kL>(p, sm1, (unsigned)grid, stream)) != cudaSuccess) return e;
        closed_second_kernel<kL><<<(unsigned)grid, kThreads, sm2, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t pairs = (int64_t)p.n_traces * p.n_cls;
    if (pairs > 0) {
        closed_final_kernel<kL><<<(unsigned)((pairs + kThreads - 1) / kThreads), kThreads, sm2, stream>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (p.n_items && p.jobs && p.log_entries && p.log_cap > 0) {
        closed_log_kernel<kL><<<(unsigned)((p.n_items + kThreads - 1) / kThreads), kThreads, sm1, stream>>>(p);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

template <bool kL, int WK>
int max_ctas_t(uint32_t ring, int K) {
    int blocks = 0;
    const size_t smem = (WK > 0 && !kL) ? 0 : smem_of<kL>(ring, 1, K);
    if (cudaFuncSetAttribute(closed_first_kernel<kL, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, closed_first_kernel<kL, WK>, kThreads, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

}  // namespace

int closed_threads_per_cta() { return kThreads; }

int closed_window(int W) {
    switch (W) {
#define MAGUS_CLOSED_HAS_W(w) \
        case w: return w;
        MAGUS_CLOSED_WINDOWS(MAGUS_CLOSED_HAS_W)
#undef MAGUS_CLOSED_HAS_W
        default: return 0;
    }
}

template <bool kL>
int max_ctas_w(uint32_t ring, int K, int window) {
    switch (window) {
#define MAGUS_CLOSED_OCC_W(w) \
        case w: return max_ctas_t<kL, w>(ring, K);
        MAGUS_CLOSED_WINDOWS(MAGUS_CLOSED_OCC_W)
#undef MAGUS_CLOSED_OCC_W
        default: return max_ctas_t<kL, 0>(ring, K);
    }
}

int closed_max_ctas_per_sm(uint32_t ring, bool ladder, int n_levels, int window) {
    return ladder ? max_ctas_w<true>(ring, n_levels, window) : max_ctas_w<false>(ring, n_levels, window);
}

cudaError_t launch_replay_closed(const ClosedParams &p, bool ladder, cudaStream_t stream) {
    return ladder ? launch_t<true>(p, stream) : launch_t<false>(p, stream);
}

}  // namespace magus
