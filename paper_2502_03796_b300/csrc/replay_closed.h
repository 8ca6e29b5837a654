// replay_closed.h - the time-parallel closed loop in jump mode (replay_closed.cu): its
// per-policy thresholds, per-segment replay records, launch parameters and host entry points.
#pragma once
#include "magus_internal.h"

namespace magus {

// Closed-loop jump mode: the monitor reads obs = min(x, C(level)).  Levels are the bottom or
// the top of the ladder (l = 0 / 1 below).  With a = delta_t, b = delta_{t-W}, a throughput is
// capped exactly when its delta exceeds cthr[level]; Alg. 1's decision is then a threshold
// test on the other delta (both capped: a constant), all found on the host by bisection
// with the FP64 expressions the oracle evaluates (plan.cu).
struct ClosedThr {
    int64_t bu[2], bd[2];  // a capped at level l, b not: +1 iff b < bu[l]; -1 iff b >= bd[l]
    int64_t au[2], ad[2];  // b capped at level l, a not: +1 iff a >= au[l]; -1 iff a < ad[l]
    uint32_t cthr[2];      // delta > cthr[l] <=> x(delta) > C(level l), exactly
    uint32_t cc;           // both capped (levels la, lb): bit 2 la + lb: +1; bit 4 + 2 la + lb: -1
    uint32_t pad;
};

// One replay of one time segment of one pair: the state it started from, what it charged
// and logged, the state it ended in.
struct ClosedSlot {
    unsigned long long s0, sm, hash;  // stretched sums at bottom / top, hash of its change entries
    uint64_t lvh_in, fl_in;           // levels (bit j: round start-1-j) and flags at its start
    uint64_t lvh_out, fl_out;         // the same after its last round
    uint32_t n0, nm, nhf, nch;        // unstretched rounds at bottom / top, hf rounds, changes
    uint32_t lv_in, lv_out;           // level bit at the start / after the last round
    uint32_t ok;                      // bit 0 replayed, bit 1 exact start, bit 2 log overflow
    uint32_t pad;
};

// A segment whose change entries the final pass could not take from a replay's scratch (it
// overflowed): replayed once more by the log pass from its true start state, writing its
// entries to the pair's log from entry `off` on.
struct ClosedJob {
    uint64_t lvh, fl;   // state at the segment start
    uint64_t off;       // index of its first entry in the pair's log
    uint32_t lv, on;    // level bit; on: replay it
};

struct ClosedParams {
    const uint32_t *traces;
    const uint64_t *offsets;
    const uint64_t *lengths;
    int32_t n_traces;
    int32_t n_pols;              // pair index = trace * n_pols + policy
    const DevPolicy *pols;
    const ClosedThr *thr;        // [n_cls]
    const int32_t *cls;          // [n_cls] policy indices replayed here
    int32_t n_cls;
    uint32_t ring;               // deltas kept per thread (a power of two >= every W)
    const uint64_t *ibase;       // [n_traces + 1]: first item of each trace
    uint64_t n_items;            // items: (trace, policy, segment), segments innermost
    uint32_t seg_len;            // rounds per segment (a multiple of 64)
    uint32_t burn;               // rounds replayed before a segment from a guessed state
    DevModel model;
    ClosedSlot *slots;           // [2][n_items]: first replay, second replay
    uint32_t *scratch;           // [2][n_items][scr_cap] change entries, or NULL
    uint64_t scr_cap;
    ClosedJob *jobs;             // [n_items], with a log: segments for the log pass
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
    int *status;
    unsigned long long *stats;   // [3]: second replays, replays in the final pass, in the log pass
};
__host__ __device__ inline bool closed_policy(const DevPolicy &d) { return d.step_mode == 2 && d.pin == 0; }
void derive_closed(const DevPolicy &pol, const DevModel &m, ClosedThr *out);
int closed_threads_per_cta();
int closed_max_ctas_per_sm(uint32_t ring);   // resident CTAs of the first-replay kernel
cudaError_t launch_replay_closed(const ClosedParams &p, cudaStream_t stream);

}  // namespace magus
