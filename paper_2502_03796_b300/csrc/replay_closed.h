// replay_closed.h - the time-parallel closed loop (replay_closed.cu), jump and one-rung
// modes: per-policy thresholds, per-segment replay records, launch parameters and host
// entry points.
#pragma once
#include "magus_internal.h"

namespace magus {

// Closed loop: the monitor reads obs = min(x, C(level in effect)).  With a = delta_t and
// b = delta_{t-W}, a throughput is capped exactly when its delta exceeds cthr[level]; Alg. 1's
// decision is then a threshold test on the other delta (both capped: a constant), all found
// on the host by bisection with the FP64 expressions the oracle evaluates (plan.cu).
// Level index l: jump mode 0 = bottom, 1 = top of the ladder; one-rung mode the rung itself.
struct ClosedThr {
    int64_t bu[MAGUS_MAX_LEVELS];   // a capped at level l, b not: +1 iff b < bu[l]
    int64_t bd[MAGUS_MAX_LEVELS];   //                              -1 iff b >= bd[l]
    int64_t au[MAGUS_MAX_LEVELS];   // b capped at level l, a not: +1 iff a >= au[l]
    int64_t ad[MAGUS_MAX_LEVELS];   //                              -1 iff a < ad[l]
    uint32_t cthr[MAGUS_MAX_LEVELS];  // delta > cthr[l] <=> x(delta) > C(level l), exactly
    uint32_t ccu[MAGUS_MAX_LEVELS];   // both capped, a at la, b at lb: bit lb of ccu[la]: +1
    uint32_t ccd[MAGUS_MAX_LEVELS];   //                                 bit lb of ccd[la]: -1
};

// One replay of one time segment of one pair: the state it started from, what it charged
// and logged, the state it ended in.  One-rung mode keeps the levels of the last W rounds in
// a separate byte array per slot (newest first) and its energy and time as FP64 totals
// (e, t), formed once per segment from integer per-rung counts and sums.
struct ClosedSlot {
    unsigned long long s0, sm, hash;  // jump: stretched sums at bottom / top; hash of its entries
    uint64_t lvh_in, fl_in;           // jump: levels (bit j: round start-1-j); flags at its start
    uint64_t lvh_out, fl_out;         // the same after its last round
    double e, t;                      // one-rung mode: energy and time charged
    uint32_t n0, nm, nhf, nch;        // jump: unstretched rounds at bottom / top; hf rounds; changes
    uint32_t lv_in, lv_out;           // level (jump: bit, one-rung: rung) at the start / at the end
    uint32_t ok;                      // bit 0 replayed, bit 1 exact start, bit 2 entries lost
    uint32_t pad;
};

// A segment whose change entries the final pass could not take from a replay's scratch (it
// overflowed): replayed once more by the log pass from its true start state, writing its
// entries to the pair's log from entry `off` on.
struct ClosedJob {
    uint64_t lvh, fl;   // state at the segment start (jump: level bits)
    uint64_t off;       // index of its first entry in the pair's log
    uint32_t lv, on;    // level; on: replay it
    uint8_t hist[MAGUS_MAX_WINDOW];   // one-rung mode: levels of the W rounds before, newest first
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
    int32_t window;              // the W every policy of the call shares where the first-replay
                                 // kernel has an instance for it, else 0
    const uint64_t *ibase;       // [n_traces + 1]: first item of each trace
    uint64_t n_items;            // items: (trace, policy, segment), segments innermost
    uint32_t seg_len;            // rounds per segment (a multiple of 64)
    uint32_t burn;               // rounds replayed before a segment from a guessed state
    DevModel model;
    ClosedSlot *slots;           // [2][n_items]: first replay, second replay
    uint8_t *lhist;              // one-rung mode: [2][n_items][2][64] level histories (start, end)
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
// Closed loop, not pinned: jump mode (step_mode 2) or one rung per decision (step_mode 3).
__host__ __device__ inline bool closed_policy(const DevPolicy &d) {
    return (d.step_mode == 2 || d.step_mode == 3) && d.pin == 0;
}
// ladder: levels 0 .. K-1 (one-rung mode), else bottom and top (jump mode).
void derive_closed(const DevPolicy &pol, const DevModel &m, bool ladder, ClosedThr *out);
int closed_threads_per_cta();
// W itself where the first-replay kernel has an instance for it, else 0
int closed_window(int W);
// resident CTAs of the first-replay kernel (window: as ClosedParams::window)
int closed_max_ctas_per_sm(uint32_t ring, bool ladder, int n_levels, int window);
cudaError_t launch_replay_closed(const ClosedParams &p, bool ladder, cudaStream_t stream);

}  // namespace magus
