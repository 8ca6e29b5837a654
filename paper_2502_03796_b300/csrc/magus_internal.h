// magus_internal.h - structures shared by the replay kernels and their host launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "magus.h"

namespace magus {

// Per-policy parameters as the kernels use them (derived on the host, plan.cu).
// Algorithm 1's "derivative > inc" is decided on the integer m = a - b
// (a = delta_t, b = delta_{t-W}) outside a narrow band around the crossover, and by the
// exact FP64 evaluation inside it.
struct alignas(16) DevPolicy {
    int64_t up_mid;        // outside the band: +1 iff m > up_mid
    int64_t dn_mid;        // outside the band: -1 iff m < dn_mid
    uint32_t up_lo, up_w;  // band test on the low word: (uint32)(m - up_lo) <= up_w
    uint32_t dn_lo, dn_w;
    double inc, dec;       // Alg. 1 thresholds for the exact path
    int32_t W, L;          // Alg. 1 window, Alg. 2 list length
    int32_t kmin;          // smallest flag count c with c / L >= high_freq_threshold
    int32_t step_mode;
    double th;             // Alg. 2 threshold (the plain kernel evaluates it literally)
    int32_t pin;           // 0: controlled; k > 0: static baseline at ladder index k - 1
    int32_t to_static;     // a pin at a ladder bound sent to the static kernel (set on the host)
    // Alg. 1 on the FP64 difference d = x_t - x_{t-W} without the division: RN(d / W) > inc
    // exactly when d > up_last, RN(d / W) < dec exactly when d <= dn_last (RN(d / W) is
    // monotone in d; both found on the host over the ordered doubles)
    double up_last, dn_last;
};

// Ladder / energy model as the kernels use it.
struct DevModel {
    double q;              // dt * 1e9 (throughput divisor)
    double bpc;            // bytes per counter unit
    double dt;
    int32_t K;
    uint32_t thr0, thrM;   // delta > thr -> interval stretched at level 0 / K-1 (0xffffffff: never)
    int32_t one;           // 1, read at run time: lets the kernels express adds as IMADs
    double a0, aM;         // seconds per stretched delta unit at level 0 / K-1
    double P0, PM;         // power at level 0 / K-1
    double cap[MAGUS_MAX_LEVELS];  // capacity per level, GB/s (plain kernel)
    double pw[MAGUS_MAX_LEVELS];   // power per level, W (plain kernel)
    uint32_t thr[MAGUS_MAX_LEVELS];  // per level: delta > thr -> stretched (ladder kernel)
    double ak[MAGUS_MAX_LEVELS];     // per level: seconds per stretched delta unit
};

struct WorkItem {
    uint32_t trace;
    uint32_t cfg0;         // first policy group of the block
};

// Policies sharing Alg. 1's parameters (W, inc, dec): their predictions coincide, so the
// batched kernel makes them once per group.
constexpr int kMaxGroup = 4;
struct PolicyGroup {
    int32_t count;                 // 1..kMaxGroup
    int32_t member[kMaxGroup];     // policy indices (unused slots repeat member[0])
    int32_t same_L;                // every member has the same Alg. 2 list length
    int32_t pad[2];
};

struct TpParams {
    const uint32_t *traces;
    const uint64_t *offsets;
    const uint64_t *lengths;
    const DevPolicy *pols;
    int32_t n_pols;
    int32_t n_items;
    const WorkItem *items;
    const PolicyGroup *groups;
    int32_t n_groups;
    int32_t pad0;
    unsigned int *queue;   // work counter (zeroed before launch)
    int *status;           // device status word (0 ok, else MAGUS_E*)
    DevModel model;
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
    // limit of each per-chunk copy wait in ns (0: the default 2 s); the wait for the copies
    // still in flight when a CTA stops always keeps the default
    uint64_t chunk_wait_ns;
};

// Traces are read through a 2-D TMA tensor map over the packed buffer viewed as
// [rows][32] uint32 (trace starts are multiples of 32 elements), 128-byte swizzle.
constexpr int kTraceAlign = 32;
int make_trace_tmap(const uint32_t *traces, uint64_t total_elems, int box_rows, CUtensorMap *out,
                    std::string *err);
int tp_box_rows(int time_groups);
// Tile: time_groups warps split a chunk in time for each of policy_slots policy groups of
// up to group_size members (time_groups * policy_slots = 8, group_size 1 or 4; or the
// 4-warp tiles 4 x 1 x 1, 1 x 4 x 4 and 2 x 2 x 4).
bool tp_tile_supported(int time_groups, int policy_slots, int group_size);
// tmap: boxes of tp_box_rows(time_groups) rows; tmap_tail: boxes of kTailRows rows, for the
// last, partial chunk of each trace (the copy stops within kTailRows - 1 rows of its end).
constexpr int kTailRows = 8;
// window: the window length W shared by every policy group of the launch, or 0; where the
// tile has an instance for that W it runs that instance (tp_kernel_window names it, 0: none).
int tp_kernel_window(int time_groups, int policy_slots, int group_size, int window);
cudaError_t launch_replay_tp(int time_groups, int policy_slots, int group_size, const TpParams &p,
                             const CUtensorMap &tmap, const CUtensorMap &tmap_tail, int grid, cudaStream_t stream,
                             int window = 0);
int tp_max_ctas_per_sm(int time_groups, int policy_slots, int group_size, int *smem_bytes, int window = 0);

// ---- segment-parallel replay (replay_seg.cu)
struct SegItem {
    uint32_t trace;
    uint32_t grp;          // policy group
    uint32_t seg;          // time segment of the trace
    uint32_t pad;
};

// What one time segment of one pair contributes; the rounds before the segment's first
// event ("prefix") are charged for both possible entering levels.
struct SegSummary {
    unsigned long long s0, sm;       // stretched delta sums at bottom / top after the first event
    unsigned long long p_s0, p_sm;   // the prefix's stretched sums if it ran at bottom / top
    unsigned long long hash;         // hash of the change entries after the first event
    uint32_t n0, nm;                 // unstretched rounds at bottom / top after the first event
    uint32_t p_n0, p_nm;             // the prefix's unstretched rounds if at bottom / top
    uint32_t nhf;                    // high-frequency rounds
    uint32_t n_det;                  // change entries after the first event
    uint32_t first_pos;              // segment round of the first event, 0xffffffff if none
    uint32_t vals;                   // bit 0 first event's level, bit 1 level at the end, bit 2 known
};

// Flags and deltas after a trace's last round (for the carried state).
struct SegTail {
    uint64_t flags;
    uint32_t hist[MAGUS_MAX_WINDOW];
};

struct SegParams {
    const uint32_t *traces;
    const uint64_t *offsets;
    const uint64_t *lengths;
    const DevPolicy *pols;
    int32_t n_pols;
    int32_t n_items;
    const PolicyGroup *groups;
    const SegItem *items;
    const uint64_t *seg_base;        // per trace: index of its first segment
    uint32_t seg_len;                // rounds per segment (a multiple of 1024)
    uint32_t pad0;
    unsigned int *queue;
    int *status;
    DevModel model;
    SegSummary *summ;                // [segments * n_pols]
    SegTail *tails;                  // [pairs]
    // Change entries after each segment's first event, before the combine kernel compacts
    // them.  Per trace, scratch_base[trace] == kInPlace: segment k of a pair writes them to
    // the pair's own log at slot k * seg_len (the log holds at least the trace's length);
    // otherwise to scratch_log + scratch_base[trace] + (k * n_pols + policy) * seg_cap.
    const uint64_t *scratch_base;    // per trace, or NULL without a log
    uint32_t *scratch_log;
    uint64_t seg_cap;
    uint32_t *log;                   // the caller's log [pairs * log_cap] or NULL
    uint64_t log_cap;
    magus_state_t *state;
};

constexpr uint64_t kInPlace = ~0ull;

int seg_warps_per_cta();
// window: as for the tile kernel (the W every policy group shares, or 0)
int seg_max_ctas_per_sm(int group_size, int window = 0);
cudaError_t launch_replay_seg(int group_size, const SegParams &p, const CUtensorMap &tmap, int grid,
                              cudaStream_t stream, int window = 0);
cudaError_t launch_combine(const SegParams &p, int64_t n_pairs, double *energy, double *edp, double *time,
                           uint64_t *n_changes, uint64_t *change_hash, uint64_t *n_hf, cudaStream_t stream);

struct PlainParams {
    const uint32_t *trace;
    uint64_t n;
    const DevPolicy *pols;
    int32_t n_pols;
    int64_t pair_base;     // output index of policy 0 of this trace
    DevModel model;
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    uint8_t *level_log;
    double *deriv_log;
};
cudaError_t launch_replay_plain(const PlainParams &p, cudaStream_t stream);

// The literal kernel over all traces for the policies listed in `lit` (one thread per pair).
struct LiteralParams {
    const uint32_t *traces;
    const uint64_t *offsets;   // device, per trace
    const uint64_t *lengths;   // device, per trace
    int32_t n_traces;
    int32_t n_pols;            // pair index = trace * n_pols + policy
    const DevPolicy *pols;
    const int32_t *lit;        // device: policy indices replayed here
    int32_t n_lit;
    int32_t skip_pinned;       // pinned policies are left to the static kernel
    DevModel model;
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
    int *status;
};
cudaError_t launch_replay_literal(const LiteralParams &p, cudaStream_t stream);

// Policies the time-parallel kernels replay: open-loop jump mode, pinned (if at all) to a
// ladder bound.  The ladder kernel takes the open-loop one-rung mode, the segmented
// closed-loop kernels the closed loop (replay_closed.h), the literal kernel the rest (pins
// inside the ladder in jump mode, pins in the other modes).  A pin at a bound joins the
// static kernel when that kernel runs anyway (to_static).
__host__ __device__ inline bool tp_policy(const DevPolicy &d, int n_levels) {
    return d.step_mode == 0 && d.to_static == 0 && (d.pin == 0 || d.pin == 1 || d.pin == n_levels);
}
__host__ __device__ inline bool ladder_policy(const DevPolicy &d) { return d.step_mode == 1 && d.pin == 0; }
// Pinned policies the tile and segment kernels do not take (a pin inside the ladder in jump
// mode, any pin in the other modes, a bound pin marked to_static): without carried state,
// the static kernel.
__host__ __device__ inline bool static_policy(const DevPolicy &d, int n_levels) {
    return d.pin > 0 && !tp_policy(d, n_levels);
}
// The static kernel's parameters and launcher: replay_static.h.

// The one-rung (ladder) kernel: one warp per (trace, policy) item.
struct LadderItem {
    uint32_t trace;
    uint32_t pol;
};
struct LadderParams {
    const uint32_t *traces;
    const uint64_t *offsets;
    const uint64_t *lengths;
    const DevPolicy *pols;
    int32_t n_pols;
    int32_t n_items;
    const LadderItem *items;
    unsigned int *queue;
    int *status;
    DevModel model;
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
};
int ladder_warps_per_cta();
// window: the W every one-rung policy of the call shares, or 0 (selects a W-specific instance)
int ladder_max_ctas_per_sm(int window = 0);
cudaError_t launch_replay_ladder(const LadderParams &p, const CUtensorMap &tmap, int grid, cudaStream_t stream,
                                 int window = 0);

// Host planning (plan.cu).
// Groups over the policies with include[i] != 0 (all when include is NULL).
void form_groups(const std::vector<DevPolicy> &pols, int gp, std::vector<PolicyGroup> *out,
                 const std::vector<char> *include = nullptr);
int derive_policy(const magus_policy_t &in, const magus_model_t &m, DevPolicy *out, std::string *err);
int derive_model(const magus_model_t &m, DevModel *out, std::string *err);

void set_error(const std::string &msg);
const char *last_error_cstr();

}  // namespace magus
