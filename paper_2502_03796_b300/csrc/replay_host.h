// replay_host.h - host side of the replay handles: the handle, workspace helpers, plans and
// the kernel launches shared by api.cu (C entry points) and launch.cu (planning, launches).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "replay_closed.h"
#include "replay_static.h"

// The replay handle (magus_replay_t of the C ABI).
struct magus_replay {
    using DevModel = magus::DevModel;
    int device = 0;
    int sms = 0;
    std::vector<double> f;
    magus_model_t model{};
    DevModel dm{};
    size_t budget = 0;
    // device memory owned by the handle
    int *status = nullptr;            // device status word
    unsigned int *queue = nullptr;    // work counter
    void *ws = nullptr;               // plan workspace (policies, items, offsets, lengths)
    size_t ws_size = 0;
    cudaEvent_t ws_ev = nullptr;      // last use of the workspace
    bool ws_ev_pending = false;
    // the tile-kernel plan now in the workspace (a repeated call with the same plan skips
    // the upload and with it the wait for the previous launch)
    std::vector<char> ws_plan;
    bool ws_plan_valid = false;
    // pinned staging ring for plan uploads
    void *pin[2] = {nullptr, nullptr};
    size_t pin_size[2] = {0, 0};
    cudaEvent_t pin_ev[2] = {nullptr, nullptr};
    bool pin_pending[2] = {false, false};
    int pin_next = 0;
    // scratch for autotuning and host-memory runs
    void *scratch = nullptr;
    size_t scratch_size = 0;
    // host-memory runs: copy / compute streams, per-slot events
    cudaStream_t hs_copy = nullptr, hs_comp = nullptr;
    cudaEvent_t hs_ready[2] = {nullptr, nullptr}, hs_done[2] = {nullptr, nullptr};
    // events around batched-kernel launches since the last magus_replay_kernel_time()
    struct KEv {
        cudaEvent_t a, m, b;          // before the main kernel, after it, after the last kernel
        int kernels;                  // kernels launched between a and b
    };
    std::vector<KEv> k_ev;
    size_t k_used = 0;
    int tile_tg = 0, tile_cw = 0;     // 0: automatic
    int seg_rounds = -1;              // -1: automatic; 0: tile kernel; > 0: segment kernel
    uint64_t chunk_wait_ns = 0;       // tile kernel's per-chunk wait limit (0: default 2 s)
    void *segbuf = nullptr;           // segment summaries, tails, log scratch
    size_t seg_size = 0;
    void *stbuf = nullptr;            // static kernel: per-trace accumulators of split traces
    size_t st_size = 0;
    // policies -> {time_groups, policy_slots, group size, segment rounds (0: tile kernel)}
    std::map<int, std::array<int, 4>> tuned;
    // closed loop: segment and burn-in rounds (0: automatic; segment -1: literal kernel);
    // per mode (jump, one rung per decision): the buffer (plan, replay slots, change-entry
    // scratch, counters), the cached automatic choice and the last call's item count
    int cls_seg = 0, cls_burn = -1;
    uint64_t cls_key[2] = {0, 0};              // workload of the cached automatic choice
    uint64_t cls_auto_seg[2] = {0, 0}, cls_auto_burn[2] = {0, 0};
    void *clsbuf[2] = {nullptr, nullptr};
    size_t cls_size[2] = {0, 0};
    unsigned long long *cls_stats[2] = {nullptr, nullptr};   // device counters of the last call
    uint64_t cls_items[2] = {0, 0};
    std::unordered_map<std::string, magus::ClosedThr> cthr_cache;   // derived policy bytes -> thresholds
};

namespace magus {
namespace host {

int cuda_fail(cudaError_t e, const char *what);

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Segment length of the automatic choice (the fastest of 8,192 / 16,384 / 32,768 rounds on
// the 4,096 x 100,000 batched workload).
constexpr int kDefaultSegRounds = 16384;

constexpr int kUseTile = 1;   // launch_seg_plan: the segment buffers exceed the budget

struct Plan {
    std::vector<DevPolicy> pols;
    std::vector<char> tp;              // per policy: replayed by the time-parallel kernels
    std::vector<int32_t> lit;          // policies for the literal kernel
    std::vector<int32_t> cls;          // closed-loop policies (replay_closed.cu)
    std::vector<ClosedThr> cthr;       // their capped-throughput thresholds
    std::vector<StaticItem> sit;       // static-kernel CTAs (pins without carried state), or none
    std::vector<LadderItem> lad;       // (trace, one-rung policy) items, longest traces first
    std::vector<PolicyGroup> groups;
    std::vector<WorkItem> items;
    std::vector<uint64_t> offsets, lengths;
    int tg = 8, cw = 1, gp = 1;
    int seg_len = 0;                   // > 0: segment kernel with this many rounds per segment
};

struct Outs {
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
};

int kev_slot(magus_replay *h, size_t *slot);
size_t align_up(size_t v, size_t a);
int ensure_ws(magus_replay *h, void **buf, size_t *size, size_t need);
int ensure_pin(magus_replay *h, int slot, size_t need);
int check_policies(magus_replay *h, const magus_policy_t *configs, int32_t n_configs, std::vector<DevPolicy> *out);
// Without carried state, when some pin takes the static kernel, the pins at a ladder bound
// join it (one pass charges every rung) instead of a replay each on the tile kernel.
void route_pins(std::vector<DevPolicy> *pols, int n_levels, bool with_state);
void choose_tile(magus_replay *h, const std::vector<DevPolicy> &pols, const uint64_t *lengths, int n_traces, int *tg,
                 int *cw, int *gp, int *seg);
int build_plan(magus_replay *h, const uint64_t *lengths, int32_t n_traces, const magus_policy_t *configs,
               int32_t n_configs, int tg, int cw, int gp, int seg, Plan *pl, bool with_state = false);
int launch_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                float *ms_out = nullptr);
// The closed-loop jump-mode policies of a plan (time-parallel, or the literal kernel when
// its buffers exceed the budget); adds the kernels it launched to *kernels.
int launch_closed_part(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, const DevPolicy *d_pols,
                       const uint64_t *d_off, const uint64_t *d_len, cudaStream_t stream, int *kernels);

}  // namespace host
}  // namespace magus
