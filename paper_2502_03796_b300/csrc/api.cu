// api.cu - C ABI of libmagus: replay handles, argument checks, planning, workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "magus_internal.h"

using namespace magus;

struct magus_replay {
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
    void *segbuf = nullptr;           // segment summaries, tails, log scratch
    size_t seg_size = 0;
    // policies -> {time_groups, policy_slots, group size, segment rounds (0: tile kernel)}
    std::map<int, std::array<int, 4>> tuned;
};

namespace {

const char *kVersion = "magus-b300 0.1 (sm_103a)";

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return MAGUS_ECUDA;
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Event slot for one timed replay (up to 4096 per kernel_time() period; later ones reuse
// the last slot).
int kev_slot(magus_replay *h, size_t *slot) {
    if (h->k_used == h->k_ev.size() && h->k_used < 4096) {
        magus_replay::KEv e{};
        CK(cudaEventCreate(&e.a), "cudaEventCreate");
        CK(cudaEventCreate(&e.m), "cudaEventCreate");
        CK(cudaEventCreate(&e.b), "cudaEventCreate");
        h->k_ev.push_back(e);
    }
    *slot = h->k_used < h->k_ev.size() ? h->k_used : h->k_ev.size() - 1;
    return MAGUS_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device-memory growth inside the handle budget.  Waits for the previous user first.
int ensure_ws(magus_replay *h, void **buf, size_t *size, size_t need) {
    if (need <= *size) return MAGUS_OK;
    size_t want = std::max(need, *size * 2);
    size_t other = h->ws_size + h->scratch_size + h->seg_size - *size;
    if (want + other > h->budget) want = need;
    if (want + other > h->budget) {
        set_error("device workspace of " + std::to_string(need) + " bytes exceeds the handle's memory budget");
        return MAGUS_ENOMEM;
    }
    if (h->ws_ev_pending) CK(cudaEventSynchronize(h->ws_ev), "cudaEventSynchronize");
    if (*buf) CK(cudaFree(*buf), "cudaFree");
    *buf = nullptr;
    *size = 0;
    cudaError_t e = cudaMalloc(buf, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of the workspace failed");
        return MAGUS_ENOMEM;
    }
    *size = want;
    return MAGUS_OK;
}

int ensure_pin(magus_replay *h, int slot, size_t need) {
    if (h->pin_pending[slot]) {
        CK(cudaEventSynchronize(h->pin_ev[slot]), "cudaEventSynchronize");
        h->pin_pending[slot] = false;
    }
    if (need <= h->pin_size[slot]) return MAGUS_OK;
    if (h->pin[slot]) CK(cudaFreeHost(h->pin[slot]), "cudaFreeHost");
    h->pin[slot] = nullptr;
    h->pin_size[slot] = 0;
    size_t want = std::max(need, (size_t)1 << 16);
    cudaError_t e = cudaMallocHost(&h->pin[slot], want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("pinned staging allocation failed");
        return MAGUS_ENOMEM;
    }
    h->pin_size[slot] = want;
    return MAGUS_OK;
}

int check_policies(magus_replay *h, const magus_policy_t *configs, int32_t n_configs,
                   std::vector<DevPolicy> *out, bool jump_only) {
    if (!configs || n_configs < 1 || n_configs > 4096) {
        set_error("configs must be non-NULL with 1 <= n_configs <= 4096");
        return MAGUS_EINVAL;
    }
    out->resize(n_configs);
    for (int c = 0; c < n_configs; c++) {
        std::string err;
        int rc = derive_policy(configs[c], h->model, &(*out)[c], &err);
        if (rc) {
            set_error("policy " + std::to_string(c) + ": " + err);
            return rc;
        }
        (void)jump_only;   // every valid policy runs: see tp_policy() for the routing
    }
    return MAGUS_OK;
}

// Segment length of the automatic choice (the fastest of 8,192 / 16,384 / 32,768 rounds on
// the 4,096 x 100,000 batched workload).
constexpr int kDefaultSegRounds = 16384;

struct Plan {
    std::vector<DevPolicy> pols;
    std::vector<char> tp;              // per policy: replayed by the time-parallel kernels
    std::vector<int32_t> lit;          // policies for the literal kernel
    std::vector<LadderItem> lad;       // (trace, one-rung policy) items, longest traces first
    std::vector<PolicyGroup> groups;
    std::vector<WorkItem> items;
    std::vector<uint64_t> offsets, lengths;
    int tg = 8, cw = 1, gp = 1;
    int seg_len = 0;                   // > 0: segment kernel with this many rounds per segment
};

// Tile for a workload: group size 4 when policies share predictions, then as many policy
// slots per CTA as there are groups (up to 8), the remaining warps splitting time.
void choose_tile(magus_replay *h, const std::vector<DevPolicy> &pols, const uint64_t *lengths, int n_traces, int *tg,
                 int *cw, int *gp, int *seg) {
    const int n_configs = (int)pols.size();
    auto it = h->tuned.find(n_configs);
    if (!h->tile_tg && h->seg_rounds < 0 && it != h->tuned.end()) {   // the autotuner's pick
        *tg = it->second[0];
        *cw = it->second[1];
        *gp = it->second[2];
        *seg = it->second[3];
        return;
    }
    std::vector<char> tp(pols.size());
    int n_tp = 0;
    for (size_t i = 0; i < pols.size(); i++) n_tp += (tp[i] = tp_policy(pols[i], h->model.n_levels) ? 1 : 0);
    std::vector<PolicyGroup> g4;
    form_groups(pols, kMaxGroup, &g4, &tp);
    *gp = (2 * g4.size() <= (size_t)n_tp) ? kMaxGroup : 1;
    const int n_groups = std::max(1, *gp == 1 ? n_tp : (int)g4.size());
    if (h->tile_tg) {
        *tg = h->tile_tg;
        *cw = h->tile_cw;
    } else {
        int c = 1;
        while (c * 2 <= std::min(8, n_groups)) c *= 2;
        *cw = c;
        *tg = 8 / c;
    }
    // an explicit tile shape selects the tile kernel unless segments were asked for as well
    if (h->seg_rounds >= 0 || h->tile_tg) {
        *seg = h->seg_rounds > 0 ? h->seg_rounds : 0;
        return;
    }
    // automatic: the tile kernel replays a trace's chunks one after another in one CTA, so
    // a few long traces leave most SMs idle; the segment kernel (about 15% more work per
    // round) splits them in time.  Take it when the longest trace's chain of chunks exceeds
    // 1.3x the chunks each resident CTA gets on average.
    *seg = 0;
    int smem = 0;
    const int per_sm = tp_max_ctas_per_sm(*tg, *cw, *gp, &smem);
    if (per_sm <= 0 || n_traces <= 0) return;
    const uint64_t chunk = (uint64_t)*tg * 1024;
    const uint64_t blocks = (uint64_t)(n_groups + *cw - 1) / *cw;
    uint64_t longest = 0, total = 0;
    for (int i = 0; i < n_traces; i++) {
        const uint64_t c = (lengths[i] + chunk - 1) / chunk;
        longest = std::max(longest, c);
        total += c * blocks;
    }
    const double per_cta = (double)total / ((double)h->sms * per_sm);
    if (!((double)longest > 1.3 * per_cta && longest * chunk >= 2 * (uint64_t)kDefaultSegRounds)) return;
    // segment length: work items are taken from a queue, so the launch lasts about
    // ceil(items / warps) items; pick the length that minimises that (plus a fixed cost of
    // 256 rounds per segment for its prehistory, summary and combine step)
    const int seg_ctas = seg_max_ctas_per_sm(*gp);
    if (seg_ctas <= 0) return;
    const double warps = (double)h->sms * seg_ctas * seg_warps_per_cta();
    double best = 1e300;
    for (int L = 2048; L <= 65536; L += 1024) {
        uint64_t items = 0;
        for (int i = 0; i < n_traces; i++) items += (lengths[i] + L - 1) / L;
        items *= (uint64_t)n_groups;
        const double cost = std::ceil((double)items / warps) * (L + 256.0);
        if (cost < best * 0.999) {   // ties go to the shorter segment
            best = cost;
            *seg = L;
        }
    }
}

int build_plan(magus_replay *h, const uint64_t *lengths, int32_t n_traces, const magus_policy_t *configs,
               int32_t n_configs, int tg, int cw, int gp, int seg, Plan *pl) {
    int rc = check_policies(h, configs, n_configs, &pl->pols, true);
    if (rc) return rc;
    pl->tg = tg;
    pl->cw = cw;
    pl->gp = gp;
    pl->seg_len = seg;
    pl->tp.resize(pl->pols.size());
    pl->lit.clear();
    std::vector<int32_t> lad_pols;
    for (size_t i = 0; i < pl->pols.size(); i++) {
        pl->tp[i] = tp_policy(pl->pols[i], h->model.n_levels) ? 1 : 0;
        if (pl->tp[i]) continue;
        if (ladder_policy(pl->pols[i])) lad_pols.push_back((int32_t)i);
        else pl->lit.push_back((int32_t)i);
    }
    form_groups(pl->pols, gp, &pl->groups, &pl->tp);
    pl->offsets.resize(n_traces);
    pl->lengths.assign(lengths, lengths + n_traces);
    uint64_t off = 0;
    for (int i = 0; i < n_traces; i++) {
        pl->offsets[i] = off;
        off += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
    }
    // longest traces first: the persistent CTAs take items in this order
    std::vector<int> order(n_traces);
    for (int i = 0; i < n_traces; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lengths[a] > lengths[b]; });
    const int n_groups = (int)pl->groups.size();
    const int blocks = (n_groups + cw - 1) / cw;
    pl->items.clear();
    pl->items.reserve((size_t)n_traces * blocks);
    for (int i : order)
        for (int b = 0; b < blocks; b++) pl->items.push_back(WorkItem{(uint32_t)i, (uint32_t)(b * cw)});
    pl->lad.clear();
    pl->lad.reserve((size_t)n_traces * lad_pols.size());
    for (int i : order)
        for (int32_t c : lad_pols) pl->lad.push_back(LadderItem{(uint32_t)i, (uint32_t)c});
    return MAGUS_OK;
}

struct Outs {
    double *energy, *edp, *time;
    uint32_t *log_entries;
    uint64_t log_cap;
    uint64_t *n_changes, *change_hash, *n_hf;
    magus_state_t *state;
};

// Upload the plan through pinned staging and launch the batched kernel on `stream`.
// The policies the time-parallel kernels do not replay: one thread per pair, all traces in
// one launch (replay_plain.cu).  d_*: the plan as uploaded to the workspace.
int launch_literal_part(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o,
                        const DevPolicy *d_pols, const uint64_t *d_off, const uint64_t *d_len, const int32_t *d_lit,
                        cudaStream_t stream) {
    LiteralParams lp;
    memset(&lp, 0, sizeof(lp));
    lp.traces = traces;
    lp.offsets = d_off;
    lp.lengths = d_len;
    lp.n_traces = (int32_t)pl.lengths.size();
    lp.n_pols = (int32_t)pl.pols.size();
    lp.pols = d_pols;
    lp.lit = d_lit;
    lp.n_lit = (int32_t)pl.lit.size();
    lp.model = h->dm;
    lp.energy = o.energy;
    lp.edp = o.edp;
    lp.time = o.time;
    lp.log_entries = o.log_entries;
    lp.log_cap = o.log_cap;
    lp.n_changes = o.n_changes;
    lp.change_hash = o.change_hash;
    lp.n_hf = o.n_hf;
    lp.state = o.state;
    lp.status = h->status;
    CK(launch_replay_literal(lp, stream), "literal kernel launch");
    return MAGUS_OK;
}

// The one-rung policies: one warp per (trace, policy) item (replay_ladder.cu).
int launch_ladder_part(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o,
                       const DevPolicy *d_pols, const uint64_t *d_off, const uint64_t *d_len,
                       const LadderItem *d_items, cudaStream_t stream) {
    uint64_t total_elems = 0;
    for (size_t i = 0; i < pl.lengths.size(); i++)
        total_elems += (pl.lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    std::string err;
    int rc = make_trace_tmap(traces, total_elems, 32, &tmap, &err);
    if (rc) { set_error(err); return rc; }
    LadderParams lp;
    memset(&lp, 0, sizeof(lp));
    lp.traces = traces;
    lp.offsets = d_off;
    lp.lengths = d_len;
    lp.pols = d_pols;
    lp.n_pols = (int32_t)pl.pols.size();
    lp.n_items = (int32_t)pl.lad.size();
    lp.items = d_items;
    lp.queue = h->queue;
    lp.status = h->status;
    lp.model = h->dm;
    lp.energy = o.energy;
    lp.edp = o.edp;
    lp.time = o.time;
    lp.log_entries = o.log_entries;
    lp.log_cap = o.log_cap;
    lp.n_changes = o.n_changes;
    lp.change_hash = o.change_hash;
    lp.n_hf = o.n_hf;
    lp.state = o.state;
    const int per_sm = ladder_max_ctas_per_sm();
    if (per_sm <= 0) {
        set_error("ladder kernel does not fit on this device");
        return MAGUS_ECUDA;
    }
    const size_t ctas = (pl.lad.size() + ladder_warps_per_cta() - 1) / ladder_warps_per_cta();
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(ctas, (size_t)h->sms * per_sm));
    CK(cudaMemsetAsync(h->queue, 0, sizeof(unsigned int), stream), "cudaMemsetAsync");
    CK(launch_replay_ladder(lp, tmap, grid, stream), "ladder kernel launch");
    return MAGUS_OK;
}

int launch_seg_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                    float *ms_out);
constexpr int kUseTile = 1;   // launch_seg_plan: the segment buffers exceed the budget

int launch_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                float *ms_out = nullptr) {
    if (pl.seg_len > 0) {
        const int rc = launch_seg_plan(h, pl, traces, o, stream, ms_out);
        if (rc != kUseTile) return rc;
    }
    const size_t n_items = pl.items.size();
    const size_t sz_pol = align_up(pl.pols.size() * sizeof(DevPolicy), 256);
    const size_t sz_grp = align_up(std::max<size_t>(pl.groups.size(), 1) * sizeof(PolicyGroup), 256);
    const size_t sz_items = align_up(std::max<size_t>(n_items, 1) * sizeof(WorkItem), 256);
    const size_t sz_off = align_up(std::max<size_t>(pl.offsets.size(), 1) * 8, 256);
    const size_t sz_lit = align_up(std::max<size_t>(pl.lit.size(), 1) * 4, 256);
    const size_t sz_lad = align_up(std::max<size_t>(pl.lad.size(), 1) * sizeof(LadderItem), 256);
    const size_t off_lad = sz_pol + sz_grp + sz_items + 2 * sz_off + sz_lit;
    const size_t total = off_lad + sz_lad;
    int rc = ensure_ws(h, &h->ws, &h->ws_size, total);
    if (rc) return rc;
    const int slot = h->pin_next;
    h->pin_next ^= 1;
    rc = ensure_pin(h, slot, total);
    if (rc) return rc;
    char *pin = (char *)h->pin[slot];
    memcpy(pin, pl.pols.data(), pl.pols.size() * sizeof(DevPolicy));
    memcpy(pin + sz_pol, pl.groups.data(), pl.groups.size() * sizeof(PolicyGroup));
    if (n_items) memcpy(pin + sz_pol + sz_grp, pl.items.data(), n_items * sizeof(WorkItem));
    if (!pl.offsets.empty()) {
        memcpy(pin + sz_pol + sz_grp + sz_items, pl.offsets.data(), pl.offsets.size() * 8);
        memcpy(pin + sz_pol + sz_grp + sz_items + sz_off, pl.lengths.data(), pl.lengths.size() * 8);
    }
    if (!pl.lit.empty()) memcpy(pin + sz_pol + sz_grp + sz_items + 2 * sz_off, pl.lit.data(), pl.lit.size() * 4);
    if (!pl.lad.empty()) memcpy(pin + off_lad, pl.lad.data(), pl.lad.size() * sizeof(LadderItem));
    if (h->ws_ev_pending) CK(cudaStreamWaitEvent(stream, h->ws_ev, 0), "cudaStreamWaitEvent");
    char *ws = (char *)h->ws;
    CK(cudaMemcpyAsync(ws, pin, total, cudaMemcpyHostToDevice, stream), "cudaMemcpyAsync(plan)");
    CK(cudaEventRecord(h->pin_ev[slot], stream), "cudaEventRecord");
    h->pin_pending[slot] = true;
    CK(cudaMemsetAsync(h->queue, 0, sizeof(unsigned int), stream), "cudaMemsetAsync");

    TpParams p;
    memset(&p, 0, sizeof(p));
    p.traces = traces;
    p.pols = (const DevPolicy *)ws;
    p.n_pols = (int32_t)pl.pols.size();
    p.groups = (const PolicyGroup *)(ws + sz_pol);
    p.n_groups = (int32_t)pl.groups.size();
    p.items = (const WorkItem *)(ws + sz_pol + sz_grp);
    p.offsets = (const uint64_t *)(ws + sz_pol + sz_grp + sz_items);
    p.lengths = (const uint64_t *)(ws + sz_pol + sz_grp + sz_items + sz_off);
    p.n_items = (int32_t)n_items;
    p.queue = h->queue;
    p.status = h->status;
    p.model = h->dm;
    p.energy = o.energy;
    p.edp = o.edp;
    p.time = o.time;
    p.log_entries = o.log_entries;
    p.log_cap = o.log_cap;
    p.n_changes = o.n_changes;
    p.change_hash = o.change_hash;
    p.n_hf = o.n_hf;
    p.state = o.state;
    int smem = 0;
    const int per_sm = tp_max_ctas_per_sm(pl.tg, pl.cw, pl.gp, &smem);
    if (per_sm <= 0) {
        set_error("tile shape does not fit on this device");
        return MAGUS_ECUDA;
    }
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(n_items, (size_t)h->sms * per_sm));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        CK(cudaEventCreate(&e0), "cudaEventCreate");
        CK(cudaEventCreate(&e1), "cudaEventCreate");
        CK(cudaEventRecord(e0, stream), "cudaEventRecord");
    }
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (n_items) {
        uint64_t total_elems = 0;
        for (size_t i = 0; i < pl.lengths.size(); i++)
            total_elems += (pl.lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
        std::string err;
        rc = make_trace_tmap(traces, total_elems, tp_box_rows(pl.tg), &tmap, &err);
        if (rc) { set_error(err); return rc; }
    }
    const bool has_lit = !pl.lit.empty() && !pl.lengths.empty();
    const bool has_lad = !pl.lad.empty();
    if (n_items || has_lit || has_lad) {
        size_t slot_k;
        rc = kev_slot(h, &slot_k);
        if (rc) return rc;
        // event m follows the first kernel: the main kernel of this call
        bool m_done = false;
        auto mark = [&]() -> int {
            if (!m_done) CK(cudaEventRecord(h->k_ev[slot_k].m, stream), "cudaEventRecord");
            m_done = true;
            return MAGUS_OK;
        };
        CK(cudaEventRecord(h->k_ev[slot_k].a, stream), "cudaEventRecord");
        if (n_items) {
            CK(launch_replay_tp(pl.tg, pl.cw, pl.gp, p, tmap, grid, stream), "replay kernel launch");
            if ((rc = mark())) return rc;
        }
        if (has_lad) {
            rc = launch_ladder_part(h, pl, traces, o, p.pols, p.offsets, p.lengths, (const LadderItem *)(ws + off_lad),
                                    stream);
            if (rc || (rc = mark())) return rc;
        }
        if (has_lit) {
            rc = launch_literal_part(h, pl, traces, o, p.pols, p.offsets, p.lengths,
                                     (const int32_t *)(ws + sz_pol + sz_grp + sz_items + 2 * sz_off), stream);
            if (rc || (rc = mark())) return rc;
        }
        CK(cudaEventRecord(h->k_ev[slot_k].b, stream), "cudaEventRecord");
        h->k_ev[slot_k].kernels = (n_items ? 1 : 0) + (has_lad ? 1 : 0) + (has_lit ? 1 : 0);
        if (h->k_used < h->k_ev.size()) h->k_used++;
    }
    if (ms_out) {
        CK(cudaEventRecord(e1, stream), "cudaEventRecord");
        CK(cudaEventSynchronize(e1), "cudaEventSynchronize");
        CK(cudaEventElapsedTime(ms_out, e0, e1), "cudaEventElapsedTime");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    CK(cudaEventRecord(h->ws_ev, stream), "cudaEventRecord");
    h->ws_ev_pending = true;
    return MAGUS_OK;
}

// Segment kernel: every warp replays one (trace, policy group, time segment) at a time; a
// combine kernel resolves each pair's segments in order (replay_seg.cu).
int launch_seg_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                    float *ms_out) {
    const int n_traces = (int)pl.lengths.size();
    const int n_pols = (int)pl.pols.size();
    const uint64_t seg_len = (uint64_t)pl.seg_len;
    std::vector<uint64_t> seg_base(std::max(n_traces, 1), 0);
    uint64_t total_segs = 0;
    for (int i = 0; i < n_traces; i++) {
        seg_base[i] = total_segs;
        total_segs += (pl.lengths[i] + seg_len - 1) / seg_len;
    }
    std::vector<int> order(n_traces);
    for (int i = 0; i < n_traces; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pl.lengths[a] > pl.lengths[b]; });
    std::vector<SegItem> items;
    items.reserve((size_t)total_segs * pl.groups.size());
    for (int i : order) {
        const uint32_t nseg = (uint32_t)((pl.lengths[i] + seg_len - 1) / seg_len);
        for (uint32_t g = 0; g < pl.groups.size(); g++)
            for (uint32_t k = 0; k < nseg; k++) items.push_back(SegItem{(uint32_t)i, g, k, 0});
    }
    const size_t n_items = items.size();
    if (n_items > (size_t)INT32_MAX) {
        set_error("too many segment work items");
        return MAGUS_EINVAL;
    }
    // change entries after each segment's first event: in the pair's own log when it holds
    // the whole trace, else in scratch (only the first log_cap of a segment can be kept)
    const bool has_log = o.log_entries && o.log_cap > 0;
    const uint64_t seg_cap = has_log ? std::min<uint64_t>(seg_len, o.log_cap) : 0;
    std::vector<uint64_t> scratch_base(std::max(n_traces, 1), 0);
    uint64_t scratch_entries = 0;
    for (int i = 0; i < n_traces && has_log; i++) {
        if (pl.lengths[i] <= o.log_cap) {
            scratch_base[i] = kInPlace;
        } else {
            scratch_base[i] = scratch_entries;
            scratch_entries += (pl.lengths[i] + seg_len - 1) / seg_len * (uint64_t)n_pols * seg_cap;
        }
    }
    // plan workspace: policies | groups | items | offsets | lengths | segment bases | scratch bases
    const size_t sz_pol = align_up(pl.pols.size() * sizeof(DevPolicy), 256);
    const size_t sz_grp = align_up(std::max<size_t>(pl.groups.size(), 1) * sizeof(PolicyGroup), 256);
    const size_t sz_items = align_up(std::max<size_t>(n_items, 1) * sizeof(SegItem), 256);
    const size_t sz_off = align_up(std::max<size_t>(n_traces, 1) * 8, 256);
    const size_t sz_lit = align_up(std::max<size_t>(pl.lit.size(), 1) * 4, 256);
    const size_t sz_lad = align_up(std::max<size_t>(pl.lad.size(), 1) * sizeof(LadderItem), 256);
    const size_t off_lad = sz_pol + sz_grp + sz_items + 4 * sz_off + sz_lit;
    const size_t total = off_lad + sz_lad;
    // device buffers: summaries | tails | change-log scratch
    const uint64_t n_pairs = (uint64_t)n_traces * n_pols;
    const size_t sz_sum = align_up(std::max<uint64_t>(total_segs * n_pols, 1) * sizeof(SegSummary), 256);
    const size_t sz_tail = align_up(std::max<uint64_t>(n_pairs, 1) * sizeof(SegTail), 256);
    const size_t sz_log = align_up(scratch_entries * 4, 256);
    const size_t seg_need = sz_sum + sz_tail + sz_log;
    // the tile kernel needs none of the segment buffers: take it when they do not fit
    if (std::max(total, h->ws_size) + h->scratch_size + std::max(seg_need, h->seg_size) > h->budget) return kUseTile;
    int rc = ensure_ws(h, &h->ws, &h->ws_size, total);
    if (rc) return rc;
    rc = ensure_ws(h, &h->segbuf, &h->seg_size, seg_need);
    if (rc) return rc;
    const int slot = h->pin_next;
    h->pin_next ^= 1;
    rc = ensure_pin(h, slot, total);
    if (rc) return rc;
    char *pin = (char *)h->pin[slot];
    memcpy(pin, pl.pols.data(), pl.pols.size() * sizeof(DevPolicy));
    memcpy(pin + sz_pol, pl.groups.data(), pl.groups.size() * sizeof(PolicyGroup));
    if (n_items) memcpy(pin + sz_pol + sz_grp, items.data(), n_items * sizeof(SegItem));
    if (n_traces) {
        memcpy(pin + sz_pol + sz_grp + sz_items, pl.offsets.data(), n_traces * 8);
        memcpy(pin + sz_pol + sz_grp + sz_items + sz_off, pl.lengths.data(), n_traces * 8);
        memcpy(pin + sz_pol + sz_grp + sz_items + 2 * sz_off, seg_base.data(), n_traces * 8);
        memcpy(pin + sz_pol + sz_grp + sz_items + 3 * sz_off, scratch_base.data(), n_traces * 8);
    }
    if (!pl.lit.empty()) memcpy(pin + sz_pol + sz_grp + sz_items + 4 * sz_off, pl.lit.data(), pl.lit.size() * 4);
    if (!pl.lad.empty()) memcpy(pin + off_lad, pl.lad.data(), pl.lad.size() * sizeof(LadderItem));
    if (h->ws_ev_pending) CK(cudaStreamWaitEvent(stream, h->ws_ev, 0), "cudaStreamWaitEvent");
    char *ws = (char *)h->ws;
    CK(cudaMemcpyAsync(ws, pin, total, cudaMemcpyHostToDevice, stream), "cudaMemcpyAsync(plan)");
    CK(cudaEventRecord(h->pin_ev[slot], stream), "cudaEventRecord");
    h->pin_pending[slot] = true;
    CK(cudaMemsetAsync(h->queue, 0, sizeof(unsigned int), stream), "cudaMemsetAsync");

    SegParams p;
    memset(&p, 0, sizeof(p));
    p.traces = traces;
    p.pols = (const DevPolicy *)ws;
    p.n_pols = n_pols;
    p.groups = (const PolicyGroup *)(ws + sz_pol);
    p.items = (const SegItem *)(ws + sz_pol + sz_grp);
    p.n_items = (int32_t)n_items;
    p.offsets = (const uint64_t *)(ws + sz_pol + sz_grp + sz_items);
    p.lengths = (const uint64_t *)(ws + sz_pol + sz_grp + sz_items + sz_off);
    p.seg_base = (const uint64_t *)(ws + sz_pol + sz_grp + sz_items + 2 * sz_off);
    p.seg_len = (uint32_t)seg_len;
    p.queue = h->queue;
    p.status = h->status;
    p.model = h->dm;
    p.summ = (SegSummary *)h->segbuf;
    p.tails = (SegTail *)((char *)h->segbuf + sz_sum);
    p.scratch_base = has_log ? (const uint64_t *)(ws + sz_pol + sz_grp + sz_items + 3 * sz_off) : nullptr;
    p.scratch_log = scratch_entries ? (uint32_t *)((char *)h->segbuf + sz_sum + sz_tail) : nullptr;
    p.seg_cap = seg_cap;
    p.log = has_log ? o.log_entries : nullptr;
    p.log_cap = has_log ? o.log_cap : 0;
    p.state = o.state;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (n_items) {
        uint64_t total_elems = 0;
        for (int i = 0; i < n_traces; i++)
            total_elems += (pl.lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
        std::string err;
        rc = make_trace_tmap(traces, total_elems, 32, &tmap, &err);
        if (rc) { set_error(err); return rc; }
    }
    const int per_sm = seg_max_ctas_per_sm(pl.gp);
    if (per_sm <= 0) {
        set_error("segment kernel does not fit on this device");
        return MAGUS_ECUDA;
    }
    const size_t warps = (size_t)h->sms * per_sm * seg_warps_per_cta();
    const int grid = (int)std::max<size_t>(1, std::min<size_t>((n_items + seg_warps_per_cta() - 1) / seg_warps_per_cta(),
                                                               warps / seg_warps_per_cta()));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        CK(cudaEventCreate(&e0), "cudaEventCreate");
        CK(cudaEventCreate(&e1), "cudaEventCreate");
        CK(cudaEventRecord(e0, stream), "cudaEventRecord");
    }
    size_t slot_k;
    rc = kev_slot(h, &slot_k);
    if (rc) return rc;
    // event m follows the main kernel: the segment kernel, else the first one launched
    bool m_done = false;
    auto mark = [&]() -> int {
        if (!m_done) CK(cudaEventRecord(h->k_ev[slot_k].m, stream), "cudaEventRecord");
        m_done = true;
        return MAGUS_OK;
    };
    CK(cudaEventRecord(h->k_ev[slot_k].a, stream), "cudaEventRecord");
    if (n_items) {
        CK(launch_replay_seg(pl.gp, p, tmap, grid, stream), "segment kernel launch");
        if ((rc = mark())) return rc;
    }
    const bool any_tp = std::count(pl.tp.begin(), pl.tp.end(), (char)1) > 0;
    if (n_pairs && any_tp) {
        CK(launch_combine(p, (int64_t)n_pairs, o.energy, o.edp, o.time, o.n_changes, o.change_hash, o.n_hf, stream),
           "combine kernel launch");
        if ((rc = mark())) return rc;
    }
    const bool has_lad = !pl.lad.empty();
    if (has_lad) {
        rc = launch_ladder_part(h, pl, traces, o, p.pols, p.offsets, p.lengths, (const LadderItem *)(ws + off_lad),
                                stream);
        if (rc || (rc = mark())) return rc;
    }
    const bool has_lit = !pl.lit.empty() && n_traces > 0;
    if (has_lit) {
        rc = launch_literal_part(h, pl, traces, o, p.pols, p.offsets, p.lengths,
                                 (const int32_t *)(ws + sz_pol + sz_grp + sz_items + 4 * sz_off), stream);
        if (rc || (rc = mark())) return rc;
    }
    if ((rc = mark())) return rc;
    CK(cudaEventRecord(h->k_ev[slot_k].b, stream), "cudaEventRecord");
    h->k_ev[slot_k].kernels = (n_items ? 1 : 0) + ((n_pairs && any_tp) ? 1 : 0) + (has_lad ? 1 : 0) + (has_lit ? 1 : 0);
    if (h->k_used < h->k_ev.size()) h->k_used++;
    if (ms_out) {
        CK(cudaEventRecord(e1, stream), "cudaEventRecord");
        CK(cudaEventSynchronize(e1), "cudaEventSynchronize");
        CK(cudaEventElapsedTime(ms_out, e0, e1), "cudaEventElapsedTime");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    CK(cudaEventRecord(h->ws_ev, stream), "cudaEventRecord");
    h->ws_ev_pending = true;
    return MAGUS_OK;
}

int check_run_args(magus_replay *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
                   const magus_freq_log_t *log, const double *e, const double *edp) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    if (n_traces < 0) { set_error("n_traces must be >= 0"); return MAGUS_EINVAL; }
    if (n_traces > 0 && (!lengths || !traces)) { set_error("traces and lengths are required"); return MAGUS_EINVAL; }
    if (((uintptr_t)traces & 15u) != 0) { set_error("traces must be 16-byte aligned"); return MAGUS_EINVAL; }
    if (n_traces > 0 && (!e || !edp)) { set_error("out_energy and out_edp are required"); return MAGUS_EINVAL; }
    if (log && log->entries && log->capacity == 0) { set_error("log capacity must be >= 1"); return MAGUS_EINVAL; }
    for (int i = 0; i < n_traces; i++) {
        if (lengths[i] >= (1ull << 40)) { set_error("trace length too large"); return MAGUS_EINVAL; }
        if (log && log->entries && lengths[i] >= (1ull << 27) - 1) {
            set_error("change-log entries hold interval indices below 2^27");
            return MAGUS_EINVAL;
        }
    }
    return MAGUS_OK;
}

Outs outs_of(const magus_freq_log_t *log, double *e, double *edp, double *t, magus_state_t *st) {
    Outs o;
    memset(&o, 0, sizeof(o));
    o.energy = e;
    o.edp = edp;
    o.time = t;
    o.state = st;
    if (log) {
        o.log_entries = log->entries;
        o.log_cap = log->entries ? log->capacity : 0;
        o.n_changes = log->n_changes;
        o.change_hash = log->change_hash;
        o.n_hf = log->n_hf;
    }
    return o;
}


// Plain kernel: one launch per trace (optionally with per-interval logs for one trace).
int plain_impl(magus_replay *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
               const magus_policy_t *configs, int32_t n_configs, const magus_freq_log_t *log, double *out_energy,
               double *out_edp, double *out_time, uint8_t *level_log, double *deriv_log, cudaStream_t s) {
    try {
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        std::vector<DevPolicy> pols;
        int rc = check_policies(h, configs, n_configs, &pols, false);
        if (rc) return rc;
        const size_t sz = pols.size() * sizeof(DevPolicy);
        rc = ensure_ws(h, &h->ws, &h->ws_size, sz);
        if (rc) return rc;
        const int slot = h->pin_next;
        h->pin_next ^= 1;
        rc = ensure_pin(h, slot, sz);
        if (rc) return rc;
        memcpy(h->pin[slot], pols.data(), sz);
        if (h->ws_ev_pending) CK(cudaStreamWaitEvent(s, h->ws_ev, 0), "cudaStreamWaitEvent");
        CK(cudaMemcpyAsync(h->ws, h->pin[slot], sz, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
        CK(cudaEventRecord(h->pin_ev[slot], s), "cudaEventRecord");
        h->pin_pending[slot] = true;
        Outs o = outs_of(log, out_energy, out_edp, out_time, nullptr);
        uint64_t off = 0;
        for (int i = 0; i < n_traces; i++) {
            PlainParams p;
            memset(&p, 0, sizeof(p));
            p.trace = traces + off;
            p.n = lengths[i];
            p.pols = (const DevPolicy *)h->ws;
            p.n_pols = n_configs;
            p.pair_base = (int64_t)i * n_configs;
            p.model = h->dm;
            p.energy = o.energy;
            p.edp = o.edp;
            p.time = o.time;
            p.log_entries = o.log_entries;
            p.log_cap = o.log_cap;
            p.n_changes = o.n_changes;
            p.change_hash = o.change_hash;
            p.n_hf = o.n_hf;
            p.level_log = level_log;
            p.deriv_log = deriv_log;
            CK(launch_replay_plain(p, s), "plain kernel launch");
            off += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
        }
        CK(cudaEventRecord(h->ws_ev, s), "cudaEventRecord");
        h->ws_ev_pending = true;
        return MAGUS_OK;
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return MAGUS_ENOMEM;
    }
}

}  // namespace

extern "C" {

const char *magus_last_error(void) { return last_error_cstr(); }
const char *magus_version(void) { return kVersion; }

int magus_packed_size(const uint64_t *lengths, int32_t n_traces, uint64_t *offsets, uint64_t *total) {
    if (n_traces < 0 || (n_traces > 0 && !lengths) || !total) {
        set_error("invalid arguments");
        return MAGUS_EINVAL;
    }
    uint64_t off = 0;
    for (int i = 0; i < n_traces; i++) {
        if (offsets) offsets[i] = off;
        off += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
    }
    *total = off;
    return MAGUS_OK;
}

int magus_policy_bounds(const magus_policy_t *policy, const magus_model_t *model, int64_t out[4]) {
    if (!policy || !model || !out) { set_error("NULL argument"); return MAGUS_EINVAL; }
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) { set_error(err); return rc; }
    DevPolicy dp;
    rc = derive_policy(*policy, *model, &dp, &err);
    if (rc) { set_error(err); return rc; }
    out[0] = dp.up_mid;
    out[1] = dp.dn_mid;
    out[2] = dp.kmin;
    out[3] = 3;
    return MAGUS_OK;
}

int magus_replay_open(magus_replay_t **out, const magus_model_t *model, int device, size_t mem_budget) {
    if (!out || !model) { set_error("NULL argument"); return MAGUS_EINVAL; }
    *out = nullptr;
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) { set_error(err); return rc; }
    magus_replay *h = new (std::nothrow) magus_replay();
    if (!h) { set_error("out of host memory"); return MAGUS_ENOMEM; }
    h->f.assign(model->f_ghz, model->f_ghz + model->n_levels);
    h->model = *model;
    h->model.f_ghz = h->f.data();
    h->dm = dm;
    h->device = device;
    h->budget = mem_budget ? mem_budget : ((size_t)1 << 30);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&h->status, 256);
    if (e == cudaSuccess) h->queue = (unsigned int *)((char *)h->status + 128);
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, 256);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ws_ev, cudaEventDisableTiming);
    for (int s = 0; s < 2 && e == cudaSuccess; s++) e = cudaEventCreateWithFlags(&h->pin_ev[s], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        magus_replay_close(h);
        return cuda_fail(e, "magus_replay_open");
    }
    *out = h;
    return MAGUS_OK;
}

int magus_replay_close(magus_replay_t *h) {
    if (!h) return MAGUS_OK;
    cudaSetDevice(h->device);
    if (h->ws_ev_pending) cudaEventSynchronize(h->ws_ev);
    for (int s = 0; s < 2; s++) {
        if (h->pin_pending[s]) cudaEventSynchronize(h->pin_ev[s]);
        if (h->pin[s]) cudaFreeHost(h->pin[s]);
        if (h->pin_ev[s]) cudaEventDestroy(h->pin_ev[s]);
    }
    for (int s = 0; s < 2; s++) {
        if (h->hs_ready[s]) cudaEventDestroy(h->hs_ready[s]);
        if (h->hs_done[s]) cudaEventDestroy(h->hs_done[s]);
    }
    if (h->hs_copy) cudaStreamDestroy(h->hs_copy);
    if (h->hs_comp) cudaStreamDestroy(h->hs_comp);
    for (auto &ev : h->k_ev) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.m);
        cudaEventDestroy(ev.b);
    }
    if (h->ws) cudaFree(h->ws);
    if (h->scratch) cudaFree(h->scratch);
    if (h->segbuf) cudaFree(h->segbuf);
    if (h->status) cudaFree(h->status);
    if (h->ws_ev) cudaEventDestroy(h->ws_ev);
    delete h;
    return MAGUS_OK;
}

int magus_replay_set_tile(magus_replay_t *h, int32_t tg, int32_t cw) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    if (tg == 0 && cw == 0) {
        h->tile_tg = h->tile_cw = 0;
        return MAGUS_OK;
    }
    if (!((tg == 8 && cw == 1) || (tg == 4 && cw == 2) || (tg == 2 && cw == 4) || (tg == 1 && cw == 8))) {
        set_error("supported tiles: (8,1) (4,2) (2,4) (1,8)");
        return MAGUS_EINVAL;
    }
    h->tile_tg = tg;
    h->tile_cw = cw;
    return MAGUS_OK;
}

int magus_replay_set_segments(magus_replay_t *h, int32_t seg_rounds) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    if (seg_rounds < -1 || (seg_rounds > 0 && (seg_rounds % 1024 != 0 || seg_rounds > (1 << 24)))) {
        set_error("segment rounds must be -1 (automatic), 0 (tile kernel) or a multiple of 1024 up to 2^24");
        return MAGUS_EINVAL;
    }
    h->seg_rounds = seg_rounds;
    return MAGUS_OK;
}

int magus_replay_run(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
                     const magus_policy_t *configs, int32_t n_configs, const magus_freq_log_t *log,
                     double *out_energy, double *out_edp, double *out_time, magus_state_t *io_state,
                     void *stream) {
    try {
        int rc = check_run_args(h, traces, lengths, n_traces, log, out_energy, out_edp);
        if (rc) return rc;
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        std::vector<DevPolicy> pols;
        rc = check_policies(h, configs, n_configs, &pols, true);
        if (rc) return rc;
        int tg, cw, gp, seg;
        choose_tile(h, pols, lengths, n_traces, &tg, &cw, &gp, &seg);
        Plan pl;
        rc = build_plan(h, lengths, n_traces, configs, n_configs, tg, cw, gp, seg, &pl);
        if (rc) return rc;
        return launch_plan(h, pl, traces, outs_of(log, out_energy, out_edp, out_time, io_state),
                           (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return MAGUS_ENOMEM;
    }
}

int magus_replay_kernel_time(magus_replay_t *h, double *total_ms, double *main_ms, int32_t *runs,
                             int32_t *kernels) {
    if (!h || !total_ms || !runs) { set_error("NULL argument"); return MAGUS_EINVAL; }
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    double tot = 0, mn = 0;
    int32_t nk = 0;
    for (size_t i = 0; i < h->k_used; i++) {
        float ms = 0, ms_main = 0;
        CK(cudaEventSynchronize(h->k_ev[i].b), "cudaEventSynchronize");
        CK(cudaEventElapsedTime(&ms, h->k_ev[i].a, h->k_ev[i].b), "cudaEventElapsedTime");
        CK(cudaEventElapsedTime(&ms_main, h->k_ev[i].a, h->k_ev[i].m), "cudaEventElapsedTime");
        tot += ms;
        mn += ms_main;
        nk += h->k_ev[i].kernels;
    }
    *total_ms = tot;
    if (main_ms) *main_ms = mn;
    *runs = (int32_t)h->k_used;
    if (kernels) *kernels = nk;
    h->k_used = 0;
    return MAGUS_OK;
}

int magus_replay_status(magus_replay_t *h, void *stream) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    int st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(status)");
    if (st) {
        CK(cudaMemset(h->status, 0, sizeof(int)), "cudaMemset");
        set_error(st == MAGUS_ETIMEDOUT ? "a bounded device wait gave up"
                                        : "a carried level was neither 0 nor K-1");
    }
    return st;
}

int magus_replay_autotune(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
                          const magus_policy_t *configs, int32_t n_configs, int32_t *out_best, float *out_ms,
                          void *stream) {
    try {
        double *dummy = (double *)16;  // validated as non-NULL; real buffers come from scratch
        int rc = check_run_args(h, traces, lengths, n_traces, nullptr, dummy, dummy);
        if (rc) return rc;
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        const size_t pairs = (size_t)std::max(n_traces, 1) * n_configs;
        rc = ensure_ws(h, &h->scratch, &h->scratch_size, pairs * 16);
        if (rc) return rc;
        Outs o;
        memset(&o, 0, sizeof(o));
        o.energy = (double *)h->scratch;
        o.edp = o.energy + pairs;
        static const int shapes[14][4] = {{8, 1, 1, 0}, {4, 2, 1, 0}, {2, 4, 1, 0}, {1, 8, 1, 0},
                                          {8, 1, 4, 0}, {4, 2, 4, 0}, {2, 4, 4, 0}, {1, 8, 4, 0},
                                          {8, 1, 1, 8192}, {8, 1, 1, 16384}, {8, 1, 1, 32768},
                                          {8, 1, 4, 8192}, {8, 1, 4, 16384}, {8, 1, 4, 32768}};
        float best = 1e30f;
        int bt = 8, bc = 1, bg = 1, bs = 0;
        std::vector<DevPolicy> pols;
        rc = check_policies(h, configs, n_configs, &pols, true);
        if (rc) return rc;
        std::vector<PolicyGroup> g4;
        form_groups(pols, kMaxGroup, &g4);
        for (auto &sh : shapes) {
            const int n_groups = sh[2] == 1 ? n_configs : (int)g4.size();
            if (sh[2] > 1 && g4.size() == (size_t)n_configs) continue;   // nothing to share
            if (sh[1] > 1 && sh[1] / 2 >= n_groups) continue;            // more slots than groups
            Plan pl;
            rc = build_plan(h, lengths, n_traces, configs, n_configs, sh[0], sh[1], sh[2], sh[3], &pl);
            if (rc) return rc;
            float ms = 0, mn = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                rc = launch_plan(h, pl, traces, o, (cudaStream_t)stream, &ms);
                if (rc) return rc;
                if (rep) mn = std::min(mn, ms);
            }
            if (mn < best) {
                best = mn;
                bt = sh[0];
                bc = sh[1];
                bg = sh[2];
                bs = sh[3];
            }
        }
        h->tuned[n_configs] = {bt, bc, bg, bs};
        if (out_best) {
            out_best[0] = bt;
            out_best[1] = bc;
            out_best[2] = bg;
            out_best[3] = bs;
        }
        if (out_ms) *out_ms = best;
        return MAGUS_OK;
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return MAGUS_ENOMEM;
    }
}

int magus_replay_plain(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
                       const magus_policy_t *configs, int32_t n_configs, const magus_freq_log_t *log,
                       double *out_energy, double *out_edp, double *out_time, void *stream) {
    int rc = check_run_args(h, traces, lengths, n_traces, log, out_energy, out_edp);
    if (rc) return rc;
    return plain_impl(h, traces, lengths, n_traces, configs, n_configs, log, out_energy, out_edp, out_time,
                      nullptr, nullptr, (cudaStream_t)stream);
}

int magus_replay_detail(magus_replay_t *h, const uint32_t *trace, uint64_t n, const magus_policy_t *config,
                        uint8_t *out_level, double *out_derivative, const magus_freq_log_t *log,
                        double *out_energy, double *out_edp, double *out_time, void *stream) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    if (n > 0 && !trace) { set_error("trace is required"); return MAGUS_EINVAL; }
    if (!out_energy || !out_edp) { set_error("out_energy and out_edp are required"); return MAGUS_EINVAL; }
    if (log && log->entries && log->capacity == 0) { set_error("log capacity must be >= 1"); return MAGUS_EINVAL; }
    if (n >= (1ull << 27) - 1 && log && log->entries) {
        set_error("change-log entries hold interval indices below 2^27");
        return MAGUS_EINVAL;
    }
    uint64_t len = n;
    return plain_impl(h, trace, &len, 1, config, 1, log, out_energy, out_edp, out_time, out_level,
                      out_derivative, (cudaStream_t)stream);
}

int magus_replay_run_host(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths, int32_t n_traces,
                          const magus_policy_t *configs, int32_t n_configs, const magus_freq_log_t *log,
                          double *out_energy, double *out_edp, double *out_time) {
    try {
        if (n_traces > 0 && !traces) {
            set_error("traces and lengths are required");
            return MAGUS_EINVAL;
        }
        // host traces need no alignment: they are copied into an aligned device buffer
        int rc = check_run_args(h, (const uint32_t *)16, lengths, n_traces, log, out_energy, out_edp);
        if (rc) return rc;
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        if (!h->hs_comp) {
            CK(cudaStreamCreateWithFlags(&h->hs_comp, cudaStreamNonBlocking), "cudaStreamCreate");
            CK(cudaStreamCreateWithFlags(&h->hs_copy, cudaStreamNonBlocking), "cudaStreamCreate");
            for (int s = 0; s < 2; s++) {
                CK(cudaEventCreateWithFlags(&h->hs_ready[s], cudaEventDisableTiming), "cudaEventCreate");
                CK(cudaEventCreateWithFlags(&h->hs_done[s], cudaEventDisableTiming), "cudaEventCreate");
            }
        }
        std::vector<DevPolicy> pols;
        rc = check_policies(h, configs, n_configs, &pols, true);
        if (rc) return rc;
        int tg, cw, gp, seg;
        choose_tile(h, pols, lengths, n_traces, &tg, &cw, &gp, &seg);
        const bool has_log = log != nullptr;
        const uint64_t cap = (has_log && log->entries) ? log->capacity : 0;
        const size_t per_pair = 16 + (out_time ? 8 : 0) +
                                (has_log ? 8 * ((log->n_changes ? 1 : 0) + (log->change_hash ? 1 : 0) +
                                                (log->n_hf ? 1 : 0)) : 0) + (size_t)cap * 4;
        // two buffer slots, each holding one batch of traces and its outputs
        const size_t slot_bytes = std::min<size_t>(h->budget / 2 > (64u << 20) ? h->budget / 2 - (32u << 20)
                                                                              : (16u << 20),
                                                   (size_t)512 << 20);
        std::vector<std::pair<int, int>> batches;
        for (int i = 0; i < n_traces;) {
            size_t bytes = 0;
            int j = i;
            while (j < n_traces) {
                size_t add = align_up((lengths[j] + kTraceAlign - 1) / kTraceAlign * kTraceAlign * 4, 256) + align_up(per_pair * n_configs, 256) + 2048;
                if (j > i && bytes + add > slot_bytes) break;
                bytes += add;
                j++;
            }
            if (bytes > slot_bytes) {
                set_error("one trace with its outputs exceeds half the memory budget");
                return MAGUS_ENOMEM;
            }
            batches.push_back({i, j});
            i = j;
        }
        rc = ensure_ws(h, &h->scratch, &h->scratch_size, 2 * slot_bytes);
        if (rc) return rc;
        std::vector<uint64_t> first_off(batches.size());
        {
            uint64_t off = 0;
            size_t b = 0;
            for (int i = 0; i < n_traces; i++) {
                if (b < batches.size() && batches[b].first == i) first_off[b++] = off;
                off += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
            }
        }
        for (size_t b = 0; b < batches.size(); b++) {
            const int slot = (int)(b & 1);
            const int i0 = batches[b].first, i1 = batches[b].second, nt = i1 - i0;
            char *base = (char *)h->scratch + slot * slot_bytes;
            uint64_t words = 0;
            for (int i = i0; i < i1; i++) words += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
            uint32_t *d_tr = (uint32_t *)base;
            char *p = base + align_up(words * 4, 256);
            const size_t np = (size_t)nt * n_configs;
            double *d_e = (double *)p; p += align_up(np * 8, 256);
            double *d_edp = (double *)p; p += align_up(np * 8, 256);
            double *d_t = nullptr;
            if (out_time) { d_t = (double *)p; p += align_up(np * 8, 256); }
            magus_freq_log_t dl;
            memset(&dl, 0, sizeof(dl));
            if (has_log) {
                if (log->n_changes) { dl.n_changes = (uint64_t *)p; p += align_up(np * 8, 256); }
                if (log->change_hash) { dl.change_hash = (uint64_t *)p; p += align_up(np * 8, 256); }
                if (log->n_hf) { dl.n_hf = (uint64_t *)p; p += align_up(np * 8, 256); }
                if (cap) { dl.entries = (uint32_t *)p; dl.capacity = cap; p += align_up(np * cap * 4, 256); }
            }
            // the copy into this slot waits until the slot's previous batch is finished
            if (b >= 2) CK(cudaStreamWaitEvent(h->hs_copy, h->hs_done[slot], 0), "cudaStreamWaitEvent");
            if (words) CK(cudaMemcpyAsync(d_tr, traces + first_off[b], words * 4, cudaMemcpyHostToDevice, h->hs_copy),
                          "cudaMemcpyAsync(traces)");
            CK(cudaEventRecord(h->hs_ready[slot], h->hs_copy), "cudaEventRecord");
            CK(cudaStreamWaitEvent(h->hs_comp, h->hs_ready[slot], 0), "cudaStreamWaitEvent");
            Plan pl;
            rc = build_plan(h, lengths + i0, nt, configs, n_configs, tg, cw, gp, seg, &pl);
            if (rc) return rc;
            rc = launch_plan(h, pl, d_tr, outs_of(has_log ? &dl : nullptr, d_e, d_edp, d_t, nullptr), h->hs_comp);
            if (rc) return rc;
            const size_t po = (size_t)i0 * n_configs;
            CK(cudaMemcpyAsync(out_energy + po, d_e, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
            CK(cudaMemcpyAsync(out_edp + po, d_edp, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
            if (out_time) CK(cudaMemcpyAsync(out_time + po, d_t, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
            if (has_log) {
                if (log->n_changes) CK(cudaMemcpyAsync(log->n_changes + po, dl.n_changes, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
                if (log->change_hash) CK(cudaMemcpyAsync(log->change_hash + po, dl.change_hash, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
                if (log->n_hf) CK(cudaMemcpyAsync(log->n_hf + po, dl.n_hf, np * 8, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
                if (cap) CK(cudaMemcpyAsync(log->entries + po * cap, dl.entries, np * cap * 4, cudaMemcpyDeviceToHost, h->hs_comp), "cudaMemcpyAsync");
            }
            CK(cudaEventRecord(h->hs_done[slot], h->hs_comp), "cudaEventRecord");
        }
        CK(cudaStreamSynchronize(h->hs_comp), "cudaStreamSynchronize");
        return magus_replay_status(h, h->hs_comp);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return MAGUS_ENOMEM;
    }
}
}  // extern "C"
