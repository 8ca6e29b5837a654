// launch.cu - planning (kernel choice, policy routing, work items) and the launches of the
// replay kernels: tile or segment kernel for the jump mode, ladder kernel for the one-rung
// mode, the segmented closed-loop kernels for the closed loop (both step modes), literal
// kernel for the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "replay_host.h"

namespace magus {
namespace host {

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
        // (4, 1) takes one-member groups only, (1, 4) and (2, 2) groups of up to four (of one
        // member each, where no policies share Algorithm 1)
        if (!tp_tile_supported(*tg, *cw, *gp)) *gp = (*gp == 1) ? kMaxGroup : 1;
    } else if (*gp > 1 && n_groups >= 2) {
        // grouped policies: a 4-warp tile, four slots from eight groups on (policy sweep,
        // 64 groups: 39.9 ms against 44.0 for 1 x 8), else two slots of two warps (uneven
        // lengths, 4 groups: 35.3 ms against 38.9 for 2 x 4)
        *cw = n_groups >= 8 ? 4 : 2;
        *tg = n_groups >= 8 ? 1 : 2;
    } else {
        int c = 1;
        while (c * 2 <= std::min(8, n_groups)) c *= 2;
        *cw = c;
        // one policy group: the 4-warp tile (six CTAs per SM, barriers among 4 warps; 3.6 %
        // faster than 8 warps on 4,096 x 100,000 at equal residency)
        *tg = (c == 1 && *gp == 1) ? 4 : 8 / c;
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

void route_pins(std::vector<DevPolicy> *pols, int n_levels, bool with_state) {
    if (with_state) return;
    bool any = false;
    for (const DevPolicy &d : *pols) any = any || static_policy(d, n_levels);
    if (!any) return;
    for (DevPolicy &d : *pols)
        if (d.pin > 0 && tp_policy(d, n_levels)) d.to_static = 1;
}

int build_plan(magus_replay *h, const uint64_t *lengths, int32_t n_traces, const magus_policy_t *configs,
               int32_t n_configs, int tg, int cw, int gp, int seg, Plan *pl, bool with_state) {
    int rc = check_policies(h, configs, n_configs, &pl->pols);
    if (rc) return rc;
    route_pins(&pl->pols, h->model.n_levels, with_state);
    pl->tg = tg;
    pl->cw = cw;
    pl->gp = gp;
    pl->seg_len = seg;
    pl->tp.resize(pl->pols.size());
    pl->lit.clear();
    std::vector<int32_t> lad_pols;
    pl->cls.clear();
    pl->cthr.clear();
    for (size_t i = 0; i < pl->pols.size(); i++) {
        pl->tp[i] = tp_policy(pl->pols[i], h->model.n_levels) ? 1 : 0;
        if (pl->tp[i]) continue;
        if (ladder_policy(pl->pols[i])) {
            lad_pols.push_back((int32_t)i);
        } else if (closed_policy(pl->pols[i])) {
            pl->cls.push_back((int32_t)i);
            // thresholds per rung take a few thousand FP64 bisection steps: kept per policy
            std::string key(reinterpret_cast<const char *>(&pl->pols[i]), sizeof(DevPolicy));
            auto it = h->cthr_cache.find(key);
            if (it == h->cthr_cache.end()) {
                if (h->cthr_cache.size() >= 16384) h->cthr_cache.clear();
                ClosedThr c;
                derive_closed(pl->pols[i], h->dm, pl->pols[i].step_mode == 3, &c);
                it = h->cthr_cache.emplace(key, c).first;
            }
            pl->cthr.push_back(it->second);
        } else {
            pl->lit.push_back((int32_t)i);
        }
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
    if (pl->items.size() > (size_t)INT32_MAX || (size_t)n_traces * lad_pols.size() > (size_t)INT32_MAX) {
        set_error("too many (trace, policy) work items");
        return MAGUS_EINVAL;
    }
    pl->lad.clear();
    pl->lad.reserve((size_t)n_traces * lad_pols.size());
    for (int i : order)
        for (int32_t c : lad_pols) pl->lad.push_back(LadderItem{(uint32_t)i, (uint32_t)c});
    // without carried state the pins among the literal policies take the static kernel
    pl->sit.clear();
    bool any_pin = false;
    for (int32_t c : pl->lit) any_pin = any_pin || pl->pols[c].pin > 0;
    if (!with_state && any_pin && n_traces > 0) {
        static_items(pl->lengths, h->sms, h->model.n_levels, &pl->sit);
        if (pl->sit.size() > (size_t)INT32_MAX) {
            set_error("too many static-kernel work items");
            return MAGUS_EINVAL;
        }
    }
    return MAGUS_OK;
}


// Upload the plan through pinned staging and launch the batched kernel on `stream`.
// The policies the time-parallel kernels do not replay: one thread per pair, all traces in
// one launch (replay_plain.cu).  d_*: the plan as uploaded to the workspace.
// Without carried state the pinned ones among them go to the static kernel (one pass over
// the trace at the pinned rung, replay_static.cu).  Adds the kernels launched to *kernels.
int launch_literal_part(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o,
                        const DevPolicy *d_pols, const uint64_t *d_off, const uint64_t *d_len, const int32_t *d_lit,
                        int32_t n_lit, const std::vector<int32_t> &lit, const StaticItem *d_sit, cudaStream_t stream,
                        int *kernels) {
    const bool split = o.state == nullptr && d_sit != nullptr;
    int n_pinned = 0;
    for (int32_t c : lit) n_pinned += pl.pols[c].pin > 0 ? 1 : 0;
    if (split && n_pinned > 0) {
        StaticParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.traces = traces;
        sp.offsets = d_off;
        sp.lengths = d_len;
        sp.n_traces = (int32_t)pl.lengths.size();
        sp.n_pols = (int32_t)pl.pols.size();
        sp.pols = d_pols;
        sp.lit = d_lit;
        sp.n_lit = n_lit;
        sp.model = h->dm;
        sp.energy = o.energy;
        sp.edp = o.edp;
        sp.time = o.time;
        sp.n_changes = o.n_changes;
        sp.change_hash = o.change_hash;
        sp.n_hf = o.n_hf;
        // a trace split into parts sums them in zeroed per-trace accumulators
        bool split_traces = false;
        for (const StaticItem &it : pl.sit) split_traces = split_traces || it.parts > 1;
        sp.items = d_sit;
        sp.n_items = (int32_t)pl.sit.size();
        if (split_traces) {
            const size_t n_tr = pl.lengths.size();
            const size_t sz_acc = align_up(n_tr * 2 * (MAGUS_MAX_LEVELS + 1) * sizeof(unsigned long long), 256);
            const size_t need = sz_acc + n_tr * sizeof(uint32_t);
            const int rc = ensure_ws(h, &h->stbuf, &h->st_size, need);
            if (rc) return rc;
            CK(cudaMemsetAsync(h->stbuf, 0, need, stream), "cudaMemsetAsync");
            sp.acc = (unsigned long long *)h->stbuf;
            sp.arrived = (uint32_t *)((char *)h->stbuf + sz_acc);
        }
        CK(launch_replay_static(sp, stream), "static kernel launch");
        *kernels += 1;
        if (n_pinned == (int)lit.size()) return MAGUS_OK;
    }
    LiteralParams lp;
    memset(&lp, 0, sizeof(lp));
    lp.traces = traces;
    lp.offsets = d_off;
    lp.lengths = d_len;
    lp.n_traces = (int32_t)pl.lengths.size();
    lp.n_pols = (int32_t)pl.pols.size();
    lp.pols = d_pols;
    lp.lit = d_lit;
    lp.n_lit = n_lit;
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
    lp.skip_pinned = split ? 1 : 0;
    CK(launch_replay_literal(lp, stream), "literal kernel launch");
    *kernels += 1;
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
    // the window length every one-rung item shares, if any
    int window = pl.lad.empty() ? 0 : pl.pols[pl.lad[0].pol].W;
    for (const LadderItem &it : pl.lad)
        if (pl.pols[it.pol].W != window) window = 0;
    const int per_sm = ladder_max_ctas_per_sm(window);
    if (per_sm <= 0) {
        set_error("ladder kernel does not fit on this device");
        return MAGUS_ECUDA;
    }
    const size_t ctas = (pl.lad.size() + ladder_warps_per_cta() - 1) / ladder_warps_per_cta();
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(ctas, (size_t)h->sms * per_sm));
    CK(cudaMemsetAsync(h->queue, 0, sizeof(unsigned int), stream), "cudaMemsetAsync");
    CK(launch_replay_ladder(lp, tmap, grid, stream, window), "ladder kernel launch");
    return MAGUS_OK;
}

int launch_seg_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                    float *ms_out);

int launch_plan(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, cudaStream_t stream,
                float *ms_out) {
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
    const size_t sz_sit = align_up(std::max<size_t>(pl.sit.size(), 1) * sizeof(StaticItem), 256);
    const size_t off_sit = off_lad + sz_lad;
    const size_t total = off_sit + sz_sit;
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
    if (!pl.sit.empty()) memcpy(pin + off_sit, pl.sit.data(), pl.sit.size() * sizeof(StaticItem));
    char *ws = (char *)h->ws;
    const bool same_plan = h->ws_plan_valid && h->ws_plan.size() == total && !memcmp(h->ws_plan.data(), pin, total);
    if (!same_plan) {
        if (h->ws_ev_pending) CK(cudaStreamWaitEvent(stream, h->ws_ev, 0), "cudaStreamWaitEvent");
        CK(cudaMemcpyAsync(ws, pin, total, cudaMemcpyHostToDevice, stream), "cudaMemcpyAsync(plan)");
        CK(cudaEventRecord(h->pin_ev[slot], stream), "cudaEventRecord");
        h->pin_pending[slot] = true;
        h->ws_plan.assign(pin, pin + total);
        h->ws_plan_valid = true;
    }
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
    p.chunk_wait_ns = h->chunk_wait_ns;
    // the window length every policy group shares, if any (selects a W-specific instance)
    int window = pl.groups.empty() ? 0 : pl.pols[pl.groups[0].member[0]].W;
    for (const PolicyGroup &g : pl.groups)
        if (pl.pols[g.member[0]].W != window) window = 0;
    int smem = 0;
    const int per_sm = tp_max_ctas_per_sm(pl.tg, pl.cw, pl.gp, &smem, window);
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
    CUtensorMap tmap, tmap_tail;
    memset(&tmap, 0, sizeof(tmap));
    memset(&tmap_tail, 0, sizeof(tmap_tail));
    if (n_items) {
        uint64_t total_elems = 0;
        for (size_t i = 0; i < pl.lengths.size(); i++)
            total_elems += (pl.lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
        std::string err;
        rc = make_trace_tmap(traces, total_elems, tp_box_rows(pl.tg), &tmap, &err);
        if (!rc) rc = make_trace_tmap(traces, total_elems, kTailRows, &tmap_tail, &err);
        if (rc) { set_error(err); return rc; }
    }
    const bool has_lit = !pl.lit.empty() && !pl.lengths.empty();
    const bool has_lad = !pl.lad.empty();
    const bool has_cls = !pl.cls.empty() && !pl.lengths.empty();
    if (n_items || has_lit || has_lad || has_cls) {
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
            CK(launch_replay_tp(pl.tg, pl.cw, pl.gp, p, tmap, tmap_tail, grid, stream, window), "replay kernel launch");
            if ((rc = mark())) return rc;
        }
        if (has_lad) {
            rc = launch_ladder_part(h, pl, traces, o, p.pols, p.offsets, p.lengths, (const LadderItem *)(ws + off_lad),
                                    stream);
            if (rc || (rc = mark())) return rc;
        }
        int lit_kernels = 0;
        if (has_lit) {
            rc = launch_literal_part(h, pl, traces, o, p.pols, p.offsets, p.lengths,
                                     (const int32_t *)(ws + sz_pol + sz_grp + sz_items + 2 * sz_off),
                                     (int32_t)pl.lit.size(), pl.lit,
                                     pl.sit.empty() ? nullptr : (const StaticItem *)(ws + off_sit), stream,
                                     &lit_kernels);
            if (rc || (rc = mark())) return rc;
        }
        int cls_kernels = 0;
        if (has_cls) {
            rc = launch_closed_part(h, pl, traces, o, p.pols, p.offsets, p.lengths, stream, &cls_kernels);
            if (rc || (rc = mark())) return rc;
        }
        CK(cudaEventRecord(h->k_ev[slot_k].b, stream), "cudaEventRecord");
        h->k_ev[slot_k].kernels = (n_items ? 1 : 0) + (has_lad ? 1 : 0) + lit_kernels + cls_kernels;
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
    const size_t sz_sit = align_up(std::max<size_t>(pl.sit.size(), 1) * sizeof(StaticItem), 256);
    const size_t off_sit = off_lad + sz_lad;
    const size_t total = off_sit + sz_sit;
    // device buffers: summaries | tails | change-log scratch
    const uint64_t n_pairs = (uint64_t)n_traces * n_pols;
    const size_t sz_sum = align_up(std::max<uint64_t>(total_segs * n_pols, 1) * sizeof(SegSummary), 256);
    const size_t sz_tail = align_up(std::max<uint64_t>(n_pairs, 1) * sizeof(SegTail), 256);
    const size_t sz_log = align_up(scratch_entries * 4, 256);
    const size_t seg_need = sz_sum + sz_tail + sz_log;
    // the tile kernel needs none of the segment buffers: take it when they do not fit
    if (std::max(total, h->ws_size) + h->scratch_size + h->cls_size[0] + h->cls_size[1] + h->st_size +
            std::max(seg_need, h->seg_size) >
        h->budget)
        return kUseTile;
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
    if (!pl.sit.empty()) memcpy(pin + off_sit, pl.sit.data(), pl.sit.size() * sizeof(StaticItem));
    if (h->ws_ev_pending) CK(cudaStreamWaitEvent(stream, h->ws_ev, 0), "cudaStreamWaitEvent");
    char *ws = (char *)h->ws;
    h->ws_plan_valid = false;
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
    // the window length every policy group shares, if any (selects a W-specific instance)
    int window = pl.groups.empty() ? 0 : pl.pols[pl.groups[0].member[0]].W;
    for (const PolicyGroup &g : pl.groups)
        if (pl.pols[g.member[0]].W != window) window = 0;
    const int per_sm = seg_max_ctas_per_sm(pl.gp, window);
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
        CK(launch_replay_seg(pl.gp, p, tmap, grid, stream, window), "segment kernel launch");
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
    int lit_kernels = 0;
    if (has_lit) {
        rc = launch_literal_part(h, pl, traces, o, p.pols, p.offsets, p.lengths,
                                 (const int32_t *)(ws + sz_pol + sz_grp + sz_items + 4 * sz_off),
                                 (int32_t)pl.lit.size(), pl.lit,
                                 pl.sit.empty() ? nullptr : (const StaticItem *)(ws + off_sit), stream, &lit_kernels);
        if (rc || (rc = mark())) return rc;
    }
    int cls_kernels = 0;
    if (!pl.cls.empty() && n_traces > 0) {
        rc = launch_closed_part(h, pl, traces, o, p.pols, p.offsets, p.lengths, stream, &cls_kernels);
        if (rc || (rc = mark())) return rc;
    }
    if ((rc = mark())) return rc;
    CK(cudaEventRecord(h->k_ev[slot_k].b, stream), "cudaEventRecord");
    h->k_ev[slot_k].kernels = (n_items ? 1 : 0) + ((n_pairs && any_tp) ? 1 : 0) + (has_lad ? 1 : 0) + lit_kernels +
                              cls_kernels;
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

// Closed-loop jump-mode policies (replay_closed.cu): every (trace, policy, time segment)
// replayed on its own thread from a guessed state, segments whose guess was wrong replayed
// again, then one thread per pair walks its segments in order.  The literal kernel takes
// them instead when the segmented replay is switched off or its buffers exceed the budget.
static int launch_closed_mode(magus_replay *h, const Plan &pl, int mode, const std::vector<int32_t> &cls,
                              const std::vector<ClosedThr> &cthr, const uint32_t *traces, const Outs &o,
                              const DevPolicy *d_pols, const uint64_t *d_off, const uint64_t *d_len,
                              cudaStream_t stream, int *kernels) {
    const int n_traces = (int)pl.lengths.size();
    const int n_cls = (int)cls.size();
    const bool ladder = mode == 1;
    int wmax = 1, wmin = 1 << 30;
    for (int32_t c : cls) {
        wmax = std::max(wmax, pl.pols[c].W);
        wmin = std::min(wmin, pl.pols[c].W);
    }
    uint32_t ring = 1;
    while ((int)ring < wmax) ring <<= 1;
    // every policy with the same W: the first-replay kernel's instance for that W
    const int window = wmin == wmax ? closed_window(wmax) : 0;
    // Every thread replays one segment (plus its burn-in) one round after another, so a
    // launch lasts about (waves of threads) x (segment + burn-in rounds).  Automatic choice:
    // for each wave count w, the shortest segment whose items fit w waves of resident
    // threads, burn-in min(512, S / 2) in jump mode and min(2048, S / 2) with one rung per
    // decision (a guessed rung takes longer to meet the true one: 512 rounds left 15 % of
    // the 4,096 x 100,000 segments to a second replay, 2,048 rounds 0.01 %); keep the
    // cheapest (cached per workload).
    auto burn_of = [&](uint64_t S) -> uint64_t {
        return h->cls_burn >= 0 ? (uint64_t)h->cls_burn
                                : std::min<uint64_t>(ladder ? 2048 : 512, S / 2 / 64 * 64);
    };
    uint64_t S = (uint64_t)h->cls_seg, G = 0;
    if (h->cls_seg > 0) {
        G = burn_of(S);
    } else {
        uint64_t key = 1469598103934665603ull ^ ((uint64_t)n_cls << 32) ^ ring ^ ((uint64_t)h->cls_burn << 48) ^
                       ((uint64_t)window << 24);
        uint64_t longest = 0;
        for (uint64_t n : pl.lengths) {
            key = (key ^ n) * 1099511628211ull;
            longest = std::max(longest, n);
        }
        if (key == h->cls_key[mode] && h->cls_auto_seg[mode]) {
            S = h->cls_auto_seg[mode];
            G = h->cls_auto_burn[mode];
        } else {
            const int ctas = closed_max_ctas_per_sm(ring, ladder, h->dm.K, window);
            const uint64_t resident = (uint64_t)h->sms * std::max(ctas, 1) * closed_threads_per_cta();
            auto items_of = [&](uint64_t L) {
                uint64_t it = 0;
                for (uint64_t n : pl.lengths) it += (n + L - 1) / L;
                return it * (uint64_t)n_cls;
            };
            const uint64_t top = std::max<uint64_t>(64, align_up(longest, 64));
            double best = 1e300;
            for (uint64_t w = 1; w <= 64; w++) {
                // shortest multiple of 64 with items_of(L) <= w * resident (non-increasing in L)
                if (items_of(top) > w * resident) continue;
                uint64_t lo = 0, hi = top / 64;   // items_of(64 * hi) fits
                while (hi - lo > 1) {
                    const uint64_t mid = (lo + hi) / 2;
                    if (items_of(64 * mid) <= w * resident) hi = mid;
                    else lo = mid;
                }
                const uint64_t L = 64 * hi;
                const double cost = (double)((items_of(L) + resident - 1) / resident) * (double)(L + burn_of(L));
                if (cost < best) {
                    best = cost;
                    S = L;
                }
                if (L <= 1024) break;
            }
            if (S == 0) S = top;   // more than 64 waves even with whole traces
            S = std::min<uint64_t>(S, (uint64_t)1 << 24);
            G = burn_of(S);
            h->cls_key[mode] = key;
            h->cls_auto_seg[mode] = S;
            h->cls_auto_burn[mode] = G;
        }
    }
    std::vector<uint64_t> ibase(n_traces + 1);
    uint64_t items = 0;
    for (int i = 0; i < n_traces; i++) {
        ibase[i] = items;
        items += (pl.lengths[i] + S - 1) / S * (uint64_t)n_cls;
    }
    ibase[n_traces] = items;
    const bool logging = o.log_entries && o.log_cap > 0;
    // buffer: policies | thresholds | item bases | counters | replay slots | rung histories
    // (one-rung mode) | log-pass jobs | entry scratch (per replay; a replay with more entries
    // leaves them to the log pass, so the scratch shrinks to what the budget holds)
    const size_t sz_cls = align_up((size_t)n_cls * 4, 256);
    const size_t sz_thr = align_up((size_t)n_cls * sizeof(ClosedThr), 256);
    const size_t sz_ib = align_up((size_t)(n_traces + 1) * 8, 256);
    const size_t plan_bytes = sz_cls + sz_thr + sz_ib;
    const size_t sz_st = 256;
    const size_t sz_slot = align_up((size_t)(2 * items) * sizeof(ClosedSlot), 256);
    const size_t sz_hist = ladder ? align_up((size_t)(4 * items) * MAGUS_MAX_WINDOW, 256) : 0;
    const size_t sz_job = logging ? align_up((size_t)items * sizeof(ClosedJob), 256) : 0;
    const size_t others = h->ws_size + h->scratch_size + h->seg_size + h->cls_size[1 - mode] + h->st_size;
    uint64_t scr_cap = logging ? std::min<uint64_t>(S, std::max<uint64_t>(64, S / 8)) : 0;
    auto need_of = [&](uint64_t cap) {
        return plan_bytes + sz_st + sz_slot + sz_hist + sz_job + align_up((size_t)(2 * items * cap) * 4, 256);
    };
    while (scr_cap > 0 && others + std::max(need_of(scr_cap), h->cls_size[mode]) > h->budget) scr_cap /= 2;
    const size_t need = need_of(scr_cap);
    const bool segmented = h->cls_seg >= 0 && items <= (uint64_t)INT32_MAX * closed_threads_per_cta() &&
                           others + std::max(need, h->cls_size[mode]) <= h->budget;
    int rc = ensure_ws(h, &h->clsbuf[mode], &h->cls_size[mode], segmented ? need : sz_cls);
    if (rc) return rc;
    char *buf = (char *)h->clsbuf[mode];
    std::vector<char> blob(segmented ? plan_bytes : sz_cls, 0);
    memcpy(blob.data(), cls.data(), (size_t)n_cls * 4);
    if (segmented) {
        memcpy(blob.data() + sz_cls, cthr.data(), (size_t)n_cls * sizeof(ClosedThr));
        memcpy(blob.data() + sz_cls + sz_thr, ibase.data(), (size_t)(n_traces + 1) * 8);
    }
    // the previous call's kernels may still read the buffer
    if (h->ws_ev_pending) CK(cudaStreamWaitEvent(stream, h->ws_ev, 0), "cudaStreamWaitEvent");
    CK(cudaMemcpyAsync(buf, blob.data(), blob.size(), cudaMemcpyHostToDevice, stream), "cudaMemcpyAsync(closed plan)");
    if (!segmented) return launch_literal_part(h, pl, traces, o, d_pols, d_off, d_len, (const int32_t *)buf, n_cls, cls,
                                               nullptr, stream, kernels);
    unsigned long long *stats = (unsigned long long *)(buf + plan_bytes);
    CK(cudaMemsetAsync(stats, 0, 3 * sizeof(unsigned long long), stream), "cudaMemsetAsync");
    // no stale log-pass jobs (the final pass sets those of every pair it completes)
    if (logging) CK(cudaMemsetAsync(buf + plan_bytes + sz_st + sz_slot + sz_hist, 0, sz_job, stream), "cudaMemsetAsync");
    ClosedParams cp;
    memset(&cp, 0, sizeof(cp));
    cp.traces = traces;
    cp.offsets = d_off;
    cp.lengths = d_len;
    cp.n_traces = n_traces;
    cp.n_pols = (int32_t)pl.pols.size();
    cp.pols = d_pols;
    cp.cls = (const int32_t *)buf;
    cp.thr = (const ClosedThr *)(buf + sz_cls);
    cp.n_cls = n_cls;
    cp.ring = ring;
    cp.window = window;
    cp.ibase = (const uint64_t *)(buf + sz_cls + sz_thr);
    cp.n_items = items;
    cp.seg_len = (uint32_t)S;
    cp.burn = (uint32_t)G;
    cp.model = h->dm;
    cp.slots = (ClosedSlot *)(buf + plan_bytes + sz_st);
    cp.lhist = ladder ? (uint8_t *)(buf + plan_bytes + sz_st + sz_slot) : nullptr;
    cp.jobs = logging ? (ClosedJob *)(buf + plan_bytes + sz_st + sz_slot + sz_hist) : nullptr;
    cp.scratch = scr_cap ? (uint32_t *)(buf + plan_bytes + sz_st + sz_slot + sz_hist + sz_job) : nullptr;
    cp.scr_cap = scr_cap;
    cp.energy = o.energy;
    cp.edp = o.edp;
    cp.time = o.time;
    cp.log_entries = o.log_entries;
    cp.log_cap = o.log_cap;
    cp.n_changes = o.n_changes;
    cp.change_hash = o.change_hash;
    cp.n_hf = o.n_hf;
    cp.state = o.state;
    cp.status = h->status;
    cp.stats = stats;
    CK(launch_replay_closed(cp, ladder, stream), "closed-loop kernel launch");
    *kernels += (items ? 3 : 1) + ((items && logging) ? 1 : 0);
    h->cls_items[mode] = items;
    h->cls_stats[mode] = stats;
    return MAGUS_OK;
}

// The closed-loop policies of a plan, jump mode and one rung per decision in turn (their own
// kernels and buffers).
int launch_closed_part(magus_replay *h, const Plan &pl, const uint32_t *traces, const Outs &o, const DevPolicy *d_pols,
                       const uint64_t *d_off, const uint64_t *d_len, cudaStream_t stream, int *kernels) {
    for (int mode = 0; mode < 2; mode++) {
        h->cls_items[mode] = 0;
        h->cls_stats[mode] = nullptr;
    }
    if (pl.cls.empty() || pl.lengths.empty()) return MAGUS_OK;
    for (int mode = 0; mode < 2; mode++) {
        std::vector<int32_t> cls;
        std::vector<ClosedThr> cthr;
        for (size_t i = 0; i < pl.cls.size(); i++)
            if ((pl.pols[pl.cls[i]].step_mode == 3) == (mode == 1)) {
                cls.push_back(pl.cls[i]);
                cthr.push_back(pl.cthr[i]);
            }
        if (cls.empty()) continue;
        const int rc = launch_closed_mode(h, pl, mode, cls, cthr, traces, o, d_pols, d_off, d_len, stream, kernels);
        if (rc) return rc;
    }
    return MAGUS_OK;
}

}  // namespace host
}  // namespace magus
