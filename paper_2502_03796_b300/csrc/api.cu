// api.cu - C ABI of libmagus: replay handles, argument checks, workspace helpers, entry points.
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

#include "replay_host.h"

using namespace magus;
using namespace magus::host;

namespace magus {
namespace host {

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return MAGUS_ECUDA;
}

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
    size_t other = h->ws_size + h->scratch_size + h->seg_size + h->cls_size[0] + h->cls_size[1] + h->st_size - *size;
    if (want + other > h->budget) want = need;
    if (want + other > h->budget) {
        set_error("device workspace of " + std::to_string(need) + " bytes exceeds the handle's memory budget");
        return MAGUS_ENOMEM;
    }
    if (h->ws_ev_pending) CK(cudaEventSynchronize(h->ws_ev), "cudaEventSynchronize");
    if (buf == &h->ws) h->ws_plan_valid = false;
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

// Derive every policy (errors name the policy); which kernel replays it is decided later
// (tp_policy / ladder_policy).
int check_policies(magus_replay *h, const magus_policy_t *configs, int32_t n_configs,
                   std::vector<DevPolicy> *out) {
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
    }
    return MAGUS_OK;
}

}  // namespace host
}  // namespace magus

namespace {

const char *kVersion = "magus-b300 0.1 (sm_103a)";

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
        int rc = check_policies(h, configs, n_configs, &pols);
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
        h->ws_plan_valid = false;
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

int magus_policy_fp64_thresholds(const magus_policy_t *policy, const magus_model_t *model, double out[2]) {
    if (!policy || !model || !out) { set_error("NULL argument"); return MAGUS_EINVAL; }
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) { set_error(err); return rc; }
    DevPolicy dp;
    rc = derive_policy(*policy, *model, &dp, &err);
    if (rc) { set_error(err); return rc; }
    out[0] = dp.up_last;
    out[1] = dp.dn_last;
    return MAGUS_OK;
}

int magus_policy_closed_thresholds(const magus_policy_t *policy, const magus_model_t *model, int64_t out[11]) {
    if (!policy || !model || !out) { set_error("NULL argument"); return MAGUS_EINVAL; }
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) { set_error(err); return rc; }
    DevPolicy dp;
    rc = derive_policy(*policy, *model, &dp, &err);
    if (rc) { set_error(err); return rc; }
    ClosedThr c;
    derive_closed(dp, dm, false, &c);
    out[10] = 0;
    for (int l = 0; l < 2; l++) {
        out[0 + l] = c.cthr[l];
        out[2 + l] = c.bu[l];
        out[4 + l] = c.bd[l];
        out[6 + l] = c.au[l];
        out[8 + l] = c.ad[l];
        for (int lb = 0; lb < 2; lb++) {
            if ((c.ccu[l] >> lb) & 1u) out[10] |= 1 << (2 * l + lb);
            if ((c.ccd[l] >> lb) & 1u) out[10] |= 1 << (4 + 2 * l + lb);
        }
    }
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
    if (h->stbuf) cudaFree(h->stbuf);
    for (int m = 0; m < 2; m++)
        if (h->clsbuf[m]) cudaFree(h->clsbuf[m]);
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
    if (!((tg == 8 && cw == 1) || (tg == 4 && cw == 2) || (tg == 2 && cw == 4) || (tg == 1 && cw == 8) ||
          (tg == 4 && cw == 1) || (tg == 1 && cw == 4) || (tg == 2 && cw == 2))) {
        set_error("supported tiles: (8,1) (4,2) (2,4) (1,8) (4,1) (1,4) (2,2)");
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

int magus_replay_set_wait(magus_replay_t *h, uint64_t chunk_wait_ns) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    h->chunk_wait_ns = chunk_wait_ns;
    return MAGUS_OK;
}

int magus_replay_set_closed(magus_replay_t *h, int32_t seg_rounds, int32_t burn_rounds) {
    if (!h) { set_error("NULL handle"); return MAGUS_EINVAL; }
    if (seg_rounds < -1 || (seg_rounds > 0 && (seg_rounds % 64 != 0 || seg_rounds > (1 << 24)))) {
        set_error("closed-loop segment rounds must be -1 (literal kernel), 0 (automatic) or a multiple of 64 up to 2^24");
        return MAGUS_EINVAL;
    }
    if (burn_rounds < -1 || (burn_rounds >= 0 && (burn_rounds % 64 != 0 || burn_rounds > (1 << 24)))) {
        set_error("burn-in rounds must be -1 (automatic) or a multiple of 64 up to 2^24");
        return MAGUS_EINVAL;
    }
    h->cls_seg = seg_rounds;
    h->cls_burn = burn_rounds;
    return MAGUS_OK;
}

int magus_replay_closed_stats(magus_replay_t *h, uint64_t *out4) {
    if (!h || !out4) { set_error("NULL argument"); return MAGUS_EINVAL; }
    out4[0] = out4[1] = out4[2] = out4[3] = 0;
    for (int m = 0; m < 2; m++) {
        if (!h->cls_stats[m]) continue;
        if (h->ws_ev_pending) CK(cudaEventSynchronize(h->ws_ev), "cudaEventSynchronize");
        unsigned long long st[3] = {0, 0, 0};
        CK(cudaMemcpy(st, h->cls_stats[m], sizeof(st), cudaMemcpyDeviceToHost), "cudaMemcpy(closed stats)");
        out4[0] += h->cls_items[m];
        out4[1] += st[0];
        out4[2] += st[1];
        out4[3] += st[2];
    }
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
        rc = check_policies(h, configs, n_configs, &pols);
        if (rc) return rc;
        route_pins(&pols, h->model.n_levels, io_state != nullptr);
        int tg, cw, gp, seg;
        choose_tile(h, pols, lengths, n_traces, &tg, &cw, &gp, &seg);
        Plan pl;
        rc = build_plan(h, lengths, n_traces, configs, n_configs, tg, cw, gp, seg, &pl, io_state != nullptr);
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
        static const int shapes[17][4] = {{8, 1, 1, 0}, {4, 1, 1, 0}, {4, 2, 1, 0}, {2, 4, 1, 0}, {1, 8, 1, 0},
                                          {8, 1, 4, 0}, {4, 2, 4, 0}, {2, 4, 4, 0}, {1, 8, 4, 0}, {1, 4, 4, 0},
                                          {2, 2, 4, 0},
                                          {8, 1, 1, 8192}, {8, 1, 1, 16384}, {8, 1, 1, 32768},
                                          {8, 1, 4, 8192}, {8, 1, 4, 16384}, {8, 1, 4, 32768}};
        float best = 1e30f;
        int bt = 8, bc = 1, bg = 1, bs = 0;
        std::vector<DevPolicy> pols;
        rc = check_policies(h, configs, n_configs, &pols);
        if (rc) return rc;
        route_pins(&pols, h->model.n_levels, false);
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
        rc = check_policies(h, configs, n_configs, &pols);
        if (rc) return rc;
        route_pins(&pols, h->model.n_levels, false);
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
