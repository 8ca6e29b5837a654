// noalloc.cu - batched replay for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they want a replay: code running
// inside another framework's memory pool, a process whose device memory is fully
// reserved up front, or a plug-in that is only handed ready-made buffers.  For them,
// magus_replay_run_static runs the same time-parallel kernel as magus_replay_run, but the
// kernel's planning scratch (policy table, work list, trace offsets and lengths, work
// counter, status word) lives in one file-scope __device__ array of fixed size instead of a
// handle's workspace.  Every GPU that loads the library holds that array until the process
// exits.  No device memory is allocated or freed by this path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "magus_internal.h"

using namespace magus;

namespace {

// 4 MiB: room for 4096 policies plus about 160,000 traces with one policy.
constexpr size_t kStaticScratchBytes = (size_t)MAGUS_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};   // device address of g_static_scratch per device

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail(const std::string &msg, int code) {
    set_error(msg);
    return code;
}

}  // namespace

extern "C" int magus_replay_run_static(const magus_model_t *model, const uint32_t *traces, const uint64_t *lengths,
                                       int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                                       const magus_freq_log_t *log, double *out_energy, double *out_edp,
                                       double *out_time, magus_state_t *io_state, void *stream) {
    if (!model) return fail("model is NULL", MAGUS_EINVAL);
    if (n_traces < 0) return fail("n_traces must be >= 0", MAGUS_EINVAL);
    if (n_traces > 0 && (!traces || !lengths)) return fail("traces and lengths are required", MAGUS_EINVAL);
    if (((uintptr_t)traces & 15u) != 0) return fail("traces must be 16-byte aligned", MAGUS_EINVAL);
    if (n_traces > 0 && (!out_energy || !out_edp)) return fail("out_energy and out_edp are required", MAGUS_EINVAL);
    if (!configs || n_configs < 1 || n_configs > 4096)
        return fail("configs must be non-NULL with 1 <= n_configs <= 4096", MAGUS_EINVAL);
    if (log && log->entries && log->capacity == 0) return fail("log capacity must be >= 1", MAGUS_EINVAL);
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) return fail(err, rc);
    std::vector<DevPolicy> pols(n_configs);
    for (int c = 0; c < n_configs; c++) {
        rc = derive_policy(configs[c], *model, &pols[c], &err);
        if (rc) return fail("policy " + std::to_string(c) + ": " + err, rc);
        if (configs[c].step_mode != 0) return fail("step_mode must be 0", MAGUS_EINVAL);
        if (configs[c].pin_level != 0 && configs[c].pin_level != 1 && configs[c].pin_level != model->n_levels)
            return fail("pin_level must be 0, 1 or n_levels", MAGUS_EINVAL);
    }
    // every trace needs at least 24 bytes of plan (offset, length, one work item): refuse a
    // trace count the scratch cannot hold before laying out the plan
    if ((size_t)n_traces * (2 * sizeof(uint64_t) + sizeof(WorkItem)) > kStaticScratchBytes)
        return fail("workload needs more than " + std::to_string(kStaticScratchBytes) +
                        " bytes of planning scratch; the static scratch holds " + std::to_string(kStaticScratchBytes) +
                        " (use magus_replay_run)",
                    MAGUS_EINVAL);
    for (int i = 0; i < n_traces; i++) {
        if (lengths[i] >= (1ull << 40)) return fail("trace length too large", MAGUS_EINVAL);
        if (log && log->entries && lengths[i] >= (1ull << 27) - 1)
            return fail("change-log entries hold interval indices below 2^27", MAGUS_EINVAL);
    }
    // policies sharing predictions form groups of up to 4; as many group slots per CTA as
    // there are groups (up to 8), the rest of the warps split time
    std::vector<PolicyGroup> groups;
    form_groups(pols, kMaxGroup, &groups);
    const int gp = (2 * groups.size() <= pols.size()) ? kMaxGroup : 1;
    if (gp == 1) form_groups(pols, 1, &groups);
    const int n_groups = (int)groups.size();
    int cw = 1;
    while (cw * 2 <= std::min(8, n_groups)) cw *= 2;
    const int tg = (cw == 1 && gp == 1) ? 4 : 8 / cw;   // the tile magus_replay_run picks
    const size_t blocks = (size_t)(n_groups + cw - 1) / cw;
    const size_t n_items = (size_t)n_traces * blocks;
    // scratch layout: [status, counter | policies | groups | items | offsets | lengths]
    const size_t off_pol = 256;
    const size_t off_grp = off_pol + align_up(pols.size() * sizeof(DevPolicy), 256);
    const size_t off_items = off_grp + align_up(groups.size() * sizeof(PolicyGroup), 256);
    const size_t off_off = off_items + align_up(std::max<size_t>(n_items, 1) * sizeof(WorkItem), 256);
    const size_t per_trace = align_up((size_t)std::max(n_traces, 1) * sizeof(uint64_t), 256);
    const size_t off_len = off_off + per_trace;
    const size_t total = off_len + per_trace;
    if (total > kStaticScratchBytes)
        return fail("workload needs " + std::to_string(total) + " bytes of planning scratch; the static scratch holds " +
                        std::to_string(kStaticScratchBytes) + " (use magus_replay_run)",
                    MAGUS_EINVAL);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(std::string("cudaGetDevice: ") + cudaGetErrorString(e), MAGUS_ECUDA);
    if (dev < 0 || dev >= kMaxDevices) return fail("device index out of range", MAGUS_EINVAL);
    char *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr)
                return fail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), MAGUS_ECUDA);
            g_scratch_ptr[dev] = ptr;
        }
        scratch = (char *)g_scratch_ptr[dev];
    }

    // host image of the plan (host memory only)
    std::vector<unsigned char> img(total, 0);
    memcpy(img.data() + off_pol, pols.data(), pols.size() * sizeof(DevPolicy));
    memcpy(img.data() + off_grp, groups.data(), groups.size() * sizeof(PolicyGroup));
    std::vector<int> order(n_traces);
    for (int i = 0; i < n_traces; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lengths[a] > lengths[b]; });
    WorkItem *items = (WorkItem *)(img.data() + off_items);
    size_t k = 0;
    for (int i : order)
        for (size_t b = 0; b < blocks; b++) items[k++] = WorkItem{(uint32_t)i, (uint32_t)(b * cw)};
    uint64_t *offs = (uint64_t *)(img.data() + off_off);
    uint64_t *lens = (uint64_t *)(img.data() + off_len);
    uint64_t o = 0;
    for (int i = 0; i < n_traces; i++) {
        offs[i] = o;
        lens[i] = lengths[i];
        o += (lengths[i] + kTraceAlign - 1) / kTraceAlign * kTraceAlign;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the copy also zeroes the status word and the work counter (first 256 bytes)
    e = cudaMemcpyAsync(scratch, img.data(), total, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e), MAGUS_ECUDA);
    if (n_items) {
        TpParams p;
        memset(&p, 0, sizeof(p));
        p.traces = traces;
        p.pols = (const DevPolicy *)(scratch + off_pol);
        p.n_pols = n_configs;
        p.groups = (const PolicyGroup *)(scratch + off_grp);
        p.n_groups = n_groups;
        p.items = (const WorkItem *)(scratch + off_items);
        p.n_items = (int32_t)n_items;
        p.offsets = (const uint64_t *)(scratch + off_off);
        p.lengths = (const uint64_t *)(scratch + off_len);
        p.queue = (unsigned int *)(scratch + 128);
        p.status = (int *)scratch;
        p.model = dm;
        p.energy = out_energy;
        p.edp = out_edp;
        p.time = out_time;
        if (log) {
            p.log_entries = log->entries;
            p.log_cap = log->entries ? log->capacity : 0;
            p.n_changes = log->n_changes;
            p.change_hash = log->change_hash;
            p.n_hf = log->n_hf;
        }
        p.state = io_state;
        // the window length every policy group shares, if any (selects a W-specific instance)
        int window = groups.empty() ? 0 : pols[groups[0].member[0]].W;
        for (const PolicyGroup &g : groups)
            if (pols[g.member[0]].W != window) window = 0;
        int smem = 0;
        const int per_sm = tp_max_ctas_per_sm(tg, cw, gp, &smem, window);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || per_sm <= 0) return fail("device query failed", MAGUS_ECUDA);
        const int grid = (int)std::max<size_t>(1, std::min<size_t>(n_items, (size_t)sms * per_sm));
        CUtensorMap tmap, tmap_tail;
        rc = make_trace_tmap(traces, o, tp_box_rows(tg), &tmap, &err);
        if (!rc) rc = make_trace_tmap(traces, o, kTailRows, &tmap_tail, &err);
        if (rc) return fail(err, rc);
        e = launch_replay_tp(tg, cw, gp, p, tmap, tmap_tail, grid, s, window);
        if (e != cudaSuccess) return fail(std::string("replay kernel launch: ") + cudaGetErrorString(e), MAGUS_ECUDA);
    }
    // synchronous: the scratch is reused by the next call, and device-side input errors
    // (a carried level that is neither 0 nor K-1) are reported here
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e), MAGUS_ECUDA);
    int status = 0;
    e = cudaMemcpy(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(std::string("cudaMemcpy(status): ") + cudaGetErrorString(e), MAGUS_ECUDA);
    if (status) return fail(status == MAGUS_ETIMEDOUT ? "a bounded device wait gave up"
                                                      : "a carried level was neither 0 nor K-1", status);
    return MAGUS_OK;
}
