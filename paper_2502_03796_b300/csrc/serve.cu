// serve.cu - online MAGUS controller over many node streams (continuous batching).
//
// Each stream keeps its replay state (intervals seen, level, the last 64 flags and deltas)
// in a device-resident table.  Requests carry new counter deltas of one stream.  A launcher
// thread packs the requests waiting at that moment into a batch (at most one request per
// stream per batch, so a stream's requests apply in submission order), copies the batch to
// the device and launches it as a CUDA graph (H2D copy -> serve kernel -> D2H results).  Up
// to two batches are in flight, so requests that arrive while one batch runs are admitted
// into the next; a completer thread waits for batches in order and publishes the results.
//
// The serve kernel runs one warp per request: the request's deltas go through shared memory
// in sub-blocks of 1024 rounds with the same row machinery as the batched replay
// (replay_core.cuh): Alg. 1 predictions, Alg. 2 high-frequency state, the jump-to-bound
// latch and the energy charge, continuing from the stream's stored state.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "magus_internal.h"
#include "replay_core.cuh"

using namespace magus;

namespace {

constexpr int SB = 1024;
constexpr int HALO = 64;
constexpr int SERVE_WARPS = 8;
constexpr uint32_t kMaxRequestDeltas = 65536;

struct alignas(16) ServeReq {
    uint32_t stream;
    uint32_t n;
    uint64_t off;        // element offset of the request's deltas in the payload area
};

struct alignas(16) ServeOut {
    uint64_t n_seen;
    uint32_t level, n_changes;
    uint64_t hash;
    uint32_t n_hf, pad;
    double energy, time;
};

struct alignas(16) ServeHeader {
    uint32_t n_req;
    uint32_t pad;
    uint64_t payload_off;  // byte offset of the payload area from the batch base
};

struct ServeParams {
    const char *batch;         // device: header, requests, payload
    ServeOut *out;             // device results [n_req]
    magus_state_t *table;      // device stream states
    DevPolicy P;
    DevModel M;
};

// One warp per request; state loaded from and stored back to the stream table.  Each warp
// owns a 5 KB shared buffer: a 1024-byte block whose last two rows hold the 64 deltas
// before the current sub-block, then 32 rows of 32 deltas in the 128-byte swizzled layout
// of replay_core.cuh (written here with plain stores).
__global__ void __launch_bounds__(SERVE_WARPS * 32) serve_kernel(const ServeParams p) {
    using namespace core;
    __shared__ __align__(1024) uint32_t buf[SERVE_WARPS][(1024 + SB * 4) / 4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const ServeHeader *hdr = (const ServeHeader *)p.batch;
    const uint32_t n_req = hdr->n_req;
    const ServeReq *reqs = (const ServeReq *)(p.batch + sizeof(ServeHeader));
    const uint32_t *payload = (const uint32_t *)(p.batch + hdr->payload_off);
    const DevPolicy &P = p.P;
    const DevModel &M = p.M;
    const uint32_t topK = (uint32_t)(M.K - 1);
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    const uint32_t base = smem_u32(buf[wib]) + 1024;   // data row 0
    for (uint32_t r = blockIdx.x * SERVE_WARPS + wib; r < n_req; r += gridDim.x * SERVE_WARPS) {
        const ServeReq rq = reqs[r];
        magus_state_t &st = p.table[rq.stream];
        const uint64_t n_seen0 = st.n_seen;
        uint64_t tailH = st.flags;
        uint32_t level = st.level ? 1u : 0u;
        if (P.pin) level = P.pin > 1 ? 1u : 0u;   // a static baseline holds its level
        for (int k = lane; k < HALO; k += 32) sts32(swz_elem(base, k - HALO), st.hist[k]);
        const uint32_t *src = payload + rq.off;
        const uint64_t n = rq.n;
        Acc acc;
        acc_zero(acc);
        uint32_t nch = 0;
        for (uint64_t c0 = 0; c0 < n; c0 += SB) {
            if (c0 > 0) {
                // rows 30, 31 become rows -2, -1 (same swizzle phase)
                __syncwarp();
                const uint32_t h0 = lds32(base + 30 * 128 + 4 * lane), h1 = lds32(base + 30 * 128 + 128 + 4 * lane);
                __syncwarp();
                sts32(base - 256 + 4 * lane, h0);
                sts32(base - 128 + 4 * lane, h1);
            }
            const uint64_t cnt = n - c0 < (uint64_t)SB ? n - c0 : (uint64_t)SB;
            for (uint32_t k = lane; k < SB; k += 32) sts32(swz_elem(base, (int)k), k < cnt ? src[c0 + k] : 0u);
            __syncwarp();
            const int64_t r0 = (int64_t)c0 + 32 * lane;
            const int64_t left = (int64_t)n - r0;
            const uint32_t vmask = valid_mask(left);
            const uint32_t pmask = predict_mask(vmask, n_seen0 + (uint64_t)r0, P.W);
            const RowPred rp = row_predict(base, lane, P, M, vmask, pmask);
            const uint32_t FL = rp.UP | rp.DN;
            const uint64_t H = row_history(FL, tailH, lane);
            const uint32_t act = P.pin ? 0u : FULL;   // static baselines run no control
            const uint32_t HF = hf_row(H, FL, P.L, P.kmin) & vmask & act;
            const uint32_t SETM = (HF | rp.UP) & act;
            const uint32_t SET0 = rp.DN & ~HF & act;
            const uint32_t EV = SETM | SET0;
            const bool has = EV != 0;
            // disjoint masks: the last event sets the top exactly when SETM > SET0
            const uint32_t exitv = SETM > SET0 ? 1u : 0u;
            const uint32_t bev = __ballot_sync(FULL, has), bex = __ballot_sync(FULL, exitv);
            const uint32_t prior = bev & lanemask_lt;
            const uint32_t pex = bex & lanemask_lt;
            const uint32_t cin = prior ? (pex > (prior ^ pex) ? 1u : 0u) : level;
            const uint32_t Lm = latch_row(SETM, SET0, cin);
            const uint32_t Flev = (Lm << 1) | cin;
            const uint32_t CHG = (Lm ^ Flev) & vmask;
            row_energy(base, lane, Flev, rp, vmask, acc);
            acc.hf += __popc(HF);
            nch += __popc(CHG);
            if (__any_sync(FULL, CHG != 0))
                emit_changes(CHG, Lm, n_seen0 + c0, topK, nullptr, 0, 0, acc.hash, lane);
            // final state of the request, written by the lane holding its last round
            if (left >= 1 && left <= 32) {
                const int pl = (int)left - 1;
                st.n_seen = n_seen0 + n;
                st.level = ((Lm >> pl) & 1u) ? topK : 0u;
                st.flags = (H >> (pl + 1)) | ((uint64_t)FL << (63 - pl));
                read_hist(base, 32 * lane + pl, st.hist);
            }
            // carry into the next sub-block
            const uint32_t fl30 = __shfl_sync(FULL, FL, 30), fl31 = __shfl_sync(FULL, FL, 31);
            tailH = (uint64_t)fl30 | ((uint64_t)fl31 << 32);
            if (bev) level = bex > (bev ^ bex) ? 1u : 0u;
        }
        __syncwarp();
        const uint32_t n0 = __reduce_add_sync(FULL, acc.n0), nm = __reduce_add_sync(FULL, acc.nm);
        const uint32_t hf = __reduce_add_sync(FULL, acc.hf), ch = __reduce_add_sync(FULL, nch);
        const unsigned long long s0 = warp_sum_u64(acc.s0), smv = warp_sum_u64(acc.sm);
        const unsigned long long hs = warp_sum_u64(acc.hash);
        if (lane == 0) {
            ServeOut o;
            double E, T;
            totals(M, n0, nm, s0, smv, &E, &T);
            o.n_seen = n_seen0 + n;
            o.level = level ? topK : 0u;
            o.n_changes = ch;
            o.hash = hs;
            o.n_hf = hf;
            o.pad = 0;
            o.energy = E;
            o.time = T;
            p.out[r] = o;
        }
        __syncwarp();
    }
}

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    uint32_t stream;
    std::vector<uint32_t> data;
    Clock::time_point t_submit;
    bool done = false;
    magus_result_t res{};
};

struct Slot {
    char *pin = nullptr;         // pinned staging: header, requests, payload
    char *dev = nullptr;         // device batch buffer
    ServeOut *dout = nullptr;    // device results
    ServeOut *hout = nullptr;    // pinned results
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<uint64_t> ids;   // requests of the batch in flight
    bool busy = false;
};

}  // namespace

struct magus_serve {
    int device = 0;
    int32_t n_streams = 0;
    size_t budget = 0;
    int32_t max_req = 0;
    int64_t max_samples = 0;
    DevPolicy pol{};
    DevModel dm{};
    magus_state_t *table = nullptr;
    cudaStream_t stream = nullptr;
    int grid = 1;
    Slot slots[2];
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_slot;
    std::deque<uint64_t> pending;                     // submitted, not yet batched (FIFO)
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    size_t admitted_bytes = 0;
    uint64_t submitted = 0, completed = 0, rejected = 0, launches = 0, samples = 0;
    std::vector<double> latencies;
    std::deque<int> inflight;                         // slot indices in launch order
    bool stop = false;
    int error = 0;
    std::thread launcher, completer;
};

namespace {

int serve_fail(magus_serve *s, const std::string &msg, int code) {
    set_error(msg);
    if (s) s->error = code;
    return code;
}

// Capture H2D -> kernel -> D2H for one slot with maximal sizes; sizes are patched per launch.
cudaError_t build_graph(magus_serve *s, Slot &sl) {
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaMemcpyAsync(sl.dev, sl.pin, sl.bytes, cudaMemcpyHostToDevice, s->stream);
    ServeParams p;
    p.batch = sl.dev;
    p.out = sl.dout;
    p.table = s->table;
    p.P = s->pol;
    p.M = s->dm;
    serve_kernel<<<s->grid, SERVE_WARPS * 32, 0, s->stream>>>(p);
    cudaMemcpyAsync(sl.hout, sl.dout, sizeof(ServeOut) * (size_t)s->max_req, cudaMemcpyDeviceToHost, s->stream);
    e = cudaStreamEndCapture(s->stream, &sl.graph);
    if (e != cudaSuccess) return e;
    size_t nn = 0;
    e = cudaGraphGetNodes(sl.graph, nullptr, &nn);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(nn);
    e = cudaGraphGetNodes(sl.graph, nodes.data(), &nn);
    if (e != cudaSuccess) return e;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nd, &t);
        if (t != cudaGraphNodeTypeMemcpy) continue;
        cudaMemcpy3DParms mp;
        cudaGraphMemcpyNodeGetParams(nd, &mp);
        if (mp.kind == cudaMemcpyHostToDevice) sl.h2d = nd;
        else sl.d2h = nd;
    }
    if (!sl.h2d || !sl.d2h) return cudaErrorUnknown;
    return cudaGraphInstantiate(&sl.exec, sl.graph, 0);
}

void complete_slot(magus_serve *s, int si) {
    Slot &sl = s->slots[si];
    cudaEventSynchronize(sl.done);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t k = 0; k < sl.ids.size(); k++) {
        auto it = s->reqs.find(sl.ids[k]);
        if (it == s->reqs.end()) continue;
        Request &rq = it->second;
        const ServeOut &o = sl.hout[k];
        rq.res.n_seen = o.n_seen;
        rq.res.level = o.level;
        rq.res.n_changes = o.n_changes;
        rq.res.change_hash = o.hash;
        rq.res.n_hf = o.n_hf;
        rq.res.energy_j = o.energy;
        rq.res.time_s = o.time;
        rq.res.latency_s = std::chrono::duration<double>(now - rq.t_submit).count();
        rq.done = true;
        s->latencies.push_back(rq.res.latency_s);
        s->admitted_bytes -= rq.data.size() * 4;
        s->samples += rq.data.size();
        std::vector<uint32_t>().swap(rq.data);
        s->completed++;
    }
    sl.ids.clear();
    sl.busy = false;
    s->cv_slot.notify_all();
    s->cv_done.notify_all();
}

void completer_main(magus_serve *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->inflight.empty(); });
        if (s->inflight.empty() && s->stop) return;
        const int si = s->inflight.front();
        lk.unlock();
        complete_slot(s, si);
        lk.lock();
        s->inflight.pop_front();
    }
}

void launcher_main(magus_serve *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    int next_slot = 0;
    while (true) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
        if (s->stop && s->pending.empty()) return;
        // a free slot (its previous batch completed)
        s->cv_slot.wait(lk, [&] { return !s->slots[next_slot].busy || s->stop; });
        if (s->stop) return;   // requests still pending at close are dropped
        Slot &sl = s->slots[next_slot];
        // form the batch: FIFO, at most one request per stream, within the caps
        std::unordered_set<uint32_t> seen;
        std::deque<uint64_t> keep;
        std::vector<Request *> batch;
        int64_t nsamp = 0;
        while (!s->pending.empty()) {
            const uint64_t id = s->pending.front();
            s->pending.pop_front();
            Request &rq = s->reqs[id];
            const bool fits = (int32_t)batch.size() < s->max_req &&
                              (batch.empty() || nsamp + (int64_t)rq.data.size() <= s->max_samples);
            if (!fits || seen.count(rq.stream)) {
                seen.insert(rq.stream);   // later requests of this stream wait as well
                keep.push_back(id);
                if (!fits && (int32_t)batch.size() >= s->max_req) {
                    while (!s->pending.empty()) { keep.push_back(s->pending.front()); s->pending.pop_front(); }
                }
                continue;
            }
            seen.insert(rq.stream);
            batch.push_back(&rq);
            nsamp += (int64_t)rq.data.size();
        }
        s->pending.swap(keep);
        if (batch.empty()) continue;
        sl.busy = true;
        sl.ids.clear();
        for (auto *rq : batch) sl.ids.push_back(rq->id);
        // pack (payload copy outside the lock is unsafe: vectors may be released only by
        // the completer after this batch completes, so packing under the lock is fine)
        ServeHeader *hdr = (ServeHeader *)sl.pin;
        ServeReq *rqs = (ServeReq *)(sl.pin + sizeof(ServeHeader));
        const size_t payload_off = (sizeof(ServeHeader) + batch.size() * sizeof(ServeReq) + 255) / 256 * 256;
        uint32_t *pay = (uint32_t *)(sl.pin + payload_off);
        uint64_t off = 0;
        for (size_t k = 0; k < batch.size(); k++) {
            rqs[k].stream = batch[k]->stream;
            rqs[k].n = (uint32_t)batch[k]->data.size();
            rqs[k].off = off;
            memcpy(pay + off, batch[k]->data.data(), batch[k]->data.size() * 4);
            off += (batch[k]->data.size() + 3) / 4 * 4;   // 16-byte aligned request payloads
        }
        hdr->n_req = (uint32_t)batch.size();
        hdr->pad = 0;
        hdr->payload_off = payload_off;
        const size_t in_bytes = payload_off + off * 4;
        const size_t out_bytes = batch.size() * sizeof(ServeOut);
        lk.unlock();
        cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(sl.exec, sl.h2d, sl.dev, sl.pin, in_bytes,
                                                            cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaGraphExecMemcpyNodeSetParams1D(sl.exec, sl.d2h, sl.hout, sl.dout, out_bytes,
                                                   cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, s->stream);
        lk.lock();
        if (e != cudaSuccess) {
            s->error = MAGUS_ECUDA;
            set_error(std::string("serve launch: ") + cudaGetErrorString(e));
        }
        s->launches++;
        s->inflight.push_back(next_slot);
        s->cv_work.notify_all();
        next_slot ^= 1;
    }
}

}  // namespace

extern "C" {

int magus_serve_open(magus_serve_t **out, const magus_model_t *model, const magus_policy_t *policy,
                     int32_t n_streams, size_t mem_budget, int device, int32_t max_batch_requests,
                     int64_t max_batch_samples) {
    if (!out || !model || !policy) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    *out = nullptr;
    if (n_streams < 1 || n_streams > (1 << 24)) return serve_fail(nullptr, "n_streams must be 1..2^24", MAGUS_EINVAL);
    std::string err;
    DevModel dm;
    int rc = derive_model(*model, &dm, &err);
    if (rc) return serve_fail(nullptr, err, rc);
    DevPolicy dp;
    rc = derive_policy(*policy, *model, &dp, &err);
    if (rc) return serve_fail(nullptr, err, rc);
    if (policy->step_mode != 0) return serve_fail(nullptr, "serving supports step_mode 0", MAGUS_EINVAL);
    if (policy->pin_level != 0 && policy->pin_level != 1 && policy->pin_level != model->n_levels)
        return serve_fail(nullptr, "serving pins to the ladder bounds only: pin_level 0, 1 or n_levels", MAGUS_EINVAL);
    magus_serve *s = new (std::nothrow) magus_serve();
    if (!s) return serve_fail(nullptr, "out of host memory", MAGUS_ENOMEM);
    s->device = device;
    s->n_streams = n_streams;
    s->budget = mem_budget ? mem_budget : ((size_t)8 << 30);
    s->max_req = max_batch_requests > 0 ? max_batch_requests : 16384;
    s->max_samples = max_batch_samples > 0 ? max_batch_samples : ((int64_t)1 << 24);
    if (s->max_samples < kMaxRequestDeltas) s->max_samples = kMaxRequestDeltas;
    s->pol = dp;
    s->dm = dm;
    cudaError_t e = cudaSetDevice(device);
    int sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, SERVE_WARPS * 32, 0);
    s->grid = std::max(1, sms * std::max(per_sm, 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->table, sizeof(magus_state_t) * (size_t)n_streams);
    if (e == cudaSuccess) e = cudaMemset(s->table, 0, sizeof(magus_state_t) * (size_t)n_streams);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        Slot &sl = s->slots[k];
        sl.bytes = 256 + (size_t)s->max_req * sizeof(ServeReq) + 256 + 4 * ((size_t)s->max_samples + 4 * (size_t)s->max_req);
        e = cudaMallocHost(&sl.pin, sl.bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.dev, sl.bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.dout, sizeof(ServeOut) * (size_t)s->max_req);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.hout, sizeof(ServeOut) * (size_t)s->max_req);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            memset(sl.pin, 0, 256);
            e = build_graph(s, sl);
        }
    }
    if (e != cudaSuccess) {
        set_error(std::string("magus_serve_open: ") + cudaGetErrorString(e));
        cudaGetLastError();
        magus_serve_close(s);
        return MAGUS_ECUDA;
    }
    s->launcher = std::thread(launcher_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return MAGUS_OK;
}

int magus_serve_submit(magus_serve_t *s, uint32_t stream_id, const uint32_t *deltas, uint32_t n, uint64_t *req_id) {
    if (!s || !req_id || (n > 0 && !deltas)) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    if (stream_id >= (uint32_t)s->n_streams) return serve_fail(nullptr, "stream_id out of range", MAGUS_EINVAL);
    if (n < 1 || n > kMaxRequestDeltas) return serve_fail(nullptr, "request size must be 1..65536", MAGUS_EINVAL);
    Request rq;
    rq.stream = stream_id;
    rq.data.assign(deltas, deltas + n);
    rq.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return serve_fail(nullptr, "serving runtime stopped after a CUDA error", s->error);
    if (s->admitted_bytes + (size_t)n * 4 > s->budget) {
        s->rejected++;
        return serve_fail(nullptr, "admission refused: memory budget exhausted", MAGUS_EBUSY);
    }
    rq.id = s->next_id++;
    *req_id = rq.id;
    s->admitted_bytes += (size_t)n * 4;
    s->submitted++;
    s->pending.push_back(rq.id);
    s->reqs.emplace(rq.id, std::move(rq));
    s->cv_work.notify_all();
    return MAGUS_OK;
}

int magus_serve_poll(magus_serve_t *s, uint64_t req_id, magus_result_t *out) {
    if (!s || !out) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return serve_fail(nullptr, "unknown request id", MAGUS_ENOTFOUND);
    if (!it->second.done) return MAGUS_EAGAIN;
    *out = it->second.res;
    s->reqs.erase(it);
    return MAGUS_OK;
}

int magus_serve_drain(magus_serve_t *s) {
    if (!s) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == s->submitted || s->error; });
    return s->error ? s->error : MAGUS_OK;
}

int magus_serve_stats(magus_serve_t *s, magus_serve_stats_t *out) {
    if (!s || !out) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->launches = s->launches;
    out->samples = s->samples;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_s = q(0.50);
        out->p99_s = q(0.99);
        out->p999_s = q(0.999);
        out->max_s = v.back();
    }
    return MAGUS_OK;
}

int magus_serve_export(magus_serve_t *s, magus_state_t *out_states) {
    if (!s || !out_states) return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    int rc = magus_serve_drain(s);
    if (rc) return rc;
    cudaSetDevice(s->device);
    cudaError_t e = cudaMemcpy(out_states, s->table, sizeof(magus_state_t) * (size_t)s->n_streams,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return serve_fail(nullptr, cudaGetErrorString(e), MAGUS_ECUDA);
    return MAGUS_OK;
}

int magus_serve_load(magus_serve_t *s, const double *arrival_s, const uint32_t *stream_id,
                     const uint32_t *size, const uint32_t *payload, const uint64_t *payload_off, int64_t n_req,
                     double *out_latency_s, double *out_wall_s, magus_result_t *out_results) {
    if (!s || !arrival_s || !stream_id || !size || !payload || !payload_off || n_req < 0)
        return serve_fail(nullptr, "NULL argument", MAGUS_EINVAL);
    std::vector<uint64_t> ids((size_t)n_req, 0);
    const auto t0 = Clock::now();
    int rc = MAGUS_OK;
    for (int64_t i = 0; i < n_req; i++) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        int r = magus_serve_submit(s, stream_id[i], payload + payload_off[i], size[i], &ids[i]);
        if (r == MAGUS_EBUSY) {
            ids[i] = 0;   // refused by admission control, counted in the stats
            continue;
        }
        if (r) { rc = r; break; }
    }
    int d = magus_serve_drain(s);
    if (out_wall_s) *out_wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    if (!rc) rc = d;
    for (int64_t i = 0; i < n_req; i++) {
        magus_result_t res;
        memset(&res, 0, sizeof(res));
        double lat = -1.0;
        if (ids[i] && magus_serve_poll(s, ids[i], &res) == MAGUS_OK) lat = res.latency_s;
        else res.latency_s = -1.0;
        if (out_latency_s) out_latency_s[i] = lat;
        if (out_results) out_results[i] = res;
    }
    return rc;
}

int magus_serve_close(magus_serve_t *s) {
    if (!s) return MAGUS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_slot.notify_all();
    }
    if (s->launcher.joinable()) s->launcher.join();
    if (s->completer.joinable()) s->completer.join();
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto &sl : s->slots) {
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.pin) cudaFreeHost(sl.pin);
        if (sl.hout) cudaFreeHost(sl.hout);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.dout) cudaFree(sl.dout);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->table) cudaFree(s->table);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return MAGUS_OK;
}

}  // extern "C"
