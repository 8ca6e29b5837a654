/*
 * magus.h - C ABI of libmagus: batched replay of the MAGUS uncore-frequency control step
 * (arXiv 2502.03796) on one B300 GPU.
 *
 * One "round" per monitored interval (dt seconds) of one trace under one policy:
 *   1. monitor (Sec. 3): counter delta (in bytes_per_count units) -> memory throughput
 *      x = bytes_per_count * delta / (dt * 1e9) GB/s;
 *   2. Phase 1 (Sec. 3.1, Algorithm 1): x joins a FIFO of W+1 throughputs; once full,
 *      derivative = (newest - oldest) / W; > inc -> +1, < dec -> -1, else 0 (a temporary
 *      decision); 0 while the FIFO fills;
 *   3. Phase 2 (Sec. 3.2, Algorithm 2): a flag (prediction != 0) joins a zero-filled
 *      FIFO of L flags; high-frequency state iff sum / L >= high_freq_threshold;
 *   4. decision (Sec. 3.2, Sec. 6.1): high-frequency -> top of the ladder; else +1 ->
 *      top, -1 -> bottom (decreases go directly to the lower bound), 0 -> hold.  The
 *      level chosen after interval t governs interval t+1; the first interval runs at the
 *      bottom of the ladder (Sec. 4: idle nodes sit at the minimum uncore frequency);
 *   5. energy model (not from the paper): interval t at level f lasts
 *      dt * max(1, x_t / C(f)) with C(f) = bw_ref * f / f_ref and draws
 *      P(f) = p_static + p_dyn * (f / f_ref)^2; E = sum P * duration, T = sum duration,
 *      EDP = E * T (Sec. 5.4 names the energy-delay product as a metric).
 *
 * Conventions
 *   - Every function returns int status: MAGUS_OK (0) or a negative MAGUS_E* code, and
 *     never throws.  magus_last_error() gives a message for the calling thread.
 *   - The caller owns every input and output buffer; the library owns handles and their
 *     device workspace (allocated lazily, within the handle's memory budget).
 *   - "device" pointers are CUDA device memory of the handle's device; "host" pointers
 *     are ordinary (pageable or pinned) host memory.
 *   - Per-pair outputs are pair-major: pair p = trace * n_configs + config.
 *   - magus_replay_run / _plain / _detail are asynchronous on the given stream
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).  Device-side input
 *     errors detected by a kernel are reported by the next magus_replay_status().
 *
 * Packed trace layout (device or host): traces are stored back to back; trace i starts at
 * element offset off_i with off_0 = 0 and off_{i+1} = off_i + round_up(n_i, 32), so every
 * trace starts on a 128-byte row of 32 deltas (the batched kernel reads rows of 32 with TMA
 * tensor copies); the buffer holds magus_packed_size() elements (padding elements are read
 * but ignored) and its base is 16-byte aligned.  Deltas are uint32 counts of
 * bytes_per_count bytes per interval.
 */
#ifndef MAGUS_H
#define MAGUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAGUS_OK 0
#define MAGUS_EINVAL (-1)    /* invalid argument */
#define MAGUS_ENOMEM (-2)    /* allocation failed or memory budget exceeded */
#define MAGUS_EBUSY (-3)     /* serving: admission refused (no slot / memory) */
#define MAGUS_EAGAIN (-4)    /* serving: result not ready yet */
#define MAGUS_ETIMEDOUT (-5) /* a bounded device-side wait gave up */
#define MAGUS_ECUDA (-6)     /* CUDA runtime error */
#define MAGUS_ENOTFOUND (-7) /* serving: unknown request id */

#define MAGUS_MAX_WINDOW 64  /* upper bound of direv_length (W) and tune_window (L) */
#define MAGUS_MAX_LEVELS 32  /* upper bound of the ladder length */

/* Policy parameters (Algorithm 1 and Algorithm 2 arguments). */
typedef struct {
    double inc_threshold;       /* Alg. 1 inc_threshold, GB/s per interval */
    double dec_threshold;       /* Alg. 1 dec_threshold, GB/s per interval */
    int32_t direv_length;       /* Alg. 1 direv_length W, 1..64 */
    int32_t tune_window;        /* Alg. 2 len(uncore_tune_ls) L, 1..64 */
    double high_freq_threshold; /* Alg. 2 high_freq_threshold (paper: 0.6) */
    int32_t step_mode;          /* bit 0 clear: jump to the ladder bounds (Sec. 6.1); set: one
                                   rung per decision.  Bit 1 set: closed loop -- the monitor
                                   reads min(demand, capacity at the level in effect), the
                                   throughput a throttled uncore delivers (Sec. 6.3), instead
                                   of the recorded demand.  magus_replay_run / _plain /
                                   _detail take 0..3 (see magus_replay_run for which kernel
                                   runs what); serving and magus_replay_run_static take 0. */
    int32_t pin_level;          /* 0: MAGUS control.  k in 1..n_levels: a static baseline that
                                   holds ladder index k-1 for every interval and runs no
                                   control (no changes, no high-frequency rounds; the
                                   predictions still feed the carried flag state).  k =
                                   n_levels is the default setting the paper compares
                                   against (uncore at its maximum, Sec. 5.3), k = 1 the
                                   minimum (Sec. 6.3).  Serving and magus_replay_run_static
                                   take 0, 1 or n_levels; magus_replay_run / _plain any k. */
} magus_policy_t;

/* Ladder and energy model. */
typedef struct {
    double dt_s;                /* monitoring interval, s (1e-9 .. 1e6) */
    int32_t n_levels;           /* K, 2..32 */
    int32_t bytes_per_count;    /* bytes per counter unit (64-byte lines), 1..2^20 */
    const double *f_ghz;        /* host, K strictly ascending frequencies */
    double p_static_w, p_dyn_w; /* P(f) = p_static + p_dyn (f / f_ref)^2 */
    double f_ref_ghz;           /* reference frequency (top of the ladder) */
    double bw_ref_gbs;          /* capacity at f_ref, GB/s */
} magus_model_t;

/* Carried per-pair state for split replay: feeding a trace in pieces with the same state
 * reproduces the whole-trace logs exactly and energies additively.  All pairs of one trace
 * in a call must carry states of the same earlier pieces (the delta history is read from
 * the state of the trace's first policy). */
typedef struct {
    uint64_t n_seen;            /* intervals consumed so far (0 for a fresh trace) */
    uint64_t flags;             /* bit q = flag of interval n_seen - 64 + q (bit 63 newest) */
    uint32_t level;             /* ladder index governing the next interval (0 or K-1 in
                                   jump mode) */
    uint32_t reserved;
    uint32_t hist[MAGUS_MAX_WINDOW]; /* deltas of intervals n_seen-64 .. n_seen-1 */
} magus_state_t;

/* Frequency-change log.  Entry = ((t + 1) << 5) | level: from interval t+1 on (global
 * interval index, counting n_seen) the uncore runs at ladder index `level`.  Entries of a
 * pair are in time order at entries[pair * capacity ...]; entries beyond capacity are
 * counted and hashed but not stored; slots past a pair's n_changes hold unspecified values
 * (the segment kernel uses them as scratch).  change_hash = sum over entries of
 * SplitMix64-mix(((t + 1) << 8) | level) mod 2^64 (order-free, additive over splits). */
typedef struct {
    uint32_t *entries;          /* device [pairs * capacity] or NULL */
    uint64_t capacity;          /* entries per pair (ignored when entries == NULL) */
    uint64_t *n_changes;        /* device [pairs] or NULL */
    uint64_t *change_hash;      /* device [pairs] or NULL */
    uint64_t *n_hf;             /* device [pairs] or NULL: rounds in the high-frequency state */
} magus_freq_log_t;

typedef struct magus_replay magus_replay_t;

/* ---------------------------------------------------------------------------------------
 * Replay handles
 * ------------------------------------------------------------------------------------- */

/* Create a replay handle on CUDA device `device`.  mem_budget bounds the handle's own
 * device workspace in bytes (0 = 1 GiB).  The model is copied.  Errors: EINVAL (bad model:
 * K out of range, ladder not strictly ascending, non-positive dt / capacities), ECUDA. */
int magus_replay_open(magus_replay_t **h, const magus_model_t *model, int device, size_t mem_budget);

/* Replay n_traces x n_configs (trace, policy) pairs (rounds above).  Policies in the open-loop
 * jump mode (step_mode 0, pin_level 0, 1 or n_levels) run on the time-parallel kernels (tile
 * or segment kernel), the one-rung mode (step_mode 1, pin_level 0) on the ladder kernel, the
 * closed loop (step_mode 2 or 3, pin_level 0) on the segmented closed-loop kernels
 * (magus_replay_set_closed); the others (a pin inside the ladder in jump mode, any pin in
 * the other modes) on the static kernel (one pass per trace at the pinned rungs), or with
 * io_state on the literal kernel, one thread per pair.  Without io_state, when the static
 * kernel runs, the pins at a ladder bound in jump mode join it.  With io_state a
 * closed-loop policy needs a fresh state (n_seen 0; else EINVAL through
 * magus_replay_status): its throughput FIFO would need past levels; in jump mode its
 * carried level must be 0 or n_levels - 1.
 *   traces     device, packed layout; base address 16-byte aligned
 *   lengths    host [n_traces] intervals per trace (0 allowed)
 *   configs    host [n_configs], 1 <= n_configs <= 4096
 *   log        optional (NULL): change log / counts / hash / hf counts (device arrays)
 *   out_energy device [pairs] J, out_edp device [pairs] J*s (both required);
 *   out_time   device [pairs] s or NULL
 *   io_state   device [pairs] or NULL: read at the start and written at the end of each pair
 * Asynchronous on `stream`.  Errors: EINVAL (argument checks), ENOMEM (budget), ECUDA. */
int magus_replay_run(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths,
                     int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                     const magus_freq_log_t *log, double *out_energy, double *out_edp,
                     double *out_time, magus_state_t *io_state, void *stream);

/* Same computation through host memory: traces (packed layout), outputs and log arrays are
 * HOST pointers.  The library streams the traces to the device in batches, overlapping the
 * copies with the replay, and returns when every output is back on the host. */
int magus_replay_run_host(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths,
                          int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                          const magus_freq_log_t *log, double *out_energy, double *out_edp,
                          double *out_time);

/* The plain form: one kernel launch per trace, one thread per policy, literal FP64
 * arithmetic in the order of the rounds above, global-memory loads.  Same arguments and
 * outputs as magus_replay_run (no io_state); supports step_mode 0..3 and any pin_level. */
int magus_replay_plain(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths,
                       int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                       const magus_freq_log_t *log, double *out_energy, double *out_edp,
                       double *out_time, void *stream);

/* One trace, one policy, per-interval detail (plain kernel): out_level[t] = ladder index
 * governing interval t, out_derivative[t] = Algorithm 1 derivative of round t (NaN while
 * the FIFO fills).  trace, out_level (uint8 [n]), out_derivative (double [n]) and the
 * log / totals are device pointers; out_level / out_derivative may be NULL. */
int magus_replay_detail(magus_replay_t *h, const uint32_t *trace, uint64_t n,
                        const magus_policy_t *config, uint8_t *out_level, double *out_derivative,
                        const magus_freq_log_t *log, double *out_energy, double *out_edp,
                        double *out_time, void *stream);

/* Wait for `stream` and report device-side input errors seen since the last call (EINVAL
 * for a carried level that is neither 0 nor K-1 in jump mode; ETIMEDOUT for a bounded
 * device wait that gave up), then clear them. */
int magus_replay_status(magus_replay_t *h, void *stream);

/* Device time of the batched replays of this handle since the previous call (CUDA events
 * recorded on the launching stream around each replay's kernels, up to 4096 replays; later
 * ones overwrite the last record).  total_ms: all kernels of those replays; main_ms
 * (optional): the replay kernel alone (tile kernel, or segment kernel without its combine
 * kernel); runs: timed replays; kernels (optional): kernels they launched.  Waits for those
 * launches, then resets. */
int magus_replay_kernel_time(magus_replay_t *h, double *total_ms, double *main_ms, int32_t *runs,
                             int32_t *kernels);

/* Tile shape of the batched kernel: warps that split a trace chunk in time (time_groups) x
 * policy groups per CTA (policy_slots); time_groups * policy_slots = 8, or a 4-warp tile:
 * (4, 1) for one-member groups (six CTAs per SM instead of three), (1, 4) and (2, 2) for
 * groups of up to 4 (five and four CTAs per SM instead of two).  Policies sharing
 * Algorithm 1's parameters (W, inc, dec) are grouped (up to 4 per group, predictions made
 * once per group) whenever that at least halves the group count.  (0, 0) restores the
 * automatic choice.  EINVAL for unsupported shapes. */
int magus_replay_set_tile(magus_replay_t *h, int32_t time_groups, int32_t policy_slots);

/* Kernel choice: seg_rounds > 0 (a multiple of 1024) selects the segment kernel -- every warp
 * replays one (trace, policy group, segment of seg_rounds rounds) on its own, a combine
 * kernel then joins each pair's segments in order; 0 selects the tile kernel (CTAs of 4 or
 * 8 warps sharing each trace chunk, shaped by magus_replay_set_tile); -1 (the default)
 * restores the automatic choice (the autotuner's pick, else the tile kernel, or the segment
 * kernel with 16,384-round segments when a few long traces would leave SMs idle).  EINVAL
 * otherwise. */
int magus_replay_set_segments(magus_replay_t *h, int32_t seg_rounds);

/* Failure detection (bounded device-side waits).  Every wait of the tile kernel for a trace
 * chunk's copy gives up after a limit: chunk_wait_ns nanoseconds in the tiles whose warps
 * wait for their stages themselves (the one-slot tiles (8, 1) and (4, 1), and (1, 4) with
 * groups), 2 s in the others and whenever chunk_wait_ns is 0 (the default).  The kernel then
 * records MAGUS_ETIMEDOUT,
 * stops issuing copies, lets the copies already in flight land (that last wait always keeps
 * the 2 s limit) and returns; magus_replay_status reports the timeout and clears it, and the
 * handle stays usable.  The outputs of a call that timed out are unspecified.  A short limit
 * detects a stalled copy engine sooner; a limit below the copy latency (about a
 * microsecond) makes the waits run out on purpose, which is how the timeout path is tested.
 * EINVAL for a NULL handle. */
int magus_replay_set_wait(magus_replay_t *h, uint64_t chunk_wait_ns);

/* Closed loop (step_mode 2 or 3, pin_level 0): replayed time-parallel.  Every
 * (trace, policy, segment of seg_rounds rounds) is replayed on its own from a guessed state
 * burn_rounds earlier; a segment whose guess did not reach the state its predecessor ended
 * in is replayed again, and a final pass per pair takes the replays that started from the
 * true state (results identical to the sequential replay whatever the guesses); with a
 * change log, segments with more entries than their scratch holds are replayed once more
 * to write them.
 * seg_rounds: 0 automatic (about four waves of threads, 1,024 .. 65,536), > 0 a multiple of
 * 64 up to 2^24, -1 the literal kernel (one thread per pair); burn_rounds: -1 automatic
 * (seg_rounds / 4), else a multiple of 64 up to 2^24.  EINVAL otherwise. */
int magus_replay_set_closed(magus_replay_t *h, int32_t seg_rounds, int32_t burn_rounds);

/* Work of the last call's time-parallel closed-loop replay (host, 4 values): segments
 * replayed, second replays, replays in the final pass, replays in the log pass (segments
 * whose change entries overflowed their scratch); all 0 when it did not run.  Waits for the
 * handle's outstanding launches. */
int magus_replay_closed_stats(magus_replay_t *h, uint64_t *out4);

/* Autotuner: time every supported tile shape (time_groups x policy_slots x group size 1 or
 * 4) of the tile kernel and the segment kernel (segments of 8,192 / 16,384 / 32,768 rounds,
 * group size 1 or 4) on the given (device, packed) workload and keep the fastest for later
 * calls with the same policy count.  out_best (host, 4 ints, optional) receives
 * {time_groups, policy_slots, group_size, segment_rounds (0: tile kernel)}; out_ms (host,
 * optional) the best time.  Outputs go to the handle's workspace only.  Synchronous. */
int magus_replay_autotune(magus_replay_t *h, const uint32_t *traces, const uint64_t *lengths,
                          int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                          int32_t *out_best, float *out_ms, void *stream);

int magus_replay_close(magus_replay_t *h);

/* Size of the fixed device scratch used by magus_replay_run_static (4 MiB). */
#define MAGUS_STATIC_SCRATCH_BYTES (4u << 20)

/* Batched replay without any device allocation (the paper has no counterpart: this is a
 * service for callers of this library).  Some callers cannot call cudaMalloc when they
 * want a replay -- code running inside another framework's memory pool, a process whose
 * device memory is reserved up front, a plug-in handed only ready-made buffers -- so they
 * cannot open a handle (magus_replay_open allocates).  This entry point takes the model
 * directly and runs the same kernel and computation as magus_replay_run on the CURRENT
 * device; its planning scratch (policy table, work list, trace offsets/lengths, work
 * counter, status word) lives in a fixed file-scope device array of
 * MAGUS_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the process
 * exits.  It calls no cudaMalloc / cudaFree.
 *   - Arguments and outputs as magus_replay_run (traces, outputs, log, io_state: device),
 *     but only for the policies the time-parallel tile kernel replays: step_mode 0 (open
 *     loop, jump to a bound) with pin_level 0, 1 or n_levels.  Any other step_mode or pin
 *     is refused with EINVAL (magus_replay_run takes them).
 *   - Workloads whose plan does not fit the scratch (about 100 B per policy, 16 B per
 *     trace and 8 B per trace for every block of up to 8 policy groups) are rejected with
 *     EINVAL and a message.
 *   - The first call on a device looks up the array's device address (set-up, once per
 *     device).
 *   - The call is synchronous: it uploads the plan on `stream` from pageable host memory,
 *     zeroes the work counter and status word, runs the kernel, waits for `stream` and
 *     reads the status word back before returning.  None of that may be captured, so no
 *     call (the first or any later one) may be made while any stream on the device is
 *     being captured.
 *   - Every call shares the one array, so sequential calls are safe, but calls that overlap
 *     on the GPU (other threads or streams at the same time) race on the scratch and give
 *     wrong results.
 *   - Returns device-side input errors (EINVAL for a carried level that is neither 0 nor
 *     K-1) directly. */
int magus_replay_run_static(const magus_model_t *model, const uint32_t *traces, const uint64_t *lengths,
                            int32_t n_traces, const magus_policy_t *configs, int32_t n_configs,
                            const magus_freq_log_t *log, double *out_energy, double *out_edp,
                            double *out_time, magus_state_t *io_state, void *stream);

/* ---------------------------------------------------------------------------------------
 * Helpers (host only, no device needed)
 * ------------------------------------------------------------------------------------- */

/* Packed layout: offsets[i] (host, may be NULL) and the total element count. */
int magus_packed_size(const uint64_t *lengths, int32_t n_traces, uint64_t *offsets, uint64_t *total);

/* Integer decision bounds the batched kernel derives for one policy (diagnostics and
 * tests).  out[0] = m_up, out[1] = m_dn, out[2] = k_min, out[3] = band half-width b:
 * with m = delta_t - delta_{t-W}, Algorithm 1 returns +1 for m > m_up + b and never for
 * m <= m_up - b (likewise -1 for m < m_dn - b and never for m >= m_dn + b); rounds inside
 * a band are decided by exact FP64.  k_min = smallest flag count c with
 * c / L >= high_freq_threshold (L + 1 if none). */
int magus_policy_bounds(const magus_policy_t *policy, const magus_model_t *model, int64_t out[4]);

/* FP64 decision thresholds the literal kernel derives for one policy (diagnostics and
 * tests).  With d = x_t - x_{t-W} the FP64 throughput difference, Algorithm 1's
 * RN(d / W) > inc holds exactly when d > out[0], and RN(d / W) < dec exactly when
 * d <= out[1] (+-infinity when never / always). */
int magus_policy_fp64_thresholds(const magus_policy_t *policy, const magus_model_t *model, double out[2]);

/* Closed-loop decision thresholds the segmented closed-loop kernels derive for one policy
 * (diagnostics and tests).  For level l = 0 (bottom) and 1 (top of the ladder), with
 * x(delta) = bytes_per_count * delta / (dt * 1e9) in FP64 and C_l the capacity there:
 *   out[0 + l]  largest delta with x(delta) <= C_l (a throughput is capped above it);
 *   out[2 + l]  Algorithm 1 gives +1 for obs_t = C_l, obs_{t-W} = x(b) exactly when b < out[2 + l];
 *   out[4 + l]  ... gives -1 there exactly when b >= out[4 + l];
 *   out[6 + l]  +1 for obs_t = x(a), obs_{t-W} = C_l exactly when a >= out[6 + l];
 *   out[8 + l]  -1 there exactly when a < out[8 + l];
 *   out[10]     both capped (levels la, lb): bit 2 la + lb set when +1, bit 4 + 2 la + lb
 *               when -1 (before Algorithm 1's preference of +1).
 * Thresholds range over 0 .. 2^32. */
int magus_policy_closed_thresholds(const magus_policy_t *policy, const magus_model_t *model, int64_t out[11]);

const char *magus_last_error(void);
const char *magus_version(void);

/* ---------------------------------------------------------------------------------------
 * Serving: an online controller over many node streams with device-resident state.
 * Requests carry new deltas of one stream; requests that arrive while others run are
 * batched into the next launch (continuous batching); each stream's state stays on the
 * device between requests.
 * ------------------------------------------------------------------------------------- */

typedef struct magus_serve magus_serve_t;

typedef struct {
    uint64_t n_seen;            /* stream intervals consumed after this request */
    uint32_t level;             /* level governing the stream's next interval */
    uint32_t n_changes;         /* change-log entries produced by this request */
    uint64_t change_hash;       /* hash of those entries (same definition as the replay log) */
    uint32_t n_hf;              /* high-frequency rounds in this request */
    uint32_t reserved;
    double energy_j, time_s;    /* energy and duration charged for this request's intervals */
    double latency_s;           /* submit -> result available on the host */
} magus_result_t;

typedef struct {
    uint64_t submitted, completed, rejected, launches;
    uint64_t samples;           /* intervals processed */
    double p50_s, p99_s, p999_s, max_s; /* latency of completed requests */
} magus_serve_stats_t;

/* Open a serving runtime: n_streams device-resident stream states (all fresh), one policy
 * (step_mode 0).  mem_budget bounds the bytes of request payload admitted but not yet
 * completed (0 = 8 GiB); max_batch_requests / max_batch_samples cap one launch (0 =
 * defaults).  A background thread forms batches, launches them and completes requests. */
int magus_serve_open(magus_serve_t **s, const magus_model_t *model, const magus_policy_t *policy,
                     int32_t n_streams, size_t mem_budget, int device,
                     int32_t max_batch_requests, int64_t max_batch_samples);

/* Submit n (1..65536) new deltas (host memory, copied) of stream_id.  Requests of one stream
 * are applied in submission order.  EBUSY when the memory budget is exhausted. */
int magus_serve_submit(magus_serve_t *s, uint32_t stream_id, const uint32_t *deltas, uint32_t n,
                       uint64_t *req_id);

/* Result of a request: EAGAIN until it is done, ENOTFOUND for unknown / already-polled ids.
 * A successful poll releases the request. */
int magus_serve_poll(magus_serve_t *s, uint64_t req_id, magus_result_t *out);

/* Block until every submitted request is complete. */
int magus_serve_drain(magus_serve_t *s);

int magus_serve_stats(magus_serve_t *s, magus_serve_stats_t *out);

/* Export all stream states (host, n_streams entries) for checkpointing. */
int magus_serve_export(magus_serve_t *s, magus_state_t *out_states);

/* Open-loop load driver (benchmarks): submit request i at arrival_s[i] seconds after the
 * call starts (host busy-wait), stream stream_id[i], size[i] deltas read from
 * payload + payload_off[i] (host); then drain and poll every request.  out_latency_s (host,
 * n_req, optional) receives each latency, -1 for requests refused by admission control;
 * out_wall_s the time from the first arrival to the end of the drain; out_results (host,
 * n_req, optional) each request's full result as magus_serve_poll returns it (all zero
 * with latency_s = -1 for a refused request). */
int magus_serve_load(magus_serve_t *s, const double *arrival_s, const uint32_t *stream_id,
                     const uint32_t *size, const uint32_t *payload, const uint64_t *payload_off,
                     int64_t n_req, double *out_latency_s, double *out_wall_s, magus_result_t *out_results);

int magus_serve_close(magus_serve_t *s);

#ifdef __cplusplus
}
#endif
#endif /* MAGUS_H */
