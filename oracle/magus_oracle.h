/*
 * magus_oracle.h - CPU oracle for MAGUS policy replay.  TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential, FP64 restatement of the per-interval uncore control step of
 * MAGUS (arXiv 2502.03796): memory-throughput monitor (Sec. 3), trend predictor
 * (Sec. 3.1, Algorithm 1), frequent-phase-change detector (Sec. 3.2, Algorithm 2),
 * aggressive actuation to the ladder bounds (Sec. 6.1), idle-at-minimum start
 * (Sec. 4), plus the stated uncore energy model used to charge each decision.
 *
 * Only tests/, the package smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no source with the CUDA replay library.
 */
#ifndef MAGUS_ORACLE_H
#define MAGUS_ORACLE_H
#include <stdint.h>

#define OR_MAX_WINDOW 64

typedef struct {
    double inc_threshold;        /* Alg. 1: derivative above this -> +1 */
    double dec_threshold;        /* Alg. 1: derivative below this -> -1 */
    int32_t direv_length;        /* Alg. 1: derivative window W (intervals), 1..64 */
    int32_t tune_window;         /* Alg. 2: length L of uncore_tune_ls, 1..64 */
    double high_freq_threshold;  /* Alg. 2: rate threshold (paper: 0.6) */
    int32_t step_mode;           /* bit 0 clear: jump to the ladder bounds (Sec. 6.1); set:
                                    one ladder step per decision.  Bit 1 set: closed loop --
                                    the monitor reads the throughput the uncore delivered,
                                    min(demand, capacity at the level in effect), instead of
                                    the recorded demand (Sec. 6.3 discusses the throttled
                                    throughput at low uncore frequency) */
    int32_t pin_level;           /* 0: MAGUS control; k in 1..K: a static baseline that holds
                                    ladder index k-1 throughout (K = the maximum, the default
                                    setting of Sec. 5.3; 1 = the minimum of Sec. 6.3) */
} or_policy;

typedef struct {
    double dt_s;                 /* monitoring interval */
    int32_t n_levels;            /* K */
    int32_t bytes_per_count;     /* bytes represented by one counter unit */
    const double *f_ghz;         /* ascending uncore ladder, K entries */
    double p_static_w, p_dyn_w;  /* P(f) = p_static + p_dyn (f / f_ref)^2 */
    double f_ref_ghz, bw_ref_gbs;/* capacity C(f) = bw_ref f / f_ref */
} or_model;

/* Carried state between calls (split replay). */
typedef struct {
    uint64_t n_seen;                            /* intervals consumed so far */
    int32_t level;                              /* ladder index in effect for the next interval */
    int32_t ls_len;                             /* entries held in mem_throughput_ls */
    double mem_throughput_ls[OR_MAX_WINDOW + 1];/* FIFO, oldest first */
    uint8_t uncore_tune_ls[OR_MAX_WINDOW];      /* FIFO of L flags, oldest first */
} or_state;

typedef struct {
    double energy_j, time_s, edp_js;
    uint64_t n_changes;          /* frequency-change log entries */
    uint64_t change_hash;        /* sum over entries of mix64(((t+1) << 8) | level) mod 2^64 */
    uint64_t n_hf;               /* rounds in the high-frequency state */
} or_result;

/* Replay one trace under one policy.
 *   state       in/out; call or_state_init first for a fresh trace
 *   log_t/log_level  optional (NULL): change entries (interval index t+1, new level),
 *               capacity log_cap; entries beyond capacity are counted but not stored
 *   level_log   optional: ladder index in effect during each interval (n entries)
 *   deriv_log   optional: Alg. 1 derivative of each round, NaN while the FIFO fills
 * Returns 0, or -1 on invalid arguments. */
int or_replay(const uint32_t *deltas, uint64_t n, const or_policy *pol, const or_model *model,
              or_state *state, or_result *res, uint64_t *log_t, uint8_t *log_level,
              uint64_t log_cap, uint8_t *level_log, double *deriv_log);

void or_state_init(or_state *s);

/* All (trace, policy) pairs, pair index = trace * n_policies + policy, OpenMP over pairs.
 * Traces are read at data + offsets[i] with lengths[i] entries.  Returns threads used. */
int or_replay_batch(const uint32_t *data, const uint64_t *offsets, const uint64_t *lengths,
                    int64_t n_traces, const or_policy *pols, int64_t n_policies,
                    const or_model *model, or_result *res, int n_threads);

uint64_t or_mix64(uint64_t z);

#endif
