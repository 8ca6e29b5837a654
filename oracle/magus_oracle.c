/*
 * magus_oracle.c - CPU oracle for MAGUS policy replay.  TEST INFRASTRUCTURE ONLY.
 *
 * Plain sequential FP64 restatement of one MAGUS decision round per monitored interval
 * (arXiv 2502.03796), kept deliberately literal: explicit FIFOs, a sum over the tune
 * list every round, the energy model evaluated from the model description each round.
 *
 * Readings taken where the paper is silent (each also listed in the design notes):
 *   - mem_throughput_ls holds W+1 samples, so the derivative spans W intervals
 *     (Alg. 1 divides ls[-1] - ls[0] by direv_length); the prediction is 0 until it is full.
 *   - uncore_tune_ls has L entries, starts all zero, and Alg. 2 divides by L.
 *   - a flag is pushed for every nonzero prediction, also while the high-frequency state
 *     holds the level (Sec. 3.2: events are still logged and inform later rounds).
 *   - Alg. 2's ">=" decides (Sec. 3.2's prose says "exceeds").
 *   - +1 jumps to the top of the ladder, -1 to the bottom (Sec. 6.1: decreases go
 *     directly to the lower bound); the start level is the bottom (Sec. 4).
 *   - the decision taken after interval t governs interval t+1.
 *   - throughput in GB/s = bytes_per_count * delta / (dt * 1e9).
 *   - energy model (not from the paper): P(f) = p_static + p_dyn (f/f_ref)^2, capacity
 *     C(f) = bw_ref f / f_ref, an interval lasts dt * max(1, x / C(f)).
 */
#include "magus_oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* SplitMix64 output function (Steele, Lea, Flood 2014), used to hash log entries. */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

void or_state_init(or_state *s) {
    memset(s, 0, sizeof(*s));
    s->level = 0; /* Sec. 4: idle nodes sit at the minimum uncore frequency */
}

/* Alg. 1 (Sec. 3.1): first derivative of the throughput FIFO against two thresholds. */
static int mem_throughput_trend_prediction(double inc_threshold, double dec_threshold,
                                           const double *mem_throughput_ls, int len,
                                           int direv_length, double *derivative_out) {
    double derivative = (mem_throughput_ls[len - 1] - mem_throughput_ls[0]) / (double)direv_length;
    *derivative_out = derivative;
    if (derivative > inc_threshold) return 1;
    else if (derivative < dec_threshold) return -1;
    else return 0;
}

/* Alg. 2 (Sec. 3.2): share of rounds in the tune list that would have scaled the uncore. */
static int high_freq_detection(double high_freq_threshold, const uint8_t *uncore_tune_ls, int len) {
    int sum = 0;
    for (int i = 0; i < len; i++) sum += uncore_tune_ls[i];
    double freq = (double)sum / (double)len;
    return freq >= high_freq_threshold;
}

int or_replay(const uint32_t *deltas, uint64_t n, const or_policy *pol, const or_model *m,
              or_state *st, or_result *res, uint64_t *log_t, uint8_t *log_level,
              uint64_t log_cap, uint8_t *level_log, double *deriv_log) {
    const int W = pol->direv_length, L = pol->tune_window, K = m->n_levels;
    if (W < 1 || W > OR_MAX_WINDOW || L < 1 || L > OR_MAX_WINDOW || K < 1 || K > 32) return -1;
    if (pol->pin_level < 0 || pol->pin_level > K) return -1;
    if (pol->step_mode < 0 || pol->step_mode > 3) return -1;
    const int ladder = pol->step_mode & 1, closed = (pol->step_mode >> 1) & 1;
    /* A static baseline (Sec. 5.3, Sec. 6.3) runs no control: its level is fixed. */
    const int pinned = pol->pin_level > 0;
    if (pinned) st->level = pol->pin_level - 1;
    const double q = m->dt_s * 1e9;
    memset(res, 0, sizeof(*res));
    double E = 0.0, T = 0.0;
    for (uint64_t t = 0; t < n; t++) {
        /* Monitor (Sec. 3): counter delta -> memory throughput in GB/s. */
        double x = ((double)m->bytes_per_count * (double)deltas[t]) / q;

        /* Charge interval t at the level in effect (energy model). */
        int f = st->level;
        double fr = m->f_ghz[f] / m->f_ref_ghz;
        double cap = m->bw_ref_gbs * fr;
        double pw = m->p_static_w + m->p_dyn_w * (fr * fr);
        double s = x / cap;
        if (s < 1.0) s = 1.0;
        double tau = m->dt_s * s;
        T += tau;
        E += pw * tau;
        if (level_log) level_log[t] = (uint8_t)f;

        /* Phase 1 (Sec. 3.1, Alg. 1): push into the fixed-size FIFO, predict the trend. */
        if (st->ls_len == W + 1) {
            memmove(st->mem_throughput_ls, st->mem_throughput_ls + 1, (size_t)W * sizeof(double));
            st->ls_len = W;
        }
        /* Closed loop: the monitor sees at most what the uncore at level f delivered. */
        st->mem_throughput_ls[st->ls_len++] = (closed && x > cap) ? cap : x;
        int pred = 0;
        double derivative = NAN;
        if (st->ls_len == W + 1)
            pred = mem_throughput_trend_prediction(pol->inc_threshold, pol->dec_threshold,
                                                   st->mem_throughput_ls, st->ls_len, W, &derivative);
        if (deriv_log) deriv_log[t] = derivative;

        /* Phase 2 (Sec. 3.2, Alg. 2): log whether this round would scale the uncore. */
        memmove(st->uncore_tune_ls, st->uncore_tune_ls + 1, (size_t)(L - 1));
        st->uncore_tune_ls[L - 1] = (uint8_t)(pred != 0);
        int hf = high_freq_detection(pol->high_freq_threshold, st->uncore_tune_ls, L);
        if (pinned) hf = 0;
        res->n_hf += (uint64_t)hf;

        /* Decision: high-frequency state overrides the temporary decision with the max. */
        int next;
        if (pinned) next = f;
        else if (hf) next = K - 1;
        else if (pred == 1) next = !ladder ? K - 1 : (f + 1 < K ? f + 1 : K - 1);
        else if (pred == -1) next = !ladder ? 0 : (f > 0 ? f - 1 : 0);
        else next = f;

        if (next != f) {
            uint64_t when = st->n_seen + t + 1; /* applies from the next interval on */
            if (log_t && res->n_changes < log_cap) {
                log_t[res->n_changes] = when;
                log_level[res->n_changes] = (uint8_t)next;
            }
            res->n_changes++;
            res->change_hash += or_mix64((when << 8) | (uint64_t)next);
        }
        st->level = next;
    }
    st->n_seen += n;
    res->energy_j = E;
    res->time_s = T;
    res->edp_js = E * T;
    return 0;
}

int or_replay_batch(const uint32_t *data, const uint64_t *offsets, const uint64_t *lengths,
                    int64_t n_traces, const or_policy *pols, int64_t n_policies,
                    const or_model *model, or_result *res, int n_threads) {
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < n_traces * n_policies; p++) {
            int64_t i = p / n_policies, c = p % n_policies;
            or_state st;
            or_state_init(&st);
            or_replay(data + offsets[i], lengths[i], &pols[c], model, &st, &res[p],
                      NULL, NULL, 0, NULL, NULL);
        }
    }
#else
    (void)n_threads;
    for (int64_t p = 0; p < n_traces * n_policies; p++) {
        int64_t i = p / n_policies, c = p % n_policies;
        or_state st;
        or_state_init(&st);
        or_replay(data + offsets[i], lengths[i], &pols[c], model, &st, &res[p], NULL, NULL, 0, NULL, NULL);
    }
#endif
    return used;
}
