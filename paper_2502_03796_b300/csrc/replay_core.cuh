// replay_core.cuh - per-row building blocks of the time-parallel MAGUS replay, shared by the
// batched kernel (replay_tp.cu) and the serving kernel (serve.cu).
//
// A "row" is 32 consecutive rounds owned by one lane; bit p of every mask is round p of the
// row.  Rows sit in shared memory with at least 64 earlier deltas before them, and lanes
// read their rows in rotated order k = (i + lane) & 31 so that the 32 lanes of a warp hit
// 32 different banks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"

namespace magus {
namespace core {

constexpr uint32_t FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t rotl(uint32_t x, int s) { return __funnelshift_l(x, x, s); }
__device__ __forceinline__ uint32_t rotr(uint32_t x, int s) { return __funnelshift_r(x, x, s); }

// SplitMix64 output function (Steele, Lea, Flood 2014): hashes change-log entries.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}

// Valid-round mask of a row with `left` rounds remaining from its start.
__device__ __forceinline__ uint32_t valid_mask(int64_t left) {
    return left >= 32 ? FULL : (left <= 0 ? 0u : ((1u << left) - 1u));
}

// Rounds of the row whose throughput FIFO already holds W+1 samples (global index >= W).
__device__ __forceinline__ uint32_t predict_mask(uint32_t vmask, uint64_t gstart, int W) {
    if (gstart >= (uint64_t)W) return vmask;
    const uint32_t wm = (uint32_t)((uint64_t)W - gstart);
    return vmask & (wm >= 32 ? 0u : (FULL << wm));
}

struct RowPred {
    uint32_t UP, DN;   // Alg. 1 returned +1 / -1
    uint32_t S0, SM;   // interval stretched at the bottom / top level (x > C(f))
};

// Alg. 1 for the 32 rounds of a row: derivative = (x_t - x_{t-W}) / W against inc / dec,
// decided on the integer difference of the deltas outside the narrow band the host derived
// (plan.cu) and by the exact FP64 evaluation inside it.
__device__ __forceinline__ RowPred row_predict(const uint32_t *row, int lane, const DevPolicy &P,
                                               const DevModel &M, uint32_t vmask, uint32_t pmask) {
    uint32_t UPr = 0, DNr = 0, S0r = 0, SMr = 0, BDr = 0;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k = (i + lane) & 31;
        const uint32_t a = row[k];
        const uint32_t b = row[k - P.W];
        const long long m = (long long)a - (long long)b;
        UPr |= (uint32_t)(m > P.up_mid) << i;
        DNr |= (uint32_t)(m < P.dn_mid) << i;
        const uint32_t m32 = a - b;
        BDr |= (uint32_t)(((m32 - P.up_lo) <= P.up_w) | ((m32 - P.dn_lo) <= P.dn_w)) << i;
        S0r |= (uint32_t)(a > M.thr0) << i;
        SMr |= (uint32_t)(a > M.thrM) << i;
    }
    uint32_t todo = BDr & rotr(pmask, lane);
    if (__any_sync(FULL, todo != 0)) {
        while (todo) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1;
            const int k = (i + lane) & 31;
            const uint32_t a = row[k], b = row[k - P.W];
            const double xa = __ddiv_rn(__dmul_rn(M.bpc, (double)a), M.q);
            const double xb = __ddiv_rn(__dmul_rn(M.bpc, (double)b), M.q);
            const double der = __ddiv_rn(__dsub_rn(xa, xb), (double)P.W);
            const uint32_t bit = 1u << i;
            UPr = (der > P.inc) ? (UPr | bit) : (UPr & ~bit);
            DNr = (der < P.dec) ? (DNr | bit) : (DNr & ~bit);
        }
    }
    RowPred r;
    r.UP = rotl(UPr, lane) & pmask;
    r.DN = rotl(DNr, lane) & pmask;
    r.S0 = rotl(S0r, lane) & vmask;
    r.SM = rotl(SMr, lane) & vmask;
    return r;
}

// Alg. 2 over one row: bit p of the result = high-frequency state of round p.
// H: flags of the 64 rounds before the row (bit q = round q - 64); FL: flags of the row.
__device__ __forceinline__ uint32_t hf_row(uint64_t H, uint32_t FL, int L, int kmin) {
    // window ending just before the row: rounds -L .. -1
    int cnt = __popcll(H >> (64 - L));
    // most flags any window ending inside the row can hold
    const int reach = (L > 1 ? __popcll(H >> (65 - L)) : 0) + __popc(FL);
    if (reach < kmin) return 0u;
    // bit p of LV = flag of round p - L (leaving the window at round p)
    const int s = 64 - L;
    const uint32_t LV = s == 0 ? (uint32_t)H : (uint32_t)((H >> s) | ((uint64_t)FL << (64 - s)));
    uint32_t HF = 0;
#pragma unroll
    for (int p = 0; p < 32; p++) {
        cnt += (int)((FL >> p) & 1u) - (int)((LV >> p) & 1u);
        HF |= (uint32_t)(cnt >= kmin) << p;
    }
    return HF;
}

// Flag history before each lane's row: lanes 0 and 1 take the 64 flags before the first
// row (tailH), the others their two predecessor rows.
__device__ __forceinline__ uint64_t row_history(uint32_t FL, uint64_t tailH, int lane) {
    const uint32_t p1 = __shfl_up_sync(FULL, FL, 1), p2 = __shfl_up_sync(FULL, FL, 2);
    return lane >= 2 ? ((uint64_t)p2 | ((uint64_t)p1 << 32))
         : lane == 1 ? ((tailH >> 32) | ((uint64_t)p1 << 32))
                     : tailH;
}

// Latch over one row: SETM = rounds that leave the level at the top, SET0 = at the bottom
// (disjoint), cin = level before the row (1 = top).  Returns Lm: bit p = level after
// round p.  Adding SETM to ~SET0 carries from every set-to-top bit through the following
// hold bits and stops at the next set-to-bottom bit.
__device__ __forceinline__ uint32_t latch_row(uint32_t SETM, uint32_t SET0, uint32_t cin) {
    const uint32_t A = ~SET0;
    const uint64_t sum = (uint64_t)A + (uint64_t)SETM + (uint64_t)cin;
    const uint32_t carry_in = (uint32_t)sum ^ A ^ SETM;  // carry into each bit position
    return (carry_in | SETM) & ~SET0;
}

// Sum of the row's deltas at the rounds selected by mask M (bit p = round p).
__device__ __forceinline__ unsigned long long row_masked_sum(const uint32_t *row, int lane, uint32_t M) {
    unsigned long long s = 0;
    const uint32_t Mr = rotr(M, lane);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const uint32_t a = row[(i + lane) & 31];
        s += ((Mr >> i) & 1u) ? a : 0u;
    }
    return s;
}

// Per-lane energy / log accumulators.
struct Acc {
    uint32_t n0, nm, hf;                 // unstretched rounds at bottom / top, hf rounds
    unsigned long long s0, sm, hash;     // stretched delta sums at bottom / top, log hash
};

__device__ __forceinline__ void acc_zero(Acc &a) {
    a.n0 = a.nm = a.hf = 0;
    a.s0 = a.sm = a.hash = 0;
}

// Energy bookkeeping of a row once its levels Flev (bit p = level during round p) are known.
__device__ __forceinline__ void row_energy(const uint32_t *row, int lane, uint32_t Flev, const RowPred &r,
                                           uint32_t vmask, Acc &acc) {
    acc.n0 += __popc(~Flev & ~r.S0 & vmask);
    acc.nm += __popc(Flev & ~r.SM & vmask);
    const uint32_t M0 = ~Flev & r.S0 & vmask;
    if (__any_sync(FULL, M0 != 0)) acc.s0 += row_masked_sum(row, lane, M0);
    const uint32_t MM = Flev & r.SM & vmask;
    if (__any_sync(FULL, MM != 0)) acc.sm += row_masked_sum(row, lane, MM);
}

// Energy and time totals from the integer accumulators (energy model: an interval at level
// f lasts dt * max(1, x / C(f)) and draws P(f)).
__device__ __forceinline__ void totals(const DevModel &M, uint64_t N0, uint64_t NM, unsigned long long S0,
                                       unsigned long long SMs, double *E, double *T) {
    const double t0 = M.dt * (double)N0 + M.a0 * (double)S0;    // seconds at the bottom
    const double tM = M.dt * (double)NM + M.aM * (double)SMs;   // seconds at the top
    *T = t0 + tM;
    *E = M.P0 * t0 + M.PM * tM;
}

}  // namespace core
}  // namespace magus
