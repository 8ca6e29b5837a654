// replay_core.cuh - per-row building blocks of the time-parallel MAGUS replay, shared by the
// batched kernel (replay_tp.cu) and the serving kernel (serve.cu).
//
// A "row" is 32 consecutive rounds owned by one lane; bit p of every mask is round p of the
// row.  Rows sit in shared memory in the 128-byte swizzled layout that a TMA tensor copy
// with CU_TENSOR_MAP_SWIZZLE_128B writes: the 16-byte chunk c of row R lives at chunk
// position c ^ (R & 7).  A lane reading its own row chunk by chunk therefore touches a
// different bank group than the 7 other lanes of its quarter-warp, and the chunk index --
// hence the register index -- stays a compile-time constant.  Data row 0 of a sub-block is
// 1024-byte aligned and rows -1 and -2 (the 64 deltas before it) are always readable.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "magus_internal.h"

namespace magus {
namespace core {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int32_t kFastLimit = 1 << 30;   // fast path: every delta below 2^30


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

// ------------------------------------------------------------------ swizzled shared memory
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte address of chunk c (0..7) of row R (may be -1, -2) relative to data row 0 at `base`
__device__ __forceinline__ uint32_t swz_chunk(uint32_t base, int R, int c) {
    return base + (uint32_t)(R * 128) + ((uint32_t)((c ^ R) & 7) << 4);
}
// byte address of element E (>= -64) relative to data row 0
__device__ __forceinline__ uint32_t swz_elem(uint32_t base, int E) {
    const int R = E >> 5;
    return swz_chunk(base, R, (E >> 2) & 7) + ((uint32_t)(E & 3) << 2);
}
__device__ __forceinline__ void lds128(uint32_t addr, uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d) {
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr));
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// the 32 deltas of row R, in order
__device__ __forceinline__ void load_row(uint32_t base, int R, uint32_t (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 8; c++) lds128(swz_chunk(base, R, c), v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
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
    bool fast;         // every delta of the row and its window below 2^30
};

// Integer decision points clamped to the fast path's reach (|m| < 2^30): beyond it the
// comparison is constant over every reachable m, so clamping does not change it.
__device__ __forceinline__ int32_t clamp_mid(int64_t v) {
    const int64_t lim = (int64_t)kFastLimit + 8;
    return (int32_t)(v > lim ? lim : (v < -lim ? -lim : v));
}
__device__ __forceinline__ int32_t clamp_thr(uint32_t t) {
    return (int32_t)(t > (uint32_t)kFastLimit + 8u ? (uint32_t)kFastLimit + 8u : t);
}

// Alg. 1 for one round, exact for any deltas: the 64-bit integer decision outside the band
// the host derived (plan.cu), the FP64 evaluation in the oracle's order inside it.
__device__ __forceinline__ void predict_exact(uint32_t a, uint32_t b, const DevPolicy &P, const DevModel &M,
                                              bool &up, bool &dn) {
    const long long m = (long long)a - (long long)b;
    up = m > P.up_mid;
    dn = m < P.dn_mid;
    const uint32_t m32 = a - b;
    if (((m32 - P.up_lo) <= P.up_w) || ((m32 - P.dn_lo) <= P.dn_w)) {
        const double xa = __ddiv_rn(__dmul_rn(M.bpc, (double)a), M.q);
        const double xb = __ddiv_rn(__dmul_rn(M.bpc, (double)b), M.q);
        const double der = __ddiv_rn(__dsub_rn(xa, xb), (double)P.W);
        up = der > P.inc;
        dn = der < P.dec;
    }
    dn = dn && !up;   // Alg. 1 tests +1 first: with inc < dec both can hold
}

// Alg. 1 for one row, exact for any deltas (the fallback of the fast path below).
static __device__ __noinline__ void row_predict_general(uint32_t base, int lane, const DevPolicy &P, const DevModel &M,
                                                 uint32_t &UP, uint32_t &DN, uint32_t &S0, uint32_t &SM) {
    UP = DN = S0 = SM = 0;
    for (int k = 0; k < 32; k++) {
        const int E = 32 * lane + k;
        const uint32_t a = lds32(swz_elem(base, E));
        const uint32_t b = lds32(swz_elem(base, E - P.W));
        bool up, dn;
        predict_exact(a, b, P, M, up, dn);
        UP |= (uint32_t)up << k;
        DN |= (uint32_t)dn << k;
        S0 |= (uint32_t)(a > M.thr0) << k;
        SM |= (uint32_t)(a > M.thrM) << k;
    }
}

// Fast path, S = (-W) mod 4.  With m = a - b, tu = (up_mid + 3) - m and td = m - (dn_mid - 2)
// are negative exactly outside the decision bands on the +1 / -1 side (no overflow while
// every delta is below 2^30), and lie in [0, 5] exactly inside the bands [up_mid - 2,
// up_mid + 3] and [dn_mid - 2, dn_mid + 3], where the caller falls back to the exact path:
// one three-input minimum tracks both bands.  A funnel shift pushes each sign bit into its
// mask, so round k ends up at bit 31 - k.  The stretch test and td (= tu + td - tu, the sum
// being constant) are written as multiply-adds with a run-time multiplier of -1 so that they
// issue on the FMA pipe: the kernel is bound by the half-rate integer ALU pipe and the issue
// rate together (measured: td as an IMAD took the batched replay from 0.512 to 0.486 ms; the
// masked sums as IMADs gained nothing).
// WC > 0: W = WC is known at compile time (WC <= 28, so W + S <= 32): the deltas W rounds
// earlier are the row's own deltas shifted by W, except the first W, which are the last
// W + S of the row before (its last (W + S) / 4 chunks) -- 8 + (W + S) / 4 loads instead of
// 17.  WC = 0: W at run time, the 36-delta window loaded separately.
template <int S, int WC = 0, bool kChunked = false>
__device__ __forceinline__ void row_predict_fast(uint32_t base, int lane, int W, uint32_t one, int32_t upc,
                                                 int32_t dnc, int32_t thr0c, uint32_t &UPr, uint32_t &DNr,
                                                 uint32_t &S0r, uint32_t &band, uint32_t &amax,
                                                 uint32_t (&v)[32]) {
    // kChunked: the row's deltas are loaded one 16-byte chunk at a time as the loop reaches
    // them, so a delta need not stay in a register for longer than W rounds (2.7 % faster on
    // the batched replay in the tile instances for one W; kernels that inline several
    // predictors load the row first, which keeps their register demand where it was)
    if constexpr (!kChunked) load_row(base, lane, v);
    // window of the deltas W rounds earlier: 36 deltas from the 4-aligned element E0
    constexpr int NP = WC > 0 ? (WC + S) / 4 : 9;
    uint32_t u[4 * NP];
    if constexpr (WC > 0) {
        static_assert(((WC + S) & 3) == 0 && WC + S <= 32, "window of the row before");
#pragma unroll
        for (int c = 0; c < NP; c++)
            lds128(swz_chunk(base, lane - 1, 8 - NP + c), u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3]);
    } else {
        const int E0 = 32 * lane - (W + S);
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const int E = E0 + 4 * c;
            lds128(swz_chunk(base, E >> 5, (E >> 2) & 7), u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3]);
        }
    }
    const uint32_t neg1 = 0u - one;
    const uint32_t up3 = (uint32_t)upc + 3u, dn2 = (uint32_t)dnc - 2u;
    const uint32_t tud = up3 - dn2;   // tu + td, the same for every round
    uint32_t bd = 0xffffffffu, mx = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) {
        // (each chunk's load one chunk ahead of its use: 0.4 % faster than at its use, and
        // than two ahead)
        if (kChunked && k == 0) lds128(swz_chunk(base, lane, 0), v[0], v[1], v[2], v[3]);
        if (kChunked && (k & 3) == 0 && k + 4 < 32)
            lds128(swz_chunk(base, lane, (k >> 2) + 1), v[k + 4], v[k + 5], v[k + 6], v[k + 7]);
        const uint32_t a = v[k];
        uint32_t b;
        if constexpr (WC > 0) b = k < WC ? u[k + S] : v[k - WC];
        else b = u[k + S];
        const uint32_t tu = up3 - a + b;                  // < 0: +1;  in [0, 5]: up band
        const uint32_t td = tu * neg1 + tud;              // = a - b - dn2: < 0: -1;  in [0, 5]: dn band
        const uint32_t ts = a * neg1 + (uint32_t)thr0c;   // < 0  <=>  a > thr0 (an IMAD)
        UPr = __funnelshift_l(tu, UPr, 1);
        DNr = __funnelshift_l(td, DNr, 1);
        S0r = __funnelshift_l(ts, S0r, 1);
        bd = __vimin3_u32(bd, tu, td);
        if (k & 1) mx = __vimax3_u32(mx, v[k - 1], a);
    }
    band = bd;
    amax = mx;
}

// kCoopSM: the top-capacity test by the whole warp, one row at a time, for the rows that need
// it (the tile kernel's one-member groups and the one-rung kernel: 1.2 % and 3.4 % faster;
// the segment kernel measured 12 % slower this way and keeps the per-lane pass).
template <int S, int WC = 0, bool kChunked = false, bool kCoopSM = false>
__device__ __forceinline__ bool row_predict_fast_dispatch(uint32_t base, int lane, const DevPolicy &P,
                                                          const DevModel &M, RowPred &r, uint32_t (&v)[32]) {
    uint32_t UPr = 0, DNr = 0, S0r = 0, band, amax;
    row_predict_fast<S, WC, kChunked>(base, lane, P.W, (uint32_t)M.one, clamp_mid(P.up_mid), clamp_mid(P.dn_mid),
                            clamp_thr(M.thr0), UPr, DNr, S0r, band, amax, v);
    // every delta of the sub-block is some lane's row element; the 64 before it (rows -1, -2)
    // are checked here: the fast path needs all of them below 2^30
    // (with W known at compile time only row -1 is read: W + S <= 32)
    const uint32_t h0 = WC > 0 ? 0u : lds32(swz_elem(base, lane - 64)), h1 = lds32(swz_elem(base, lane - 32));
    const uint32_t hx = max(max(h0, h1), amax);
    // fall back when a delta reaches 2^30 or a round lies in a decision band
    if (__any_sync(FULL, hx >= (uint32_t)kFastLimit || band <= 5u)) return false;
    r.UP = __brev(UPr);
    r.DN = __brev(DNr);
    r.S0 = __brev(S0r);
    r.SM = 0;
    if constexpr (kCoopSM) {
        // rows holding a delta above the top capacity are rare (a lane or two per warp where
        // any): lane j tests element j of such a row, and the ballot is the row's mask
        uint32_t need = __ballot_sync(FULL, amax > M.thrM);
        while (need) {
            const int L = __ffs(need) - 1;
            need &= need - 1;
            const uint32_t bits = __ballot_sync(FULL, lds32(swz_elem(base, 32 * L + lane)) > M.thrM);
            if (lane == L) r.SM = bits;
        }
    } else if (__any_sync(FULL, amax > M.thrM)) {
        if constexpr (kChunked) load_row(base, lane, v);
        uint32_t SMr = 0;
        const int32_t tm = clamp_thr(M.thrM);
        const uint32_t neg1 = 0u - (uint32_t)M.one;
#pragma unroll
        for (int k = 0; k < 32; k++) SMr = __funnelshift_l(v[k] * neg1 + (uint32_t)tm, SMr, 1);
        r.SM = __brev(SMr);
    }
    return true;
}

// Alg. 1 predictions and stretch bits of this lane's row (rows of the sub-block at `base`).
// WC > 0: W = WC, known at compile time.  Otherwise kSpecW: the common window lengths take
// the compile-time-W path through a switch per row (more code per kernel, so only kernels
// with one policy per slot use it; grouped tiles keep the run-time path).
template <int WC = -1, bool kSpecW = false, bool kCoopSM = false>
__device__ __forceinline__ RowPred row_predict(uint32_t base, int lane, const DevPolicy &P, const DevModel &M,
                                               uint32_t vmask, uint32_t pmask) {
    RowPred r;
    uint32_t v[32];
    bool ok = false;
    if constexpr (WC > 0) {
        ok = row_predict_fast_dispatch<(-WC) & 3, WC, true, kCoopSM>(base, lane, P, M, r, v);
    } else switch (kSpecW ? P.W : 0) {
#define MAGUS_PRED_W(w) \
        case w: ok = row_predict_fast_dispatch<(-(w)) & 3, w, false, kCoopSM>(base, lane, P, M, r, v); break;
        MAGUS_PRED_W(1) MAGUS_PRED_W(2) MAGUS_PRED_W(3) MAGUS_PRED_W(4) MAGUS_PRED_W(5) MAGUS_PRED_W(6)
        MAGUS_PRED_W(7) MAGUS_PRED_W(8) MAGUS_PRED_W(10) MAGUS_PRED_W(12) MAGUS_PRED_W(16)
#undef MAGUS_PRED_W
        default:
            switch ((-P.W) & 3) {
                case 0: ok = row_predict_fast_dispatch<0, 0, false, kCoopSM>(base, lane, P, M, r, v); break;
                case 1: ok = row_predict_fast_dispatch<1, 0, false, kCoopSM>(base, lane, P, M, r, v); break;
                case 2: ok = row_predict_fast_dispatch<2, 0, false, kCoopSM>(base, lane, P, M, r, v); break;
                default: ok = row_predict_fast_dispatch<3, 0, false, kCoopSM>(base, lane, P, M, r, v); break;
            }
    }
    r.fast = ok;
    if (!ok) row_predict_general(base, lane, P, M, r.UP, r.DN, r.S0, r.SM);
    r.UP &= pmask;
    r.DN &= pmask & ~r.UP;   // Alg. 1 tests +1 first: with inc < dec both comparisons can hold
    r.S0 &= vmask;
    r.SM &= vmask;
    return r;
}

// Alg. 2 over one row: bit p of the result = high-frequency state of round p, i.e. at
// least kmin flags among rounds p-L+1 .. p.  H: flags of the 64 rounds before the row
// (bit q = round q - 64); FL: flags of the row.
// The counts of rounds p, p+8, p+16, p+24 advance together, one per byte of a 32-bit word
// holding count + 128 - kmin: the top bit of a byte is set exactly when count >= kmin
// (counts <= 64, so bytes never carry into each other).  (A nibble-wide variant with 8
// counts per word measured slower: it needs twice the population counts to seed.)
__device__ __forceinline__ uint32_t hf_row(uint64_t H, uint32_t FL, int L, int kmin) {
    const int s = 64 - L;
    // bit p of LV = flag of round p - L (leaving the window at round p)
    const uint32_t LV = s == 0 ? (uint32_t)H : (uint32_t)((H >> s) | ((uint64_t)FL << (64 - s)));
    const uint32_t c0 = __popcll(H >> s);                    // window ending at round -1
    uint32_t HF = 0;
    const uint32_t d0 = __popc(FL & 0xffu) - __popc(LV & 0xffu);
    const uint32_t d1 = __popc(FL & 0xff00u) - __popc(LV & 0xff00u);
    const uint32_t d2 = __popc(FL & 0xff0000u) - __popc(LV & 0xff0000u);
    const uint32_t c1 = c0 + d0, c2 = c1 + d1, c3 = c2 + d2; // windows ending at 7, 15, 23
    // byte b holds count + 128 - kmin: bit 7 of the byte <=> count >= kmin
    uint32_t e4 = (c0 | (c1 << 8) | (c2 << 16) | (c3 << 24)) + (uint32_t)(128 - kmin) * 0x01010101u;
#pragma unroll
    for (int p = 0; p < 8; p++) {
        e4 = e4 + ((FL >> p) & 0x01010101u) - ((LV >> p) & 0x01010101u);
        HF = (HF >> 1) | (e4 & 0x80808080u);
    }
    return HF;
}

// Algorithm 2 for several policies sharing L (a policy group of the sweep): the sliding
// counts are formed once -- byte b of w[p] holds the flag count of the window ending at
// round 8b + p (0..64) -- and each policy only compares them with its own kmin.
__device__ __forceinline__ void hf_counts(uint64_t H, uint32_t FL, int L, uint32_t (&w)[8]) {
    const int s = 64 - L;
    const uint32_t LV = s == 0 ? (uint32_t)H : (uint32_t)((H >> s) | ((uint64_t)FL << (64 - s)));
    const uint32_t c0 = __popcll(H >> s);
    const uint32_t d0 = __popc(FL & 0xffu) - __popc(LV & 0xffu);
    const uint32_t d1 = __popc(FL & 0xff00u) - __popc(LV & 0xff00u);
    const uint32_t d2 = __popc(FL & 0xff0000u) - __popc(LV & 0xff0000u);
    const uint32_t c1 = c0 + d0, c2 = c1 + d1, c3 = c2 + d2;
    uint32_t e4 = c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
#pragma unroll
    for (int p = 0; p < 8; p++) {
        e4 = e4 + ((FL >> p) & 0x01010101u) - ((LV >> p) & 0x01010101u);
        w[p] = e4;
    }
}
// bit p of the result: count of the window ending at round p >= kmin (byte + 128 - kmin
// sets bit 7 exactly then; counts <= 64 and kmin <= 65 keep every byte in 0..192)
__device__ __forceinline__ uint32_t hf_from_counts(const uint32_t (&w)[8], int kmin) {
    const uint32_t bias = (uint32_t)(128 - kmin) * 0x01010101u;
    uint32_t HF = 0;
#pragma unroll
    for (int p = 0; p < 8; p++) HF = (HF >> 1) | ((w[p] + bias) & 0x80808080u);
    return HF;
}

// Algorithm 2 for a 10-round tune window, bit-sliced.  S_i (bit p = flag of round p - i,
// i = 0..9) are summed position by position by a carry-save adder tree (full adders: sum =
// three-input xor, carry = majority) into the 4-bit count c3 c2 c1 c0 of every round's
// window; the comparison with kmin is then a fixed boolean form of those four words.
struct Count4 {
    uint32_t c0, c1, c2, c3;
};
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }
__device__ __forceinline__ Count4 window10_counts(uint64_t H, uint32_t FL) {
    const uint32_t Hh = (uint32_t)(H >> 32);   // flags of rounds -32 .. -1
    uint32_t S[10];
    S[0] = FL;
#pragma unroll
    for (int i = 1; i < 10; i++) S[i] = __funnelshift_l(Hh, FL, i);
    const uint32_t s1 = S[0] ^ S[1] ^ S[2], k1 = maj3(S[0], S[1], S[2]);
    const uint32_t s2 = S[3] ^ S[4] ^ S[5], k2 = maj3(S[3], S[4], S[5]);
    const uint32_t s3 = S[6] ^ S[7] ^ S[8], k3 = maj3(S[6], S[7], S[8]);
    const uint32_t s4 = s1 ^ s2 ^ s3, k4 = maj3(s1, s2, s3);
    Count4 r;
    r.c0 = s4 ^ S[9];
    const uint32_t k5 = s4 & S[9];
    const uint32_t s6 = k1 ^ k2 ^ k3, k6 = maj3(k1, k2, k3);
    r.c1 = k4 ^ k5 ^ s6;
    const uint32_t k7 = maj3(k4, k5, s6);
    r.c2 = k6 ^ k7;
    r.c3 = k6 & k7;
    return r;
}
// bit p: count of round p's window >= kmin (counts are at most 10): the carry out of the
// 4-bit sum count + (16 - kmin), one majority per bit (measured faster than a switch over
// fixed boolean forms per kmin)
__device__ __forceinline__ uint32_t count4_ge(const Count4 &c, int kmin) {
    if (kmin <= 0) return 0xffffffffu;
    if (kmin > 10) return 0u;
    const uint32_t a = 16u - (uint32_t)kmin;   // 6 .. 15
    const uint32_t A0 = 0u - (a & 1u), A1 = 0u - ((a >> 1) & 1u), A2 = 0u - ((a >> 2) & 1u), A3 = 0u - ((a >> 3) & 1u);
    uint32_t cy = c.c0 & A0;
    cy = maj3(c.c1, cy, A1);
    cy = maj3(c.c2, cy, A2);
    return maj3(c.c3, cy, A3);
}

// Algorithm 2 for any window length: the bit-sliced form for 10 rounds, else byte counts
// (the one-rung kernel: 1.7 % faster on 4,096 x 100,000; the segment kernel 3.4 % on
// 16 x 4,000,000 once the threshold became a carry chain)
__device__ __forceinline__ uint32_t hf_row_any(uint64_t H, uint32_t FL, int L, int kmin) {
    return L == 10 ? count4_ge(window10_counts(H, FL), kmin) : hf_row(H, FL, L, kmin);
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

// Change-log entries of a warp's 32 rows.  Up to 32 changes: one pass, lane i takes the
// warp's i-th change (rows in order, rounds in order within a row), found by a binary search
// over the inclusive prefix counts of the rows; more changes: each lane walks its own row.  CHG / Lv: this lane's change mask and level
// after each round; row0: global interval index of round 0 of row 0 (rows follow every 32
// rounds); log: the pair's log (NULL: hash only); first: entries of the pair before this
// warp's rows.  Entries are written to consecutive slots (coalesced stores).
__device__ __forceinline__ void emit_changes(uint32_t CHG, uint32_t Lv, uint64_t row0, uint32_t topK,
                                             uint32_t *log, uint64_t log_cap, uint64_t first,
                                             unsigned long long &hash, int lane) {
    if (!log) {
        // hash only: the sum is order-free and no slot is needed, so every lane hashes its
        // own row's changes (no scan, no search; measured 5-6 % faster on the many-policy
        // workloads, which write no entries)
        uint32_t bits = CHG;
        while (bits) {
            const int q = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint64_t when = row0 + 32u * (uint32_t)lane + (uint32_t)q + 1u;
            const uint32_t lv = ((Lv >> q) & 1u) ? topK : 0u;
            hash += mix64((when << 8) | lv);
        }
        return;
    }
    const uint32_t nch = __popc(CHG);
    uint32_t incl = nch;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total > 32) {
        // dense changes: every lane walks its own row (fewer steps than several passes)
        uint64_t off = first + (incl - nch);
        uint32_t bits = CHG;
        while (bits) {
            const int q = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint64_t when = row0 + 32u * (uint32_t)lane + (uint32_t)q + 1u;
            const uint32_t lv = ((Lv >> q) & 1u) ? topK : 0u;
            if (log && off < log_cap) log[off] = (uint32_t)(when << 5) | lv;
            hash += mix64((when << 8) | lv);
            off++;
        }
        return;
    }
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t idx = base + (uint32_t)lane;
        // row r: the first row whose inclusive count exceeds idx
        int r = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t v = __shfl_sync(FULL, incl, r + step - 1);
            if (v <= idx) r += step;
        }
        r = r > 31 ? 31 : r;
        const uint32_t chg_r = __shfl_sync(FULL, CHG, r);
        const uint32_t lv_r = __shfl_sync(FULL, Lv, r);
        const uint32_t excl_r = __shfl_sync(FULL, incl - nch, r);
        if (idx < total) {
            uint32_t m = chg_r;
            for (uint32_t j = excl_r; j < idx; j++) m &= m - 1;   // drop the earlier changes
            const int q = __ffs(m) - 1;
            const uint64_t when = row0 + 32u * (uint32_t)r + (uint32_t)q + 1u;
            const uint32_t lv = ((lv_r >> q) & 1u) ? topK : 0u;
            const uint64_t off = first + idx;
            if (log && off < log_cap) log[off] = (uint32_t)(when << 5) | lv;
            hash += mix64((when << 8) | lv);
        }
    }
}

// The fallback of the staged path (more than 32 changes in a warp's rows, or interval indices
// past 2^31), out of line: it is rare, and inline its code lengthened the hot loop of the
// kernels that stage (measured 1.5 % slower on the batched replay).
static __device__ __noinline__ unsigned long long emit_changes_cold(uint32_t CHG, uint32_t Lv, uint64_t row0,
                                                                   uint32_t topK, uint32_t *log, uint64_t log_cap,
                                                                   uint64_t first, int lane) {
    unsigned long long h = 0;
    emit_changes(CHG, Lv, row0, topK, log, log_cap, first, h, lane);
    return h;
}

// Change-log staging (one warp, one pair).  A staged entry keeps the pair's log slot and
// (interval index << 1 | at the top).  Entries wait in the warp's table until 32 are
// pending; then lane i takes entry i, so the log stores and the hash run on full warps and
// the stores leave as whole lines, where emitting each sub-block's few changes at once keeps
// most lanes idle.  Usable while interval indices stay below 2^31.
struct Staged {
    uint32_t slot;   // index in the pair's log
    uint32_t tw;     // (t + 1) << 1 | level is the top
};
constexpr int kStageCap = 64;   // up to 31 waiting + up to 32 of one sub-block

// Append the changes of a warp's 32 rows (CHG / Lv as in emit_changes; `excl`: this lane's
// changes before it, in the warp's order) behind the `pending` entries already waiting.
__device__ __forceinline__ void stage_changes(uint32_t CHG, uint32_t Lv, uint32_t row0, uint32_t slot0,
                                              Staged *tab, uint32_t pending, uint32_t excl, int lane) {
    uint32_t bits = CHG;
    uint32_t k = excl;
    while (bits) {
        const int q = __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t when = row0 + 32u * (uint32_t)lane + (uint32_t)q + 1u;
        Staged e;
        e.slot = slot0 + k;
        e.tw = (when << 1) | ((Lv >> q) & 1u);
        tab[pending + k] = e;
        k++;
    }
}

// Store and hash the first `count` (<= 32) staged entries: lane i takes entry i.
__device__ __forceinline__ void flush_staged(const Staged *tab, uint32_t count, uint32_t topK, uint32_t *log,
                                             uint64_t log_cap, unsigned long long &hash, int lane) {
    if ((uint32_t)lane < count) {
        const Staged e = tab[lane];
        const uint32_t when = e.tw >> 1;
        const uint32_t lv = (e.tw & 1u) ? topK : 0u;
        if (log && e.slot < log_cap) log[e.slot] = (when << 5) | lv;
        hash += mix64(((uint64_t)when << 8) | lv);
    }
}

// part + v if bit K of M is set: the bit test sets a predicate and the add is predicated
// (two instructions; the select form costs more).
template <int K>
__device__ __forceinline__ uint32_t add_if_bit(uint32_t part, uint32_t M, uint32_t v) {
    asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "and.b32 t, %1, %3;\n\t"
        "setp.ne.b32 p, t, 0;\n\t"
        "@p add.u32 %0, %0, %2;\n\t}"
        : "+r"(part)
        : "r"(M), "r"(v), "n"(1u << K));
    return part;
}
template <int C>
__device__ __forceinline__ unsigned long long add_masked4(unsigned long long s, uint32_t M, const uint32_t (&v)[32]) {
    uint32_t part = 0;   // four deltas below 2^30 fit 32 bits
    part = add_if_bit<4 * C + 0>(part, M, v[4 * C + 0]);
    part = add_if_bit<4 * C + 1>(part, M, v[4 * C + 1]);
    part = add_if_bit<4 * C + 2>(part, M, v[4 * C + 2]);
    part = add_if_bit<4 * C + 3>(part, M, v[4 * C + 3]);
    return s + part;
}

// Sum of the row's deltas at the rounds selected by mask Msel (bit p = round p).
__device__ __forceinline__ unsigned long long row_masked_sum(uint32_t base, int lane, uint32_t Msel, bool fast) {
    uint32_t v[32];
    unsigned long long s = 0;
    if (fast) {
        // every delta < 2^30; one 16-byte chunk at a time (fewer registers live)
#define MAGUS_MASKED_CHUNK(C)                                                    \
        lds128(swz_chunk(base, lane, C), v[4 * C], v[4 * C + 1], v[4 * C + 2], v[4 * C + 3]); \
        s = add_masked4<C>(s, Msel, v);
        MAGUS_MASKED_CHUNK(0) MAGUS_MASKED_CHUNK(1) MAGUS_MASKED_CHUNK(2) MAGUS_MASKED_CHUNK(3)
        MAGUS_MASKED_CHUNK(4) MAGUS_MASKED_CHUNK(5) MAGUS_MASKED_CHUNK(6) MAGUS_MASKED_CHUNK(7)
#undef MAGUS_MASKED_CHUNK
    } else {
        load_row(base, lane, v);
#pragma unroll
        for (int k = 0; k < 32; k++) s += ((Msel >> k) & 1u) ? v[k] : 0u;
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
// kSparseTop: stretched rounds at the top (throughput above the top capacity, rare) are
// added one by one instead of a pass over the whole row (every caller now: with four warps
// the grouped tiles run the policy sweep 1.2 % faster this way; with eight, the loop had
// raised their register demand).
template <bool kSparseTop = true>
__device__ __forceinline__ void row_energy(uint32_t base, int lane, uint32_t Flev, const RowPred &r,
                                           uint32_t vmask, Acc &acc) {
    acc.n0 += __popc(~Flev & ~r.S0 & vmask);
    acc.nm += __popc(Flev & ~r.SM & vmask);
    const bool fast = __all_sync(FULL, r.fast);
    const uint32_t M0 = ~Flev & r.S0 & vmask;
    if (__any_sync(FULL, M0 != 0)) acc.s0 += row_masked_sum(base, lane, M0, fast);
    uint32_t MM = Flev & r.SM & vmask;
    if (!kSparseTop) {
        if (__any_sync(FULL, MM != 0)) acc.sm += row_masked_sum(base, lane, MM, fast);
    } else if (__any_sync(FULL, MM != 0)) {
        unsigned long long sm = 0;
        while (MM) {
            const int q = __ffs(MM) - 1;
            MM &= MM - 1;
            sm += lds32(swz_elem(base, 32 * lane + q));
        }
        acc.sm += sm;
    }
}

// Rounds of a row whose level is not known yet (before the first event of a time segment):
// their charge is kept for both possible levels.
struct PAcc {
    uint32_t n0, nm;                     // unstretched rounds if at the bottom / at the top
    unsigned long long s0, sm;           // stretched delta sums if at the bottom / at the top
};

__device__ __forceinline__ void pacc_zero(PAcc &a) {
    a.n0 = a.nm = 0;
    a.s0 = a.sm = 0;
}

__device__ __forceinline__ void row_energy_prefix(uint32_t base, int lane, uint32_t PM, const RowPred &r, PAcc &pa) {
    pa.n0 += __popc(PM & ~r.S0);
    pa.nm += __popc(PM & ~r.SM);
    const bool fast = __all_sync(FULL, r.fast);
    if (__any_sync(FULL, (PM & r.S0) != 0)) pa.s0 += row_masked_sum(base, lane, PM & r.S0, fast);
    if (__any_sync(FULL, (PM & r.SM) != 0)) pa.sm += row_masked_sum(base, lane, PM & r.SM, fast);
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

// The 64 deltas ending at element `last` (relative to data row 0), oldest first.
__device__ __forceinline__ void read_hist(uint32_t base, int last, uint32_t *out) {
    for (int k = 0; k < 64; k++) out[k] = lds32(swz_elem(base, last - 63 + k));
}

}  // namespace core
}  // namespace magus
