// plan.cu - host-side derivation of kernel parameters from a policy and a model.
//
// Algorithm 1 (Sec. 3.1) compares derivative = (x_t - x_{t-W}) / W with inc / dec, where
// x = RN(bpc * delta / q) and every operation rounds to nearest in FP64.  Let
// m = delta_t - delta_{t-W} (an integer) and r(m) = bpc * m / (q * W) the exact real value.
// Each of the three roundings moves the result by at most half an ulp of quantities no
// larger than bpc * 2^32 / q, so |derivative - r(m)| <= 6 * bpc * 2^32 * 2^-53 / (q * W),
// while consecutive integers m differ by bpc / (q * W) in r(m): the rounding error is below
// 2^-18 of one integer step.  Hence with c = inc * q * W / bpc:
//     m >= floor(c) + 4  ->  derivative > inc          (r(m) >= inc + 3 steps)
//     m <= floor(c) - 3  ->  derivative <= inc         (r(m) <= inc - 3 steps)
// and only the six integers floor(c) - 2 .. floor(c) + 3 need the FP64 evaluation.  The same
// holds for dec.  c itself is computed in long double (relative error ~2^-63, so floor(c)
// is off by at most one for |c| < 2^33, absorbed by the margins above).
#include <cmath>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "replay_closed.h"

namespace magus {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

static const long double kReach = 8589934592.0L;  // 2^33 > any |m| = |a - b| < 2^32

// Doubles in order as integers (-0 and +0 share 0) and back.
static int64_t dkey(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return (b >> 63) ? -(int64_t)(b & 0x7fffffffffffffffull) : (int64_t)b;
}
static double dval(int64_t k) {
    const uint64_t b = k >= 0 ? (uint64_t)k : ((uint64_t)(-k) | 0x8000000000000000ull);
    double x;
    memcpy(&x, &b, 8);
    return x;
}
// The largest finite d with pred(d) true, for pred true on a prefix of the finite doubles;
// -inf when it holds for none, +inf when for all.
template <class Pred>
static double last_true(Pred pred) {
    const double lo_d = -1.7976931348623157e308, hi_d = 1.7976931348623157e308;
    if (!pred(lo_d)) return -INFINITY;
    if (pred(hi_d)) return INFINITY;
    int64_t lo = dkey(lo_d), hi = dkey(hi_d);   // pred(lo) true, pred(hi) false
    // the span of the keys exceeds INT64_MAX: step in unsigned arithmetic
    while ((uint64_t)hi - (uint64_t)lo > 1u) {
        const int64_t mid = (int64_t)((uint64_t)lo + ((uint64_t)hi - (uint64_t)lo) / 2u);
        if (pred(dval(mid))) lo = mid;
        else hi = mid;
    }
    return dval(lo);
}

int derive_model(const magus_model_t &m, DevModel *out, std::string *err) {
    if (m.n_levels < 2 || m.n_levels > MAGUS_MAX_LEVELS) { *err = "n_levels must be 2..32"; return MAGUS_EINVAL; }
    if (!m.f_ghz) { *err = "f_ghz is NULL"; return MAGUS_EINVAL; }
    if (!(m.dt_s >= 1e-9 && m.dt_s <= 1e6)) { *err = "dt_s must be in [1e-9, 1e6]"; return MAGUS_EINVAL; }
    if (m.bytes_per_count < 1 || m.bytes_per_count > (1 << 20)) { *err = "bytes_per_count must be 1..2^20"; return MAGUS_EINVAL; }
    if (!(m.f_ref_ghz > 0) || !std::isfinite(m.f_ref_ghz)) { *err = "f_ref_ghz must be positive"; return MAGUS_EINVAL; }
    if (!(m.bw_ref_gbs > 0) || !std::isfinite(m.bw_ref_gbs)) { *err = "bw_ref_gbs must be positive"; return MAGUS_EINVAL; }
    if (!std::isfinite(m.p_static_w) || !std::isfinite(m.p_dyn_w)) { *err = "powers must be finite"; return MAGUS_EINVAL; }
    for (int k = 0; k < m.n_levels; k++) {
        if (!(m.f_ghz[k] > 0) || !std::isfinite(m.f_ghz[k])) { *err = "frequencies must be positive"; return MAGUS_EINVAL; }
        if (k && !(m.f_ghz[k] > m.f_ghz[k - 1])) { *err = "ladder must be strictly ascending"; return MAGUS_EINVAL; }
    }
    DevModel d;
    memset(&d, 0, sizeof(d));
    d.q = m.dt_s * 1e9;
    d.bpc = (double)m.bytes_per_count;
    d.dt = m.dt_s;
    d.K = m.n_levels;
    d.one = 1;
    for (int k = 0; k < m.n_levels; k++) {
        double fr = m.f_ghz[k] / m.f_ref_ghz;
        d.cap[k] = m.bw_ref_gbs * fr;
        d.pw[k] = m.p_static_w + m.p_dyn_w * (fr * fr);
    }
    auto thr = [&](double cap) -> uint32_t {
        // x > C  <=>  delta > C q / bpc; the boundary interval itself has x / C within
        // one rounding of 1, where max(1, x / C) is 1 either way up to an ulp.
        double v = std::floor(cap * d.q / d.bpc);
        if (v >= 4294967295.0) return 0xffffffffu;
        if (v < 0) return 0;
        return (uint32_t)v;
    };
    const int top = m.n_levels - 1;
    for (int k = 0; k < m.n_levels; k++) {
        d.thr[k] = thr(d.cap[k]);
        d.ak[k] = d.dt * d.bpc / (d.q * d.cap[k]);
    }
    d.thr0 = thr(d.cap[0]);
    d.thrM = thr(d.cap[top]);
    d.a0 = d.dt * d.bpc / (d.q * d.cap[0]);
    d.aM = d.dt * d.bpc / (d.q * d.cap[top]);
    d.P0 = d.pw[0];
    d.PM = d.pw[top];
    *out = d;
    return MAGUS_OK;
}

int derive_policy(const magus_policy_t &p, const magus_model_t &m, DevPolicy *out, std::string *err) {
    if (p.direv_length < 1 || p.direv_length > MAGUS_MAX_WINDOW) { *err = "direv_length must be 1..64"; return MAGUS_EINVAL; }
    if (p.tune_window < 1 || p.tune_window > MAGUS_MAX_WINDOW) { *err = "tune_window must be 1..64"; return MAGUS_EINVAL; }
    if (std::isnan(p.inc_threshold) || std::isnan(p.dec_threshold) || std::isnan(p.high_freq_threshold)) {
        *err = "thresholds must not be NaN"; return MAGUS_EINVAL;
    }
    if (p.step_mode < 0 || p.step_mode > 3) { *err = "step_mode must be 0..3"; return MAGUS_EINVAL; }
    if (p.pin_level < 0 || p.pin_level > m.n_levels) { *err = "pin_level must be 0..n_levels"; return MAGUS_EINVAL; }
    DevPolicy d;
    memset(&d, 0, sizeof(d));
    d.W = p.direv_length;
    d.L = p.tune_window;
    d.inc = p.inc_threshold;
    d.dec = p.dec_threshold;
    d.th = p.high_freq_threshold;
    d.step_mode = p.step_mode;
    d.pin = p.pin_level;
    // q is the FP64 product dt * 1e9 that both the oracle and the kernels divide by
    const long double qd = (long double)(m.dt_s * 1e9);
    auto crossing = [&](double thr, int64_t *mid, uint32_t *lo, uint32_t *w) {
        long double c = (long double)thr * qd * (long double)p.direv_length / (long double)m.bytes_per_count;
        if (c >= kReach) { *mid = (int64_t)kReach; *lo = 0x7fffffffu; *w = 0; return; }
        if (c <= -kReach) { *mid = -(int64_t)kReach; *lo = 0x7fffffffu; *w = 0; return; }
        int64_t f = (int64_t)floorl(c);
        *mid = f;
        *lo = (uint32_t)(uint64_t)(f - 2);
        *w = 5;
    };
    crossing(p.inc_threshold, &d.up_mid, &d.up_lo, &d.up_w);
    crossing(p.dec_threshold, &d.dn_mid, &d.dn_lo, &d.dn_w);
    const double Wd = (double)p.direv_length, inc = p.inc_threshold, dec = p.dec_threshold;
    d.up_last = last_true([&](double x) { return !(x / Wd > inc); });
    d.dn_last = last_true([&](double x) { return x / Wd < dec; });
    // Alg. 2: freq = sum / len >= threshold, sum in 0..L
    d.kmin = d.L + 1;
    for (int c = 0; c <= d.L; c++) {
        if ((double)c / (double)d.L >= p.high_freq_threshold) { d.kmin = c; break; }
    }
    *out = d;
    return MAGUS_OK;
}

// Closed loop: x(delta) exactly as the oracle and the kernels evaluate it, and the smallest
// v in [0, 2^32] with pred(v) for pred false on a prefix of 0 .. 2^32 - 1 and true after it
// (2^32 when it holds for none).
static double xval(const DevModel &m, uint32_t delta) { return (m.bpc * (double)delta) / m.q; }
template <class Pred>
static int64_t first_true_u32(Pred pred) {
    int64_t lo = -1, hi = (int64_t)1 << 32;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (pred((uint32_t)mid)) hi = mid;
        else lo = mid;
    }
    return hi;
}

// Alg. 1 in the closed loop when a throughput in its window is capped (Sec. 3.1; the
// monitor reads min(x, C) at the level in effect).  x is non-decreasing in delta and each
// FP64 difference below is monotone in the free delta, so every decision is a threshold on
// that delta; the decision itself is the division-free test on d (up_last / dn_last).
void derive_closed(const DevPolicy &P, const DevModel &M, bool ladder, ClosedThr *out) {
    ClosedThr c;
    memset(&c, 0, sizeof(c));
    const int n = ladder ? M.K : 2;
    auto level = [&](int l) { return ladder ? l : (l ? M.K - 1 : 0); };
    auto up_of = [&](double d) { return d > P.up_last; };
    auto dn_of = [&](double d) { return d <= P.dn_last; };
    for (int l = 0; l < n; l++) {
        const double C = M.cap[level(l)];
        const int64_t f = first_true_u32([&](uint32_t v) { return xval(M, v) > C; });
        c.cthr[l] = (uint32_t)(f - 1);   // C > 0 = x(0), so f >= 1
        // a capped: d = C - x(b), non-increasing in b
        c.bu[l] = first_true_u32([&](uint32_t b) { return !up_of(C - xval(M, b)); });
        c.bd[l] = first_true_u32([&](uint32_t b) { return dn_of(C - xval(M, b)); });
        // b capped: d = x(a) - C, non-decreasing in a
        c.au[l] = first_true_u32([&](uint32_t a) { return up_of(xval(M, a) - C); });
        c.ad[l] = first_true_u32([&](uint32_t a) { return !dn_of(xval(M, a) - C); });
    }
    for (int la = 0; la < n; la++)
        for (int lb = 0; lb < n; lb++) {
            const double d = M.cap[level(la)] - M.cap[level(lb)];
            if (up_of(d)) c.ccu[la] |= 1u << lb;
            if (dn_of(d)) c.ccd[la] |= 1u << lb;
        }
    *out = c;
}

// Group policies whose Alg. 1 parameters coincide (same W, inc, dec: identical predictions),
// at most gp members per group, keeping the policies' order within each group.
void form_groups(const std::vector<DevPolicy> &pols, int gp, std::vector<PolicyGroup> *out,
                 const std::vector<char> *include) {
    out->clear();
    std::vector<int> order;
    order.reserve(pols.size());
    for (size_t i = 0; i < pols.size(); i++)
        if (!include || (*include)[i]) order.push_back((int)i);
    auto key_less = [&](int a, int b) {
        const DevPolicy &x = pols[a], &y = pols[b];
        if (x.W != y.W) return x.W < y.W;
        if (x.up_mid != y.up_mid) return x.up_mid < y.up_mid;
        if (x.dn_mid != y.dn_mid) return x.dn_mid < y.dn_mid;
        if (memcmp(&x.inc, &y.inc, 8)) return memcmp(&x.inc, &y.inc, 8) < 0;
        if (memcmp(&x.dec, &y.dec, 8)) return memcmp(&x.dec, &y.dec, 8) < 0;
        return a < b;
    };
    auto same = [&](int a, int b) {
        const DevPolicy &x = pols[a], &y = pols[b];
        return x.W == y.W && x.up_mid == y.up_mid && x.dn_mid == y.dn_mid && !memcmp(&x.inc, &y.inc, 8) &&
               !memcmp(&x.dec, &y.dec, 8);
    };
    if (gp > 1) std::stable_sort(order.begin(), order.end(), key_less);
    for (size_t i = 0; i < order.size();) {
        PolicyGroup g;
        memset(&g, 0, sizeof(g));
        g.count = 0;
        size_t j = i;
        while (j < order.size() && g.count < gp && (g.count == 0 || same(order[i], order[j])))
            g.member[g.count++] = order[j++];
        for (int m = g.count; m < kMaxGroup; m++) g.member[m] = g.member[0];
        g.same_L = 1;
        for (int m = 1; m < g.count; m++) g.same_L &= pols[g.member[m]].L == pols[g.member[0]].L ? 1 : 0;
        out->push_back(g);
        i = j;
    }
}

}  // namespace magus
