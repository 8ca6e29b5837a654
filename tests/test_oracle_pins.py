"""Pins for the CPU oracle against closed forms, exact arithmetic and invariants.

Every expected value here comes from the paper's definitions worked out by hand
(Sec. 3.1 / Algorithm 1, Sec. 3.2 / Algorithm 2, Sec. 4, Sec. 6.1) or from exact
rational arithmetic, never from the oracle itself.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import tracegen

K = 17
TOP = K - 1


def exact_model(model):
    f = [Fraction(v) for v in model["f_ghz"]]
    fref = Fraction(model["f_ref_ghz"])
    cap = [Fraction(model["bw_ref_gbs"]) * fi / fref for fi in f]
    pw = [Fraction(model["p_static_w"]) + Fraction(model["p_dyn_w"]) * (fi / fref) ** 2 for fi in f]
    return cap, pw


def exact_energy(deltas, levels, model):
    """Energy and time of a level sequence, in exact rationals (energy model definition)."""
    cap, pw = exact_model(model)
    dt = Fraction(model["dt_s"])
    q = dt * 10**9
    E = Fraction(0)
    T = Fraction(0)
    for d, lv in zip(deltas, levels):
        x = Fraction(model["bytes_per_count"]) * int(d) / q
        s = max(Fraction(1), x / cap[lv])
        T += dt * s
        E += pw[lv] * dt * s
    return E, T


def close(a, b, rel=1e-12):
    return abs(float(a) - float(b)) <= rel * max(abs(float(b)), 1e-300)


# ----------------------------------------------------------------------------- Sec. 4
def test_constant_trace_stays_at_minimum(model, policy):
    n = 5000
    d = np.full(n, 123_456_789, dtype=np.uint32)     # 79.0 GB/s, above C(0.8 GHz)
    r = oracle.replay(d, policy, model, detail=True)
    assert r["n_changes"] == 0 and r["n_hf"] == 0 and r["change_hash"] == 0
    assert np.all(r["level_log"] == 0)
    # closed form: every interval at 0.8 GHz, stretched by x / C
    x = Fraction(64 * 123_456_789, 10**8)
    cap = Fraction(200) * Fraction(0.8) / Fraction(2.4)
    pw = Fraction(15) + Fraction(10) * (Fraction(0.8) / Fraction(2.4)) ** 2
    T = n * Fraction(0.1) * (x / cap)
    assert close(r["time_s"], T) and close(r["energy_j"], pw * T)
    assert close(r["edp_js"], pw * T * T)
    # derivative is exactly 0 once W+1 samples are held, NaN before (warm-up reading)
    assert np.all(np.isnan(r["deriv_log"][:policy["direv_length"]]))
    assert np.all(r["deriv_log"][policy["direv_length"]:] == 0.0)


def test_constant_trace_below_capacity_is_unstretched(model, policy):
    n = 1000
    d = np.full(n, 1_000_000, dtype=np.uint32)       # 0.64 GB/s
    r = oracle.replay(d, policy, model)
    pw0 = 15 + 10 * (0.8 / 2.4) ** 2
    assert r["n_changes"] == 0
    assert math.isclose(r["time_s"], n * 0.1, rel_tol=1e-13)
    assert math.isclose(r["energy_j"], n * 0.1 * pw0, rel_tol=1e-12)


# ----------------------------------------------------------------------------- Alg. 1
def step_trace(n, t0, lo, hi):
    d = np.full(n, lo, dtype=np.uint32)
    d[t0:] = hi
    return d


@pytest.mark.parametrize("W", [1, 2, 5, 8, 13])
def test_single_step_up(model, W):
    pol = dict(tracegen.default_policy(), direv_length=W)
    n, t0, lo, hi = 400, 100, 10_000_000, 200_000_000   # 6.4 -> 128 GB/s
    r = oracle.replay(step_trace(n, t0, lo, hi), pol, model, detail=True)
    # one +1 at round t0 -> top of the ladder from interval t0+1 on, nothing else
    assert r["n_changes"] == 1
    assert r["log_t"].tolist() == [t0 + 1] and r["log_level"].tolist() == [TOP]
    lv = r["level_log"]
    assert np.all(lv[:t0 + 1] == 0) and np.all(lv[t0 + 1:] == TOP)
    # the derivative is (hi - lo) x 64e-8 / W on exactly the W rounds t0 .. t0+W-1
    dv = r["deriv_log"]
    jump = (hi - lo) * 64 / 1e8 / W
    assert np.all(dv[t0:t0 + W] > 5.0) and np.all(dv[W:t0] == 0.0) and np.all(dv[t0 + W:] == 0.0)
    assert abs(dv[t0] - jump) < 1e-9
    # Alg. 2 with L = 10, threshold 0.6: W flags in a row reach hf iff W >= 6; the count
    # at round t is |[t0, t0+W-1] & [t-9, t]|
    n_hf = sum(1 for t in range(n) if len(set(range(t0, t0 + W)) & set(range(t - 9, t + 1))) >= 6)
    assert r["n_hf"] == n_hf
    E, T = exact_energy(step_trace(n, t0, lo, hi), [0] * (t0 + 1) + [TOP] * (n - t0 - 1), model)
    assert close(r["energy_j"], E) and close(r["time_s"], T)


def test_step_down_goes_directly_to_lower_bound(model, policy):
    # Sec. 6.1: decreases jump straight to the bottom of the ladder
    n = 600
    d = np.full(n, 10_000_000, dtype=np.uint32)
    d[100:300] = 250_000_000
    r = oracle.replay(d, policy, model, detail=True)
    assert r["log_t"].tolist() == [101, 301]
    assert r["log_level"].tolist() == [TOP, 0]
    lv = r["level_log"]
    assert set(np.unique(lv).tolist()) == {0, TOP}
    assert np.all(lv[101:301] == TOP) and np.all(lv[301:] == 0)


def test_strict_comparison_at_threshold(model, policy):
    # W = 5, inc = 5: delta 39,062,500 lines = exactly 25.0 GB/s, derivative exactly 5.0
    n, t0 = 50, 20
    for hi, expect in [(39_062_500, 0), (39_062_501, 1)]:
        d = step_trace(n, t0, 0, hi)
        r = oracle.replay(d, policy, model, detail=True)
        assert r["deriv_log"][t0] == (5.0 if expect == 0 else r["deriv_log"][t0])
        assert r["n_changes"] == expect
    # decrease side: reach the top with a large step, ramp down at -4 GB/s per interval
    # (never below dec = -5), hold, then drop to 0: derivative exactly -5.0 does not
    # trigger, one line more does
    for hi, expect in [(39_062_500, [TOP]), (39_062_501, [TOP, 0])]:
        ramp = list(range(250_000_000, hi, -6_250_000))
        d = np.array([0] * 10 + ramp + [hi] * 10 + [0] * 10, dtype=np.uint32)
        t_drop = 10 + len(ramp) + 10
        r = oracle.replay(d, policy, model, detail=True)
        assert r["deriv_log"][t_drop] == -(hi * 64 / 1e8) / 5
        assert r["log_level"].tolist() == expect
        assert r["log_t"].tolist()[0] == 11


# ----------------------------------------------------------------------------- Alg. 2
@pytest.mark.parametrize("W,hf_expected", [(5, False), (6, True), (7, True)])
def test_six_of_ten_is_high_frequency(model, W, hf_expected):
    # Sec. 3.2: threshold 0.6 on a 10-entry list ("more than six times per second" at
    # 10 rounds/s); Alg. 2 compares with >=, so six flagged rounds out of ten suffice.
    pol = dict(tracegen.default_policy(), direv_length=W)
    r = oracle.replay(step_trace(300, 100, 10_000_000, 200_000_000), pol, model)
    assert (r["n_hf"] > 0) == hf_expected
    if hf_expected:
        # hf holds on rounds where >= 6 of the last 10 flagged: t0+5 .. t0+W-1+4
        assert r["n_hf"] == (100 + W - 1 + 4) - (100 + 5) + 1


def test_square_wave_locks_at_max_and_releases(model, policy):
    # Sec. 6.3 behaviour (SRAD): rapid alternation -> locked at the top.  Period-2 wave,
    # W = 5, L = 10, k = 6, wave stops at even round ts.
    lo, hi, ts, n = 10_000_000, 200_000_000, 60, 200
    d = np.array([lo if t % 2 == 0 else hi for t in range(n)], dtype=np.uint32)
    d[ts:] = lo
    r = oracle.replay(d, policy, model, detail=True)
    # rounds 5..9 alternate +1/-1 before the list fills to 6 flags at round 10
    assert r["log_t"].tolist() == [6, 7, 8, 9, 10]
    assert r["log_level"].tolist() == [TOP, 0, TOP, 0, TOP]
    # after the wave stops, rounds ts, ts+2, ts+4 still flag (window reaches back into the
    # wave); the count falls to 6 at ts+6 and to 5 at ts+7, so hf covers rounds 10..ts+6
    assert r["n_hf"] == (ts + 6) - 10 + 1
    lv = r["level_log"]
    assert np.all(lv[10:] == TOP)
    levels = [0] * 6 + [TOP, 0, TOP, 0] + [TOP] * (n - 10)
    E, T = exact_energy(d, levels, model)
    assert close(r["energy_j"], E) and close(r["time_s"], T)


def test_flags_recorded_while_locked(model):
    # Sec. 3.2: predictions keep filling the tune list while the level is held at max.
    # A one-step ladder mode makes the difference visible: identical trace, the -1s seen
    # while locked are not executed.
    pol = dict(tracegen.default_policy(), direv_length=1, step_mode=0)
    d = np.array([10_000_000, 200_000_000] * 20 + [10_000_000] * 30, dtype=np.uint32)
    r = oracle.replay(d, pol, model, detail=True)
    # W = 1: every wave round flags; hf from round 6 (rounds 1..6 flagged) to the round
    # where the count drops below 6: the last flagged round is 40 (200M -> 10M), so the
    # count at round t >= 40 is 40 - (t - 9) + 1 = 50 - t, >= 6 up to t = 44
    assert r["n_hf"] == 44 - 6 + 1
    # round 40 predicts -1 while hf holds: no change until... never (pred 0 afterwards)
    assert r["log_level"].tolist()[-1] == TOP


def test_threshold_boundary_variants(model):
    # th <= 0: Alg. 2 is true even with an empty list -> top of the ladder after round 0
    pol = dict(tracegen.default_policy(), high_freq_threshold=0.0)
    r = oracle.replay(np.full(10, 5, dtype=np.uint32), pol, model)
    assert r["log_t"].tolist() == [1] and r["n_hf"] == 10
    # th > 1: never high-frequency
    pol = dict(tracegen.default_policy(), high_freq_threshold=1.5, direv_length=12)
    r = oracle.replay(step_trace(200, 50, 0, 300_000_000), pol, model)
    assert r["n_hf"] == 0 and r["n_changes"] == 1


def test_ladder_step_mode(model):
    pol = dict(tracegen.default_policy(), step_mode=1, high_freq_threshold=2.0)
    r = oracle.replay(step_trace(100, 20, 0, 250_000_000), pol, model)
    # W = 5 consecutive +1 rounds move five rungs, one per round
    assert r["log_level"].tolist() == [1, 2, 3, 4, 5]
    assert r["log_t"].tolist() == [21, 22, 23, 24, 25]


# ----------------------------------------------------------------------------- brute force
def naive_exact(deltas, W, L, inc, dec, th, model, pin=0, closed=False, ladder=False, top=None):
    """Second, naive restatement in exact rationals: the window is rebuilt from the raw
    trace every round, the comparisons are exact.  pin > 0: a static baseline that holds
    ladder index pin - 1 and runs no control (Sec. 5.3, Sec. 6.3).  closed: the monitor
    sees min(demand, capacity at the level in effect).  ladder: one rung per decision."""
    q = Fraction(model["dt_s"]) * 10**9
    bpc = model["bytes_per_count"]
    cap, _ = exact_model(model)
    xs = [Fraction(bpc * int(d)) / q for d in deltas]
    obs = []
    inc, dec, th = Fraction(inc), Fraction(dec), Fraction(th)
    level, preds, levels, log = (pin - 1 if pin else 0), [], [], []
    n_hf = 0
    top = len(model["f_ghz"]) - 1 if top is None else top
    for t in range(len(deltas)):
        levels.append(level)
        obs.append(min(xs[t], cap[level]) if closed else xs[t])
        if t >= W:
            der = (obs[t] - obs[t - W]) / W
            pred = 1 if der > inc else (-1 if der < dec else 0)
        else:
            pred = 0
        preds.append(pred)
        window = [1 if p != 0 else 0 for p in preds[max(0, t - L + 1):t + 1]]
        hf = Fraction(sum(window), L) >= th and not pin
        n_hf += hf
        up, dn = (min(level + 1, top), max(level - 1, 0)) if ladder else (top, 0)
        nxt = level if pin else (top if hf else (up if pred == 1 else (dn if pred == -1 else level)))
        if nxt != level:
            log.append((t + 1, nxt))
        level = nxt
    return levels, log, n_hf


def test_brute_force_tiny_traces(model):
    # alphabet chosen so that no derivative / W lands within 1e-9 of a threshold: the
    # FP64 oracle must then agree exactly with exact arithmetic on every decision
    alphabet = [0, 10_000_000, 30_000_000, 100_000_000]
    cases = 0
    for n in range(1, 7):
        for tr in itertools.product(alphabet, repeat=n):
            d = np.array(tr, dtype=np.uint32)
            for W, L, th in [(1, 2, 0.5), (2, 3, 0.6), (3, 4, 0.75), (1, 4, 0.3), (2, 2, 1.0)]:
                pol = dict(inc_threshold=5.0, dec_threshold=-3.3, direv_length=W, tune_window=L,
                           high_freq_threshold=th, step_mode=0)
                r = oracle.replay(d, pol, model, detail=True)
                levels, log, n_hf = naive_exact(tr, W, L, 5.0, -3.3, th, model)
                assert r["level_log"].tolist() == levels
                assert list(zip(r["log_t"].tolist(), r["log_level"].tolist())) == log
                assert r["n_hf"] == n_hf
                if n <= 3:
                    E, T = exact_energy(tr, levels, model)
                    assert close(r["energy_j"], E) and close(r["time_s"], T)
                cases += 1
    assert cases > 20000


def test_brute_force_ladder_open_loop(model):
    """One rung per decision in the open loop (step_mode 1) on every short trace, on the
    default 17-rung ladder and on a 3-rung ladder where runs of +1 / -1 reach both ends (the
    clamp at the top and at the bottom), against the exact-rational restatement."""
    alphabet = [0, 10_000_000, 30_000_000, 100_000_000]
    small = dict(model, f_ghz=[0.8, 1.6, 2.4], f_ref_ghz=2.4)
    cases = 0
    for mdl, max_n in ((model, 5), (small, 6)):
        for n in range(1, max_n + 1):
            for tr in itertools.product(alphabet, repeat=n):
                d = np.array(tr, dtype=np.uint32)
                for W, L, th in [(1, 2, 0.5), (2, 3, 0.6), (1, 4, 1.0), (3, 4, 0.75)]:
                    pol = dict(inc_threshold=5.0, dec_threshold=-3.3, direv_length=W, tune_window=L,
                               high_freq_threshold=th, step_mode=1)
                    r = oracle.replay(d, pol, mdl, detail=True)
                    levels, log, n_hf = naive_exact(tr, W, L, 5.0, -3.3, th, mdl, ladder=True)
                    assert r["level_log"].tolist() == levels
                    assert list(zip(r["log_t"].tolist(), r["log_level"].tolist())) == log
                    assert r["n_hf"] == n_hf
                    if n <= 3:
                        E, T = exact_energy(tr, levels, mdl)
                        assert close(r["energy_j"], E) and close(r["time_s"], T)
                    cases += 1
    assert cases > 20000
    # a rising ramp climbs one rung per round and stays at the top of the small ladder (a +1
    # there changes nothing); the oracle agrees with the hand-derived sequence
    ramp = [0, 100_000_000, 200_000_000, 300_000_000, 400_000_000]
    lv, lg, _ = naive_exact(ramp, 1, 2, 5.0, -3.3, 2.0, small, ladder=True)
    assert lv == [0, 0, 1, 2, 2] and lg == [(2, 1), (3, 2)]
    r = oracle.replay(np.array(ramp, dtype=np.uint32), dict(inc_threshold=5.0, dec_threshold=-3.3, direv_length=1,
                      tune_window=2, high_freq_threshold=2.0, step_mode=1), small, detail=True)
    assert r["level_log"].tolist() == lv and r["log_t"].tolist() == [2, 3] and r["log_level"].tolist() == [1, 2]


def test_brute_force_inverted_thresholds(model):
    """inc below dec: a derivative between them satisfies both comparisons of Alg. 1, which
    tests +1 first.  Exact-rational restatement on every trace of length <= 6."""
    alphabet = [0, 10_000_000, 30_000_000, 100_000_000]
    for n in range(1, 7):
        for tr in itertools.product(alphabet, repeat=n):
            d = np.array(tr, dtype=np.uint32)
            for W, L, th in [(1, 2, 1.5), (2, 3, 0.6), (3, 4, 1.0)]:
                pol = dict(inc_threshold=-1.0, dec_threshold=2.0, direv_length=W, tune_window=L,
                           high_freq_threshold=th, step_mode=0)
                r = oracle.replay(d, pol, model, detail=True)
                levels, log, n_hf = naive_exact(tr, W, L, -1.0, 2.0, th, model)
                assert r["level_log"].tolist() == levels
                assert list(zip(r["log_t"].tolist(), r["log_level"].tolist())) == log
                assert r["n_hf"] == n_hf


def test_brute_force_closed_loop(model):
    """Closed loop on every trace of length <= 6 over an alphabet whose larger demands
    exceed the bottom capacity (66.7 GB/s) but not the top one (200 GB/s), jump and
    ladder modes, against the exact-rational restatement."""
    alphabet = [0, 10_000_000, 150_000_000, 250_000_000]   # 0, 6.4, 96, 160 GB/s
    cases = 0
    for n in range(1, 7):
        for tr in itertools.product(alphabet, repeat=n):
            d = np.array(tr, dtype=np.uint32)
            for W, L, th, mode in [(1, 2, 0.5, 2), (2, 3, 0.6, 2), (3, 4, 0.75, 3), (1, 4, 1.0, 3)]:
                pol = dict(inc_threshold=5.0, dec_threshold=-3.3, direv_length=W, tune_window=L,
                           high_freq_threshold=th, step_mode=mode)
                r = oracle.replay(d, pol, model, detail=True)
                levels, log, n_hf = naive_exact(tr, W, L, 5.0, -3.3, th, model, closed=True,
                                                ladder=bool(mode & 1))
                assert r["level_log"].tolist() == levels
                assert list(zip(r["log_t"].tolist(), r["log_level"].tolist())) == log
                assert r["n_hf"] == n_hf
                if n <= 3:
                    E, T = exact_energy(tr, levels, model)
                    assert close(r["energy_j"], E) and close(r["time_s"], T)
                cases += 1
    assert cases > 10000


def test_closed_loop_equals_open_loop_below_capacity(model, policy):
    """When no demand exceeds the bottom capacity the uncore never throttles, so the
    closed and open loops see the same throughput and decide alike."""
    d = tracegen.single_trace().trace(0)
    capped = np.minimum(d, np.uint32(100_000_000))          # <= 64 GB/s < 66.7 GB/s
    a = oracle.replay(capped, policy, model)
    b = oracle.replay(capped, dict(policy, step_mode=2), model)
    assert a["n_changes"] > 0 and a["change_hash"] == b["change_hash"] and a["energy_j"] == b["energy_j"]
    # with demand above it, the closed loop decides differently on the generated trace
    c = oracle.replay(d, dict(policy, step_mode=2), model)
    o = oracle.replay(d, policy, model)
    assert c["change_hash"] != o["change_hash"]


def test_brute_force_static_baselines(model):
    """Pinned policies on every trace of length <= 4 over the alphabet: constant level,
    no log, no high-frequency rounds, exact energy of that level (Sec. 5.3, Sec. 6.3)."""
    alphabet = [0, 10_000_000, 30_000_000, 100_000_000]
    for n in range(1, 5):
        for tr in itertools.product(alphabet, repeat=n):
            d = np.array(tr, dtype=np.uint32)
            for pin, step_mode in [(1, 0), (K, 0), (9, 1), (2, 1)]:
                pol = dict(inc_threshold=5.0, dec_threshold=-3.3, direv_length=1, tune_window=2,
                           high_freq_threshold=0.5, step_mode=step_mode, pin_level=pin)
                r = oracle.replay(d, pol, model, detail=True)
                levels, log, n_hf = naive_exact(tr, 1, 2, 5.0, -3.3, 0.5, model, pin=pin)
                assert levels == [pin - 1] * n and log == [] and n_hf == 0
                assert r["level_log"].tolist() == levels
                assert r["n_changes"] == 0 and r["n_hf"] == 0
                E, T = exact_energy(tr, levels, model)
                assert close(r["energy_j"], E) and close(r["time_s"], T)


def test_static_max_closed_form_and_carried_level(model, policy):
    """Default setting of Sec. 5.3: uncore at the maximum for the whole run; it ignores a
    carried level and stays additive over split replays."""
    d = tracegen.single_trace().trace(0)
    pol = dict(policy, pin_level=K)
    x = 64.0 * d.astype(np.float64) / 1e8
    capM = 200 * 2.4 / 2.4
    pwM = 15 + 10 * (2.4 / 2.4) ** 2
    T = math.fsum(0.1 * np.maximum(1.0, x / capM))
    st = oracle.new_state()
    r = oracle.replay(d, pol, model, state=st)
    assert r["n_changes"] == 0 and r["n_hf"] == 0
    assert math.isclose(r["time_s"], T, rel_tol=1e-11)
    assert math.isclose(r["energy_j"], pwM * T, rel_tol=1e-11)
    # split at 7,000 with a state whose level was left at the bottom by a controlled run
    st2 = oracle.new_state()
    a = oracle.replay(d[:7000], policy, model, state=st2)
    b = oracle.replay(d[7000:], pol, model, state=st2)
    Tb = math.fsum(0.1 * np.maximum(1.0, x[7000:] / capM))
    assert math.isclose(b["time_s"], Tb, rel_tol=1e-11) and b["n_changes"] == 0
    assert a["n_changes"] > 0


def test_static_baselines_bracket_controlled_energy(model, policy):
    """Static minimum draws the least power but stretches the most; static maximum never
    stretches more than any other level (capacity grows with the level)."""
    d = tracegen.single_trace().trace(0)
    lo = oracle.replay(d, dict(policy, pin_level=1), model)
    hi = oracle.replay(d, dict(policy, pin_level=K), model)
    mg = oracle.replay(d, policy, model)
    assert hi["time_s"] <= mg["time_s"] <= lo["time_s"]
    pw0, pwM = 15 + 10 * (0.8 / 2.4) ** 2, 25.0
    assert lo["energy_j"] / lo["time_s"] == pytest.approx(pw0, rel=1e-12)
    assert hi["energy_j"] / hi["time_s"] == pytest.approx(pwM, rel=1e-12)


# ----------------------------------------------------------------------------- invariants
def test_split_replay_equals_whole(model, policy):
    ts = tracegen.single_trace()
    d = ts.trace(0)
    whole = oracle.replay(d, policy, model)
    for cut in [1, 3, 5, 6, 777, 10_000, 19_999]:
        st = oracle.new_state()
        a = oracle.replay(d[:cut], policy, model, state=st)
        b = oracle.replay(d[cut:], policy, model, state=st)
        assert np.array_equal(np.concatenate([a["log_t"], b["log_t"]]), whole["log_t"])
        assert np.array_equal(np.concatenate([a["log_level"], b["log_level"]]), whole["log_level"])
        assert a["n_hf"] + b["n_hf"] == whole["n_hf"]
        assert (a["change_hash"] + b["change_hash"]) % 2**64 == whole["change_hash"]
        assert math.isclose(a["energy_j"] + b["energy_j"], whole["energy_j"], rel_tol=1e-12)
        assert math.isclose(a["time_s"] + b["time_s"], whole["time_s"], rel_tol=1e-12)


def test_generated_trace_invariants(model, policy):
    ts = tracegen.single_trace()
    d = ts.trace(0)
    r = oracle.replay(d, policy, model, detail=True)
    n = len(d)
    assert set(np.unique(r["level_log"]).tolist()) <= {0, TOP}
    assert set(np.unique(r["log_level"]).tolist()) <= {0, TOP}
    pw0 = 15 + 10 * (0.8 / 2.4) ** 2
    assert r["time_s"] >= n * 0.1 * (1 - 1e-12)
    assert r["energy_j"] >= n * 0.1 * pw0 * (1 - 1e-12)
    # consecutive log entries alternate and their times increase
    assert np.all(np.diff(r["log_t"].astype(np.int64)) > 0)
    assert np.all(r["log_level"][1:] != r["log_level"][:-1])
    # the derivative log is Alg. 1's (x_t - x_{t-W}) / W with x = 64 delta / 1e8
    x = (64.0 * d.astype(np.float64)) / 1e8
    W = policy["direv_length"]
    assert np.array_equal(r["deriv_log"][W:], (x[W:] - x[:-W]) / float(W))
    # hash is the sum of SplitMix64 mixes of (t << 8 | level)
    h = sum(oracle.mix64((int(t) << 8) | int(lv)) for t, lv in zip(r["log_t"], r["log_level"])) % 2**64
    assert h == r["change_hash"]
    # exact energy of the level sequence
    E, T = exact_energy(d[:2000], r["level_log"][:2000].tolist(), model)
    r2 = oracle.replay(d[:2000], policy, model)
    assert close(r2["energy_j"], E, 1e-12) and close(r2["time_s"], T, 1e-12)


def test_static_policy_closed_form(model):
    pol = dict(inc_threshold=float("inf"), dec_threshold=float("-inf"), direv_length=3,
               tune_window=10, high_freq_threshold=2.0, step_mode=0)
    d = tracegen.single_trace().trace(0)
    r = oracle.replay(d, pol, model)
    assert r["n_changes"] == 0
    x = 64.0 * d.astype(np.float64) / 1e8
    cap0 = 200 * 0.8 / 2.4
    pw0 = 15 + 10 * (0.8 / 2.4) ** 2
    T = math.fsum(0.1 * np.maximum(1.0, x / cap0))
    assert math.isclose(r["time_s"], T, rel_tol=1e-11)
    assert math.isclose(r["energy_j"], pw0 * T, rel_tol=1e-11)


def test_mix64_published_vector():
    # SplitMix64 (Steele, Lea, Flood 2014): first output for seed 0 is 0xE220A8397B1DCDAF
    assert oracle.mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_batch_matches_single(model, policy):
    ts = tracegen.batched(6, 3000)
    pols = [policy, dict(policy, direv_length=2, inc_threshold=2.0, dec_threshold=-2.0)]
    out, used = oracle.replay_batch(ts.data, ts.offsets, ts.lengths, pols, model)
    assert used >= 1
    for i in range(6):
        for c, p in enumerate(pols):
            r = oracle.replay(ts.trace(i), p, model)
            k = i * 2 + c
            assert out["n_changes"][k] == r["n_changes"] and out["change_hash"][k] == r["change_hash"]
            assert out["energy_j"][k] == r["energy_j"]
