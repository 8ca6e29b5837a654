"""Host-side checks of the C ABI (no GPU needed): the library loads and exports every
symbol include/magus.h declares; host helpers (packed layout, decision bounds) are right."""
import ctypes
import os
import re

import numpy as np
import pytest

import tracegen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mg():
    from paper_2502_03796_b300 import build, magus
    build.build()
    return magus


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "magus.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(magus_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(mg):
    lib = ctypes.CDLL(mg.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding knows every one of them
    assert set(names) <= set(mg.SIGNATURES), set(names) - set(mg.SIGNATURES)


def test_version_and_error_strings(mg):
    assert b"sm_103a" in mg.lib().magus_version()
    with pytest.raises(mg.MagusError):
        mg.policy_bounds(dict(tracegen.default_policy(), direv_length=0), tracegen.default_model())
    assert b"direv_length" in mg.lib().magus_last_error()


def test_packed_layout(mg):
    off, tot = mg.packed_offsets([0, 1, 5, 8, 3])
    assert off.tolist() == [0, 0, 32, 64, 96] and tot == 128
    ts = tracegen.make_traces(np.array([3, 9, 1], dtype=np.uint64))
    off, tot = mg.packed_offsets(ts.lengths)
    assert np.array_equal(off, ts.offsets) and tot == len(ts.data)


def exact_decision(a, b, W, thr, model, up=True):
    """Algorithm 1 comparison evaluated in IEEE double (Python floats), as the oracle does."""
    q = model["dt_s"] * 1e9
    bpc = float(model["bytes_per_count"])
    d = ((bpc * a) / q - (bpc * b) / q) / float(W)
    return d > thr if up else d < thr


@pytest.mark.parametrize("model_kind", ["default", "odd"])
def test_decision_bounds_against_ieee_double(mg, model_kind):
    """Outside the band the integer rule must equal the FP64 rule for every base value."""
    model = tracegen.default_model()
    if model_kind == "odd":
        model = dict(model, dt_s=0.037, bytes_per_count=3)
    rng = np.random.default_rng(1)
    base = tracegen.default_policy()
    for pol in [base, dict(base, direv_length=7, inc_threshold=3.3, dec_threshold=-0.7),
                dict(base, direv_length=64, inc_threshold=1e-7, dec_threshold=-123.456),
                dict(base, direv_length=1, inc_threshold=-2.0, dec_threshold=-9.0)]:
        m_up, m_dn, kmin, band = (int(x) for x in mg.policy_bounds(pol, model))
        W = pol["direv_length"]
        for _ in range(300):
            b = int(rng.integers(0, 2**32 - 2**20))
            for m in range(m_up - band - 4, m_up + band + 6):
                a = b + m
                if not 0 <= a < 2**32:
                    continue
                ref = exact_decision(a, b, W, pol["inc_threshold"], model, up=True)
                if m > m_up + band:
                    assert ref, (pol, a, b)
                elif m <= m_up - band:
                    assert not ref, (pol, a, b)
            for m in range(m_dn - band - 6, m_dn + band + 4):
                a = b + m
                if not 0 <= a < 2**32:
                    continue
                ref = exact_decision(a, b, W, pol["dec_threshold"], model, up=False)
                if m < m_dn - band:
                    assert ref, (pol, a, b)
                elif m >= m_dn + band:
                    assert not ref, (pol, a, b)


def test_kmin_matches_algorithm_2(mg):
    model = tracegen.default_model()
    for L in (1, 2, 3, 10, 33, 64):
        for th in (-1.0, 0.0, 0.05, 0.3, 0.5, 0.6, 0.6000000001, 0.7, 1.0, 1.5):
            k = int(mg.policy_bounds(dict(tracegen.default_policy(), tune_window=L, high_freq_threshold=th),
                                     model)[2])
            ref = next((c for c in range(L + 1) if c / L >= th), L + 1)
            assert k == ref, (L, th)


def test_model_validation(mg):
    bad = dict(tracegen.default_model(), f_ghz=[1.0, 0.9])
    with pytest.raises(mg.MagusError):
        mg.policy_bounds(tracegen.default_policy(), bad)
    with pytest.raises(mg.MagusError):
        mg.policy_bounds(tracegen.default_policy(), dict(tracegen.default_model(), dt_s=0.0))


def test_policy_field_validation(mg):
    """Host-side checks of the mode fields (no device needed): step_mode 0..3, pin_level
    0..n_levels; the ABI struct keeps the C layout."""
    import ctypes
    assert ctypes.sizeof(mg.Policy) == 40
    assert mg.Policy.pin_level.offset == 36 and mg.Policy.step_mode.offset == 32
    model = tracegen.default_model()
    for ok in (dict(step_mode=3), dict(pin_level=17), dict(pin_level=1, step_mode=1)):
        mg.policy_bounds(dict(tracegen.default_policy(), **ok), model)
    for bad, word in ((dict(step_mode=4), b"step_mode"), (dict(step_mode=-1), b"step_mode"),
                      (dict(pin_level=18), b"pin_level"), (dict(pin_level=-1), b"pin_level")):
        with pytest.raises(mg.MagusError):
            mg.policy_bounds(dict(tracegen.default_policy(), **bad), model)
        assert word in mg.lib().magus_last_error()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp64_thresholds_reproduce_algorithm_1(mg, seed):
    """The literal kernel's division-free test of Algorithm 1: d > up_last exactly when
    RN(d / W) > inc, d <= dn_last exactly when RN(d / W) < dec -- checked with numpy's IEEE
    division on the thresholds' neighbours and on random differences."""
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    for _ in range(40):
        W = int(rng.integers(1, 65))
        inc = float(rng.choice([rng.uniform(-50, 50), np.inf, -np.inf, 0.0]))
        dec = float(rng.choice([rng.uniform(-50, 50), np.inf, -np.inf, 0.0]))
        pol = dict(tracegen.default_policy(), direv_length=W, inc_threshold=inc, dec_threshold=dec)
        up, dn = mg.policy_fp64_thresholds(pol, model)
        Wd = np.float64(W)
        probes = [up, dn] + rng.uniform(-200 * W, 200 * W, size=400).tolist()
        for t in (up, dn):
            if np.isfinite(t):
                probes += [np.nextafter(t, np.inf), np.nextafter(t, -np.inf)]
        for d in probes:
            d = np.float64(d)
            if not np.isfinite(d):
                continue
            assert (d / Wd > inc) == (d > up), (W, inc, d, up)
            assert (d / Wd < dec) == (d <= dn), (W, dec, d, dn)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_closed_thresholds_reproduce_algorithm_1(mg, seed):
    """The closed loop's integer tests: a throughput is capped (obs = C) exactly when its
    delta exceeds out[l], and with one throughput capped Algorithm 1's outcome is a
    threshold on the other delta -- checked against numpy's IEEE evaluation of
    x = bpc * delta / q, d = obs_t - obs_{t-W}, d / W > inc and d / W < dec on the
    thresholds' neighbours and on random deltas; both capped against the constant."""
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    bpc, q = np.float64(model["bytes_per_count"]), np.float64(model["dt_s"] * 1e9)
    caps = [np.float64(model["bw_ref_gbs"] * (f / model["f_ref_ghz"])) for f in (model["f_ghz"][0], model["f_ghz"][-1])]

    def x(v):
        return (bpc * np.float64(v)) / q

    for _ in range(30):
        W = int(rng.integers(1, 65))
        inc = float(rng.choice([rng.uniform(-50, 50), np.inf, -np.inf, 0.0]))
        dec = float(rng.choice([rng.uniform(-50, 50), np.inf, -np.inf, 0.0]))
        pol = dict(tracegen.default_policy(), direv_length=W, inc_threshold=inc, dec_threshold=dec, step_mode=2)
        t = mg.policy_closed_thresholds(pol, model)
        Wd = np.float64(W)
        up = lambda d: bool(d / Wd > inc)
        dn = lambda d: bool(d / Wd < dec)
        for l, C in enumerate(caps):
            c = int(t[l])
            assert x(c) <= C and (c == 2**32 - 1 or x(c + 1) > C)
            probes = rng.integers(0, 2**32, size=200).tolist()
            for k in (2, 4, 6, 8):
                v = int(t[k + l])
                probes += [v - 2, v - 1, v, v + 1]
            for v in probes:
                if not 0 <= v < 2**32:
                    continue
                assert up(C - x(v)) == (v < t[2 + l]), (pol, l, v)
                assert dn(C - x(v)) == (v >= t[4 + l]), (pol, l, v)
                assert up(x(v) - C) == (v >= t[6 + l]), (pol, l, v)
                assert dn(x(v) - C) == (v < t[8 + l]), (pol, l, v)
        for la in range(2):
            for lb in range(2):
                d = caps[la] - caps[lb]
                assert bool((int(t[10]) >> (2 * la + lb)) & 1) == up(d)
                assert bool((int(t[10]) >> (4 + 2 * la + lb)) & 1) == dn(d)
