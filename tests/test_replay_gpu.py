"""GPU parity: the CUDA replay path (through the C ABI) against the CPU oracle.

Decision logs, change counts, change hashes and high-frequency counts must match
bit-exactly; energy / time / EDP within 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import REL_TOL, assert_pair, oracle_pairs, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILES = [(8, 1), (4, 1), (4, 2), (2, 4), (1, 8), (1, 4), (2, 2)]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


@pytest.fixture(scope="module")
def rp(mg, ):
    r = mg.Replay(tracegen.default_model())
    yield r
    r.close()


def edge_policies():
    base = tracegen.default_policy()
    return [
        base,
        dict(base, direv_length=1, tune_window=1, high_freq_threshold=1.0),     # hf <=> flag
        dict(base, direv_length=64, tune_window=64, inc_threshold=0.5, dec_threshold=-0.5),
        dict(base, direv_length=2, inc_threshold=2.0, dec_threshold=-2.0, high_freq_threshold=0.4),
        dict(base, high_freq_threshold=0.0),                                     # always hf
        dict(base, high_freq_threshold=1.5, direv_length=12),                    # never hf
        dict(base, inc_threshold=float("inf"), dec_threshold=float("-inf")),     # static
        dict(base, direv_length=7, tune_window=33, inc_threshold=3.3, dec_threshold=-1.25,
             high_freq_threshold=0.3),
        dict(base, inc_threshold=-1.0, dec_threshold=-2.0),                      # negative inc
        dict(base, inc_threshold=-2.0, dec_threshold=3.0, direv_length=9),       # inc < dec: +1 first
        dict(base, pin_level=17),                                                # static maximum
        dict(base, direv_length=7, high_freq_threshold=0.0, pin_level=1),        # static minimum
    ]


RAGGED = [0, 1, 3, 4, 5, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 2047, 4097, 8191, 8192, 8193,
          16385, 20000, 24577, 33000]


def ragged_set(seed=3):
    return tracegen.make_traces(np.array(RAGGED, dtype=np.uint64), seed=seed, mean_phase=12.0)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_single_trace_detail_matches_oracle(rp, mode):
    """Per-interval levels and derivatives bit-exact: open / closed loop, jump / ladder."""
    ts = tracegen.single_trace()
    model, pol = tracegen.default_model(), dict(tracegen.default_policy(), step_mode=mode)
    d = to_device(ts)
    n = int(ts.lengths[0])
    out = rp.detail(d, n, pol, log_capacity=n)
    torch.cuda.synchronize()
    ref = oracle.replay(ts.trace(0), pol, model, detail=True)
    o = to_numpy(out)
    assert np.array_equal(o["level_log"][:n], ref["level_log"])
    assert np.array_equal(o["deriv_log"][:n].view(np.uint64), ref["deriv_log"].view(np.uint64))
    assert_pair(o, 0, ref, cap=n, tag="detail")


@pytest.mark.parametrize("tile", TILES)
def test_ragged_batch_all_tiles(rp, tile):
    ts = ragged_set()
    model = tracegen.default_model()
    pols = edge_policies()
    cap = 40_000
    rp.set_tile(*tile)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_tile(0, 0)
    assert rp.status() == 0
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"tile{tile}")


def grouped_policies():
    """Three Alg. 1 settings x four Alg. 2 settings: policy groups of 4 share predictions."""
    out = []
    for W, inc, dec in [(5, 5.0, -5.0), (3, 2.0, -1.5), (40, 0.4, -0.4)]:
        for L, th in [(10, 0.6), (1, 1.0), (64, 0.05), (7, 0.0)]:
            out.append(dict(inc_threshold=inc, dec_threshold=dec, direv_length=W, tune_window=L,
                            high_freq_threshold=th, step_mode=0))
    # interleave so that group members are not adjacent in the caller's order
    return out[::2] + out[1::2]


@pytest.mark.parametrize("tile", TILES)
def test_grouped_policies_all_tiles(rp, tile):
    ts = ragged_set(seed=8)
    model = tracegen.default_model()
    pols = grouped_policies()
    cap = 40_000
    rp.set_tile(*tile)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_tile(0, 0)
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"grouped tile{tile}")


@pytest.mark.parametrize("tile", [(4, 1), (8, 1)])
def test_window10_every_kmin(rp, tile):
    """A 10-round tune window with every flag-count threshold 0..11 (the bit-sliced Alg. 2
    path of one-member groups), on two predictor settings."""
    ts = ragged_set(seed=21)
    model = tracegen.default_model()
    pols = []
    for W, inc, dec in [(5, 5.0, -5.0), (2, 1.0, -1.0)]:
        for th in (0.0, 0.1, 0.15, 0.3, 0.4, 0.45, 0.6, 0.7, 0.8, 0.9, 1.0, 1.05):
            pols.append(dict(inc_threshold=inc, dec_threshold=dec, direv_length=W, tune_window=10,
                             high_freq_threshold=th, step_mode=0))
    cap = 40_000
    rp.set_tile(*tile)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_tile(0, 0)
    assert rp.status() == 0
    ref = oracle_pairs(ts, pols, model)
    assert len({r["n_hf"] for r in ref.values()}) > 12   # the thresholds make different detectors
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"window10 tile{tile}")


@pytest.mark.parametrize("kernel", ["tile", "segments", "ladder"])
@pytest.mark.parametrize("W", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 33, 64])
def test_window_instances(rp, W, kernel):
    """One policy group per call, so every group shares W: the tile, segment and one-rung
    kernels run their instance for that W where they have one (1-8, 10, 12, 16) and the any-W
    instance otherwise; two policies with different W in one call share none."""
    ts = ragged_set(seed=30 + W)
    model = tracegen.default_model()
    mode = 1 if kernel == "ladder" else 0
    pols = [dict(tracegen.default_policy(), direv_length=W, inc_threshold=0.5 * W, dec_threshold=-0.5 * W,
                 step_mode=mode)]
    if W == 64:
        pols.append(dict(tracegen.default_policy(), direv_length=5, step_mode=mode))
    cap = 40_000
    if kernel == "tile":
        rp.set_tile(4, 1)   # the 4-warp one-slot tile (the automatic one for one policy group)
    elif kernel == "segments":
        rp.set_segments(2048)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_tile(0, 0)
        rp.set_segments(-1)
    assert rp.status() == 0
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"W={W} {kernel}")


@pytest.mark.parametrize("kernel", ["tile", "segments", "ladder"])
@pytest.mark.parametrize("W", [1, 3, 5, 8, 16])
def test_fast_limit_in_window_before_sub_block(rp, W, kernel):
    """A delta at or above 2^30 among the W rounds just before a 1,024-round sub-block (the
    row before it, whose deltas the sub-block's first row reads as the values W rounds
    earlier) must send that sub-block to the exact path: placed before sub-block and chunk
    starts, one placement per trace, against the oracle."""
    n = 12 * 1024 + 77
    cases = [(k, j, v) for k in (1, 2, 3, 4, 5, 8, 9) for j in sorted({1, (W + 1) // 2, W})
             for v in (2**30, 2**31 + 7, 2**32 - 5)]
    ts = tracegen.make_traces(np.full(len(cases), n, dtype=np.uint64), seed=70 + W, mean_phase=20.0)
    data = np.array(ts.data, copy=True)
    for i, (k, j, v) in enumerate(cases):
        data[int(ts.offsets[i]) + 1024 * k - j] = v
    ts = tracegen.TraceSet(lengths=ts.lengths, offsets=ts.offsets, data=data)
    model = tracegen.default_model()
    mode = 1 if kernel == "ladder" else 0
    pols = [dict(tracegen.default_policy(), direv_length=W, inc_threshold=0.5 * W, dec_threshold=-0.5 * W,
                 step_mode=mode)]
    cap = 20_000
    if kernel == "tile":
        rp.set_tile(4, 1)
    elif kernel == "segments":
        rp.set_segments(2048)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_tile(0, 0)
        rp.set_segments(-1)
    assert rp.status() == 0
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"W={W} {kernel} case {cases[p]}")


def test_autotune_picks_a_tile(rp):
    ts = tracegen.sweep(n_traces=8, n=30_000, seed=2)
    pols = tracegen.sweep_policies()[:32]
    (tg, cw, gp, seg), ms = rp.autotune(to_device(ts), ts.lengths, pols)
    assert ((tg * cw == 8) or (tg, cw) in ((4, 1), (1, 4), (2, 2))) and gp in (1, 4) and seg in (0, 8192, 16384, 32768) and ms > 0
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols))
    ref, _ = oracle.replay_batch(ts.data, ts.offsets, ts.lengths, pols, tracegen.default_model())
    assert np.array_equal(out["change_hash"], ref["change_hash"].astype(np.uint64))
    np.testing.assert_allclose(out["energy_j"], ref["energy_j"], rtol=REL_TOL)


def test_plain_kernel_matches_oracle(rp):
    ts = tracegen.make_traces(np.array([0, 1, 7, 100, 5000, 20000], dtype=np.uint64), seed=11)
    pols = edge_policies() + [dict(tracegen.default_policy(), step_mode=1, high_freq_threshold=0.9),
                              dict(tracegen.default_policy(), step_mode=1, pin_level=9),   # mid-ladder pin
                              dict(tracegen.default_policy(), step_mode=2),                # closed loop
                              dict(tracegen.default_policy(), step_mode=3, high_freq_threshold=0.9,
                                   direv_length=3)]                                        # closed, ladder
    cap = 20_000
    out = to_numpy(rp.plain(to_device(ts), ts.lengths, pols, log_capacity=cap))
    ref = oracle_pairs(ts, pols, tracegen.default_model())
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag="plain")


def band_trace(W, ms, bases):
    """Blocks [b]*W + [b+m]*W: rounds in the second block see delta_t - delta_{t-W} = m, the
    next block's rounds see -m."""
    parts = []
    for b in bases:
        for m in ms:
            a = b + m
            if 0 <= a <= 0xFFFFFFFF and 0 <= b <= 0xFFFFFFFF:
                parts += [b] * W + [a] * W
    return np.array(parts, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("model_kind", ["default", "odd"])
def test_decision_band_exhaustive(rp, mg, model_kind):
    """Every integer difference within 8 of each decision crossover, at small, large and
    > 2^31 base values: exact FP64 agreement of Alg. 1 on both sides."""
    model = tracegen.default_model()
    if model_kind == "odd":
        model = dict(model, dt_s=0.037, bytes_per_count=3)
    handle = rp if model_kind == "default" else mg.Replay(model)
    base = tracegen.default_policy()
    pols = [dict(base, direv_length=5), dict(base, direv_length=7, inc_threshold=3.3, dec_threshold=-0.7),
            dict(base, direv_length=3, inc_threshold=1e-7, dec_threshold=-2.5e-3)]
    bases = [0, 7, 1_000_000, 123_456_789, 2**31 - 50, 2**31 + 3, 2**32 - 2**20]
    traces, lengths = [], []
    for pol in pols:
        b = mg.policy_bounds(pol, model)
        ms = sorted(set(int(x) for c in (b[0], b[1]) for x in range(c - 8, c + 9)))
        for flagpol in (dict(pol, tune_window=1, high_freq_threshold=1.0),
                        dict(pol, tune_window=1, high_freq_threshold=2.0)):
            tr = band_trace(pol["direv_length"], ms, bases)
            traces.append((tr, flagpol))
    for tr, pol in traces:
        ts = tracegen.single_trace_set(tr)
        out = to_numpy(handle.run(to_device(ts), ts.lengths, [pol], log_capacity=len(tr)))
        ref = oracle.replay(tr, pol, model)
        assert_pair(out, 0, ref, cap=len(tr), tag=f"band {pol}")
    if handle is not rp:
        handle.close()


@pytest.mark.parametrize("seg", [0, 1024, 16384])
@pytest.mark.parametrize("grouped", [False, True])
def test_split_replay_with_state(rp, mg, grouped, seg):
    """Feeding a trace in pieces with carried state reproduces the whole-trace log and
    additive energies (against the oracle's whole-trace replay); tile kernel (seg 0) and
    segment kernel."""
    rp.set_segments(seg)
    try:
        _split_replay(rp, mg, grouped)
    finally:
        rp.set_segments(-1)


def _split_replay(rp, mg, grouped):
    model = tracegen.default_model()
    ts_all = tracegen.make_traces(np.array([30_000], dtype=np.uint64), seed=5, mean_phase=9.0)
    full = ts_all.trace(0)
    pols = [tracegen.default_policy(), dict(tracegen.default_policy(), direv_length=40, tune_window=50,
                                            high_freq_threshold=0.1),
            dict(tracegen.default_policy(), pin_level=17)]
    if grouped:
        pols = grouped_policies()
    cuts = [0, 3, 4, 37, 64, 65, 1100, 8192, 8200, 20000, 30_000]
    state = torch.zeros(len(pols) * mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    E = np.zeros(len(pols))
    T = np.zeros(len(pols))
    logs = [[] for _ in pols]
    nhf = np.zeros(len(pols), dtype=np.int64)
    hsh = [0] * len(pols)
    for a, b in zip(cuts[:-1], cuts[1:]):
        piece = full[a:b]
        ts = tracegen.single_trace_set(piece)
        cap = max(len(piece), 1)
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap, state=state))
        for c in range(len(pols)):
            E[c] += out["energy_j"][c]
            T[c] += out["time_s"][c]
            nhf[c] += int(out["n_hf"][c])
            hsh[c] = (hsh[c] + int(out["change_hash"][c])) % 2**64
            k = int(out["n_changes"][c])
            logs[c].append(out["log"][c * cap:c * cap + k])
    assert rp.status() == 0
    for c, pol in enumerate(pols):
        ref = oracle.replay(full, pol, model)
        ent = np.concatenate(logs[c]).astype(np.uint32)
        assert np.array_equal((ent >> 5).astype(np.uint64), ref["log_t"])
        assert np.array_equal((ent & 31).astype(np.uint8), ref["log_level"])
        assert nhf[c] == ref["n_hf"] and hsh[c] == ref["change_hash"]
        assert abs(E[c] - ref["energy_j"]) <= REL_TOL * ref["energy_j"]
        assert abs(T[c] - ref["time_s"]) <= REL_TOL * ref["time_s"]
    st = state.cpu().numpy().view(np.uint64)
    assert int(st[0]) == 30_000


SEGS = [1024, 2048, 16384]


@pytest.mark.parametrize("seg", SEGS)
def test_ragged_batch_segments(rp, seg):
    """Segment kernel: ragged lengths across segment and sub-block borders, edge policies."""
    ts = ragged_set()
    model = tracegen.default_model()
    pols = edge_policies()
    cap = 40_000
    rp.set_segments(seg)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_segments(-1)
    assert rp.status() == 0
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"seg{seg}")


@pytest.mark.parametrize("seg", [1024, 8192])
def test_grouped_policies_segments(rp, seg):
    ts = ragged_set(seed=8)
    model = tracegen.default_model()
    pols = grouped_policies()
    cap = 40_000
    rp.set_segments(seg)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_segments(-1)
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"grouped seg{seg}")


@pytest.mark.parametrize("seg", [0, 1024])
def test_short_log_capacity(rp, seg):
    """A log shorter than the pair's changes keeps the first entries; counts, hash and
    energy still cover every change."""
    ts = tracegen.make_traces(np.array([5000, 12000, 3], dtype=np.uint64), seed=21, mean_phase=3.0)
    model = tracegen.default_model()
    pols = edge_policies()[:4]
    cap = 37
    rp.set_segments(seg)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
    finally:
        rp.set_segments(-1)
    ref = oracle_pairs(ts, pols, model)
    assert max(r["n_changes"] for r in ref.values()) > cap
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"short log seg{seg}")


@pytest.mark.parametrize("extra", [0, 5, -1000])
def test_dense_changes_segment_log(rp, mg, extra):
    """A change at every round (square wave, no high-frequency state): a segment's log
    entries are compacted right behind all earlier ones.  The second piece starts with a
    change (carried state), so each segment's entries move one slot to the right of where the
    segment kernel wrote them in the caller's log (extra >= 0: the log holds the trace);
    extra < 0 takes the scratch path."""
    model = tracegen.default_model()
    pol = dict(tracegen.default_policy(), high_freq_threshold=1.5)
    n, cut = 6000, 3001
    full = np.array([10_000_000 if t % 2 == 0 else 200_000_000 for t in range(n)], dtype=np.uint32)
    ref = oracle.replay(full, pol, model)
    assert ref["n_changes"] == n - 5
    state = torch.zeros(mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    rp.set_segments(1024)
    logs, E = [], 0.0
    try:
        for a, b in ((0, cut), (cut, n)):
            ts = tracegen.single_trace_set(full[a:b])
            cap = (b - a) + extra
            out = to_numpy(rp.run(to_device(ts), ts.lengths, [pol], log_capacity=cap, state=state))
            k = int(out["n_changes"][0])
            assert k == min(b, n) - max(a, 5)
            logs.append(out["log"][:min(k, cap)])
            E += out["energy_j"][0]
    finally:
        rp.set_segments(-1)
    assert rp.status() == 0
    ent = np.concatenate(logs).astype(np.uint32)
    t = (ent >> 5).astype(np.uint64)
    if extra >= 0:
        assert np.array_equal(t, ref["log_t"])
        assert np.array_equal((ent & 31).astype(np.uint8), ref["log_level"])
    else:
        k0 = cut - 5
        assert np.array_equal(t[:len(logs[0])], ref["log_t"][:len(logs[0])])
        assert np.array_equal(t[len(logs[0]):], ref["log_t"][k0:k0 + len(logs[1])])
    assert abs(E - ref["energy_j"]) <= REL_TOL * ref["energy_j"]


def literal_policies():
    """Policies outside the time-parallel kernels' scope, replayed in the same call by the
    literal kernel: one rung per decision, closed loop, a pin inside the ladder."""
    base = tracegen.default_policy()
    return [dict(base, step_mode=1, high_freq_threshold=0.9), dict(base, step_mode=2),
            dict(base, step_mode=3, direv_length=3, high_freq_threshold=0.8), dict(base, pin_level=9),
            dict(base, step_mode=1, pin_level=4)]


@pytest.mark.parametrize("seg", [0, 1024])
def test_mixed_modes_one_call(rp, seg):
    """Jump-mode policies (tile or segment kernel) and literal-path policies in one call:
    every pair against the oracle."""
    ts = tracegen.make_traces(np.array([0, 1, 33, 1025, 5000, 20000], dtype=np.uint64), seed=13, mean_phase=20.0)
    model = tracegen.default_model()
    pols = [p for pair in zip(edge_policies()[:5], literal_policies()) for p in pair]
    cap = 20_000
    rp.set_segments(seg)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
        tot, main, runs, kernels = rp.kernel_time(detail=True)
    finally:
        rp.set_segments(-1)
    assert rp.status() == 0 and kernels >= 2
    ref = oracle_pairs(ts, pols, model)
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag=f"mixed seg{seg}")


def ladder_policies():
    base = dict(tracegen.default_policy(), step_mode=1)
    return [base,
            dict(base, high_freq_threshold=1.5),                                   # never hf: pure walk
            dict(base, direv_length=1, tune_window=1, high_freq_threshold=1.0),    # hf <=> flag
            dict(base, direv_length=2, inc_threshold=2.0, dec_threshold=-2.0, high_freq_threshold=0.9),
            dict(base, direv_length=64, tune_window=64, inc_threshold=0.5, dec_threshold=-0.5),
            dict(base, inc_threshold=-1.0, dec_threshold=-2.0, high_freq_threshold=0.95)]


@pytest.mark.parametrize("n_levels", [2, 17, 32])
def test_ladder_kernel_matches_oracle(mg, n_levels):
    """One rung per decision on the time-parallel ladder kernel: ragged lengths, ladders of
    2, 17 and 32 rungs (2 rungs: the jump mode's outcome), full and short logs."""
    model = dict(tracegen.default_model(), f_ghz=[0.8 + 1.6 * k / (n_levels - 1) for k in range(n_levels)])
    ts = ragged_set(seed=17)
    pols = ladder_policies()
    h = mg.Replay(model)
    try:
        for cap in (40_000, 9):
            out = to_numpy(h.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
            assert h.status() == 0
            ref = oracle_pairs(ts, pols, model)
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"ladder K={n_levels} cap={cap}")
        tot, main, runs, kernels = h.kernel_time(detail=True)
        assert runs == 2 and kernels == 2
    finally:
        h.close()


@pytest.mark.parametrize("ladder", ["two", "thirty-two", "close rungs", "saturating", "never stretched"])
def test_static_kernel_ladders(mg, ladder):
    """The static kernel's rung lookup on ladders of 2 and 32 rungs, two rungs 1e-7 GHz
    apart (their thresholds share every cell the lookup table could use: the binary-search
    variant), capacities whose upper thresholds exceed the 32-bit counter range (never
    stretched there) and a ladder where no delta is ever stretched: every rung pinned, ragged
    lengths (the longest trace split over four CTAs), against the oracle; one static-kernel
    launch."""
    f17 = tracegen.default_model()["f_ghz"]
    models = {
        "two": dict(tracegen.default_model(), f_ghz=[0.8, 2.4]),
        "thirty-two": dict(tracegen.default_model(), f_ghz=[0.8 + 1.6 * k / 31 for k in range(32)]),
        "close rungs": dict(tracegen.default_model(), f_ghz=[0.8, 0.8000001] + f17[1:]),
        "saturating": dict(tracegen.default_model(), bw_ref_gbs=4000.0),
        "never stretched": dict(tracegen.default_model(), bw_ref_gbs=1e6),
    }
    model = models[ladder]
    K = len(model["f_ghz"])
    ts = tracegen.make_traces(np.array([0, 1, 33, 2047, 2048, 2049, 30_001, 100_003], dtype=np.uint64), seed=23,
                              mean_phase=30.0)
    if ladder == "saturating":
        ts.data[:] = np.minimum(ts.data.astype(np.uint64) * 16, 0xFFFFFFFF).astype(ts.data.dtype)
    base = tracegen.default_policy()
    pols = [dict(base, pin_level=k) for k in range(1, K + 1)] + [dict(base, step_mode=3, pin_level=K // 2 + 1)]
    ref = oracle_pairs(ts, pols, model)
    h = mg.Replay(model)
    try:
        h.kernel_time()
        out = to_numpy(h.run(to_device(ts), ts.lengths, pols, log_capacity=8))
        tot, main, runs, kernels = h.kernel_time(detail=True)
        assert h.status() == 0
        for p, r in ref.items():
            assert_pair(out, p, r, cap=8, tag=f"static, {ladder}")
        assert runs == 1 and kernels == 1
    finally:
        h.close()


@pytest.mark.parametrize("seg", [0, 2048])
def test_controlled_policies_beside_pins(rp, seg):
    """Controlled jump-mode policies next to pins at the bounds and inside the ladder, on the
    tile kernel (seg 0) and on the segment kernel (seg 2048: its plan carries the static
    kernel's items too): the bound pins join the static kernel once an inner pin makes it
    run; every pair against the oracle, ragged lengths, with logs."""
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    ts = tracegen.make_traces(np.array([0, 5, 2048, 9_001, 70_003], dtype=np.uint64), seed=37, mean_phase=20.0)
    base = tracegen.default_policy()
    pols = [base, dict(base, pin_level=1), dict(base, inc_threshold=3.0, dec_threshold=-3.0),
            dict(base, pin_level=7), dict(base, pin_level=K)]
    ref = oracle_pairs(ts, pols, model)
    rp.set_segments(seg)
    try:
        rp.kernel_time()
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=300))
        tot, main, runs, kernels = rp.kernel_time(detail=True)
    finally:
        rp.set_segments(-1)
    assert rp.status() == 0
    for p, r in ref.items():
        assert_pair(out, p, r, cap=300, tag=f"pins beside controlled, seg {seg}")
    # tile kernel + static kernel, or segment kernel + combine + static kernel
    assert runs == 1 and kernels == (2 if seg == 0 else 3)


def test_static_kernel_long_traces_in_many_parts(mg):
    """A few long traces (1.5M and 0.9M intervals and a short one): the static kernel splits
    each long trace into tens of CTAs whose per-rung totals meet in the trace's accumulators;
    the last part to arrive charges the rungs.  Pins at the bottom, middle and top rung in
    jump mode (the bound pins join the static kernel), against the oracle, twice in a row (the
    accumulators start from zero every call)."""
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    ts = tracegen.make_traces(np.array([1_500_001, 900_000, 4_097], dtype=np.uint64), seed=29, mean_phase=40.0)
    base = tracegen.default_policy()
    pols = [dict(base, pin_level=k) for k in (1, 9, K)]
    ref = oracle_pairs(ts, pols, model, log=False)
    h = mg.Replay(model)
    try:
        for rep in range(2):
            h.kernel_time()
            out = to_numpy(h.run(to_device(ts), ts.lengths, pols, log_capacity=0))
            tot, main, runs, kernels = h.kernel_time(detail=True)
            assert h.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=0, check_log=False, tag=f"static long, call {rep}")
            assert runs == 1 and kernels == 1
    finally:
        h.close()


def test_literal_split_replay_with_state(rp, mg):
    """Ladder mode and an inner pin carry their state across calls (open loop); a closed
    loop can only start from a fresh state (EINVAL otherwise)."""
    model = tracegen.default_model()
    full = tracegen.make_traces(np.array([12_000], dtype=np.uint64), seed=6, mean_phase=9.0).trace(0)
    base = tracegen.default_policy()
    pols = [dict(base, step_mode=1, high_freq_threshold=0.9), dict(base, pin_level=9), base]
    state = torch.zeros(len(pols) * mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    E = np.zeros(len(pols))
    logs = [[] for _ in pols]
    for a, b in zip([0, 5, 70, 4000], [5, 70, 4000, 12_000]):
        ts = tracegen.single_trace_set(full[a:b])
        cap = b - a
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap, state=state))
        for c in range(len(pols)):
            E[c] += out["energy_j"][c]
            logs[c].append(out["log"][c * cap:c * cap + int(out["n_changes"][c])])
    assert rp.status() == 0
    for c, pol in enumerate(pols):
        ref = oracle.replay(full, pol, model)
        ent = np.concatenate(logs[c]).astype(np.uint32)
        assert np.array_equal((ent >> 5).astype(np.uint64), ref["log_t"])
        assert np.array_equal((ent & 31).astype(np.uint8), ref["log_level"])
        assert abs(E[c] - ref["energy_j"]) <= REL_TOL * ref["energy_j"]
    ts = tracegen.single_trace_set(full[:100])
    rp.run(to_device(ts), ts.lengths, [dict(base, step_mode=2)] * 3, state=state)
    assert rp.status() == mg.EINVAL


def test_invalid_carried_level_reports_einval(rp, mg):
    ts = tracegen.make_traces(np.array([100], dtype=np.uint64), seed=1)
    state = torch.zeros(mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    state.view(torch.int32)[4] = 3   # level field (offset 16): neither 0 nor K-1
    rp.run(to_device(ts), ts.lengths, [tracegen.default_policy()], state=state)
    assert rp.status() == mg.EINVAL
    assert rp.status() == 0


def test_argument_errors(rp, mg):
    ts = tracegen.make_traces(np.array([100], dtype=np.uint64), seed=1)
    d = to_device(ts)
    with pytest.raises(mg.MagusError) as e:
        rp.run(d, ts.lengths, [dict(tracegen.default_policy(), direv_length=65)])
    assert e.value.code == mg.EINVAL
    with pytest.raises(mg.MagusError):
        rp.run(d, ts.lengths, [dict(tracegen.default_policy(), step_mode=4)])
    with pytest.raises(mg.MagusError):
        rp.run(d[1:], ts.lengths, [tracegen.default_policy()])   # misaligned base
    with pytest.raises(mg.MagusError):
        rp.run(d, ts.lengths, [dict(tracegen.default_policy(), inc_threshold=float("nan"))])
    for bad in (-2, 1000, 1025, 1 << 25):
        with pytest.raises(mg.MagusError):
            rp.set_segments(bad)
    for pin in (-1, 18):
        with pytest.raises(mg.MagusError):
            rp.run(d, ts.lengths, [dict(tracegen.default_policy(), pin_level=pin)])


def test_empty_inputs(rp):
    ts = tracegen.make_traces(np.array([0, 0], dtype=np.uint64), seed=1)
    out = to_numpy(rp.run(to_device(ts) if ts.data.size else torch.zeros(4, dtype=torch.int32, device="cuda"),
                          ts.lengths, [tracegen.default_policy()]))
    assert np.all(out["energy_j"] == 0) and np.all(out["n_changes"] == 0)
    out = rp.run(torch.zeros(4, dtype=torch.int32, device="cuda"), np.zeros(0, dtype=np.uint64),
                 [tracegen.default_policy()])
    assert out["energy_j"].numel() == 0


def same_outputs(host, dev, cap):
    """run_host against run: every output, the log up to each pair's change count (slots
    past it are unspecified)."""
    for k in ("energy_j", "edp_js", "time_s", "n_changes", "change_hash", "n_hf"):
        assert np.array_equal(np.asarray(host[k]).view(dev[k].dtype), dev[k]), k
    hl = np.asarray(host["log"]).view(np.uint32)
    for p, k in enumerate(dev["n_changes"]):
        k = min(int(k), cap)
        assert np.array_equal(hl[p * cap:p * cap + k], dev["log"][p * cap:p * cap + k]), ("log", p)


def test_run_host_matches_device(rp):
    ts = tracegen.batched(64, 10_000, seed=2)
    pols = tracegen.sweep_policies()[:5]
    dev = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=2000))
    host = rp.run_host(ts.data, ts.lengths, pols, log_capacity=2000)
    same_outputs(host, dev, 2000)


def test_run_host_mixed_modes(rp):
    """Host-buffer replay routes every mode the same way as the device call."""
    ts = tracegen.batched(24, 9_000, seed=5)
    pols = [tracegen.default_policy()] + literal_policies()
    dev = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=3000))
    host = rp.run_host(ts.data, ts.lengths, pols, log_capacity=3000)
    same_outputs(host, dev, 3000)


def test_segment_buffers_over_budget_fall_back_to_tiles(mg):
    """Asked for the segment kernel with a log scratch larger than the handle's budget, the
    call runs the tile kernel instead (one kernel per replay) with the same results."""
    model = tracegen.default_model()
    ts = tracegen.batched(64, 60_000, seed=9)
    pols = [tracegen.default_policy()]
    cap = 20_000                            # < n: scratch of 4 segments x 16,384 x 4 B per pair
    small = mg.Replay(model, mem_budget=8 << 20)
    try:
        small.set_segments(16384)
        out = to_numpy(small.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
        tot, main, runs, kernels = small.kernel_time(detail=True)
        assert small.status() == 0 and runs == 1 and kernels == 1
    finally:
        small.close()
    ref = oracle_pairs(ts, pols, model, pairs=range(0, 64, 7))
    for p, r in ref.items():
        assert_pair(out, p, r, cap=cap, tag="budget fallback")


def test_sweep_grid_scaled(rp):
    ts = tracegen.sweep(n_traces=6, n=40_000, seed=0)
    pols = tracegen.sweep_policies()
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=16_000))
    ref, _ = oracle.replay_batch(ts.data, ts.offsets, ts.lengths, pols, tracegen.default_model())
    assert np.array_equal(out["n_changes"], ref["n_changes"].astype(np.uint64))
    assert np.array_equal(out["change_hash"], ref["change_hash"].astype(np.uint64))
    assert np.array_equal(out["n_hf"], ref["n_hf"].astype(np.uint64))
    np.testing.assert_allclose(out["energy_j"], ref["energy_j"], rtol=REL_TOL)
    np.testing.assert_allclose(out["edp_js"], ref["edp_js"], rtol=REL_TOL)
    sample = oracle_pairs(ts, pols, tracegen.default_model(), pairs=range(0, 6 * 256, 37))
    for p, r in sample.items():
        assert_pair(out, p, r, cap=16_000)


def test_uneven_lengths_scaled(rp):
    ts = tracegen.uneven(n_traces=96, lo=1e2, hi=6e4, seed=4)
    pols = tracegen.sweep_policies()[:16]
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols))
    ref, _ = oracle.replay_batch(ts.data, ts.offsets, ts.lengths, pols, tracegen.default_model())
    assert np.array_equal(out["n_changes"], ref["n_changes"].astype(np.uint64))
    assert np.array_equal(out["change_hash"], ref["change_hash"].astype(np.uint64))
    assert np.array_equal(out["n_hf"], ref["n_hf"].astype(np.uint64))
    np.testing.assert_allclose(out["energy_j"], ref["energy_j"], rtol=REL_TOL)


def test_full_size_batched_workload(rp):
    """4,096 traces x 100,000 intervals, one policy, the launch the benchmark times: every
    pair's counts / hash / energy against the oracle, full logs of sampled pairs."""
    ts = tracegen.batched()
    pol = [tracegen.default_policy()]
    cap = 8192
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pol, log_capacity=cap))
    ref, _ = oracle.replay_batch(ts.data, ts.offsets, ts.lengths, pol, tracegen.default_model())
    assert np.array_equal(out["n_changes"], ref["n_changes"].astype(np.uint64))
    assert np.array_equal(out["change_hash"], ref["change_hash"].astype(np.uint64))
    assert np.array_equal(out["n_hf"], ref["n_hf"].astype(np.uint64))
    np.testing.assert_allclose(out["energy_j"], ref["energy_j"], rtol=REL_TOL)
    np.testing.assert_allclose(out["time_s"], ref["time_s"], rtol=REL_TOL)
    for p, r in oracle_pairs(ts, pol, tracegen.default_model(), pairs=[0, 1, 777, 2048, 4095]).items():
        assert_pair(out, p, r, cap=cap)


def _sampled_pairs(n_pairs, k, seed):
    return sorted(int(x) for x in np.random.default_rng(seed).choice(n_pairs, k, replace=False))


def _any_size_properties(out, ts, n_pols, dt):
    """Bounds that hold for every pair at any size: a round lasts at least dt, changes and
    high-frequency rounds are at most one per round, energy and EDP are positive."""
    n = np.repeat(ts.lengths.astype(np.float64), n_pols)
    assert np.all(out["time_s"] >= n * dt * (1 - 1e-12))
    assert np.all(out["n_changes"] <= n.astype(np.uint64))
    assert np.all(out["n_hf"] <= n.astype(np.uint64))
    assert np.all(out["energy_j"][n > 0] > 0) and np.all(out["edp_js"][n > 0] > 0)


def test_full_size_sweep_sampled(rp):
    """The policy sweep at full size (1,024 traces x 200,000 intervals x 256 policies, the
    automatic tile, as the benchmark times it): 48 sampled pairs against the oracle, and the
    any-size bounds on every pair."""
    ts = tracegen.sweep()
    pols = tracegen.sweep_policies()
    model = tracegen.default_model()
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=0))
    assert rp.status() == 0
    _any_size_properties(out, ts, len(pols), model["dt_s"])
    pairs = _sampled_pairs(ts.n_traces * len(pols), 48, seed=5)
    for p, r in oracle_pairs(ts, pols, model, pairs=pairs, log=False).items():
        assert_pair(out, p, r, cap=0, tag="full-size sweep")


def test_full_size_uneven_sampled(rp):
    """The uneven-length workload at full size (16,384 traces, 1e3 .. 1e6 intervals, 16
    policies, 2.35e9 intervals): 32 sampled pairs against the oracle, and the any-size bounds
    on every pair."""
    ts = tracegen.uneven(n_traces=16_384, seed=0)
    pols = tracegen.sweep_policies()[:16]
    model = tracegen.default_model()
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=0))
    assert rp.status() == 0
    _any_size_properties(out, ts, len(pols), model["dt_s"])
    pairs = _sampled_pairs(ts.n_traces * len(pols), 32, seed=6)
    for p, r in oracle_pairs(ts, pols, model, pairs=pairs, log=False).items():
        assert_pair(out, p, r, cap=0, tag="full-size uneven")


def test_full_size_static_workload(rp):
    """4,096 traces x 100,000 intervals pinned at each of the 17 rungs, the call
    `bench.py --workload static` times (one static-kernel launch, every trace in parts):
    the pairs of four traces against the oracle; for every trace, time does not grow with
    the rung (more capacity stretches no more intervals: the same deltas, higher thresholds)
    and energy / time is the rung's power, P(f) = 15 W + 10 W (f / 2.4 GHz)^2."""
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    ts = tracegen.batched()
    pols = [dict(tracegen.default_policy(), pin_level=k) for k in range(1, K + 1)]
    rp.kernel_time()
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=0))
    tot, main, runs, kernels = rp.kernel_time(detail=True)
    assert rp.status() == 0
    assert runs == 1 and kernels == 1
    pairs = [t * K + k for t in (0, 1, 2047, 4095) for k in range(K)]
    for p, r in oracle_pairs(ts, pols, model, pairs=pairs, log=False).items():
        assert_pair(out, p, r, cap=0, check_log=False, tag="static full size")
    T = out["time_s"].reshape(ts.n_traces, K)
    E = out["energy_j"].reshape(ts.n_traces, K)
    assert np.all(np.diff(T, axis=1) <= 0)
    assert np.all(T[:, -1] >= 100_000 * model["dt_s"] * (1 - 1e-12))
    f = np.array(model["f_ghz"])
    np.testing.assert_allclose(E / T, np.broadcast_to(15.0 + 10.0 * (f / 2.4) ** 2, E.shape), rtol=1e-12)
    assert not np.any(out["n_changes"]) and not np.any(out["n_hf"]) and not np.any(out["change_hash"])


def test_static_baselines_every_rung_every_mode(rp, mg):
    """Static baselines (pin_level 1..K) in all four step modes, ragged lengths, in one call:
    without carried state the pins outside the tile kernel's reach take the static kernel
    (one pass at the pinned rung), with carried state the literal kernel (which also writes
    the flag history); both against the oracle, and the kernels launched are counted."""
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    ts = tracegen.make_traces(np.array([0, 1, 33, 1000, 40_001], dtype=np.uint64), seed=19, mean_phase=25.0)
    base = tracegen.default_policy()
    pols = [dict(base, step_mode=m, pin_level=k) for m in range(4) for k in (1, 2, 9, K - 1, K)]
    ref = oracle_pairs(ts, pols, model)
    rp.set_segments(0)
    try:
        rp.kernel_time()
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=50))
        tot, main, runs, kernels = rp.kernel_time(detail=True)
    finally:
        rp.set_segments(-1)
    assert rp.status() == 0
    for p, r in ref.items():
        assert_pair(out, p, r, cap=50, tag="static, no state")
    assert runs == 1 and kernels == 1   # the static kernel takes every pin, those at the bounds too
    state = torch.zeros(ts.n_traces * len(pols) * mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=50, state=state))
    assert rp.status() == 0
    for p, r in ref.items():
        assert_pair(out, p, r, cap=50, tag="static, with state")
    # jump mode, controlled with pins at the bounds: those stay on the tile kernel, and join
    # the static kernel once an inner pin makes it run
    for mix, n_k in (([base, dict(base, pin_level=1), dict(base, pin_level=K)], 1),
                     ([base, dict(base, pin_level=K), dict(base, pin_level=5), dict(base, pin_level=1)], 2)):
        ref = oracle_pairs(ts, mix, model)
        rp.set_segments(0)
        try:
            rp.kernel_time()
            out = to_numpy(rp.run(to_device(ts), ts.lengths, mix, log_capacity=50))
            tot, main, runs, kernels = rp.kernel_time(detail=True)
        finally:
            rp.set_segments(-1)
        assert rp.status() == 0
        for p, r in ref.items():
            assert_pair(out, p, r, cap=50, tag=f"mix of {len(mix)}")
        assert runs == 1 and kernels == n_k


@pytest.mark.parametrize("tile", [(8, 1), (1, 4)])
def test_chunk_wait_timeout_reports_etimedout(mg, tile):
    """Failure detection without a fault: a per-chunk wait limit below the copy latency
    makes the tile kernel's bounded waits run out (a one-slot tile, and the grouped tile
    with four single-warp slots, three of them used).  The kernel records MAGUS_ETIMEDOUT,
    lets the copies in flight land and returns; the status is reported once, and the next
    call on the same handle with the default limit is exact against the oracle."""
    model = tracegen.default_model()
    ts = tracegen.batched(64, 40_000, seed=9)
    d = to_device(ts)
    pols = [tracegen.default_policy()] if tile == (8, 1) else grouped_policies()
    h = mg.Replay(model)
    try:
        h.set_segments(0)
        h.set_tile(*tile)
        h.set_wait(1)
        seen = False
        for _ in range(3):
            h.run(d, ts.lengths, pols, log_capacity=64)
            st = h.status()
            assert st in (0, mg.ETIMEDOUT), st
            if st == mg.ETIMEDOUT:
                seen = True
                break
        assert seen, "a 1 ns chunk-wait limit never ran out"
        assert h.status() == 0
        h.set_wait(0)
        cap = 4000
        out = to_numpy(h.run(d, ts.lengths, pols, log_capacity=cap))
        assert h.status() == 0
        for p, ref in oracle_pairs(ts, pols, model, pairs=range(0, 64 * len(pols), 7)).items():
            assert_pair(out, p, ref, cap=cap, tag="after a timed-out call")
    finally:
        h.close()
