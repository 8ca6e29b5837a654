"""GPU parity at the trace lengths the long-trace paths run at full size: traces of about a
million intervals (the uneven workload's longest, 1e6) through the segment kernel in jump
mode (many segments per pair, so many-segment combines), the segmented closed-loop kernels
in both step modes, and the automatic routing on an uneven mix; change-log indices next to
the 2^27 limit of a log entry (global interval index, carried state).  Every pair is
compared with the CPU oracle: logs element by element, counts and hashes bit-exactly,
energy / time / EDP within 1e-9 relative."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import REL_TOL, assert_pair, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LONG = [1_200_000, 2 ** 20 + 17, 1_000_005]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


@pytest.fixture(scope="module")
def long_set():
    return tracegen.make_traces(np.array(LONG, dtype=np.uint64), seed=31, mean_phase=40.0)


def open_policies():
    base = tracegen.default_policy()
    return [base,
            dict(base, direv_length=12, tune_window=10, inc_threshold=2.0, dec_threshold=-2.0,
                 high_freq_threshold=0.4),
            dict(base, direv_length=3, inc_threshold=8.0, dec_threshold=-8.0, high_freq_threshold=0.7)]


_REFS = {}


def refs(ts, pols, key):
    """Oracle results with full logs for every pair (cached per module run)."""
    if key not in _REFS:
        _REFS[key] = {i * len(pols) + c: oracle.replay(ts.trace(i), pol, tracegen.default_model())
                      for i in range(ts.n_traces) for c, pol in enumerate(pols)}
    return _REFS[key]


@pytest.mark.parametrize("seg", [16384, 2048])
def test_segment_kernel_million_interval_traces(mg, long_set, seg):
    ts, pols = long_set, open_policies()
    ref = refs(ts, pols, "open")
    full_cap = max(r["n_changes"] for r in ref.values()) + 16
    tight_cap = ref[0]["n_changes"]            # pair 0's log exactly full, others overflow
    rp = mg.Replay(tracegen.default_model(), mem_budget=4 << 30)
    try:
        rp.set_segments(seg)
        d = to_device(ts)
        for cap in (full_cap, tight_cap):
            rp.kernel_time()
            out = to_numpy(rp.run(d, ts.lengths, pols, log_capacity=cap))
            assert rp.status() == 0
            _, _, runs, kernels = rp.kernel_time(detail=True)
            assert kernels > runs, "the segment kernel and its combine kernel ran"
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"segment {seg} cap {cap}")
    finally:
        rp.close()


@pytest.mark.parametrize("seg,burn", [(0, -1), (4096, 512)])
def test_closed_loop_million_interval_traces(mg, long_set, seg, burn):
    ts = long_set
    base = tracegen.default_policy()
    pols = [dict(base, step_mode=2), dict(base, step_mode=3, high_freq_threshold=0.9),
            dict(base, step_mode=2, direv_length=12, inc_threshold=2.0, dec_threshold=-2.0)]
    ref = refs(ts, pols, "closed")
    cap = max(r["n_changes"] for r in ref.values()) + 16
    rp = mg.Replay(tracegen.default_model(), mem_budget=4 << 30)
    try:
        rp.set_closed(seg, burn)
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
        assert rp.status() == 0
        segs, second, final, logged = rp.closed_stats()
        assert segs > 3 * len(pols), "several segments per pair"
        for p, r in ref.items():
            assert_pair(out, p, r, cap=cap, tag=f"closed seg {seg} burn {burn}")
    finally:
        rp.close()


def test_uneven_mix_automatic_routing(mg):
    """Lengths from the uneven workload's range (1e3 .. 1e6) in one call with its 16
    policies, kernels chosen automatically (a long trace next to many short ones)."""
    lengths = np.array([1_000_000, 3_000, 250_017, 1_000, 64_999, 7_777, 999_983] + [2_000 + 97 * i for i in range(25)],
                       dtype=np.uint64)
    ts = tracegen.make_traces(lengths, seed=17, mean_phase=40.0)
    pols = tracegen.sweep_policies()[:16]
    model = tracegen.default_model()
    cap = 40_000
    rp = mg.Replay(model, mem_budget=4 << 30)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
        assert rp.status() == 0
    finally:
        rp.close()
    npol = len(pols)
    # every pair's totals against the oracle; full logs on the long traces and a sample
    for i in range(ts.n_traces):
        for c in range(npol):
            if i >= 7 and c % 5:
                continue
            r = oracle.replay(ts.trace(i), pols[c], model)
            assert_pair(out, i * npol + c, r, cap=cap, tag="uneven mix")


@pytest.mark.parametrize("seg", [0, 1024])
def test_log_indices_next_to_the_entry_limit(mg, seg):
    """Carried state puts the trace just below interval 2^27 (the largest index a log entry
    holds): entries near the limit match the oracle started from the same state."""
    model = tracegen.default_model()
    base = tracegen.default_policy()
    pols = [base, dict(base, direv_length=2, inc_threshold=1.0, dec_threshold=-1.0, high_freq_threshold=0.9)]
    n = 20_000
    start = (1 << 27) - 1 - n - 5
    ts = tracegen.make_traces(np.array([n], dtype=np.uint64), seed=44, mean_phase=8.0)
    state = torch.zeros(len(pols) * mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    sv = state.view(torch.int64)
    for c in range(len(pols)):
        sv[c * (mg.STATE_BYTES // 8)] = start            # n_seen; flags, level, history zero
    rp = mg.Replay(model)
    try:
        rp.set_segments(seg)
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=n, state=state))
        assert rp.status() == 0
    finally:
        rp.close()
    for c, pol in enumerate(pols):
        st = oracle.new_state()
        st.n_seen = start
        st.ls_len = pol["direv_length"] + 1       # a full FIFO of zero throughputs (zero deltas)
        r = oracle.replay(ts.trace(0), pol, model, state=st)
        assert r["n_changes"] > 100
        assert int(r["log_t"][-1]) > (1 << 27) - 2 * n
        assert_pair(out, c, r, cap=n, tag=f"near 2^27 seg {seg}")
