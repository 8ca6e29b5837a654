"""GPU parity of the closed loop (step_mode 2: jump mode, 3: one rung per decision) on the
segmented kernels.

Every (trace, policy, segment) is replayed from a guessed state; segments whose guess was
wrong are replayed again and a final pass per pair keeps only replays that started from the
true state.  These tests make the guesses fail on purpose (short segments, no burn-in),
overflow the per-segment change-entry scratch, and check every pair against the oracle:
decision logs, counts and hashes bit-exact, energy / time / EDP within 1e-9 relative.
"""

import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import assert_pair, oracle_pairs, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


@pytest.fixture()
def rp(mg):
    r = mg.Replay(tracegen.default_model())
    yield r
    r.close()


def closed_policies(step_mode=2):
    base = dict(tracegen.default_policy(), step_mode=step_mode)
    return [
        base,
        dict(base, direv_length=1, tune_window=1, high_freq_threshold=1.0),        # hf <=> flag
        dict(base, direv_length=64, tune_window=64, inc_threshold=0.5, dec_threshold=-0.5),
        dict(base, inc_threshold=-1.0, dec_threshold=2.0),                         # +1 and -1 overlap
        dict(base, inc_threshold=np.inf, dec_threshold=-np.inf),                   # never predicts
        dict(base, high_freq_threshold=0.1),                                       # mostly locked high
        dict(base, direv_length=7, tune_window=33, inc_threshold=2.0, dec_threshold=-2.0,
             high_freq_threshold=0.5),
    ]


def ragged():
    lengths = np.array([0, 1, 5, 63, 64, 65, 300, 1000, 4097, 20_000, 33_333], dtype=np.uint64)
    return tracegen.make_traces(lengths, seed=23, mean_phase=20.0)


@pytest.mark.parametrize("seg,burn", [(0, -1), (256, 64), (512, 0), (64, 0), (-1, -1)])
def test_closed_loop_matches_oracle(rp, seg, burn):
    """Ragged lengths, edge policies of both step modes, open-loop and literal-path policies
    in the same call, full and short logs; segments down to 64 rounds with no burn-in (most
    guesses wrong)."""
    ts = ragged()
    model = tracegen.default_model()
    base = tracegen.default_policy()
    pols = closed_policies(2) + closed_policies(3)[:5] + [base, dict(base, step_mode=3, pin_level=5)]
    ref = oracle_pairs(ts, pols, model)
    rp.set_closed(seg, burn)
    for cap in (40_000, 7):
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
        assert rp.status() == 0
        for p, r in ref.items():
            assert_pair(out, p, r, cap=cap, tag=f"closed seg={seg} burn={burn} cap={cap}")
    items, second, final, logged = rp.closed_stats()
    n_cls = len(closed_policies(2)) + 5
    if seg > 0:
        assert items == sum((int(n) + seg - 1) // seg for n in ts.lengths) * n_cls
        if burn == 0:
            assert second > 0   # guesses failed and were replayed again
    if seg < 0:
        assert items == 0


@pytest.mark.parametrize("step_mode", [2, 3])
@pytest.mark.parametrize("W", [1, 2, 3, 4, 5, 8, 9, 12, 16])
def test_closed_loop_window_instances(rp, W, step_mode):
    """Every policy of the call at one W: the first-replay kernel runs its instance for that W
    (1-8, 10, 12, 16; 9 takes the any-W kernel), both step modes, with ragged lengths, failed
    guesses (64-round segments, no burn-in) and the automatic segments."""
    ts = ragged()
    model = tracegen.default_model()
    base = dict(tracegen.default_policy(), step_mode=step_mode, direv_length=W)
    pols = [base, dict(base, inc_threshold=0.5 * W, dec_threshold=-0.5 * W, high_freq_threshold=0.3),
            dict(base, tune_window=33, high_freq_threshold=0.5)]
    ref = oracle_pairs(ts, pols, model)
    for seg, burn in ((0, -1), (256, 64), (64, 0)):
        rp.set_closed(seg, burn)
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=40_000))
        assert rp.status() == 0
        for p, r in ref.items():
            assert_pair(out, p, r, cap=40_000, tag=f"closed mode={step_mode} W={W} seg={seg} burn={burn}")


def test_closed_loop_entry_scratch_overflow(rp):
    """More change entries in a segment than its scratch holds: the log pass replays those
    segments straight into the log."""
    ts = tracegen.make_traces(np.array([6000, 9001], dtype=np.uint64), seed=5, mean_phase=2.0)
    model = tracegen.default_model()
    pols = [dict(tracegen.default_policy(), step_mode=2, inc_threshold=0.2, dec_threshold=-0.2,
                 direv_length=1, high_freq_threshold=1.5)]
    ref = oracle_pairs(ts, pols, model)
    assert max(r["n_changes"] for r in ref.values()) > 2000   # > 64 per 256-round segment
    rp.set_closed(256, 0)
    out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=20_000))
    assert rp.status() == 0
    for p, r in ref.items():
        assert_pair(out, p, r, cap=20_000, tag="scratch overflow")
    items, second, final, logged = rp.closed_stats()
    assert logged > 0


def oracle_state(level, flags64, L):
    """The oracle's state before round 0 with the given level and the flags of rounds
    -L .. -1 taken from the carried 64-bit flag word (bit 63 newest)."""
    st = oracle.new_state()
    st.level = level
    for i in range(L):   # oldest first: element L-1 is round -1 (bit 63)
        st.uncore_tune_ls[i] = (flags64 >> (64 - L + i)) & 1
    return st


def test_closed_loop_carried_state(rp, mg):
    """A fresh carried state (no rounds seen) with the top level and a flag history: the
    segmented path matches the oracle started from the same state, and its written state
    equals the literal kernel's byte for byte.  A level inside the ladder is invalid in
    jump mode, and a state that has seen rounds is refused (closed loop)."""
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    ts = tracegen.make_traces(np.array([3000, 70, 12_345], dtype=np.uint64), seed=8, mean_phase=15.0)
    pols = [dict(tracegen.default_policy(), step_mode=2), dict(tracegen.default_policy(), step_mode=2, tune_window=5)]
    flags = 0xA5F00F0F12345678
    n_pairs = ts.n_traces * len(pols)

    def fresh_states():
        st = np.zeros(n_pairs * mg.STATE_BYTES, dtype=np.uint8)
        v = st.view(np.uint64).reshape(n_pairs, -1)
        v[:, 1] = flags
        st.view(np.uint32).reshape(n_pairs, -1)[:, 4] = K - 1
        return torch.from_numpy(st).cuda()

    written = []
    for seg in (256, -1):
        rp.set_closed(seg, 0)
        state = fresh_states()
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=20_000, state=state))
        assert rp.status() == 0
        for p in range(n_pairs):
            i, c = divmod(p, len(pols))
            r = oracle.replay(ts.trace(i), pols[c], model, state=oracle_state(K - 1, flags, pols[c]["tune_window"]))
            assert_pair(out, p, r, cap=20_000, tag=f"carried state seg={seg}")
        written.append(state.cpu().numpy())
    assert np.array_equal(written[0], written[1])

    rp.set_closed(256, 0)
    bad = fresh_states()
    bad.view(torch.int32)[4] = 3   # pair 0: a level inside the ladder
    rp.run(to_device(ts), ts.lengths, pols, state=bad)
    assert rp.status() == mg.EINVAL
    seen = fresh_states()
    seen.view(torch.int64)[0] = 10  # pair 0 has seen rounds
    rp.run(to_device(ts), ts.lengths, pols, state=seen)
    assert rp.status() == mg.EINVAL
    assert rp.status() == 0


def test_closed_loop_batched_full_size_sampled(mg):
    """The closed-loop benchmark workload (4,096 traces x 100,000 intervals, one policy) in
    the launch configuration the benchmark uses: sampled pairs against the oracle."""
    ts = tracegen.batched(4096, 100_000)
    model = tracegen.default_model()
    pols = [dict(tracegen.default_policy(), step_mode=2)]
    rp = mg.Replay(model, mem_budget=8 << 30)
    try:
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=0))
        assert rp.status() == 0
        items, second, final, logged = rp.closed_stats()
        assert items > 4096 and logged == 0
    finally:
        rp.close()
    for p in (0, 1, 2047, 4095):
        r = oracle.replay(ts.trace(p), pols[0], model, log_cap=0)
        assert_pair(out, p, r, tag="closed batched sampled")


@pytest.mark.parametrize("seed", [31, 32, 33, 34])
def test_closed_loop_random(mg, seed):
    """Random closed-loop policies of both step modes (windows, lists, thresholds including
    infinities and inc < dec), random lengths and phase means, random segment / burn-in
    lengths and log capacities: every pair against the oracle."""
    from test_fuzz_gpu import random_policy
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    lengths = rng.integers(0, 60_000, size=7).astype(np.uint64)
    ts = tracegen.make_traces(lengths, seed=seed, mean_phase=float(rng.uniform(2, 80)))
    pols = []
    while len(pols) < 6:
        p = random_policy(rng, K)
        p["step_mode"], p["pin_level"] = int(rng.choice([2, 3])), 0
        pols.append(p)
    ref = oracle_pairs(ts, pols, model)
    rp = mg.Replay(model)
    try:
        for _ in range(2):
            seg, burn = [(64, 0), (128, 64), (256, 0), (512, 128), (0, -1)][int(rng.integers(0, 5))]
            cap = int(rng.choice([0, 13, 60_000]))
            rp.set_closed(seg, burn)
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"seed {seed} seg {seg} burn {burn} policy {pols[p % len(pols)]}")
    finally:
        rp.close()


@pytest.mark.parametrize("n_levels", [2, 5, 32])
def test_closed_loop_one_rung(mg, n_levels):
    """One rung per decision in the closed loop on ladders of 2, 5 and 32 rungs (2 rungs: the
    jump mode's outcome), a carried inner rung and flag history, short segments with no
    burn-in; every pair and the written state against the oracle and the literal kernel."""
    model = dict(tracegen.default_model(), f_ghz=[0.8 + 1.6 * k / (n_levels - 1) for k in range(n_levels)])
    ts = tracegen.make_traces(np.array([0, 3, 700, 5000, 21_111], dtype=np.uint64), seed=41, mean_phase=12.0)
    pols = closed_policies(3)
    ref = oracle_pairs(ts, pols, model)
    rp = mg.Replay(model)
    try:
        for seg, burn in ((128, 0), (0, -1)):
            rp.set_closed(seg, burn)
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=25_000))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=25_000, tag=f"one rung K={n_levels} seg={seg}")
        # carried state: an inner rung and a flag history (no rounds seen)
        n_pairs = ts.n_traces * len(pols)
        rung, flags = n_levels // 2, 0x0F0F00FF12345678
        written = []
        for seg in (128, -1):
            st = np.zeros(n_pairs * mg.STATE_BYTES, dtype=np.uint8)
            st.view(np.uint64).reshape(n_pairs, -1)[:, 1] = flags
            st.view(np.uint32).reshape(n_pairs, -1)[:, 4] = rung
            state = torch.from_numpy(st).cuda()
            rp.set_closed(seg, 0)
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=25_000, state=state))
            assert rp.status() == 0
            for p in range(n_pairs):
                i, c = divmod(p, len(pols))
                r = oracle.replay(ts.trace(i), pols[c], model,
                                  state=oracle_state(rung, flags, pols[c]["tune_window"]))
                assert_pair(out, p, r, cap=25_000, tag=f"one rung state K={n_levels} seg={seg}")
            written.append(state.cpu().numpy())
        assert np.array_equal(written[0], written[1])
    finally:
        rp.close()


@pytest.mark.parametrize("step_mode", [2, 3])
def test_closed_loop_threshold_edges(mg, step_mode):
    """Traces built around the closed loop's decision points -- deltas at and next to the
    capping thresholds of the bottom and top levels, at and next to the capped-case
    thresholds of Algorithm 1, zero and 2^32 - 1 -- in random order and as steps, so that
    capped and uncapped throughputs meet at every boundary: every pair against the oracle."""
    model = tracegen.default_model()
    rng = np.random.default_rng(7 + step_mode)
    pols = [dict(tracegen.default_policy(), step_mode=step_mode),
            dict(tracegen.default_policy(), step_mode=step_mode, direv_length=2, inc_threshold=1.0,
                 dec_threshold=-1.0, high_freq_threshold=0.9),
            dict(tracegen.default_policy(), step_mode=step_mode, direv_length=9, inc_threshold=40.0,
                 dec_threshold=-60.0, tune_window=3)]
    vals = {0, 1, 2**32 - 1, 2**32 - 2}
    for p in pols:
        t = [int(v) for v in mg.policy_closed_thresholds(p, model)]
        for v in t[:10]:
            for d in (-2, -1, 0, 1, 2):
                if 0 <= v + d < 2**32:
                    vals.add(v + d)
    # every rung's capacity in deltas (the one-rung mode caps at inner rungs too)
    q = model["dt_s"] * 1e9
    for f in model["f_ghz"]:
        c = int(model["bw_ref_gbs"] * (f / model["f_ref_ghz"]) * q / model["bytes_per_count"])
        vals.update(v for v in range(c - 2, c + 3) if 0 <= v < 2**32)
    vals = np.array(sorted(vals), dtype=np.uint64)
    pieces = [rng.choice(vals, size=3000)]                        # random order
    for v in vals:                                                # steps: runs of one value
        pieces.append(np.full(int(rng.integers(1, 12)), v, dtype=np.uint64))
    data = np.concatenate(pieces).astype(np.uint32)
    ts = tracegen.single_trace_set(data)
    ref = oracle_pairs(ts, pols, model)
    rp = mg.Replay(model)
    try:
        for seg, burn in ((64, 0), (0, -1), (-1, -1)):
            rp.set_closed(seg, burn)
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=len(data)))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=len(data), tag=f"edges mode {step_mode} seg={seg}")
    finally:
        rp.close()


def test_closed_loop_with_autotune_and_host_buffers(mg):
    """Closed-loop policies of both modes next to open-loop ones through the autotuner (which
    times the tile shapes with the closed-loop kernels in the same calls) and through the
    host-buffer entry point (traces streamed in batches): every pair against the oracle."""
    model = tracegen.default_model()
    ts = tracegen.make_traces(np.array([7000, 300, 12_345, 64, 2048], dtype=np.uint64), seed=61, mean_phase=18.0)
    base = tracegen.default_policy()
    pols = [base, dict(base, step_mode=2), dict(base, step_mode=3), dict(base, direv_length=3),
            dict(base, step_mode=2, tune_window=20, high_freq_threshold=0.3)]
    ref = oracle_pairs(ts, pols, model)
    rp = mg.Replay(model)
    try:
        rp.autotune(to_device(ts), ts.lengths, pols)
        out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=13_000))
        assert rp.status() == 0
        for p, r in ref.items():
            assert_pair(out, p, r, cap=13_000, tag="after autotune")
        host = rp.run_host(ts.data.view(np.uint32), ts.lengths, pols, log_capacity=13_000)
        for p, r in ref.items():
            assert_pair(host, p, r, cap=13_000, tag="host buffers")
    finally:
        rp.close()
