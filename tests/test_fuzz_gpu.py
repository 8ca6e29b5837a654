"""Randomised parity: random policies of every mode and random trace lengths through one
call (tile or segment kernel for the jump mode, ladder kernel for one rung per decision,
literal kernel for the rest), every pair against the oracle."""
import numpy as np
import pytest

import tracegen
from gpu_util import assert_pair, oracle_pairs, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def random_policy(rng, K):
    W = int(rng.integers(1, 65))
    inc = float(rng.choice([rng.uniform(-3, 12), np.inf, 0.0]))
    dec = float(rng.choice([rng.uniform(-12, 3), -np.inf, 0.0]))
    pol = dict(inc_threshold=inc, dec_threshold=dec, direv_length=W, tune_window=int(rng.integers(1, 65)),
               high_freq_threshold=float(rng.choice([rng.uniform(0, 1), 0.0, 1.0, 1.5])),
               step_mode=int(rng.choice([0, 0, 0, 1, 1, 2, 3])), pin_level=0)
    r = rng.uniform()
    if r < 0.1:
        pol["pin_level"] = int(rng.choice([1, K]))
    elif r < 0.15:
        pol["pin_level"] = int(rng.integers(1, K + 1))
    return pol


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_random_policies_and_lengths(seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    lengths = rng.integers(0, 40_000, size=9).astype(np.uint64)
    lengths[rng.integers(0, 9)] = 0
    ts = tracegen.make_traces(lengths, seed=seed, mean_phase=float(rng.uniform(3, 80)))
    pols = [random_policy(rng, K) for _ in range(int(rng.integers(3, 12)))]
    cap = int(rng.choice([0, 17, 40_000]))
    ref = oracle_pairs(ts, pols, model)
    rp = magus.Replay(model)
    try:
        for seg in (-1, int(rng.choice([1024, 4096]))):
            rp.set_segments(seg)
            out = to_numpy(rp.run(to_device(ts) if ts.data.size else torch.zeros(4, dtype=torch.int32, device="cuda"),
                                  ts.lengths, pols, log_capacity=cap))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"seed {seed} seg {seg} policy {pols[p % len(pols)]}")
    finally:
        rp.close()


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_random_split_replay_with_state(seed):
    """Random cuts of random traces replayed piece by piece with carried state, policies of
    every mode that can resume (the closed loop starts fresh only): concatenated logs and
    summed energies equal the oracle's whole-trace replay."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    import oracle
    from gpu_util import REL_TOL
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    n = int(rng.integers(2000, 30_000))
    full = tracegen.make_traces(np.array([n], dtype=np.uint64), seed=seed, mean_phase=float(rng.uniform(3, 60))).trace(0)
    pols = []
    while len(pols) < 6:
        p = random_policy(rng, K)
        if not p["step_mode"] & 2:
            pols.append(p)
    cuts = sorted(set([0, n] + rng.integers(1, n, size=int(rng.integers(1, 8))).tolist()))
    state = torch.zeros(len(pols) * magus.STATE_BYTES, dtype=torch.uint8, device="cuda")
    E = np.zeros(len(pols))
    logs = [[] for _ in pols]
    rp = magus.Replay(model)
    try:
        rp.set_segments(int(rng.choice([-1, 1024])))
        for a, b in zip(cuts[:-1], cuts[1:]):
            ts = tracegen.single_trace_set(full[a:b])
            cap = b - a
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap, state=state))
            for c in range(len(pols)):
                E[c] += out["energy_j"][c]
                logs[c].append(out["log"][c * cap:c * cap + int(out["n_changes"][c])])
        assert rp.status() == 0
    finally:
        rp.close()
    for c, pol in enumerate(pols):
        ref = oracle.replay(full, pol, model)
        ent = np.concatenate(logs[c]).astype(np.uint32)
        assert np.array_equal((ent >> 5).astype(np.uint64), ref["log_t"]), (seed, pol, cuts)
        assert np.array_equal((ent & 31).astype(np.uint8), ref["log_level"]), (seed, pol, cuts)
        assert abs(E[c] - ref["energy_j"]) <= REL_TOL * ref["energy_j"], (seed, pol)


@pytest.mark.parametrize("seed", [21, 22])
def test_random_serving_streams(seed):
    """A serving handle with a random jump-mode policy: random request sizes on a few
    streams, every result against the oracle's split replay."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    import oracle
    from gpu_util import REL_TOL
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    pol = random_policy(rng, K)
    pol["step_mode"] = 0
    if pol["pin_level"] not in (0, 1, K):
        pol["pin_level"] = 0
    ts = tracegen.make_traces(np.full(5, 7000, dtype=np.uint64), seed=seed, mean_phase=float(rng.uniform(3, 60)))
    sv = magus.Serve(model, pol, 5)
    try:
        for s in range(5):
            t, st = 0, oracle.new_state()
            ids = []
            while t < 7000:
                k = int(min(7000 - t, np.exp(rng.uniform(0, np.log(4096)))))
                ids.append((sv.submit(s, ts.trace(s)[t:t + k]), oracle.replay(ts.trace(s)[t:t + k], pol, model, state=st)))
                t += k
            sv.drain()
            for rid, ref in ids:
                r = sv.poll(rid)
                assert r["n_changes"] == ref["n_changes"] and r["change_hash"] == ref["change_hash"], (seed, pol)
                assert r["n_hf"] == ref["n_hf"]
                assert abs(r["energy_j"] - ref["energy_j"]) <= REL_TOL * max(ref["energy_j"], 1e-300)
    finally:
        sv.close()


@pytest.mark.parametrize("seed", [21, 22, 23, 24, 25])
def test_random_grouped_policies(seed):
    """Random policy groups (members sharing Alg. 1's W, inc, dec; half of them with a
    10-round tune window, whose counts are bit-sliced and shared) on random lengths, through
    the automatic tile and each grouped and one-slot tile shape: every pair against the
    oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    lengths = rng.integers(0, 30_000, size=7).astype(np.uint64)
    ts = tracegen.make_traces(lengths, seed=seed, mean_phase=float(rng.uniform(3, 80)))
    pols = []
    for _ in range(int(rng.integers(1, 11))):
        W = int(rng.choice([int(rng.integers(1, 65)), 5, 10]))
        thr = float(rng.uniform(0.3, 8.0))
        L = 10 if rng.uniform() < 0.5 else int(rng.integers(1, 65))
        for _ in range(int(rng.integers(1, 5))):
            pols.append(dict(inc_threshold=thr, dec_threshold=-thr, direv_length=W, tune_window=L,
                             high_freq_threshold=float(rng.choice([rng.uniform(0, 1), 0.0, 1.0, 1.2])),
                             step_mode=0, pin_level=0))
    order = rng.permutation(len(pols))
    pols = [pols[i] for i in order]
    cap = int(rng.choice([0, 40_000]))
    ref = oracle_pairs(ts, pols, model)
    rp = magus.Replay(model)
    try:
        for tile in ((0, 0), (1, 4), (2, 2), (8, 1), (1, 8), (4, 1)):
            rp.set_segments(0 if tile != (0, 0) else -1)
            rp.set_tile(*tile)
            out = to_numpy(rp.run(to_device(ts), ts.lengths, pols, log_capacity=cap))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"seed {seed} tile {tile}")
    finally:
        rp.close()


@pytest.mark.parametrize("seed", [41, 42, 43, 44, 45, 46])
def test_random_one_window_calls(seed):
    """Random policies of every mode that all share one W (drawn from the lengths with kernel
    instances and a few without), so the tile, segment, one-rung and closed-loop first-replay
    kernels run their instance for that W: random lengths, automatic and forced closed-loop
    segments (64 rounds, no burn-in: most guesses wrong), every pair against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    rng = np.random.default_rng(seed)
    model = tracegen.default_model()
    K = len(model["f_ghz"])
    W = int(rng.choice([1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 9, 24]))
    lengths = rng.integers(0, 30_000, size=6).astype(np.uint64)
    ts = tracegen.make_traces(lengths, seed=seed, mean_phase=float(rng.uniform(3, 80)))
    pols = []
    for _ in range(int(rng.integers(1, 5))):
        p = random_policy(rng, K)
        p.update(direv_length=W, pin_level=0, step_mode=int(rng.choice([0, 1, 2, 3, 2, 3])))
        pols.append(p)
    cap = int(rng.choice([0, 17, 40_000]))
    ref = oracle_pairs(ts, pols, model)
    rp = magus.Replay(model)
    try:
        for seg, burn in ((0, -1), (256, 64), (64, 0)):
            rp.set_closed(seg, burn)
            out = to_numpy(rp.run(to_device(ts) if ts.data.size else torch.zeros(4, dtype=torch.int32, device="cuda"),
                                  ts.lengths, pols, log_capacity=cap))
            assert rp.status() == 0
            for p, r in ref.items():
                assert_pair(out, p, r, cap=cap, tag=f"seed {seed} W {W} closed {seg},{burn}")
    finally:
        rp.close()
