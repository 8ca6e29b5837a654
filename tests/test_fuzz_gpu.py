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
