"""GPU tests of the serving runtime: per-request results against the oracle's split replay,
identical results alone and in a mix of many streams (continuous batching), admission
control and state export."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import REL_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


def stream_requests(trace, rng, lo=1, hi=4096):
    """Cut one stream's trace into consecutive requests of log-uniform sizes."""
    cuts, t = [], 0
    while t < len(trace):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        n = max(1, min(n, len(trace) - t))
        cuts.append((t, t + n))
        t += n
    return cuts


def oracle_split(trace, cuts, policy, model):
    st = oracle.new_state()
    return [oracle.replay(trace[a:b], policy, model, state=st) for a, b in cuts]


def same(r, ref, exact_energy=False):
    assert r["n_changes"] == ref["n_changes"]
    assert r["change_hash"] == ref["change_hash"]
    assert r["n_hf"] == ref["n_hf"]
    if exact_energy:
        assert r["energy_j"] == ref["energy_j"] and r["time_s"] == ref["time_s"]
    else:
        assert abs(r["energy_j"] - ref["energy_j"]) <= REL_TOL * max(ref["energy_j"], 1e-300)
        assert abs(r["time_s"] - ref["time_s"]) <= REL_TOL * max(ref["time_s"], 1e-300)


def test_requests_match_oracle_and_mix(mg):
    model, pol = tracegen.default_model(), tracegen.default_policy()
    rng = np.random.default_rng(7)
    n_streams = 300
    ts = tracegen.make_traces(np.full(n_streams, 6000, dtype=np.uint64), seed=9, mean_phase=15.0)
    plans = {s: stream_requests(ts.trace(s), rng) for s in range(n_streams)}
    # interleave requests of all streams (round-robin over each stream's sequence)
    order = []
    idx = {s: 0 for s in plans}
    while any(idx[s] < len(plans[s]) for s in plans):
        for s in plans:
            if idx[s] < len(plans[s]):
                order.append((s, idx[s]))
                idx[s] += 1
    sv = mg.Serve(model, pol, n_streams, max_batch_requests=64)
    ids = {}
    for s, k in order:
        a, b = plans[s][k]
        ids[(s, k)] = sv.submit(s, ts.trace(s)[a:b])
    sv.drain()
    mix = {key: sv.poll(rid) for key, rid in ids.items()}
    st = sv.stats()
    assert st["completed"] == len(order) and st["launches"] > 1
    states = sv.export().view(np.uint64)
    sv.close()
    for s in range(n_streams):
        refs = oracle_split(ts.trace(s), plans[s], pol, model)
        for k, ref in enumerate(refs):
            r = mix[(s, k)]
            same(r, ref)
            assert r["n_seen"] == plans[s][k][1]
    # every stream's exported state counts all its intervals
    per = mg.STATE_BYTES // 8
    assert all(int(states[s * per]) == 6000 for s in range(n_streams))
    # alone: the same requests of a few streams, one stream at a time, one request per launch
    for s in (1, 17):
        alone = mg.Serve(model, pol, n_streams, max_batch_requests=1)
        for k, (a, b) in enumerate(plans[s]):
            rid = alone.submit(s, ts.trace(s)[a:b])
            alone.drain()
            same(alone.poll(rid), mix[(s, k)], exact_energy=True)
        alone.close()


@pytest.mark.parametrize("pin", [1, 17])
def test_static_baseline_stream(mg, pin):
    """A serving handle pinned to a ladder bound (the static baselines of Sec. 5.3 and
    Sec. 6.3): no changes, no high-frequency rounds, the oracle's energy per request."""
    model = tracegen.default_model()
    pol = dict(tracegen.default_policy(), pin_level=pin)
    rng = np.random.default_rng(3)
    ts = tracegen.make_traces(np.full(4, 5000, dtype=np.uint64), seed=4, mean_phase=10.0)
    sv = mg.Serve(model, pol, 4)
    for s in range(4):
        cuts = stream_requests(ts.trace(s), rng)
        ids = [sv.submit(s, ts.trace(s)[a:b]) for a, b in cuts]
        sv.drain()
        for rid, ref in zip(ids, oracle_split(ts.trace(s), cuts, pol, model)):
            r = sv.poll(rid)
            same(r, ref)
            assert r["n_changes"] == 0 and r["level"] == pin - 1
    sv.close()
    with pytest.raises(mg.MagusError):
        mg.Serve(model, dict(pol, pin_level=5), 4)


def test_admission_and_errors(mg):
    model, pol = tracegen.default_model(), tracegen.default_policy()
    sv = mg.Serve(model, pol, 4, mem_budget=4 * 1000)
    d = np.arange(600, dtype=np.uint32)
    r1 = sv.try_submit(0, d)
    assert r1 > 0
    # 2400 + 2400 bytes > 4000: refused unless the first already completed
    r2 = sv.try_submit(1, d)
    assert r2 > 0 or r2 == mg.EBUSY
    sv.drain()
    assert sv.poll(r1) is not None
    with pytest.raises(mg.MagusError) as e:
        sv.poll(r1)
    assert e.value.code == mg.ENOTFOUND
    with pytest.raises(mg.MagusError):
        sv.submit(4, d)                     # stream out of range
    with pytest.raises(mg.MagusError):
        sv.submit(0, np.zeros(0, dtype=np.uint32))
    sv.close()


def test_load_driver_smoke(mg):
    model, pol = tracegen.default_model(), tracegen.default_policy()
    rq = tracegen.requests(2000, rate_per_s=50_000.0, n_streams=1000, seed=3)
    pool = tracegen.batched(4, 100_000, seed=1).data
    rng = np.random.default_rng(0)
    off = rng.integers(0, len(pool) - 4096, size=len(rq.size)).astype(np.uint64)
    sv = mg.Serve(model, pol, 1000)
    lat, wall = sv.load(rq.arrival_s, rq.stream_id, rq.size, pool, off)
    st = sv.stats()
    sv.close()
    assert st["completed"] == 2000 and np.all(lat > 0)
    assert wall >= rq.arrival_s[-1]


def test_load_20k_streams_sampled_against_oracle(mg):
    """The serving load driver over 20,000 streams: Poisson arrivals at 200k requests/s,
    request sizes log-uniform in 1..4096, continuous batching.  For a sample of 300 streams,
    every request's result (counts, hash, high-frequency rounds, energy, time, intervals
    seen, level) equals the oracle replaying that stream's requests in submission order with
    carried state."""
    model, pol = tracegen.default_model(), tracegen.default_policy()
    n_streams = 20_000
    rq = tracegen.requests(60_000, rate_per_s=200_000.0, n_streams=n_streams, seed=5)
    pool = tracegen.batched(16, 100_000, seed=2).data
    rng = np.random.default_rng(1)
    off = rng.integers(0, len(pool) - 4096, size=len(rq.size)).astype(np.uint64)
    sv = mg.Serve(model, pol, n_streams, mem_budget=8 << 30)
    lat, wall, res = sv.load(rq.arrival_s, rq.stream_id, rq.size, pool, off, results=True)
    st = sv.stats()
    sv.close()
    assert st["rejected"] == 0 and st["completed"] == len(rq.size) and st["launches"] > 1
    assert np.all(lat > 0)
    active = np.unique(rq.stream_id)
    sample = rng.choice(active, size=300, replace=False)
    for s in sample:
        idx = np.nonzero(rq.stream_id == s)[0]
        ost = oracle.new_state()
        seen = 0
        for i in idx:
            a, n = int(off[i]), int(rq.size[i])
            ref = oracle.replay(pool[a:a + n], pol, model, state=ost)
            seen += n
            r = {k: res[k][i] for k in ("n_changes", "change_hash", "n_hf", "energy_j", "time_s")}
            r = dict(n_changes=int(r["n_changes"]), change_hash=int(r["change_hash"]), n_hf=int(r["n_hf"]),
                     energy_j=float(r["energy_j"]), time_s=float(r["time_s"]))
            same(r, ref)
            assert int(res["n_seen"][i]) == seen
            assert int(res["level"][i]) == ost.level
