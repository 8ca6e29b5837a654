"""magus_replay_run_static: the replay entry point for callers that cannot allocate
device memory (for example code living inside another framework's memory pool, or a
process whose device memory is all reserved up front).  It keeps its planning scratch in a
fixed device array instead of a handle's workspace.

Checked here through the C ABI against the CPU oracle and against magus_replay_run on the
same inputs, on calls in a row with different workloads (the shared scratch must not leak
from one call into the next), with state carried across calls, with policies pinned to the
bottom and top of the ladder, and on the arguments it refuses.  This file is collected last
on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import REL_TOL, assert_pair, oracle_pairs, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


def run_static(mg, model_holder, d_traces, lengths, policies, log_capacity, state=None, check=True):
    n_pairs = len(lengths) * len(policies)
    dev = torch.device("cuda")
    out = dict(energy_j=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               edp_js=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               time_s=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               n_changes=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               change_hash=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               n_hf=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               log=torch.zeros(max(n_pairs * log_capacity, 1), dtype=torch.int32, device=dev))
    log = mg.FreqLog(out["log"].data_ptr(), log_capacity, out["n_changes"].data_ptr(),
                     out["change_hash"].data_ptr(), out["n_hf"].data_ptr())
    pols = mg.policy_array(policies)
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    rc = mg.lib().magus_replay_run_static(
        ctypes.byref(model_holder.m), d_traces.data_ptr(), ln.ctypes.data, len(ln), ctypes.cast(pols, mg.P),
        len(policies), ctypes.byref(log), out["energy_j"].data_ptr(), out["edp_js"].data_ptr(),
        out["time_s"].data_ptr(), None if state is None else state.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    if not check:
        return rc
    mg.check(rc)
    return to_numpy(out)


def compare(a, b):
    for k in ("n_changes", "change_hash", "n_hf", "log"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("energy_j", "edp_js", "time_s"):
        np.testing.assert_allclose(a[k], b[k], rtol=REL_TOL)


def check_oracle(got, ts, pols, model, cap, tag):
    for p, ref in oracle_pairs(ts, pols, model).items():
        assert_pair(got, p, ref, cap=cap, tag=tag)


def test_static_scratch_matches_run_and_oracle_twice(mg):
    model = tracegen.default_model()
    mh = mg.ModelHolder(model)
    rp = mg.Replay(model)
    cap = 6000
    # call 1: ragged lengths, several policies (bottom and top pins among them)
    ts1 = tracegen.make_traces(np.array([0, 1, 33, 1025, 8193, 20000, 4097, 64], dtype=np.uint64), seed=21,
                               mean_phase=12.0)
    K = len(model["f_ghz"])
    pols1 = tracegen.sweep_policies()[::37] + [dict(tracegen.default_policy(), pin_level=1),
                                                dict(tracegen.default_policy(), pin_level=K)]
    d1 = to_device(ts1)
    ref1 = to_numpy(rp.run(d1, ts1.lengths, pols1, log_capacity=cap))
    got1 = run_static(mg, mh, d1, ts1.lengths, pols1, cap)
    compare(got1, ref1)
    check_oracle(got1, ts1, pols1, model, cap, "static scratch, call 1")
    # call 2: a different workload through the same scratch
    ts2 = tracegen.batched(40, 12_345, seed=4)
    pols2 = [tracegen.default_policy()]
    d2 = to_device(ts2)
    ref2 = to_numpy(rp.run(d2, ts2.lengths, pols2, log_capacity=cap))
    got2 = run_static(mg, mh, d2, ts2.lengths, pols2, cap)
    compare(got2, ref2)
    check_oracle(got2, ts2, pols2, model, cap, "static scratch, call 2")
    rp.close()


def test_static_scratch_split_replay_with_state(mg):
    """A trace fed in pieces through consecutive calls with carried state (io_state on the
    device) reproduces the oracle's whole-trace log exactly and its energies additively;
    controlled policies and both bound pins."""
    model = tracegen.default_model()
    mh = mg.ModelHolder(model)
    K = len(model["f_ghz"])
    full = tracegen.make_traces(np.array([30_000], dtype=np.uint64), seed=5, mean_phase=9.0).trace(0)
    base = tracegen.default_policy()
    pols = [base, dict(base, direv_length=40, tune_window=50, high_freq_threshold=0.1),
            dict(base, pin_level=1), dict(base, pin_level=K)]
    state = torch.zeros(len(pols) * mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    cuts = [0, 3, 64, 65, 1100, 8192, 8200, 20000, 30_000]
    E = np.zeros(len(pols))
    T = np.zeros(len(pols))
    nhf = np.zeros(len(pols), dtype=np.int64)
    hsh = [0] * len(pols)
    logs = [[] for _ in pols]
    for a, b in zip(cuts[:-1], cuts[1:]):
        ts = tracegen.single_trace_set(full[a:b])
        cap = b - a
        out = run_static(mg, mh, to_device(ts), ts.lengths, pols, cap, state=state)
        for c in range(len(pols)):
            E[c] += out["energy_j"][c]
            T[c] += out["time_s"][c]
            nhf[c] += int(out["n_hf"][c])
            hsh[c] = (hsh[c] + int(out["change_hash"][c])) % 2**64
            logs[c].append(out["log"][c * cap:c * cap + int(out["n_changes"][c])])
    for c, pol in enumerate(pols):
        ref = oracle.replay(full, pol, model)
        ent = np.concatenate(logs[c]).astype(np.uint32)
        assert np.array_equal((ent >> 5).astype(np.uint64), ref["log_t"]), c
        assert np.array_equal((ent & 31).astype(np.uint8), ref["log_level"]), c
        assert nhf[c] == ref["n_hf"] and hsh[c] == ref["change_hash"], c
        assert abs(E[c] - ref["energy_j"]) <= REL_TOL * ref["energy_j"], c
        assert abs(T[c] - ref["time_s"]) <= REL_TOL * ref["time_s"], c
    st = state.cpu().numpy().view(np.uint64)
    assert int(st[0]) == 30_000


def test_static_scratch_refusals(mg):
    """Policies outside the time-parallel kernel's reach are refused on the host; a carried
    level that is neither 0 nor K-1 is reported by the kernel; a following call is clean."""
    model = tracegen.default_model()
    mh = mg.ModelHolder(model)
    ts = tracegen.make_traces(np.array([100], dtype=np.uint64), seed=1)
    d = to_device(ts)
    base = tracegen.default_policy()
    for bad in (dict(base, step_mode=1), dict(base, step_mode=2), dict(base, pin_level=9)):
        assert run_static(mg, mh, d, ts.lengths, [bad], 10, check=False) == mg.EINVAL
    state = torch.zeros(mg.STATE_BYTES, dtype=torch.uint8, device="cuda")
    state.view(torch.int32)[4] = 3   # level field (offset 16): neither 0 nor K-1
    assert run_static(mg, mh, d, ts.lengths, [base], 10, state=state, check=False) == mg.EINVAL
    assert b"carried level" in mg.lib().magus_last_error()
    got = run_static(mg, mh, d, ts.lengths, [base], 100)
    check_oracle(got, ts, [base], model, 100, "after a refused call")


def test_static_scratch_rejects_oversized_plan(mg):
    model = tracegen.default_model()
    mh = mg.ModelHolder(model)
    n = 200_000   # 200,000 traces x 24 B of plan > 4 MiB
    lengths = np.ones(n, dtype=np.uint64)
    d = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    pols = mg.policy_array([tracegen.default_policy()])
    rc = mg.lib().magus_replay_run_static(ctypes.byref(mh.m), d.data_ptr(), lengths.ctypes.data, n,
                                          ctypes.cast(pols, mg.P), 1, None, e.data_ptr(), e.data_ptr(), None,
                                          None, None)
    assert rc == mg.EINVAL
    assert b"static scratch" in mg.lib().magus_last_error()
