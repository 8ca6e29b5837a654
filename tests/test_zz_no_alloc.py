"""magus_replay_run_static: the replay entry point for callers that cannot allocate
device memory (for example code living inside another framework's memory pool, or a
process whose device memory is all reserved up front).  It keeps its planning scratch in a
fixed device array instead of a handle's workspace.

Checked here through the C ABI against magus_replay_run on the same inputs, on two calls
in a row with different workloads (the shared scratch must not leak from one call into
the next).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import tracegen
from gpu_util import REL_TOL, to_device, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    magus.lib()
    return magus


def run_static(mg, model_holder, d_traces, lengths, policies, log_capacity):
    n_pairs = len(lengths) * len(policies)
    dev = torch.device("cuda")
    out = dict(energy_j=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               edp_js=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               time_s=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
               n_changes=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               change_hash=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               n_hf=torch.zeros(n_pairs, dtype=torch.int64, device=dev),
               log=torch.zeros(n_pairs * log_capacity, dtype=torch.int32, device=dev))
    log = mg.FreqLog(out["log"].data_ptr(), log_capacity, out["n_changes"].data_ptr(),
                     out["change_hash"].data_ptr(), out["n_hf"].data_ptr())
    pols = mg.policy_array(policies)
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    rc = mg.lib().magus_replay_run_static(
        ctypes.byref(model_holder.m), d_traces.data_ptr(), ln.ctypes.data, len(ln), ctypes.cast(pols, mg.P),
        len(policies), ctypes.byref(log), out["energy_j"].data_ptr(), out["edp_js"].data_ptr(),
        out["time_s"].data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    mg.check(rc)
    return to_numpy(out)


def compare(a, b):
    for k in ("n_changes", "change_hash", "n_hf", "log"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("energy_j", "edp_js", "time_s"):
        np.testing.assert_allclose(a[k], b[k], rtol=REL_TOL)


def test_static_scratch_matches_run_twice(mg):
    model = tracegen.default_model()
    mh = mg.ModelHolder(model)
    rp = mg.Replay(model)
    cap = 6000
    # call 1: ragged lengths, several policies
    ts1 = tracegen.make_traces(np.array([0, 1, 33, 1025, 8193, 20000, 4097, 64], dtype=np.uint64), seed=21,
                               mean_phase=12.0)
    pols1 = tracegen.sweep_policies()[::37]
    d1 = to_device(ts1)
    ref1 = to_numpy(rp.run(d1, ts1.lengths, pols1, log_capacity=cap))
    got1 = run_static(mg, mh, d1, ts1.lengths, pols1, cap)
    compare(got1, ref1)
    # call 2: a different workload through the same scratch
    ts2 = tracegen.batched(40, 12_345, seed=4)
    pols2 = [tracegen.default_policy()]
    d2 = to_device(ts2)
    ref2 = to_numpy(rp.run(d2, ts2.lengths, pols2, log_capacity=cap))
    got2 = run_static(mg, mh, d2, ts2.lengths, pols2, cap)
    compare(got2, ref2)
    rp.close()


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
