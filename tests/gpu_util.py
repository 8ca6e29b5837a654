"""Helpers for the GPU parity tests: move generated inputs to the device, compare with the
oracle.  Inputs come from tracegen only; expected values from oracle only."""
import numpy as np

import oracle
import tracegen

REL_TOL = 1e-9   # energy / time / EDP, relative (FP64 sums in different orders)


def to_device(ts: tracegen.TraceSet):
    import torch
    return torch.from_numpy(ts.data.view(np.int32)).cuda()


def oracle_pairs(ts: tracegen.TraceSet, policies, model, pairs=None, log=True):
    """Oracle results for (trace, policy) pairs, pair index = trace * n_policies + policy."""
    npol = len(policies)
    if pairs is None:
        pairs = range(ts.n_traces * npol)
    res = {}
    for p in pairs:
        i, c = divmod(int(p), npol)
        res[int(p)] = oracle.replay(ts.trace(i), policies[c], model, log_cap=-1 if log else 0)
    return res


def assert_pair(out_np, p, ref, cap=0, check_log=True, tag=""):
    msg = f"{tag} pair {p}"
    assert int(out_np["n_changes"][p]) == ref["n_changes"], msg + " n_changes"
    assert int(out_np["change_hash"][p]) % 2**64 == ref["change_hash"], msg + " hash"
    assert int(out_np["n_hf"][p]) == ref["n_hf"], msg + " n_hf"
    for k in ("energy_j", "edp_js", "time_s"):
        if k in out_np:
            a, b = float(out_np[k][p]), ref[k]
            assert abs(a - b) <= REL_TOL * max(abs(b), 1e-300), f"{msg} {k}: {a} vs {b}"
    if cap and check_log:
        k = min(ref["n_changes"], cap)
        ent = out_np["log"][p * cap:p * cap + k].astype(np.uint32)
        t = (ent >> 5).astype(np.uint64)
        lv = (ent & 31).astype(np.uint8)
        assert np.array_equal(t, ref["log_t"][:k].astype(np.uint64)), msg + " log times"
        assert np.array_equal(lv, ref["log_level"][:k]), msg + " log levels"


def to_numpy(out):
    r = {}
    for k, v in out.items():
        a = v.cpu().numpy()
        if k in ("n_changes", "change_hash", "n_hf"):
            a = a.view(np.uint64)
        if k == "log":
            a = a.view(np.uint32)
        r[k] = a
    return r
