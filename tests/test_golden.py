"""Hand-derived worked examples (tests/golden/*.txt, each with its derivation from the
paper's definitions): the oracle must reproduce them, and so must the CUDA paths."""
import glob
import os

import numpy as np
import pytest

import oracle
import tracegen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_cases():
    cases = []
    for path in sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))):
        for k, block in enumerate(open(path).read().split("\n---\n")):
            kv = {}
            for line in block.splitlines():
                if not line.strip() or line.startswith("#"):
                    continue
                key, _, val = line.partition(":")
                kv[key.strip()] = val.strip()
            cases.append((f"{os.path.basename(path)}#{k}", kv))
    return cases


def build(kv):
    pol = dict(step_mode=0)
    for item in kv["policy"].split():
        name, val = item.split("=")
        key = {"W": "direv_length", "inc": "inc_threshold", "dec": "dec_threshold", "L": "tune_window",
               "th": "high_freq_threshold"}[name]
        pol[key] = int(val) if name in ("W", "L") else float(val)
    kind, *args = kv["trace"].split()
    a = {x.split("=")[0]: int(x.split("=")[1]) for x in args}
    n = a["n"]
    if kind == "square":
        d = np.array([a["lo"] if t % 2 == 0 else a["hi"] for t in range(n)], dtype=np.uint32)
        d[a["stop"]:] = a["lo"]
    elif kind == "step":
        d = np.full(n, a["lo"], dtype=np.uint32)
        d[a["t0"]:] = a["hi"]
    else:
        raise ValueError(kind)
    log = [tuple(int(v) for v in e.split(":")) for e in kv.get("log", "").split()]
    return pol, d, log, int(kv["n_changes"]), int(kv["n_hf"])


CASES = parse_cases()


def test_golden_fixtures_exist():
    assert len(CASES) >= 5


@pytest.mark.parametrize("name,kv", CASES, ids=[c[0] for c in CASES])
def test_oracle_reproduces_golden(name, kv, model):
    pol, d, log, nch, nhf = build(kv)
    r = oracle.replay(d, pol, model)
    assert list(zip(r["log_t"].tolist(), r["log_level"].tolist())) == log
    assert r["n_changes"] == nch and r["n_hf"] == nhf


@pytest.mark.gpu
@pytest.mark.parametrize("name,kv", CASES, ids=[c[0] for c in CASES])
def test_cuda_paths_reproduce_golden(name, kv, model):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03796_b300 import magus
    from gpu_util import to_device, to_numpy
    pol, d, log, nch, nhf = build(kv)
    ts = tracegen.single_trace_set(d)
    rp = magus.Replay(model)
    for out in (rp.run(to_device(ts), ts.lengths, [pol], log_capacity=len(d)),
                rp.plain(to_device(ts), ts.lengths, [pol], log_capacity=len(d))):
        o = to_numpy(out)
        k = int(o["n_changes"][0])
        ent = o["log"][:k].astype(np.uint32)
        assert list(zip((ent >> 5).tolist(), (ent & 31).tolist())) == log
        assert k == nch and int(o["n_hf"][0]) == nhf
    rp.close()
