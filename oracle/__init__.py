"""CPU oracle for MAGUS policy replay -- TEST INFRASTRUCTURE ONLY.

A plain sequential FP64 C restatement of the MAGUS per-interval control step
(arXiv 2502.03796: Sec. 3 monitor, Sec. 3.1 / Algorithm 1 predictor, Sec. 3.2 /
Algorithm 2 detector, Sec. 6.1 jump-to-bound actuation, Sec. 4 start at minimum) plus
the stated uncore energy model.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import this module; the CUDA replay
library never does, and the two share no source.

Pins (see tests/test_oracle_pins.py): closed forms for constant traces, single steps,
square waves and threshold ties; exact-rational brute force on tiny traces; split-replay
and ladder invariants.  Energy totals are pinned by closed forms and exact rationals
only; the paper prints no energy numbers for this model (parity of those against the
paper is unpinned by construction: the paper measured real hardware).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "magus_oracle.c")
_HDR = os.path.join(_HERE, "magus_oracle.h")
_LIB = os.path.join(_HERE, "libmagus_oracle.so")
MAX_WINDOW = 64


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Policy(ctypes.Structure):
    _fields_ = [("inc_threshold", ctypes.c_double), ("dec_threshold", ctypes.c_double),
                ("direv_length", ctypes.c_int32), ("tune_window", ctypes.c_int32),
                ("high_freq_threshold", ctypes.c_double), ("step_mode", ctypes.c_int32),
                ("pin_level", ctypes.c_int32)]


class Model(ctypes.Structure):
    _fields_ = [("dt_s", ctypes.c_double), ("n_levels", ctypes.c_int32),
                ("bytes_per_count", ctypes.c_int32), ("f_ghz", ctypes.POINTER(ctypes.c_double)),
                ("p_static_w", ctypes.c_double), ("p_dyn_w", ctypes.c_double),
                ("f_ref_ghz", ctypes.c_double), ("bw_ref_gbs", ctypes.c_double)]


class State(ctypes.Structure):
    _fields_ = [("n_seen", ctypes.c_uint64), ("level", ctypes.c_int32), ("ls_len", ctypes.c_int32),
                ("mem_throughput_ls", ctypes.c_double * (MAX_WINDOW + 1)),
                ("uncore_tune_ls", ctypes.c_uint8 * MAX_WINDOW)]


class Result(ctypes.Structure):
    _fields_ = [("energy_j", ctypes.c_double), ("time_s", ctypes.c_double),
                ("edp_js", ctypes.c_double), ("n_changes", ctypes.c_uint64),
                ("change_hash", ctypes.c_uint64), ("n_hf", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.or_replay.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Policy), ctypes.POINTER(Model),
                                   ctypes.POINTER(State), ctypes.POINTER(Result), P, P,
                                   ctypes.c_uint64, P, P]
        _lib.or_replay.restype = ctypes.c_int
        _lib.or_state_init.argtypes = [ctypes.POINTER(State)]
        _lib.or_replay_batch.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int64,
                                         ctypes.POINTER(Model), P, ctypes.c_int]
        _lib.or_replay_batch.restype = ctypes.c_int
        _lib.or_mix64.argtypes = [ctypes.c_uint64]
        _lib.or_mix64.restype = ctypes.c_uint64
    return _lib


def _policy(d: Dict) -> Policy:
    return Policy(float(d["inc_threshold"]), float(d["dec_threshold"]), int(d["direv_length"]),
                  int(d["tune_window"]), float(d["high_freq_threshold"]), int(d.get("step_mode", 0)),
                  int(d.get("pin_level", 0)))


class _ModelHolder:
    def __init__(self, d: Dict):
        self.f = np.ascontiguousarray(d["f_ghz"], dtype=np.float64)
        self.m = Model(float(d["dt_s"]), len(self.f), int(d["bytes_per_count"]),
                       self.f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       float(d["p_static_w"]), float(d["p_dyn_w"]), float(d["f_ref_ghz"]),
                       float(d["bw_ref_gbs"]))


def new_state() -> State:
    s = State()
    _load().or_state_init(ctypes.byref(s))
    return s


def replay(deltas, policy: Dict, model: Dict, state: Optional[State] = None, log_cap: int = -1,
           detail: bool = False) -> Dict:
    """Replay one trace.  Returns energy/time/edp, change count/hash, n_hf, the change log
    (``log_t`` = interval index from which the new level applies, ``log_level``) and, with
    ``detail``, the per-interval level and Alg. 1 derivative (NaN while the FIFO fills)."""
    lib = _load()
    d = np.ascontiguousarray(deltas, dtype=np.uint32)
    n = int(d.shape[0])
    if state is None:
        state = new_state()
    cap = n if log_cap < 0 else int(log_cap)
    lt = np.zeros(max(cap, 1), dtype=np.uint64)
    ll = np.zeros(max(cap, 1), dtype=np.uint8)
    lv = np.zeros(max(n, 1), dtype=np.uint8) if detail else None
    dv = np.zeros(max(n, 1), dtype=np.float64) if detail else None
    mh = _ModelHolder(model)
    pol = _policy(policy)
    res = Result()
    rc = lib.or_replay(d.ctypes.data, n, ctypes.byref(pol), ctypes.byref(mh.m), ctypes.byref(state),
                       ctypes.byref(res), lt.ctypes.data, ll.ctypes.data, cap,
                       lv.ctypes.data if detail else None, dv.ctypes.data if detail else None)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    k = min(int(res.n_changes), cap)
    out = dict(energy_j=res.energy_j, time_s=res.time_s, edp_js=res.edp_js,
               n_changes=int(res.n_changes), change_hash=int(res.change_hash), n_hf=int(res.n_hf),
               log_t=lt[:k].copy(), log_level=ll[:k].copy(), state=state)
    if detail:
        out["level_log"] = lv[:n].copy()
        out["deriv_log"] = dv[:n].copy()
    return out


def replay_batch(data: np.ndarray, offsets: np.ndarray, lengths: np.ndarray,
                 policies: Sequence[Dict], model: Dict, n_threads: int = 0):
    """All (trace, policy) pairs, pair-major [trace][policy].  Returns (dict of arrays,
    threads used)."""
    lib = _load()
    data = np.ascontiguousarray(data, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    pols = (Policy * len(policies))(*[_policy(p) for p in policies])
    mh = _ModelHolder(model)
    n_pairs = len(lengths) * len(policies)
    res = (Result * max(n_pairs, 1))()
    used = lib.or_replay_batch(data.ctypes.data, offsets.ctypes.data, lengths.ctypes.data,
                               len(lengths), ctypes.cast(pols, ctypes.c_void_p), len(policies),
                               ctypes.byref(mh.m), ctypes.cast(res, ctypes.c_void_p), n_threads)
    arr = np.ctypeslib.as_array(res)[:n_pairs]
    out = {k: np.array(arr[k]) for k in ("energy_j", "time_s", "edp_js", "n_changes", "change_hash", "n_hf")}
    return out, used


def mix64(z: int) -> int:
    return int(_load().or_mix64(z))
