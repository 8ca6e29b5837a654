"""Seeded synthetic inputs for MAGUS policy replay (input synthesis only).

This module generates uint32 memory-traffic counter deltas, policy-config grids, the
uncore ladder/energy model description and serving request streams.  It holds none of
the control method's arithmetic: both the CPU oracle (``oracle/``) and the CUDA replay
library consume what it produces.

Workloads (sizes of the paper-derived replay study; the paper's own telemetry from
Altis / ECP proxies / MLPerf runs is not available, so these synthetic traces stand in):

* ``single_trace``  1 trace x 20,000 intervals, phase mean 40, seed 0, default policy.
* ``batched``       4,096 traces x 100,000 intervals, phase mean 40, 1 policy.
* ``sweep``         1,024 traces x 200,000 intervals, bursty (mean 10) / long (mean 500)
                    regimes of mean length 5,000, 256 policies (8 thresholds x 8 windows
                    x 4 hysteresis counts of a 10-entry tune window).
* ``uneven``        16,384 traces, lengths log-uniform in [1e3, 1e6], 16 policies.
* ``requests``      Poisson arrivals at 200k req/s over 100,000 streams, sizes
                    log-uniform in [1, 4096].
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tracegen.c")
_LIB = os.path.join(_HERE, "libtracegen.so")


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("mean_phase", ctypes.c_double), ("mean_phase_b", ctypes.c_double),
                ("regime_mean", ctypes.c_double), ("level_lo", ctypes.c_double),
                ("level_hi", ctypes.c_double), ("sigma", ctypes.c_double),
                ("dt_s", ctypes.c_double), ("line_bytes", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        u64 = ctypes.c_uint64
        _lib.tg_trace.argtypes = [ctypes.POINTER(_Params), u64, u64, P, u64]
        _lib.tg_traces.argtypes = [ctypes.POINTER(_Params), u64, P, P, P, u64, P]
        _lib.tg_lengths_loguniform.argtypes = [u64, u64, ctypes.c_double, ctypes.c_double, P]
        _lib.tg_requests.argtypes = [u64, u64, ctypes.c_double, u64, ctypes.c_double,
                                     ctypes.c_double, P, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------------------- model
def default_model() -> dict:
    """Uncore ladder 0.8-2.4 GHz in 0.1 GHz steps (17 levels), dt = 100 ms, and the
    stated energy model: P(f) = 15 W + 10 W (f / 2.4 GHz)^2, capacity 200 GB/s f / 2.4 GHz,
    64-byte counted lines."""
    return dict(dt_s=0.1, f_ghz=[(8 + k) / 10.0 for k in range(17)], p_static_w=15.0,
                p_dyn_w=10.0, f_ref_ghz=2.4, bw_ref_gbs=200.0, bytes_per_count=64)


def default_policy() -> dict:
    """Project defaults for the predictor / detector parameters (the paper fixes only the
    0.6 high-frequency threshold and, through 'six times per second' at 10 rounds/s, a
    10-entry tune window)."""
    return dict(inc_threshold=5.0, dec_threshold=-5.0, direv_length=5, tune_window=10,
                high_freq_threshold=0.6, step_mode=0)


def sweep_policies() -> List[dict]:
    """256 configs: |inc| = |dec| in 8 values x window W in 8 values x hysteresis count
    k in {4,5,6,7} of a 10-entry tune window (threshold k/10)."""
    out = []
    for thr in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0):
        for w in (2, 3, 4, 5, 6, 8, 10, 12):
            for k in (4, 5, 6, 7):
                out.append(dict(inc_threshold=thr, dec_threshold=-thr, direv_length=w,
                                tune_window=10, high_freq_threshold=k / 10.0, step_mode=0))
    return out


# ----------------------------------------------------------------------------- traces
@dataclasses.dataclass
class TraceSet:
    """Traces stored back to back; trace i occupies data[offsets[i] : offsets[i] + lengths[i]].
    Every offset is a multiple of 32 elements (128 bytes) and the buffer is padded to a
    multiple of 32 elements."""
    lengths: np.ndarray   # uint64 [n_traces]
    offsets: np.ndarray   # uint64 [n_traces]
    data: np.ndarray      # uint32 [total]

    @property
    def n_traces(self) -> int:
        return int(self.lengths.shape[0])

    @property
    def n_samples(self) -> int:
        return int(self.lengths.sum())

    def trace(self, i: int) -> np.ndarray:
        o = int(self.offsets[i])
        return self.data[o:o + int(self.lengths[i])]

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(self.lengths.tobytes())
        for i in range(self.n_traces):
            h.update(self.trace(i).tobytes())
        return h.hexdigest()


def aligned_offsets(lengths: np.ndarray, align: int = 32) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.uint64)
    padded = (lengths + np.uint64(align - 1)) // np.uint64(align) * np.uint64(align)
    off = np.zeros_like(padded)
    if len(padded) > 1:
        off[1:] = np.cumsum(padded[:-1], dtype=np.uint64)
    return off


def make_traces(lengths, seed: int = 0, mean_phase: float = 40.0, mean_phase_b: float = 0.0,
                regime_mean: float = 0.0, ids: Optional[np.ndarray] = None,
                level_lo: float = 2.0, level_hi: float = 180.0, sigma: float = 0.05,
                dt_s: float = 0.1, line_bytes: float = 64.0, out: Optional[np.ndarray] = None
                ) -> TraceSet:
    lib = _load()
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    offsets = aligned_offsets(lengths)
    total = int(offsets[-1] + ((lengths[-1] + 31) // 32) * 32) if len(lengths) else 0
    if out is None:
        data = np.zeros(max(total, 32), dtype=np.uint32)
    else:
        data = out[:total]
    if ids is None:
        ids = np.arange(len(lengths), dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    p = _Params(mean_phase, mean_phase_b, regime_mean, level_lo, level_hi, sigma, dt_s, line_bytes)
    lib.tg_traces(ctypes.byref(p), seed, _ptr(ids), _ptr(lengths), _ptr(offsets), len(lengths),
                  _ptr(data))
    return TraceSet(lengths=lengths, offsets=offsets, data=data)


def loguniform_lengths(n: int, lo: float, hi: float, seed: int = 0) -> np.ndarray:
    lib = _load()
    out = np.zeros(n, dtype=np.uint64)
    lib.tg_lengths_loguniform(seed, n, lo, hi, _ptr(out))
    return out


# ----------------------------------------------------------------------------- workloads
def single_trace(seed: int = 0, n: int = 20_000) -> TraceSet:
    return make_traces(np.array([n], dtype=np.uint64), seed=seed, mean_phase=40.0)


def batched(n_traces: int = 4096, n: int = 100_000, seed: int = 0, first_id: int = 0) -> TraceSet:
    ids = np.arange(first_id, first_id + n_traces, dtype=np.uint64)
    return make_traces(np.full(n_traces, n, dtype=np.uint64), seed=seed, mean_phase=40.0, ids=ids)


def sweep(n_traces: int = 1024, n: int = 200_000, seed: int = 0, first_id: int = 0) -> TraceSet:
    ids = np.arange(first_id, first_id + n_traces, dtype=np.uint64)
    return make_traces(np.full(n_traces, n, dtype=np.uint64), seed=seed, mean_phase=10.0,
                       mean_phase_b=500.0, regime_mean=5000.0, ids=ids)


def uneven(n_traces: int = 16_384, lo: float = 1e3, hi: float = 1e6, seed: int = 0) -> TraceSet:
    lengths = loguniform_lengths(n_traces, lo, hi, seed=seed)
    return make_traces(lengths, seed=seed, mean_phase=40.0)


@dataclasses.dataclass
class RequestStream:
    arrival_s: np.ndarray   # float64 [n]
    stream_id: np.ndarray   # uint32 [n]
    size: np.ndarray        # uint32 [n]


def requests(n_req: int, rate_per_s: float = 200_000.0, n_streams: int = 100_000,
             size_lo: float = 1.0, size_hi: float = 4096.0, seed: int = 0) -> RequestStream:
    lib = _load()
    a = np.zeros(n_req, dtype=np.float64)
    s = np.zeros(n_req, dtype=np.uint32)
    z = np.zeros(n_req, dtype=np.uint32)
    lib.tg_requests(seed, n_req, rate_per_s, n_streams, size_lo, size_hi, _ptr(a), _ptr(s), _ptr(z))
    return RequestStream(a, s, z)


def single_trace_set(deltas) -> TraceSet:
    """Wrap one hand-built trace in the packed layout (zero padding to 32 elements)."""
    d = np.asarray(deltas, dtype=np.uint32)
    n = len(d)
    data = np.zeros(max((n + 31) // 32 * 32, 32), dtype=np.uint32)
    data[:n] = d
    return TraceSet(lengths=np.array([n], dtype=np.uint64), offsets=np.zeros(1, dtype=np.uint64), data=data)
