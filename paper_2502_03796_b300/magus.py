"""ctypes binding of libmagus (include/magus.h).

Argument marshalling only: every step of the replay runs in the library's CUDA kernels.
PyTorch supplies device buffers and streams.  Importing works without a GPU; creating a
handle needs the built library (``python -m paper_2502_03796_b300.build``) and a CUDA
device, and raises otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmagus.so")

OK, EINVAL, ENOMEM, EBUSY, EAGAIN, ETIMEDOUT, ECUDA, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
MAX_WINDOW = 64


class MagusError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmagus error {code}: {msg}")
        self.code = code


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
    _fields_ = [("n_seen", ctypes.c_uint64), ("flags", ctypes.c_uint64), ("level", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("hist", ctypes.c_uint32 * MAX_WINDOW)]


STATE_BYTES = ctypes.sizeof(State)


class FreqLog(ctypes.Structure):
    _fields_ = [("entries", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("n_changes", ctypes.c_void_p), ("change_hash", ctypes.c_void_p),
                ("n_hf", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("n_seen", ctypes.c_uint64), ("level", ctypes.c_uint32), ("n_changes", ctypes.c_uint32),
                ("change_hash", ctypes.c_uint64), ("n_hf", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("energy_j", ctypes.c_double), ("time_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("samples", ctypes.c_uint64), ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double),
                ("p999_s", ctypes.c_double), ("max_s", ctypes.c_double)]


# every symbol include/magus.h declares, with its ctypes signature
P = ctypes.c_void_p
_I32, _U32, _I64, _U64, _SZ = ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
SIGNATURES = {
    "magus_replay_open": ([P, ctypes.POINTER(Model), ctypes.c_int, _SZ], ctypes.c_int),
    "magus_replay_run": ([P, P, P, _I32, P, _I32, P, P, P, P, P, P], ctypes.c_int),
    "magus_replay_run_host": ([P, P, P, _I32, P, _I32, P, P, P, P], ctypes.c_int),
    "magus_replay_plain": ([P, P, P, _I32, P, _I32, P, P, P, P, P], ctypes.c_int),
    "magus_replay_detail": ([P, P, _U64, P, P, P, P, P, P, P, P], ctypes.c_int),
    "magus_replay_status": ([P, P], ctypes.c_int),
    "magus_replay_set_tile": ([P, _I32, _I32], ctypes.c_int),
    "magus_replay_set_segments": ([P, _I32], ctypes.c_int),
    "magus_replay_set_wait": ([P, _U64], ctypes.c_int),
    "magus_replay_set_closed": ([P, _I32, _I32], ctypes.c_int),
    "magus_replay_closed_stats": ([P, P], ctypes.c_int),
    "magus_replay_kernel_time": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "magus_replay_autotune": ([P, P, P, _I32, P, _I32, P, P, P], ctypes.c_int),
    "magus_replay_close": ([P], ctypes.c_int),
    "magus_replay_run_static": ([ctypes.POINTER(Model), P, P, _I32, P, _I32, P, P, P, P, P, P], ctypes.c_int),
    "magus_packed_size": ([P, _I32, P, P], ctypes.c_int),
    "magus_policy_bounds": ([ctypes.POINTER(Policy), ctypes.POINTER(Model), P], ctypes.c_int),
    "magus_policy_fp64_thresholds": ([ctypes.POINTER(Policy), ctypes.POINTER(Model), P], ctypes.c_int),
    "magus_policy_closed_thresholds": ([ctypes.POINTER(Policy), ctypes.POINTER(Model), P], ctypes.c_int),
    "magus_last_error": ([], ctypes.c_char_p),
    "magus_version": ([], ctypes.c_char_p),
    "magus_serve_open": ([P, ctypes.POINTER(Model), ctypes.POINTER(Policy), _I32, _SZ, ctypes.c_int, _I32, _I64],
                         ctypes.c_int),
    "magus_serve_submit": ([P, _U32, P, _U32, P], ctypes.c_int),
    "magus_serve_poll": ([P, _U64, ctypes.POINTER(Result)], ctypes.c_int),
    "magus_serve_drain": ([P], ctypes.c_int),
    "magus_serve_stats": ([P, ctypes.POINTER(ServeStats)], ctypes.c_int),
    "magus_serve_export": ([P, P], ctypes.c_int),
    "magus_serve_load": ([P, P, P, P, P, P, _I64, P, P, P], ctypes.c_int),
    "magus_serve_close": ([P], ctypes.c_int),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libmagus.so (in-tree build).  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2502_03796_b300.build` (nvcc, sm_103a)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            if not hasattr(l, name):   # tests/test_abi.py checks that every symbol exists
                continue
            fn = getattr(l, name)
            fn.argtypes = args
            fn.restype = res
        _lib = l
    return _lib


def check(rc: int) -> int:
    if rc != OK:
        raise MagusError(rc, lib().magus_last_error().decode())
    return rc


def make_policy(d: Dict) -> Policy:
    return Policy(float(d["inc_threshold"]), float(d["dec_threshold"]), int(d["direv_length"]),
                  int(d["tune_window"]), float(d["high_freq_threshold"]), int(d.get("step_mode", 0)),
                  int(d.get("pin_level", 0)))


def policy_array(pols: Sequence[Dict]):
    arr = (Policy * len(pols))(*[make_policy(p) for p in pols])
    return arr


class ModelHolder:
    """Keeps the ladder array alive for the Model struct that points at it."""

    def __init__(self, d: Dict):
        self.f = np.ascontiguousarray(d["f_ghz"], dtype=np.float64)
        self.m = Model(float(d["dt_s"]), len(self.f), int(d["bytes_per_count"]),
                       self.f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(d["p_static_w"]),
                       float(d["p_dyn_w"]), float(d["f_ref_ghz"]), float(d["bw_ref_gbs"]))


def packed_offsets(lengths) -> tuple:
    """magus_packed_size: (offsets uint64 array, total elements)."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    off = np.zeros(max(len(ln), 1), dtype=np.uint64)
    tot = ctypes.c_uint64()
    check(lib().magus_packed_size(ln.ctypes.data, len(ln), off.ctypes.data, ctypes.byref(tot)))
    return off[:len(ln)], int(tot.value)


def policy_bounds(policy: Dict, model: Dict) -> np.ndarray:
    mh = ModelHolder(model)
    pol = make_policy(policy)
    out = np.zeros(4, dtype=np.int64)
    check(lib().magus_policy_bounds(ctypes.byref(pol), ctypes.byref(mh.m), out.ctypes.data))
    return out


def policy_fp64_thresholds(policy: Dict, model: Dict):
    """magus_policy_fp64_thresholds: (up_last, dn_last) -- +1 iff d > up_last, -1 iff
    d <= dn_last, with d the FP64 throughput difference over W intervals."""
    mh = ModelHolder(model)
    pol = make_policy(policy)
    out = np.zeros(2, dtype=np.float64)
    check(lib().magus_policy_fp64_thresholds(ctypes.byref(pol), ctypes.byref(mh.m), out.ctypes.data))
    return float(out[0]), float(out[1])


def policy_closed_thresholds(policy: Dict, model: Dict) -> np.ndarray:
    """magus_policy_closed_thresholds: 11 int64 (capped-throughput thresholds per level)."""
    mh = ModelHolder(model)
    pol = make_policy(policy)
    out = np.zeros(11, dtype=np.int64)
    check(lib().magus_policy_closed_thresholds(ctypes.byref(pol), ctypes.byref(mh.m), out.ctypes.data))
    return out


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Replay:
    """A replay handle (magus_replay_open / _close) with thin wrappers of the entry points.
    Device buffers are torch tensors on the handle's device; traces are int32/uint32
    tensors in the packed layout."""

    def __init__(self, model: Dict, device: int = 0, mem_budget: int = 0):
        self._mh = ModelHolder(model)
        self.model = model
        self.device = device
        h = ctypes.c_void_p()
        check(lib().magus_replay_open(ctypes.byref(h), ctypes.byref(self._mh.m), device, mem_budget))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().magus_replay_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- output allocation helpers (torch, on the handle's device) ------------------------
    def _outputs(self, n_pairs: int, log_capacity: int, counts: bool, want_time: bool):
        import torch
        dev = torch.device("cuda", self.device)
        out = dict(energy_j=torch.zeros(n_pairs, dtype=torch.float64, device=dev),
                   edp_js=torch.zeros(n_pairs, dtype=torch.float64, device=dev))
        if want_time:
            out["time_s"] = torch.zeros(n_pairs, dtype=torch.float64, device=dev)
        log = None
        if counts or log_capacity:
            log = FreqLog()
            if counts:
                for k in ("n_changes", "change_hash", "n_hf"):
                    out[k] = torch.zeros(n_pairs, dtype=torch.int64, device=dev)
                log.n_changes, log.change_hash, log.n_hf = (out["n_changes"].data_ptr(),
                                                            out["change_hash"].data_ptr(), out["n_hf"].data_ptr())
            if log_capacity:
                out["log"] = torch.zeros(n_pairs * log_capacity, dtype=torch.int32, device=dev)
                log.entries = out["log"].data_ptr()
                log.capacity = log_capacity
        return out, log

    def run(self, traces, lengths, policies: Sequence[Dict], log_capacity: int = 0, counts: bool = True,
            want_time: bool = True, state=None, stream=None, out=None) -> Dict:
        """magus_replay_run.  ``state``: optional uint8 tensor of n_pairs * STATE_BYTES."""
        ln = np.ascontiguousarray(lengths, dtype=np.uint64)
        pols = policy_array(policies)
        n_pairs = len(ln) * len(policies)
        if out is None:
            out, log = self._outputs(n_pairs, log_capacity, counts, want_time)
        else:
            out, log = out
        check(lib().magus_replay_run(self.h, _ptr(traces), ln.ctypes.data, len(ln), ctypes.cast(pols, P),
                                     len(policies), ctypes.byref(log) if log is not None else None,
                                     out["energy_j"].data_ptr(), out["edp_js"].data_ptr(),
                                     _ptr(out.get("time_s")), _ptr(state), _stream(stream)))
        return out

    def alloc(self, n_pairs: int, log_capacity: int = 0, counts: bool = True, want_time: bool = True):
        """Preallocate outputs for repeated run(..., out=...) calls."""
        return self._outputs(n_pairs, log_capacity, counts, want_time)

    def plain(self, traces, lengths, policies: Sequence[Dict], log_capacity: int = 0, counts: bool = True,
              want_time: bool = True, stream=None, out=None) -> Dict:
        ln = np.ascontiguousarray(lengths, dtype=np.uint64)
        pols = policy_array(policies)
        n_pairs = len(ln) * len(policies)
        if out is None:
            out, log = self._outputs(n_pairs, log_capacity, counts, want_time)
        else:
            out, log = out
        check(lib().magus_replay_plain(self.h, _ptr(traces), ln.ctypes.data, len(ln), ctypes.cast(pols, P),
                                       len(policies), ctypes.byref(log) if log is not None else None,
                                       out["energy_j"].data_ptr(), out["edp_js"].data_ptr(),
                                       _ptr(out.get("time_s")), _stream(stream)))
        return out

    def detail(self, trace, n: int, policy: Dict, log_capacity: int = 0, stream=None) -> Dict:
        import torch
        dev = torch.device("cuda", self.device)
        out, log = self._outputs(1, log_capacity, True, True)
        out["level_log"] = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
        out["deriv_log"] = torch.zeros(max(n, 1), dtype=torch.float64, device=dev)
        pol = make_policy(policy)
        check(lib().magus_replay_detail(self.h, _ptr(trace), n, ctypes.byref(pol), out["level_log"].data_ptr(),
                                        out["deriv_log"].data_ptr(), ctypes.byref(log), out["energy_j"].data_ptr(),
                                        out["edp_js"].data_ptr(), out["time_s"].data_ptr(), _stream(stream)))
        return out

    def run_host(self, traces: np.ndarray, lengths, policies: Sequence[Dict], log_capacity: int = 0,
                 counts: bool = True, out: Optional[Dict] = None) -> Dict:
        """magus_replay_run_host: numpy (ideally pinned) host buffers in and out."""
        ln = np.ascontiguousarray(lengths, dtype=np.uint64)
        pols = policy_array(policies)
        n_pairs = len(ln) * len(policies)
        if out is None:
            out = dict(energy_j=np.zeros(n_pairs), edp_js=np.zeros(n_pairs), time_s=np.zeros(n_pairs))
            if counts:
                for k in ("n_changes", "change_hash", "n_hf"):
                    out[k] = np.zeros(n_pairs, dtype=np.uint64)
            if log_capacity:
                out["log"] = np.zeros(n_pairs * log_capacity, dtype=np.uint32)
        log = None
        if "n_changes" in out or "log" in out:
            log = FreqLog()
            if "n_changes" in out:
                log.n_changes, log.change_hash, log.n_hf = (out["n_changes"].ctypes.data,
                                                            out["change_hash"].ctypes.data, out["n_hf"].ctypes.data)
            if "log" in out:
                log.entries = out["log"].ctypes.data
                log.capacity = len(out["log"]) // max(n_pairs, 1)
        check(lib().magus_replay_run_host(self.h, traces.ctypes.data, ln.ctypes.data, len(ln), ctypes.cast(pols, P),
                                          len(policies), ctypes.byref(log) if log is not None else None,
                                          out["energy_j"].ctypes.data, out["edp_js"].ctypes.data,
                                          out["time_s"].ctypes.data if "time_s" in out else None))
        return out

    def status(self, stream=None) -> int:
        return lib().magus_replay_status(self.h, _stream(stream))

    def kernel_time(self, detail: bool = False):
        """(total ms, replays) of the batched replays since the previous call; with detail,
        (total ms, replay-kernel ms, replays, kernels launched)."""
        ms = ctypes.c_double()
        main = ctypes.c_double()
        n = ctypes.c_int32()
        k = ctypes.c_int32()
        check(lib().magus_replay_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(main), ctypes.byref(n),
                                             ctypes.byref(k)))
        if detail:
            return ms.value, main.value, n.value, k.value
        return ms.value, n.value

    def set_segments(self, seg_rounds: int):
        """-1 automatic, 0 tile kernel, > 0 segment kernel with that many rounds per segment."""
        check(lib().magus_replay_set_segments(self.h, seg_rounds))

    def set_wait(self, chunk_wait_ns: int = 0):
        """Limit of the tile kernel's per-chunk copy waits in ns (0: the default 2 s)."""
        check(lib().magus_replay_set_wait(self.h, chunk_wait_ns))

    def set_closed(self, seg_rounds: int = 0, burn_rounds: int = -1):
        """Closed loop in jump mode: 0 automatic segments, > 0 rounds per segment (multiple
        of 64), -1 the literal kernel; burn_rounds -1 automatic."""
        check(lib().magus_replay_set_closed(self.h, seg_rounds, burn_rounds))

    def closed_stats(self):
        """(segments replayed, second replays, final-pass replays, log-pass replays) of the
        last call."""
        out = (ctypes.c_uint64 * 4)()
        check(lib().magus_replay_closed_stats(self.h, out))
        return tuple(int(v) for v in out)

    def set_tile(self, time_groups: int, policy_slots: int):
        check(lib().magus_replay_set_tile(self.h, time_groups, policy_slots))

    def autotune(self, traces, lengths, policies: Sequence[Dict], stream=None):
        ln = np.ascontiguousarray(lengths, dtype=np.uint64)
        pols = policy_array(policies)
        best = (ctypes.c_int32 * 4)()
        ms = ctypes.c_float()
        check(lib().magus_replay_autotune(self.h, _ptr(traces), ln.ctypes.data, len(ln), ctypes.cast(pols, P),
                                          len(policies), ctypes.cast(best, P), ctypes.byref(ms), _stream(stream)))
        return (best[0], best[1], best[2], best[3]), ms.value


def decode_log(entries: np.ndarray):
    """Split FULL-log entries into (interval index t+1, level)."""
    e = np.asarray(entries, dtype=np.uint32)
    return (e >> 5).astype(np.uint64), (e & 31).astype(np.uint8)


class Serve:
    """Serving runtime handle (magus_serve_open / _close) with thin wrappers."""

    def __init__(self, model: Dict, policy: Dict, n_streams: int, mem_budget: int = 0, device: int = 0,
                 max_batch_requests: int = 0, max_batch_samples: int = 0):
        self._mh = ModelHolder(model)
        self._pol = make_policy(policy)
        self.n_streams = n_streams
        h = ctypes.c_void_p()
        check(lib().magus_serve_open(ctypes.byref(h), ctypes.byref(self._mh.m), ctypes.byref(self._pol),
                                     n_streams, mem_budget, device, max_batch_requests, max_batch_samples))
        self.h = h

    def submit(self, stream_id: int, deltas: np.ndarray) -> int:
        d = np.ascontiguousarray(deltas, dtype=np.uint32)
        rid = ctypes.c_uint64()
        check(lib().magus_serve_submit(self.h, stream_id, d.ctypes.data, len(d), ctypes.byref(rid)))
        return rid.value

    def try_submit(self, stream_id: int, deltas: np.ndarray):
        """Returns the request id, or the negative status (e.g. EBUSY) without raising."""
        d = np.ascontiguousarray(deltas, dtype=np.uint32)
        rid = ctypes.c_uint64()
        rc = lib().magus_serve_submit(self.h, stream_id, d.ctypes.data, len(d), ctypes.byref(rid))
        return rid.value if rc == OK else rc

    def poll(self, req_id: int):
        """Result dict, or None while the request is not done (EAGAIN)."""
        r = Result()
        rc = lib().magus_serve_poll(self.h, req_id, ctypes.byref(r))
        if rc == EAGAIN:
            return None
        check(rc)
        return {k: getattr(r, k) for k, _ in Result._fields_ if k != "reserved"}

    def drain(self):
        check(lib().magus_serve_drain(self.h))

    def stats(self) -> Dict:
        st = ServeStats()
        check(lib().magus_serve_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def export(self) -> np.ndarray:
        out = np.zeros(self.n_streams * STATE_BYTES, dtype=np.uint8)
        check(lib().magus_serve_export(self.h, out.ctypes.data))
        return out

    def load(self, arrival_s, stream_id, size, payload, payload_off, results: bool = False):
        """magus_serve_load: (latencies, wall seconds[, per-request result dicts as arrays])."""
        a = np.ascontiguousarray(arrival_s, dtype=np.float64)
        sid = np.ascontiguousarray(stream_id, dtype=np.uint32)
        sz = np.ascontiguousarray(size, dtype=np.uint32)
        pay = np.ascontiguousarray(payload, dtype=np.uint32)
        off = np.ascontiguousarray(payload_off, dtype=np.uint64)
        lat = np.zeros(len(a))
        wall = ctypes.c_double()
        res = (Result * max(len(a), 1))() if results else None
        check(lib().magus_serve_load(self.h, a.ctypes.data, sid.ctypes.data, sz.ctypes.data, pay.ctypes.data,
                                     off.ctypes.data, len(a), lat.ctypes.data, ctypes.byref(wall),
                                     ctypes.cast(res, P) if results else None))
        if not results:
            return lat, wall.value
        arr = np.ctypeslib.as_array(res)[:len(a)]
        return lat, wall.value, {k: np.array(arr[k]) for k, _ in Result._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "h", None):
            lib().magus_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
