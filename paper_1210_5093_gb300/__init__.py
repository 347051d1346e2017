"""GB300 speculative chunked DFA membership test (Ko, Jung, Han & Burgstaller).

Thin ctypes binding over the C ABI in include/dfamatch.h (libdfamatch.so,
built in-tree by ``paper_1210_5093_gb300.build``).  Every step of the
membership test runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch is used for device memory and streams.  There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DFA_DEBUG_BOUNDS=1 loads the build with device-side bounds checks instead
# (libdfamatch_debug.so: the same kernels, every index checked; a failed check
# is reported as DFA_EBOUNDS in the test's result)
DEBUG_BOUNDS = os.environ.get("DFA_DEBUG_BOUNDS", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "libdfamatch_debug.so" if DEBUG_BOUNDS else "libdfamatch.so")

OK, EINVAL, ESYMBOL, ENOMEM, ECUDA, ETIMEOUT, EBUDGET, EAGAIN, ENOSPACE, EHOSTONLY, EBOUNDS = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10

_lib = None


class DfaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = strerror(status) if _lib is not None else str(status)
        super().__init__("%s: %s (%d)" % (what or "dfamatch", msg, status))


class Result(ctypes.Structure):
    _fields_ = [("final_state", ctypes.c_uint32), ("accept", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8 * 3), ("status", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("num_states", ctypes.c_uint32), ("num_symbols", ctypes.c_uint32),
                ("num_states_ext", ctypes.c_uint32), ("num_classes", ctypes.c_uint32),
                ("i_max", ctypes.c_uint32), ("num_excluded", ctypes.c_uint32),
                ("state_bytes", ctypes.c_uint32), ("placement", ctypes.c_uint32),
                ("states_per_thread", ctypes.c_uint32), ("q0", ctypes.c_uint32),
                ("table_bytes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("gamma", ctypes.c_double), ("mean_iset", ctypes.c_double),
                ("byte_rows", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("states_per_thread", ctypes.c_uint32), ("tiles_per_cta", ctypes.c_uint32),
                ("min_chunk_bytes", ctypes.c_uint32), ("batch_chunk_bytes", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("host_segment_bytes", ctypes.c_uint32),
                ("grid_waves", ctypes.c_uint32)]


class MatchOpts(ctypes.Structure):
    _fields_ = [("num_chunks", ctypes.c_uint32), ("multiplicity", ctypes.c_uint32),
                ("lookahead", ctypes.c_uint32), ("boundary_window", ctypes.c_uint32),
                ("match_begin_event", ctypes.c_void_p), ("match_end_event", ctypes.c_void_p)]


class GroupInfo(ctypes.Structure):
    _fields_ = [("num_dfas", ctypes.c_uint32), ("joint_classes", ctypes.c_uint32),
                ("state_bytes", ctypes.c_uint32), ("states_per_thread", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("max_states_ext", ctypes.c_uint32),
                ("sum_max_set", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("table_bytes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64)]


class GroupOpts(ctypes.Structure):
    _fields_ = [("num_chunks", ctypes.c_uint32), ("states_per_thread", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("dev_work", ctypes.c_void_p), ("match_begin_event", ctypes.c_void_p),
                ("match_end_event", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("result", Result), ("submit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("bytes_matched", ctypes.c_uint64), ("bytes_in_flight", ctypes.c_uint64),
                ("max_bytes_in_flight", ctypes.c_uint64), ("max_concurrent", ctypes.c_uint64)]


# name -> (restype, argtypes); the complete exported surface of include/dfamatch.h
_P, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "dfa_create": (_I, [_U32, _U32, _P, _U32, _P, _U32, _P, _P]),
    "dfa_create_host": (_I, [_U32, _U32, _P, _U32, _P, _U32, _P, _P]),
    "dfa_destroy": (None, [_P]),
    "dfa_info": (_I, [_P, _P]),
    "dfa_class_of_bytes": (_I, [_P, _P]),
    "dfa_get_tuning": (_I, [_P, _P]),
    "dfa_set_tuning": (_I, [_P, _P]),
    "dfa_autotune": (_I, [_P, _P, _U64, _P, _P, _P]),
    "dfa_get_tuning_opts": (_I, [_P, _P, _P]),
    "dfa_set_tuning_opts": (_I, [_P, _P, _P]),
    "dfa_autotune_opts": (_I, [_P, _P, _U64, _P, _P, _P, _P]),
    "dfa_iset": (_I, [_P, _U32, _P, _U32, _P]),
    "dfa_partition": (_I, [_U64, _U32, _U32, _P]),
    "dfa_match": (_I, [_P, _P, _U64, _P, _P]),
    "dfa_plan_chunks": (_I, [_P, _U64, _P, _P]),
    "dfa_match_num_kernels": (_I, [_P, _U64, _P, _P]),
    "dfa_plan_sets": (_I, [_P, _P, _U64, _P, _P, _U32, _P]),
    "dfa_plan_starts": (_I, [_P, _P, _U64, _P, _P, _U32, _P]),
    "dfa_debug_chunk_maps": (_I, [_P, _P, _U64, _P, _P, _U32, _P, _P]),
    "dfa_match_workspace_size": (_I, [_P, _U64, _P, _P]),
    "dfa_match_async": (_I, [_P, _P, _U64, _P, _P, _P, _U64, _P]),
    "dfa_match_noalloc": (_I, [_P, _P, _U64, _P, _P, _P]),
    "dfa_noalloc_scratch_bytes": (_U64, []),
    "dfa_probe_lookup_rate": (_I, [_P, _U32, _P, _P]),
    "dfa_match_batch": (_I, [_U32, _P, _P, _P, _P, _P, _P]),
    "dfa_batch_prepare": (_I, [_U32, _P, _P, _P, _P, _P]),
    "dfa_batch_launch": (_I, [_P, _P, _P]),
    "dfa_batch_graph_launch": (_I, [_P, _P, _P]),
    "dfa_batch_num_kernels": (_I, [_P, _P]),
    "dfa_batch_set_events": (_I, [_P, _P, _P]),
    "dfa_batch_destroy": (None, [_P]),
    "dfa_strerror": (ctypes.c_char_p, [_I]),
    "dfa_group_create": (_I, [_P, _U32, _P]),
    "dfa_group_destroy": (None, [_P]),
    "dfa_group_info": (_I, [_P, _P]),
    "dfa_group_joint_classes": (_I, [_P, _P]),
    "dfa_group_autotune": (_I, [_P, _P, _U64, _P, _P, _P, _P]),
    "dfa_group_plan_chunks": (_I, [_P, _U64, _P, _P]),
    "dfa_group_workspace_size": (_I, [_P, _U64, _P, _P]),
    "dfa_group_match_async": (_I, [_P, _P, _U64, _P, _P, _P, _U64, _P]),
    "dfa_group_match": (_I, [_P, _P, _U64, _P, _P]),
    "dfa_group_debug_chunk_maps": (_I, [_P, _P, _U64, _P, _P, _U32, _P, _P]),
    "dfa_server_create": (_I, [_U64, _U32, _P]),
    "dfa_server_set_opts": (_I, [_P, _P]),
    "dfa_server_submit": (_I, [_P, _P, _P, _U64, _P]),
    "dfa_server_poll": (_I, [_P, _P, _U32, _P]),
    "dfa_server_drain": (_I, [_P, ctypes.c_double]),
    "dfa_server_stats": (_I, [_P, _P]),
    "dfa_server_destroy": (None, [_P]),
}


def lib():
    """Load libdfamatch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built; run paper_1210_5093_gb300.build.build()"
                               % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().dfa_strerror(status).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise DfaError(rc, what)


def _opts(num_chunks=0, multiplicity=0, lookahead=1, events=None, boundary_window=0) -> MatchOpts:
    """boundary_window: Sec. 4.2 placement of the chunk starts (0: Eqs. 6-7)."""
    ev = (None, None) if events is None else (events[0].cuda_event, events[1].cuda_event)
    return MatchOpts(int(num_chunks), int(multiplicity), int(lookahead), int(boundary_window),
                     ev[0], ev[1])


def partition(n: int, P: int, m: int = 1) -> np.ndarray:
    """Chunk boundaries of Eqs. (6)-(7) with unit weights (P+1 entries)."""
    out = np.zeros(P + 1, dtype=np.uint64)
    _check(lib().dfa_partition(n, P, m, out.ctypes.data), "dfa_partition")
    return out


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def results_from(buf) -> list:
    """Decode a uint8 tensor/array of 12*count bytes into (final, accept, status) tuples."""
    a = buf.cpu().numpy() if hasattr(buf, "cpu") else np.asarray(buf)
    a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1, 12)
    final = a[:, 0:4].copy().view(np.uint32).ravel()
    acc = a[:, 4]
    st = a[:, 8:12].copy().view(np.int32).ravel()
    return [(int(f), bool(x), int(s)) for f, x, s in zip(final, acc, st)]


class Dfa:
    """A compiled DFA (dfa_t).  delta[q, a] in [0, num_states) or -1 (error state)."""

    def __init__(self, num_states: int, num_symbols: int, delta, q0: int, finals,
                 byte_to_symbol=None, host_only: bool = False):
        L = lib()
        self._delta = np.ascontiguousarray(np.asarray(delta, dtype=np.int32))
        if self._delta.size != num_states * num_symbols:
            raise ValueError("delta must have num_states*num_symbols entries")
        self._finals = np.ascontiguousarray(np.asarray(finals, dtype=np.uint32).ravel())
        self._map = None if byte_to_symbol is None else np.ascontiguousarray(
            np.asarray(byte_to_symbol, dtype=np.uint8))
        self.num_states, self.num_symbols, self.q0 = int(num_states), int(num_symbols), int(q0)
        h = ctypes.c_void_p()
        fn = L.dfa_create_host if host_only else L.dfa_create
        rc = fn(num_states, num_symbols, self._delta.ctypes.data, q0,
                self._finals.ctypes.data if len(self._finals) else None, len(self._finals),
                None if self._map is None else self._map.ctypes.data, ctypes.byref(h))
        _check(rc, "dfa_create")
        self._h = h
        self.host_only = host_only

    @classmethod
    def from_spec(cls, spec, host_only: bool = False) -> "Dfa":
        return cls(spec.num_states, spec.num_symbols, spec.delta, spec.q0, spec.finals,
                   spec.byte_to_symbol, host_only=host_only)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dfa_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> Info:
        out = Info()
        _check(lib().dfa_info(self._h, ctypes.byref(out)), "dfa_info")
        return out

    def tuning(self, lookahead: int = 1, boundary_window: int = 0) -> Tuning:
        """The tuning record used for launches with this lookahead (1: the base
        record) and, with boundary_window > 0, Sec. 4.2 placement."""
        t = Tuning()
        o = _opts(lookahead=lookahead, boundary_window=boundary_window)
        _check(lib().dfa_get_tuning_opts(self._h, ctypes.byref(o), ctypes.byref(t)),
               "dfa_get_tuning_opts")
        return t

    def set_tuning(self, states_per_thread: int = 0, tiles_per_cta: int = 0,
                   min_chunk_bytes: int = 0, batch_chunk_bytes: int = 0, ctas_per_sm: int = 0,
                   host_segment_bytes: int = 0, lookahead: int = 1, boundary_window: int = 0,
                   grid_waves: int = 0):
        """host_segment_bytes: first segment of dfa_match's copy/match pipeline for
        host input (0 = automatic, 0xFFFFFFFF = copy the whole string first).
        lookahead: the depth whose record is set (1: the base record)."""
        t = Tuning(states_per_thread, tiles_per_cta, min_chunk_bytes, batch_chunk_bytes, ctas_per_sm,
                   host_segment_bytes, grid_waves)
        o = _opts(lookahead=lookahead, boundary_window=boundary_window)
        _check(lib().dfa_set_tuning_opts(self._h, ctypes.byref(o), ctypes.byref(t)),
               "dfa_set_tuning_opts")

    def autotune(self, dev_sample, stream=None, lookahead: int = 1, boundary_window: int = 0):
        """Time the candidate tunings on a device sample (launches with this
        lookahead and placement window) and keep the fastest in that record.
        Returns (Tuning, best_ms)."""
        t = Tuning()
        ms = ctypes.c_double()
        n = dev_sample.numel()
        o = _opts(lookahead=lookahead, boundary_window=boundary_window)
        _check(lib().dfa_autotune_opts(self._h, dev_sample.data_ptr() if n else None, n,
                                       ctypes.byref(o), _stream_ptr(stream), ctypes.byref(t),
                                       ctypes.byref(ms)),
               "dfa_autotune_opts")
        return t, float(ms.value)

    def class_of_bytes(self) -> np.ndarray:
        out = np.zeros(256, dtype=np.uint16)
        _check(lib().dfa_class_of_bytes(self._h, out.ctypes.data), "dfa_class_of_bytes")
        return out

    def iset(self, c: int) -> list:
        n = ctypes.c_uint32()
        _check(lib().dfa_iset(self._h, c, None, 0, ctypes.byref(n)), "dfa_iset")
        out = np.zeros(max(1, n.value), dtype=np.uint32)
        _check(lib().dfa_iset(self._h, c, out.ctypes.data, n.value, ctypes.byref(n)), "dfa_iset")
        return out[: n.value].tolist()

    # -------------------------------------------------------------- matching
    def match(self, data, num_chunks: int = 0, multiplicity: int = 0, lookahead: int = 1,
              events=None, boundary_window: int = 0):
        """Synchronous test.  data: bytes / numpy uint8 / a (pinned) CPU tensor, or a
        CUDA uint8 tensor.  Returns (status, final_state, accept)."""
        res = Result()
        o = _opts(num_chunks, multiplicity, lookahead, events, boundary_window)
        if hasattr(data, "data_ptr"):
            ptr, n, keep = data.data_ptr(), data.numel(), data
        else:
            keep = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8)
                                        if isinstance(data, (bytes, bytearray)) else
                                        np.asarray(data, dtype=np.uint8))
            ptr, n = keep.ctypes.data, keep.size
        rc = lib().dfa_match(self._h, ptr if n else None, n, ctypes.byref(o), ctypes.byref(res))
        del keep
        if rc == EBOUNDS:   # debug build: final_state holds the source line of the failed check
            raise DfaError(rc, "dfa_match (check at dfa_kernels.cu line %d)" % res.final_state)
        if rc not in (OK, ESYMBOL):
            raise DfaError(rc, "dfa_match")
        if rc == ESYMBOL:
            return ESYMBOL, None, None
        return OK, int(res.final_state), bool(res.accept)

    def plan_chunks(self, n: int, num_chunks: int = 0, multiplicity: int = 0,
                    lookahead: int = 1, boundary_window: int = 0) -> int:
        out = ctypes.c_uint32()
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        _check(lib().dfa_plan_chunks(self._h, n, ctypes.byref(o), ctypes.byref(out)),
               "dfa_plan_chunks")
        return int(out.value)

    def num_kernels(self, n: int, num_chunks: int = 0, lookahead: int = 1,
                    boundary_window: int = 0) -> int:
        out = ctypes.c_uint32()
        o = _opts(num_chunks, 0, lookahead, None, boundary_window)
        _check(lib().dfa_match_num_kernels(self._h, n, ctypes.byref(o), ctypes.byref(out)),
               "dfa_match_num_kernels")
        return int(out.value)

    def chunk_maps(self, dev_data, num_chunks: int = 0, lookahead: int = 1,
                   boundary_window: int = 0):
        """(L maps [P, |Q|+1] uint16, final_state): the chunk maps of Sec. 4.1 as the
        match kernel computed them (identity outside each chunk's I_k)."""
        o = _opts(num_chunks, 0, lookahead, None, boundary_window)
        n = dev_data.numel()
        P = ctypes.c_uint32()
        ptr = dev_data.data_ptr() if n else None
        _check(lib().dfa_debug_chunk_maps(self._h, ptr, n, ctypes.byref(o), None, 0, ctypes.byref(P),
                                          None), "dfa_debug_chunk_maps")
        qe = self.num_states + 1
        out = np.zeros((P.value, qe), dtype=np.uint16)
        fs = ctypes.c_uint32()
        _check(lib().dfa_debug_chunk_maps(self._h, ptr, n, ctypes.byref(o), out.ctypes.data, P.value,
                                          ctypes.byref(P), ctypes.byref(fs)), "dfa_debug_chunk_maps")
        return out, int(fs.value)

    def plan_sets(self, dev_data, num_chunks: int = 0, multiplicity: int = 0,
                  lookahead: int = 1, boundary_window: int = 0) -> np.ndarray:
        """|I_k| of every chunk of a single test on dev_data (planning kernels only)."""
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        n = dev_data.numel()
        P = ctypes.c_uint32()
        _check(lib().dfa_plan_sets(self._h, dev_data.data_ptr() if n else None, n, ctypes.byref(o),
                                   None, 0, ctypes.byref(P)), "dfa_plan_sets")
        out = np.zeros(max(1, P.value), dtype=np.uint32)
        _check(lib().dfa_plan_sets(self._h, dev_data.data_ptr() if n else None, n, ctypes.byref(o),
                                   out.ctypes.data, P.value, ctypes.byref(P)), "dfa_plan_sets")
        return out[: P.value]

    def plan_starts(self, dev_data, num_chunks: int = 0, multiplicity: int = 0,
                    lookahead: int = 1, boundary_window: int = 0) -> np.ndarray:
        """Chunk boundaries [0, start_1, ..., start_{P-1}, n] of a single test on
        dev_data: Eqs. (6)-(7), or the Sec. 4.2 placement with boundary_window."""
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        n = dev_data.numel()
        ptr = dev_data.data_ptr() if n else None
        P = ctypes.c_uint32()
        _check(lib().dfa_plan_starts(self._h, ptr, n, ctypes.byref(o), None, 0, ctypes.byref(P)),
               "dfa_plan_starts")
        out = np.zeros(P.value + 1, dtype=np.uint64)
        _check(lib().dfa_plan_starts(self._h, ptr, n, ctypes.byref(o), out.ctypes.data, P.value + 1,
                                     ctypes.byref(P)), "dfa_plan_starts")
        return out

    def workspace_size(self, n: int, num_chunks: int = 0, multiplicity: int = 0,
                       lookahead: int = 1, boundary_window: int = 0) -> int:
        out = ctypes.c_uint64()
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        _check(lib().dfa_match_workspace_size(self._h, n, ctypes.byref(o), ctypes.byref(out)),
               "dfa_match_workspace_size")
        return int(out.value)

    def match_async(self, dev_data, dev_out, workspace, stream=None, num_chunks: int = 0,
                    multiplicity: int = 0, lookahead: int = 1, events=None,
                    boundary_window: int = 0):
        """Enqueue a test on `stream` (torch stream; default: current).  dev_data: CUDA
        uint8 tensor; dev_out: CUDA uint8 tensor of >= 12 bytes; workspace: CUDA uint8
        tensor of >= workspace_size() bytes; events: optional (begin, end) torch.cuda.Event
        pair recorded around the match kernel."""
        o = _opts(num_chunks, multiplicity, lookahead, events, boundary_window)
        n = dev_data.numel()
        rc = lib().dfa_match_async(self._h, dev_data.data_ptr() if n else None, n, ctypes.byref(o),
                                   dev_out.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                   _stream_ptr(stream))
        _check(rc, "dfa_match_async")

    def match_noalloc(self, dev_data, dev_out, stream=None, num_chunks: int = 0,
                      multiplicity: int = 0, lookahead: int = 1, boundary_window: int = 0):
        """Enqueue a test that uses the library's fixed scratch array instead of a
        workspace (see dfa_match_noalloc: calls sharing a device must not overlap)."""
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        n = dev_data.numel()
        rc = lib().dfa_match_noalloc(self._h, dev_data.data_ptr() if n else None, n,
                                     ctypes.byref(o), dev_out.data_ptr(), _stream_ptr(stream))
        _check(rc, "dfa_match_noalloc")


def probe_lookup_rate(dfa: "Dfa", steps: int = 4096, stream=None) -> float:
    """Lookups per second of one dependent table lookup on dfa's own table and
    placement (dfa_probe_lookup_rate)."""
    r = ctypes.c_double()
    _check(lib().dfa_probe_lookup_rate(dfa.handle, steps, _stream_ptr(stream), ctypes.byref(r)),
           "dfa_probe_lookup_rate")
    return float(r.value)


def noalloc_scratch_bytes() -> int:
    return int(lib().dfa_noalloc_scratch_bytes())


def _ptr_array(vals):
    arr = (ctypes.c_void_p * len(vals))(*[ctypes.c_void_p(int(v)) for v in vals])
    return arr


class Batch:
    """A prepared batch of membership tests (dfa_batch_t): planned once, launched
    many times as one persistent launch (optionally replayed from a CUDA graph)."""

    def __init__(self, dfas: Sequence[Dfa], tensors, num_chunks: int = 0, multiplicity: int = 0,
                 lookahead: int = 1, boundary_window: int = 0):
        self._dfas = list(dfas)
        self._tensors = list(tensors)
        n = len(self._tensors)
        dp = _ptr_array([d.handle.value for d in self._dfas])
        sp = _ptr_array([t.data_ptr() if t.numel() else 0 for t in self._tensors])
        lens = np.array([t.numel() for t in self._tensors], dtype=np.uint64)
        o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
        h = ctypes.c_void_p()
        _check(lib().dfa_batch_prepare(n, dp, sp, lens.ctypes.data, ctypes.byref(o),
                                       ctypes.byref(h)), "dfa_batch_prepare")
        self._h = h
        self.count = n

    def launch(self, dev_out, stream=None, graph: bool = False):
        fn = lib().dfa_batch_graph_launch if graph else lib().dfa_batch_launch
        _check(fn(self._h, dev_out.data_ptr(), _stream_ptr(stream)), "dfa_batch_launch")

    def set_events(self, events):
        ev = (None, None) if events is None else (events[0].cuda_event, events[1].cuda_event)
        _check(lib().dfa_batch_set_events(self._h, ev[0], ev[1]), "dfa_batch_set_events")

    def num_kernels(self) -> int:
        n = ctypes.c_uint32()
        _check(lib().dfa_batch_num_kernels(self._h, ctypes.byref(n)), "dfa_batch_num_kernels")
        return int(n.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dfa_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match_batch(dfas: Sequence[Dfa], tensors, stream=None, num_chunks: int = 0,
                multiplicity: int = 0, lookahead: int = 1, boundary_window: int = 0):
    """One-shot batched test through dfa_match_batch; returns (final, accept, status) tuples."""
    torch = _torch()
    n = len(tensors)
    out = torch.zeros(12 * n, dtype=torch.uint8, device="cuda")
    dp = _ptr_array([d.handle.value for d in dfas])
    sp = _ptr_array([t.data_ptr() if t.numel() else 0 for t in tensors])
    lens = np.array([t.numel() for t in tensors], dtype=np.uint64)
    o = _opts(num_chunks, multiplicity, lookahead, None, boundary_window)
    _check(lib().dfa_match_batch(n, dp, sp, lens.ctypes.data, ctypes.byref(o), out.data_ptr(),
                                 _stream_ptr(stream)), "dfa_match_batch")
    return results_from(out)


def _gopts(num_chunks=0, states_per_thread=0, ctas_per_sm=0, work=None, events=None) -> GroupOpts:
    ev = (None, None) if events is None else (events[0].cuda_event, events[1].cuda_event)
    return GroupOpts(int(num_chunks), int(states_per_thread), int(ctas_per_sm), 0,
                     None if work is None else work.data_ptr(), ev[0], ev[1])


class Group:
    """Several DFAs matched together on one input, the input staged once for
    all of them (dfa_group_t).  The Dfa objects are kept alive with the group."""

    def __init__(self, dfas: Sequence[Dfa]):
        self._dfas = list(dfas)
        dp = _ptr_array([d.handle.value for d in self._dfas])
        h = ctypes.c_void_p()
        _check(lib().dfa_group_create(dp, len(self._dfas), ctypes.byref(h)), "dfa_group_create")
        self._h = h
        self.count = len(self._dfas)

    def info(self) -> GroupInfo:
        out = GroupInfo()
        _check(lib().dfa_group_info(self._h, ctypes.byref(out)), "dfa_group_info")
        return out

    def joint_classes(self) -> np.ndarray:
        out = np.zeros(256, dtype=np.uint16)
        _check(lib().dfa_group_joint_classes(self._h, out.ctypes.data), "dfa_group_joint_classes")
        return out

    def autotune(self, dev_sample, stream=None):
        """Time the candidate K and CTAs per SM on a device sample and keep the
        fastest as the group's default.  Returns (K, ctas_per_sm, best_ms)."""
        K, c, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
        n = dev_sample.numel()
        _check(lib().dfa_group_autotune(self._h, dev_sample.data_ptr() if n else None, n,
                                        _stream_ptr(stream), ctypes.byref(K), ctypes.byref(c),
                                        ctypes.byref(ms)), "dfa_group_autotune")
        return int(K.value), int(c.value), float(ms.value)

    def plan_chunks(self, n: int, num_chunks: int = 0, states_per_thread: int = 0,
                    ctas_per_sm: int = 0) -> int:
        P = ctypes.c_uint32()
        o = _gopts(num_chunks, states_per_thread, ctas_per_sm)
        _check(lib().dfa_group_plan_chunks(self._h, n, ctypes.byref(o), ctypes.byref(P)),
               "dfa_group_plan_chunks")
        return int(P.value)

    def workspace_size(self, n: int, num_chunks: int = 0, states_per_thread: int = 0,
                       ctas_per_sm: int = 0) -> int:
        out = ctypes.c_uint64()
        o = _gopts(num_chunks, states_per_thread, ctas_per_sm)
        _check(lib().dfa_group_workspace_size(self._h, n, ctypes.byref(o), ctypes.byref(out)),
               "dfa_group_workspace_size")
        return int(out.value)

    def match_async(self, dev_data, dev_out, workspace, stream=None, num_chunks: int = 0,
                    states_per_thread: int = 0, ctas_per_sm: int = 0, work=None, events=None):
        """Enqueue the group's tests on dev_data (CUDA uint8 tensor); dev_out: CUDA
        uint8 tensor of >= 12*count bytes; work: optional CUDA int64 tensor that
        receives the launch's lookups; events: optional (begin, end) pair."""
        o = _gopts(num_chunks, states_per_thread, ctas_per_sm, work, events)
        n = dev_data.numel()
        _check(lib().dfa_group_match_async(self._h, dev_data.data_ptr() if n else None, n,
                                           ctypes.byref(o), dev_out.data_ptr(), workspace.data_ptr(),
                                           workspace.numel(), _stream_ptr(stream)),
               "dfa_group_match_async")

    def match(self, data, num_chunks: int = 0, states_per_thread: int = 0,
              ctas_per_sm: int = 0) -> list:
        """Synchronous (dfa_group_match): data is bytes / numpy uint8 / a (pinned)
        CPU tensor, or a CUDA uint8 tensor.  One (status, final_state, accept)
        per DFA, in order (final_state and accept are None for a failed test)."""
        if hasattr(data, "data_ptr"):
            ptr, n, keep = data.data_ptr(), data.numel(), data
            if data.is_cuda:   # the call runs on the legacy default stream
                _torch().cuda.current_stream().synchronize()
        else:
            keep = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8)
                                        if isinstance(data, (bytes, bytearray)) else
                                        np.asarray(data, dtype=np.uint8))
            ptr, n = keep.ctypes.data, keep.size
        out = (Result * self.count)()
        o = _gopts(num_chunks, states_per_thread, ctas_per_sm)
        _check(lib().dfa_group_match(self._h, ptr if n else None, n, ctypes.byref(o), out),
               "dfa_group_match")
        del keep
        res = []
        for r in out:
            f, a, st = int(r.final_state), bool(r.accept), int(r.status)
            if st == EBOUNDS:
                raise DfaError(st, "dfa_group_match (check at dfa_group.cu line %d)" % f)
            res.append((st, f, a) if st == OK else (st, None, None))
        return res

    def chunk_maps(self, dev_data, num_chunks: int = 0, states_per_thread: int = 0):
        """(maps [count, P, max_states_ext] uint16, final states): every DFA's
        chunk maps L_k as the match kernel computed them."""
        o = _gopts(num_chunks, states_per_thread)
        n = dev_data.numel()
        ptr = dev_data.data_ptr() if n else None
        P = ctypes.c_uint32()
        _check(lib().dfa_group_debug_chunk_maps(self._h, ptr, n, ctypes.byref(o), None, 0,
                                                ctypes.byref(P), None), "dfa_group_debug_chunk_maps")
        stride = self.info().max_states_ext
        out = np.zeros((self.count, P.value, stride), dtype=np.uint16)
        fs = np.zeros(self.count, dtype=np.uint32)
        _check(lib().dfa_group_debug_chunk_maps(self._h, ptr, n, ctypes.byref(o), out.ctypes.data,
                                                P.value, ctypes.byref(P), fs.ctypes.data),
               "dfa_group_debug_chunk_maps")
        return out, fs

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dfa_group_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (dfa_server_t)."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 8, lookahead: int = 1,
                 boundary_window: int = 0):
        h = ctypes.c_void_p()
        _check(lib().dfa_server_create(hbm_budget_bytes, max_inflight, ctypes.byref(h)),
               "dfa_server_create")
        self._h = h
        self._keep = {}
        if lookahead != 1 or boundary_window:
            self.set_opts(lookahead, boundary_window)

    def set_opts(self, lookahead: int = 1, boundary_window: int = 0):
        """Lookahead depth and Sec. 4.2 placement window of the batches formed from now on."""
        o = _opts(lookahead=lookahead, boundary_window=boundary_window)
        _check(lib().dfa_server_set_opts(self._h, ctypes.byref(o)), "dfa_server_set_opts")

    def submit(self, dfa: Dfa, host_data: np.ndarray) -> int:
        """host_data must stay alive until its completion is polled (kept here)."""
        t = ctypes.c_uint64()
        buf = host_data
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        n = buf.numel() if hasattr(buf, "numel") else buf.size
        _check(lib().dfa_server_submit(self._h, dfa.handle, ptr if n else None, n,
                                       ctypes.byref(t)), "dfa_server_submit")
        self._keep[int(t.value)] = buf
        return int(t.value)

    def poll(self, max_n: int = 1024) -> list:
        arr = (Completion * max_n)()
        n = ctypes.c_uint32()
        _check(lib().dfa_server_poll(self._h, arr, max_n, ctypes.byref(n)), "dfa_server_poll")
        out = []
        for i in range(n.value):
            c = arr[i]
            self._keep.pop(int(c.ticket), None)
            out.append((int(c.ticket), int(c.result.final_state), bool(c.result.accept),
                        int(c.result.status), float(c.submit_s), float(c.done_s)))
        return out

    def drain(self, timeout_s: float = 600.0):
        _check(lib().dfa_server_drain(self._h, timeout_s), "dfa_server_drain")

    def stats(self) -> ServerStats:
        s = ServerStats()
        _check(lib().dfa_server_stats(self._h, ctypes.byref(s)), "dfa_server_stats")
        return s

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dfa_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
