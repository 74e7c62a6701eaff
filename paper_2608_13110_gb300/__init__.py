"""GB300 (sm_103a) temporal-boundary sweep for exact amplitudes of open 1D
brickwork circuits (arXiv 2608.13110, Sec. 3.1, Algorithm 1).

Thin ctypes binding over ``libtbsweep.so`` (C-ABI in ``include/tbsweep.h``):
argument marshalling only, every step of the sweep runs in the library's CUDA
kernels. PyTorch supplies device memory and streams. There is no CPU
fallback: if the library is missing, importing this package raises.

Usage::

    import paper_2608_13110_gb300 as tb
    plan = tb.Plan(n, d, cliff, tmask)          # host planner (no GPU needed)
    amps = plan.amplitudes(bits)                # host in / host out, complex128
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtbsweep.so")

TB_OK, TB_EINVAL, TB_EDOMAIN, TB_ENOMEM, TB_ECUDA, TB_ETIMEOUT = range(6)

class _Gate1q(ctypes.Structure):
    _fields_ = [("qubit", ctypes.c_int32), ("slot", ctypes.c_int32), ("m", ctypes.c_double * 8)]


class _Opts(ctypes.Structure):
    _fields_ = [("window_bits", ctypes.c_int32), ("bottom_bits", ctypes.c_int32),
                ("top_bits", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("d", ctypes.c_int32), ("width", ctypes.c_int32),
                ("boundary_bits", ctypes.c_int32), ("log2_cost", ctypes.c_double),
                ("boundary_bytes", ctypes.c_int64), ("n_steps", ctypes.c_int32),
                ("n_passes", ctypes.c_int32), ("table_bytes", ctypes.c_int64),
                ("open_k", ctypes.c_int32), ("open_width", ctypes.c_int32),
                ("pass_madds", ctypes.c_int32)]


_vp = ctypes.c_void_p
_u8p = ctypes.POINTER(ctypes.c_uint8)
_dp = ctypes.POINTER(ctypes.c_double)
_sig = {
    "tb_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, _u8p, ctypes.POINTER(_Gate1q),
                                      ctypes.c_int, ctypes.POINTER(_Opts), ctypes.POINTER(_vp)]),
    "tb_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(_Info)]),
    "tb_workspace_bytes": (ctypes.c_int64, [_vp, ctypes.c_int64]),
    "tb_workspace_min_bytes": (ctypes.c_int64, [_vp]),
    "tb_plan_upload": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    "tb_amplitudes_device": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp, _vp]),
    "tb_amplitudes": (ctypes.c_int, [_vp, _u8p, ctypes.c_int64, _vp, ctypes.c_int64, _dp, _vp]),
    "tb_amplitudes_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp]),
    "tb_plan_schedule": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]),
    "tb_batch_workspace_bytes": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int]),
    "tb_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _vp, ctypes.c_int64, ctypes.c_int, _vp,
                                       ctypes.POINTER(_vp)]),
    "tb_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "tb_batch_destroy": (None, [_vp]),
    "tb_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_vp)]),
    "tb_server_submit": (ctypes.c_int, [_vp, _vp, _u8p, ctypes.c_int64, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "tb_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]),
    "tb_server_stats": (ctypes.c_int, [_vp, ctypes.c_void_p]),
    "tb_server_destroy": (None, [_vp]),
    "tb_profile_begin": (ctypes.c_int, []),
    "tb_profile_end": (ctypes.c_int, [ctypes.c_void_p]),
    "tb_log_xeb": (ctypes.c_int, [_dp, ctypes.c_int64, ctypes.c_int, _dp]),
    "tb_log_xeb_device": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int, _vp, _vp]),
    "tb_clifford_matrix": (ctypes.c_int, [ctypes.c_int, _dp]),
    "tb_plan_destroy": (None, [_vp]),
    "tb_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tb_last_error": (ctypes.c_char_p, []),
    "tb_device_faults": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "tb_selftest_bounded_wait": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "tb_plan_create_open": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, _u8p, ctypes.POINTER(_Gate1q),
                                           ctypes.c_int, ctypes.POINTER(_Opts), ctypes.c_int,
                                           ctypes.POINTER(_vp)]),
    "tb_plan_create_cphase": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u8p, _u8p, ctypes.POINTER(_Gate1q),
                                             ctypes.c_int, _dp, ctypes.POINTER(_Opts), ctypes.c_int,
                                             ctypes.POINTER(_vp)]),
    "tb_batched_sample": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int64, _dp,
                                         ctypes.POINTER(ctypes.c_int32), _dp]),
}

class _Lib:
    """The CUDA library, loaded on first use. A missing library is an error:
    there is no CPU fallback."""

    def __init__(self):
        self._dll = None

    def _load(self):
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2608_13110_gb300.build` "
                "(there is no CPU fallback)")
        dll = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _sig.items():
            f = getattr(dll, name)
            f.restype = res
            f.argtypes = args
        self._dll = dll

    def __getattr__(self, name):
        if self._dll is None:
            self._load()
        return getattr(self._dll, name)


_lib = _Lib()

EXPORTED = tuple(_sig)


class TbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.tb_last_error().decode() or _lib.tb_status_str(status).decode()
        super().__init__(f"{where}: {_lib.tb_status_str(status).decode()} ({msg})")


def _check(rc: int, where: str) -> None:
    if rc != TB_OK:
        raise TbError(rc, where)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


PRECISIONS = {"fp32": 0, "tf32x3": 1, "bf16x3": 2}


def _precision_code(p) -> int:
    """Pass arithmetic: "fp32" (FMA staircase), "tf32x3" or "bf16x3"
    (tensor-core dense blocks, three split products), or the integer code."""
    if isinstance(p, str):
        if p not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        return PRECISIONS[p]
    return int(p)


def batched_sample(amps, u):
    """Batched sampling (Sec. 4): amps (na, 2^k) complex from an open plan and
    uniform variates u (na,) in [0, 1) -> (suffix indices b (na,), Q_a (na,))."""
    a = np.ascontiguousarray(np.asarray(amps, np.complex128))
    if a.ndim == 1:
        a = a.reshape(1, -1)
    na, B = a.shape
    k = int(B).bit_length() - 1
    if 1 << k != B:
        raise ValueError("rows must hold 2^k amplitudes")
    uu = np.ascontiguousarray(np.asarray(u, np.float64).reshape(-1))
    if uu.size != na:
        raise ValueError("one uniform variate per prefix")
    b = np.empty(na, np.int32)
    q = np.empty(na, np.float64)
    av = a.view(np.float64)
    _check(_lib.tb_batched_sample(av.ctypes.data_as(_dp), k, na, uu.ctypes.data_as(_dp),
                                  b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), q.ctypes.data_as(_dp)),
           "tb_batched_sample")
    return b, q


def sample(plan, n_samples: int, rng, ws=None):
    """Batched sampling (Sec. 4) with an open plan (``open_k = k``): draw
    n_samples uniform prefixes a in {0,1}^(n-k), evaluate the 2^k
    amplitudes of each on the device (one sweep per prefix), and draw one
    suffix b per prefix from p(b | a) = |<a,b|U|0^n>|^2 / Q_a. ``rng`` is a
    numpy Generator (the prefixes and the uniform variates come from it).
    Returns (bitstrings (n_samples, n) uint8 with x_q = bits[:, q],
    their amplitudes (n_samples,), Q_a (n_samples,))."""
    k = plan.open_k
    if k <= 0:
        raise ValueError("batched sampling needs an open plan (open_k > 0)")
    prefixes = rng.integers(0, 2, size=(int(n_samples), plan.n - k), dtype=np.uint8)
    amps = plan.amplitudes(prefixes, ws=ws)
    b, q = batched_sample(amps, rng.random(int(n_samples)))
    bits = np.zeros((int(n_samples), plan.n), np.uint8)
    bits[:, : plan.n - k] = prefixes
    for j in range(k):
        bits[:, plan.n - k + j] = (b >> j) & 1
    return bits, amps[np.arange(int(n_samples)), b], q


def selftest_bounded_wait() -> int:
    """Run a small evaluation whose device waits are made to run out on
    purpose (see tb_selftest_bounded_wait); returns how many gave up."""
    c = ctypes.c_int32()
    _check(_lib.tb_selftest_bounded_wait(ctypes.byref(c)), "tb_selftest_bounded_wait")
    return int(c.value)


def device_faults() -> int:
    """Bounded device waits that gave up since the last call (and clear)."""
    c = ctypes.c_int32()
    _check(_lib.tb_device_faults(ctypes.byref(c)), "tb_device_faults")
    return int(c.value)


class Plan:
    """A planned circuit: folded gates, step tables and pass schedule.

    cliff: (d+1, n) Clifford indices (None = identity); tmask: (d, n) 0/1
    (None = no T); extra: iterable of (qubit, slot, 2x2 complex matrix);
    cphase: None (CZ entanglers) or (d, n-1) angles, cphase[l, i] the
    controlled phase diag(1, 1, 1, e^(i phi)) on (i, i+1) in layer l."""

    def __init__(self, n: int, d: int, cliff=None, tmask=None, extra=None, *,
                 window_bits: int = 0, bottom_bits: int = 0, top_bits: int = 0,
                 hbm_budget_bytes: int = 0, precision=0, open_k: int = 0, cphase=None):
        self.n, self.d = int(n), int(d)
        self._cliff = None if cliff is None else _u8(cliff).reshape(-1)
        self._tmask = None if tmask is None else _u8(tmask).reshape(-1)
        if self._cliff is not None and self._cliff.size != (d + 1) * n:
            raise ValueError("cliff must have (d+1)*n entries")
        if self._tmask is not None and self._tmask.size != d * n:
            raise ValueError("tmask must have d*n entries")
        ex = list(extra or [])
        arr = (_Gate1q * max(1, len(ex)))()
        for i, (q, t, m) in enumerate(ex):
            m = np.asarray(m, np.complex128).reshape(2, 2)
            arr[i].qubit, arr[i].slot = int(q), int(t)
            for k, z in enumerate(m.reshape(-1)):
                arr[i].m[2 * k] = z.real
                arr[i].m[2 * k + 1] = z.imag
        opts = _Opts(window_bits, bottom_bits, top_bits, _precision_code(precision), hbm_budget_bytes)
        self.precision = _precision_code(precision)
        h = _vp()
        cp = None if self._cliff is None else self._cliff.ctypes.data_as(_u8p)
        tp = None if self._tmask is None else self._tmask.ctypes.data_as(_u8p)
        self.open_k = int(open_k)
        if cphase is not None:
            ph = np.ascontiguousarray(np.asarray(cphase, np.float64).reshape(-1))
            if ph.size != self.d * max(self.n - 1, 0):
                raise ValueError("cphase must have d*(n-1) entries")
            self._cphase = ph
            _check(_lib.tb_plan_create_cphase(self.n, self.d, cp, tp, arr if ex else None, len(ex),
                                              ph.ctypes.data_as(_dp), ctypes.byref(opts), self.open_k,
                                              ctypes.byref(h)), "tb_plan_create_cphase")
        elif self.open_k:
            _check(_lib.tb_plan_create_open(self.n, self.d, cp, tp, arr if ex else None, len(ex),
                                            ctypes.byref(opts), self.open_k, ctypes.byref(h)),
                   "tb_plan_create_open")
        else:
            _check(_lib.tb_plan_create(self.n, self.d, cp, tp, arr if ex else None, len(ex),
                                       ctypes.byref(opts), ctypes.byref(h)), "tb_plan_create")
        self._h = h

    @classmethod
    def from_circuit(cls, circ, **kw) -> "Plan":
        return cls(circ.n, circ.d, circ.cliff, circ.tmask, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.tb_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def info(self) -> dict:
        inf = _Info()
        _check(_lib.tb_plan_info(self._h, ctypes.byref(inf)), "tb_plan_info")
        return {f: getattr(inf, f) for f, _ in _Info._fields_}

    PASS_SHAPES = ("fwd", "rev", "top", "bot", "bot_start", "bot_end", "top_end", "tensor")

    @property
    def schedule(self) -> list:
        """[(shape, window_bits, low_address_bit)] for every HBM pass."""
        npass = _lib.tb_plan_schedule(self._h, None, 0)
        buf = (ctypes.c_int32 * max(1, 3 * npass))()
        _lib.tb_plan_schedule(self._h, buf, npass)
        return [(self.PASS_SHAPES[buf[3 * i]], buf[3 * i + 1], buf[3 * i + 2]) for i in range(npass)]

    def workspace_bytes(self, nb: int) -> int:
        v = _lib.tb_workspace_bytes(self._h, int(nb))
        if v < 0:
            raise ValueError("bad nb")
        return int(v)

    def workspace_min_bytes(self) -> int:
        return int(_lib.tb_workspace_min_bytes(self._h))

    def alloc_workspace(self, nb: int, device="cuda"):
        import torch
        return torch.empty(self.workspace_bytes(nb), dtype=torch.uint8, device=device)

    def upload(self, ws, stream=None) -> None:
        _check(_lib.tb_plan_upload(self._h, ws.data_ptr(), ws.numel(), _stream_handle(stream)),
               "tb_plan_upload")

    def amplitudes_device(self, d_bits, ws, d_out, stream=None) -> None:
        """Enqueue the sweep: d_bits (nb, n) uint8 and d_out (nb, 2) float64 are
        CUDA tensors; ``ws`` must hold this plan's tables (``upload``)."""
        nb = d_bits.shape[0] if d_bits.dim() > 1 else d_bits.numel() // self.row_bytes
        _check(_lib.tb_amplitudes_device(self._h, d_bits.data_ptr(), nb, ws.data_ptr(), ws.numel(),
                                         d_out.data_ptr(), _stream_handle(stream)),
               "tb_amplitudes_device")

    def amplitudes_noalloc(self, d_bits, d_out, stream=None) -> None:
        """Like ``amplitudes_device`` but with the library's fixed scratch
        instead of a workspace (no device allocation; see tb_amplitudes_noalloc
        in include/tbsweep.h for its size limit and sharing rules)."""
        nb = d_bits.shape[0] if d_bits.dim() > 1 else d_bits.numel() // self.n
        _check(_lib.tb_amplitudes_noalloc(self._h, d_bits.data_ptr(), nb, d_out.data_ptr(),
                                          _stream_handle(stream)), "tb_amplitudes_noalloc")

    @property
    def row_bytes(self) -> int:
        """Bytes of one input row: a bitstring (n), or an open plan's prefix (n - k)."""
        return self.n - self.open_k

    def amplitudes(self, bits, ws=None, stream=None, out=None) -> np.ndarray:
        """Host bitstrings (nb, n) -> host complex128 amplitudes (nb,);
        synchronous. For an open plan the rows are prefixes (nb, n - k) and
        the result is (nb, 2^k): entry [i, y] = <a_i, b|U|0^n>,
        y = sum_j b_j 2^j."""
        b = _u8(bits)
        if b.ndim == 1:
            b = b.reshape(1, -1)
        nb = b.shape[0]
        na = 1 << self.open_k
        if out is None:
            out = np.empty((nb * na, 2), np.float64)
        if ws is None:
            ws = self.alloc_workspace(nb)
        _check(_lib.tb_amplitudes(self._h, b.ctypes.data_as(_u8p), nb, ws.data_ptr(), ws.numel(),
                                  out.ctypes.data_as(_dp), _stream_handle(stream)), "tb_amplitudes")
        z = out.view(np.complex128).reshape(-1)
        return z.reshape(nb, na) if self.open_k else z


class _BatchItem(ctypes.Structure):
    _fields_ = [("plan", _vp), ("d_bits", _vp), ("nb", ctypes.c_int64), ("d_out", _vp)]


class Batch:
    """Many circuits recorded into one CUDA graph (tb_batch_* in the C-ABI).

    items: list of (Plan, d_bits, d_out) with d_bits (nb, n) uint8 and d_out
    (nb, 2) float64 CUDA tensors; the tensors and plans must stay alive and
    keep their storage while the batch exists. ``launch()`` replays it."""

    def __init__(self, items, nbranches: int = 0, stream=None):
        import torch
        self._keep = list(items)
        arr = (_BatchItem * len(items))()
        for i, (plan, d_bits, d_out) in enumerate(items):
            nb = d_bits.shape[0] if d_bits.dim() > 1 else d_bits.numel() // plan.n
            arr[i].plan = plan.handle.value
            arr[i].d_bits = d_bits.data_ptr()
            arr[i].nb = nb
            arr[i].d_out = d_out.data_ptr()
        self._arr = arr
        need = _lib.tb_batch_workspace_bytes(ctypes.byref(arr), len(items))
        if need < 0:
            raise ValueError("bad batch item")
        dev = items[0][1].device
        self.ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
        h = _vp()
        _check(_lib.tb_batch_create(ctypes.byref(arr), len(items), self.ws.data_ptr(), self.ws.numel(),
                                    int(nbranches), _stream_handle(stream), ctypes.byref(h)), "tb_batch_create")
        self._h = h

    def launch(self, stream=None) -> None:
        _check(_lib.tb_batch_launch(self._h, _stream_handle(stream)), "tb_batch_launch")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.tb_batch_destroy(h)
            self._h = None


class _ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32), ("device", ctypes.c_int32),
                ("pinned_bytes", ctypes.c_int64)]


class _ReqStats(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double), ("run_s", ctypes.c_double),
                ("status", ctypes.c_int32), ("slot", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("amplitudes", ctypes.c_int64), ("peak_concurrent", ctypes.c_int64),
                ("peak_bytes_in_use", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("mean_latency_s", ctypes.c_double)]


class Server:
    """Amplitude server (tb_server_* in the C-ABI): resident plan tables, an
    HBM budget allocated once, ``slots`` requests running concurrently and
    queued requests admitted as slots and memory free up."""

    def __init__(self, hbm_budget_bytes: int = 16 << 30, slots: int = 4, device: int = 0,
                 pinned_bytes: int = 64 << 20):
        o = _ServerOpts(int(hbm_budget_bytes), int(slots), int(device), int(pinned_bytes))
        h = _vp()
        _check(_lib.tb_server_create(ctypes.byref(o), ctypes.byref(h)), "tb_server_create")
        self._h = h
        self._pending = {}

    def submit(self, plan: "Plan", bits) -> int:
        b = _u8(bits)
        if b.ndim == 1:
            b = b.reshape(1, -1)
        out = np.empty((b.shape[0], 2), np.float64)
        t = ctypes.c_int64(0)
        _check(_lib.tb_server_submit(self._h, plan.handle, b.ctypes.data_as(_u8p), b.shape[0],
                                     out.ctypes.data_as(_dp), ctypes.byref(t)), "tb_server_submit")
        self._pending[t.value] = (plan, out)
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0):
        """(complex128 amplitudes, {latency_s, queue_s, run_s, slot})."""
        st = _ReqStats()
        st.status = -1  # left as is while the request is still running
        rc = _lib.tb_server_wait(self._h, ticket, float(timeout), ctypes.byref(st))
        if rc == TB_ETIMEOUT and st.status == -1:
            raise TimeoutError(f"request {ticket} still running")
        plan, out = self._pending.pop(ticket)
        _check(rc, "tb_server_wait")
        return out.view(np.complex128).reshape(-1), {f: getattr(st, f) for f, _ in _ReqStats._fields_}

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_lib.tb_server_stats(self._h, ctypes.byref(st)), "tb_server_stats")
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.tb_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class _Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 7), ("ms", ctypes.c_double * 7),
                ("bytes", ctypes.c_double * 7)]


PROFILE_CLASSES = ("pass", "init", "reduce", "finalize", "narrow", "join", "late")


def profile_begin() -> None:
    """Bracket every kernel launch with CUDA events from now on."""
    _check(_lib.tb_profile_begin(), "tb_profile_begin")


def profile_end() -> dict:
    """Stop recording; {class: {"launches", "ms", "bytes"}} for the launches
    recorded since profile_begin()."""
    p = _Profile()
    _check(_lib.tb_profile_end(ctypes.byref(p)), "tb_profile_end")
    return {c: {"launches": int(p.launches[i]), "ms": float(p.ms[i]), "bytes": float(p.bytes[i])}
            for i, c in enumerate(PROFILE_CLASSES)}


def log_xeb(amps, n: int) -> float:
    a = np.ascontiguousarray(np.asarray(amps, np.complex128)).view(np.float64)
    out = ctypes.c_double(0.0)
    _check(_lib.tb_log_xeb(a.ctypes.data_as(_dp), a.size // 2, int(n), ctypes.byref(out)), "tb_log_xeb")
    return float(out.value)


def log_xeb_device(d_amps, n: int, d_out, stream=None) -> None:
    """Enqueue the FP64 log-XEB reduction of device amplitudes ``d_amps``
    (torch float64 tensor of shape (nb, 2), e.g. the output of
    ``Plan.amplitudes_device``) into ``d_out`` (torch float64 tensor, one
    element) on ``stream`` (default: the current stream). No synchronisation."""
    import torch
    if d_amps.dtype != torch.float64 or d_out.dtype != torch.float64 or not d_amps.is_contiguous():
        raise TypeError("d_amps and d_out must be contiguous float64 device tensors")
    st = stream if stream is not None else torch.cuda.current_stream(d_amps.device)
    _check(_lib.tb_log_xeb_device(d_amps.data_ptr(), d_amps.numel() // 2, int(n), d_out.data_ptr(),
                                  st.cuda_stream), "tb_log_xeb_device")


def clifford_matrix(k: int) -> np.ndarray:
    m = np.empty(8, np.float64)
    _check(_lib.tb_clifford_matrix(int(k), m.ctypes.data_as(_dp)), "tb_clifford_matrix")
    return m.view(np.complex128).reshape(2, 2)
