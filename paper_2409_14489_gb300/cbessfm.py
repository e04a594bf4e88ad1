"""Thin Python binding of ``libcbessfm.so`` (declared in ``include/cbessfm.h``).

Argument marshalling only: every step of the DBP chain runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  Importing this module loads the library and raises
``ImportError`` if it has not been built -- there is no CPU fallback.

Field tensors are complex64 of shape ``(L, 2)`` or ``(batch, L, 2)`` (polarization-minor), which
is exactly the library's float4-per-sample layout; plans with FP16/BF16 storage take float16 /
bfloat16 tensors of shape ``(L, 4)`` or ``(batch, L, 4)`` holding (x.re, x.im, y.re, y.im).
Every call checks its fields' dtype, shape and memory before the library reads them.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB


class CBESSFMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"cbessfm status {status} ({STATUS_NAMES.get(status, '?')}): {message}")
        self.status = status


STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "ALIAS", 4: "CUDA", 5: "OOM",
                6: "TIMEOUT", 7: "NOT_IMPLEMENTED"}
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_ALIAS, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, \
    ERR_NOT_IMPLEMENTED = range(8)
STORAGE_C64, STORAGE_F16X4, STORAGE_BF16X4 = 0, 1, 2


class LinkStruct(ctypes.Structure):
    _fields_ = [("beta2", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("span_length", ctypes.c_double),
                ("n_spans", ctypes.c_int), ("sample_rate", ctypes.c_double)]


class JobStruct(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n_samples", ctypes.c_int64)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built: run __graft_entry__.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(_LIB_PATH)
    c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
    P = ctypes.c_void_p
    lib.cbessfm_plan_create.argtypes = [ctypes.POINTER(LinkStruct), c_int, c_int, c_double,
                                        ctypes.POINTER(ctypes.c_float), c_int, c_int, c_int, c_int,
                                        ctypes.POINTER(P)]
    lib.cbessfm_plan_create.restype = c_int
    lib.cbessfm_plan_destroy.argtypes = [P]
    lib.cbessfm_plan_destroy.restype = c_int
    lib.cbessfm_set_coeffs.argtypes = [P, c_void_p, c_int, c_void_p]
    lib.cbessfm_set_coeffs.restype = c_int
    lib.cbessfm_set_ratio.argtypes = [P, c_double, c_void_p]
    lib.cbessfm_set_ratio.restype = c_int
    lib.cbessfm_backpropagate.argtypes = [P, c_void_p, c_void_p, c_int64, c_int, c_void_p]
    lib.cbessfm_backpropagate.restype = c_int
    lib.cbessfm_get_status.argtypes = [P, c_void_p]
    lib.cbessfm_get_status.restype = c_int
    lib.cbessfm_last_error.argtypes = []
    lib.cbessfm_last_error.restype = ctypes.c_char_p
    lib.cbessfm_version.argtypes = []
    lib.cbessfm_version.restype = ctypes.c_char_p
    lib.cbessfm_grad_workspace_size.argtypes = [P, c_int64, c_int, ctypes.POINTER(ctypes.c_size_t)]
    lib.cbessfm_grad_workspace_size.restype = c_int
    lib.cbessfm_backpropagate_checkpointed.argtypes = [P, c_void_p, c_void_p, c_int64, c_int,
                                                       c_void_p, ctypes.c_size_t, c_void_p]
    lib.cbessfm_backpropagate_checkpointed.restype = c_int
    lib.cbessfm_grad.argtypes = [P, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 ctypes.c_size_t, c_int64, c_int, c_void_p]
    lib.cbessfm_grad.restype = c_int
    lib.cbessfm_batch_create.argtypes = [ctypes.POINTER(JobStruct), c_int, ctypes.POINTER(P)]
    lib.cbessfm_batch_create.restype = c_int
    lib.cbessfm_batch_run.argtypes = [P, c_void_p]
    lib.cbessfm_batch_run.restype = c_int
    lib.cbessfm_batch_info.argtypes = [P, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_longlong)]
    lib.cbessfm_batch_info.restype = c_int
    lib.cbessfm_batch_destroy.argtypes = [P]
    lib.cbessfm_batch_destroy.restype = c_int
    lib.cbessfm_streamed_workspace_size.argtypes = [P, c_int64, c_int,
                                                    ctypes.POINTER(ctypes.c_size_t)]
    lib.cbessfm_streamed_workspace_size.restype = c_int
    lib.cbessfm_backpropagate_streamed.argtypes = [P, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                                   c_int64, c_int, c_void_p]
    lib.cbessfm_backpropagate_streamed.restype = c_int
    lib.cbessfm_backpropagate_host.argtypes = [P, c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_int64, c_int, c_int, c_void_p]
    lib.cbessfm_backpropagate_host.restype = c_int
    lib.cbessfm_set_wait_limit.argtypes = [P, ctypes.c_longlong]
    lib.cbessfm_set_wait_limit.restype = c_int
    lib.cbessfm_set_nlpr_mode.argtypes = [P, c_int]
    lib.cbessfm_set_nlpr_mode.restype = c_int
    lib.cbessfm_analytic_taps.argtypes = [ctypes.POINTER(LinkStruct), c_int, c_int, c_int,
                                          c_void_p, c_int, c_int, c_void_p, c_void_p]
    lib.cbessfm_analytic_taps.restype = c_int
    lib.cbessfm_measure_fp32_peak.argtypes = [c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_int),
                                              c_void_p]
    lib.cbessfm_measure_fp32_peak.restype = c_int
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(status: int):
    if status != OK:
        raise CBESSFMError(status, _lib.cbessfm_last_error().decode())


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_link(beta2: float, span_length: float, n_spans: int, sample_rate: float,
              gamma: float = 0.0, alpha: float = 0.0) -> LinkStruct:
    return LinkStruct(beta2, gamma, alpha, span_length, n_spans, sample_rate)


def analytic_taps(link: LinkStruct, bands: int, steps: int, step_power, ntaps: int,
                  grid: int = 64, spans_per_step: int = 1, with_response: bool = False):
    """Analytic CB-ESSFM taps ``[steps][bands][bands][ntaps]`` (float64) from
    ``cbessfm_analytic_taps``; with ``with_response`` also the complex responses c_d[m]
    ``[2 bands - 1][ntaps]`` for d = l - i = -(bands - 1) .. bands - 1."""
    pw = np.ascontiguousarray(np.broadcast_to(np.asarray(step_power, dtype=np.float64),
                                              (steps,)))
    taps = np.zeros((steps, bands, bands, ntaps), dtype=np.float64)
    resp = np.zeros((2 * bands - 1, ntaps, 2), dtype=np.float64) if with_response else None
    _check(_lib.cbessfm_analytic_taps(ctypes.byref(link), bands, steps, spans_per_step,
                                      pw.ctypes.data, ntaps, grid, taps.ctypes.data,
                                      resp.ctypes.data if resp is not None else None))
    if with_response:
        return taps, resp[..., 0] + 1j * resp[..., 1]
    return taps


class Plan:
    """A CB-ESSFM DBP plan (``cbessfm_plan_create``).

    ``coeffs``: effective taps ``[steps][bands][bands][ntaps]`` (float32, host).
    """

    def __init__(self, link: LinkStruct, bands: int, steps: int, ratio: float, coeffs,
                 n_fft: int, overlap: int, storage: int = STORAGE_C64):
        ntaps = 1
        cptr = None
        self._coeffs = None
        if steps > 0:
            c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float32))
            if c.ndim != 4 or c.shape[:3] != (steps, bands, bands):
                raise ValueError(f"coeffs must have shape ({steps}, {bands}, {bands}, ntaps)")
            ntaps = int(c.shape[3])
            self._coeffs = c
            cptr = c.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        elif coeffs is not None and np.asarray(coeffs).ndim == 4:
            ntaps = int(np.asarray(coeffs).shape[3])
        self._h = ctypes.c_void_p()
        self.link = link
        self.bands, self.steps, self.ratio = bands, steps, ratio
        self.ntaps, self.n_fft, self.overlap, self.storage = ntaps, n_fft, overlap, storage
        _check(_lib.cbessfm_plan_create(ctypes.byref(link), bands, steps, float(ratio), cptr,
                                        ntaps, n_fft, overlap, storage, ctypes.byref(self._h)))

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def block(self) -> int:
        return self.bands * self.n_fft

    @property
    def valid(self) -> int:
        return self.bands * (self.n_fft - self.overlap)

    def n_blocks(self, n_samples: int) -> int:
        return -(-n_samples // self.valid)

    def _field_dtype(self):
        import torch
        return {STORAGE_C64: torch.complex64, STORAGE_F16X4: torch.float16,
                STORAGE_BF16X4: torch.bfloat16}[self.storage]

    def _field(self, t, name: str, like=None, c64: bool = False, host: bool = False):
        """(batch, L) of a contiguous field in the plan's storage (complex64 when ``c64``) of
        shape (L, k) or (batch, L, k), k = 2 for complex64 and 4 for 16-bit storage, on the
        device (in host memory when ``host``); ``like`` is a field it must match in shape.  The
        library reads and writes whole samples from these shapes, so a wrong one is refused here."""
        import torch
        want = torch.complex64 if c64 else self._field_dtype()
        last = 2 if want == torch.complex64 else 4
        ok = (isinstance(t, torch.Tensor) and t.is_cuda != host and t.dtype == want
              and t.is_contiguous() and t.dim() in (2, 3) and t.shape[-1] == last
              and (like is None or t.shape == like.shape))
        if not ok:
            where = "host" if host else "CUDA"
            raise ValueError(f"{name} must be a contiguous {want} {where} tensor of shape "
                             f"(L, {last}) or (batch, L, {last})"
                             + ("" if like is None else ", the same as x"))
        return self._shape(t)

    def backpropagate(self, x, out=None, stream=None):
        """Run DBP on a contiguous CUDA tensor in the plan's storage: complex64 of shape (L, 2) or
        (batch, L, 2); for fp16/bf16 storage, float16/bfloat16 of shape (L, 4) or (batch, L, 4)
        holding (x.re, x.im, y.re, y.im)."""
        import torch
        batch, L = self._field(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._field(out, "out", like=x)
        _check(_lib.cbessfm_backpropagate(self._h, x.data_ptr(), out.data_ptr(), L, batch,
                                          _stream_handle(stream)))
        return out

    def backpropagate_ptr(self, in_ptr: int, out_ptr: int, n_samples: int, batch: int,
                          stream_handle: int):
        """Raw-pointer form of ``cbessfm_backpropagate`` (device addresses)."""
        _check(_lib.cbessfm_backpropagate(self._h, in_ptr, out_ptr, n_samples, batch,
                                          stream_handle))

    # ---- differentiation form -------------------------------------------------------------
    def workspace_size(self, n_samples: int, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        _check(_lib.cbessfm_grad_workspace_size(self._h, int(n_samples), int(batch), ctypes.byref(n)))
        return n.value

    def new_workspace(self, n_samples: int, batch: int = 1):
        import torch
        return torch.empty(self.workspace_size(n_samples, batch), dtype=torch.uint8, device="cuda")

    @staticmethod
    def _workspace(workspace):
        """(device address, bytes) of a workspace, which must be a contiguous CUDA tensor (the
        kernels write it; a host address there would fault the device)."""
        import torch
        if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda
                and workspace.is_contiguous()):
            raise ValueError("workspace must be a contiguous CUDA tensor")
        return workspace.data_ptr(), workspace.numel() * workspace.element_size()

    @staticmethod
    def _shape(x):
        return (1, x.shape[0]) if x.dim() == 2 else (x.shape[0], x.shape[1])

    def backpropagate_checkpointed(self, x, workspace, out=None, stream=None):
        """Forward chain that also stores the adjoint's checkpoints in ``workspace``."""
        import torch
        batch, L = self._field(x, "x")          # the plan's storage; checkpoints are complex64
        if out is None:
            out = torch.empty_like(x)
        self._field(out, "out", like=x)
        ws_ptr, ws_bytes = self._workspace(workspace)
        _check(_lib.cbessfm_backpropagate_checkpointed(
            self._h, x.data_ptr(), out.data_ptr(), L, batch, ws_ptr, ws_bytes,
            _stream_handle(stream)))
        return out

    def grad(self, grad_out, workspace, want_input: bool = True, want_ratio: bool = True,
             stream=None):
        """Adjoint of the last checkpointed forward: returns (dL/dtaps [steps, bands, bands,
        ntaps] float64, dL/dratio float64 scalar or None, dL/din complex64 or None).  Leaving
        out the ratio gradient skips its per-step work in the adjoint kernel."""
        import torch
        if not (isinstance(grad_out, torch.Tensor) and grad_out.is_cuda
                and grad_out.dtype == torch.complex64):
            raise ValueError("grad_out must be a complex64 CUDA tensor")
        ws_ptr, ws_bytes = self._workspace(workspace)
        # temporaries and outputs are made on the call's stream, so their fills and their
        # memory's reuse are ordered with the kernels (a no-op without an explicit stream)
        with torch.cuda.stream(stream):
            g = grad_out.contiguous()
            batch, L = self._field(g, "grad_out", c64=True)
            gc = torch.zeros((max(self.steps, 0), self.bands, self.bands, self.ntaps),
                             dtype=torch.float64, device="cuda")
            gr = torch.zeros((), dtype=torch.float64, device="cuda") if want_ratio else None
            gi = torch.empty_like(g) if want_input else None
            _check(_lib.cbessfm_grad(self._h, g.data_ptr(), gc.data_ptr() if gc.numel() else None,
                                     gr.data_ptr() if gr is not None else None,
                                     gi.data_ptr() if gi is not None else None,
                                     ws_ptr, ws_bytes, L, batch, _stream_handle(stream)))
        return gc, gr, gi

    def set_coeffs(self, coeffs, stream=None):
        """Replace the taps: ``[steps][bands][bands][ntaps]`` as at creation, a host array (the
        copy is synchronous) or a CUDA tensor (copied on ``stream``)."""
        import torch
        want = (self.steps, self.bands, self.bands, self.ntaps)
        if self.steps > 0 and tuple(coeffs.shape) != want:
            raise ValueError(f"coeffs must have shape {want}, not {tuple(coeffs.shape)}")
        if isinstance(coeffs, torch.Tensor) and coeffs.is_cuda:
            with torch.cuda.stream(stream):   # a converted copy is freed in order with the copy
                c = coeffs.detach().to(torch.float32).contiguous()
                _check(_lib.cbessfm_set_coeffs(self._h, c.data_ptr(), 1, _stream_handle(stream)))
            return c
        c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float32))
        _check(_lib.cbessfm_set_coeffs(self._h, c.ctypes.data, 0, _stream_handle(stream)))
        return c

    def backpropagate_host(self, h_in, h_out, d_in, d_out, launch_blocks: int = 0, stream=None):
        """Host-resident fields with overlapped transfers (``cbessfm_backpropagate_host``):
        ``h_in``/``h_out`` pinned CPU tensors, ``d_in``/``d_out`` CUDA tensors of the same shape;
        ``launch_blocks`` OLS blocks per kernel launch (0: one wave of the device).  Completion is
        ordered on ``stream`` (the current stream by default)."""
        batch, L = self._field(h_in, "h_in", host=True)
        self._field(h_out, "h_out", like=h_in, host=True)
        self._field(d_in, "d_in", like=h_in)
        self._field(d_out, "d_out", like=h_in)
        _check(_lib.cbessfm_backpropagate_host(self._h, h_in.data_ptr(), h_out.data_ptr(),
                                               d_in.data_ptr(), d_out.data_ptr(), L, batch,
                                               launch_blocks, _stream_handle(stream)))
        return h_out

    def streamed_workspace_size(self, n_samples: int, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        _check(_lib.cbessfm_streamed_workspace_size(self._h, n_samples, batch, ctypes.byref(n)))
        return n.value

    def backpropagate_streamed(self, x, out=None, workspace=None, stream=None):
        """Per-step streamed form (``cbessfm_backpropagate_streamed``); the fields between
        passes are complex64 whatever the plan's storage."""
        import torch
        batch, L = self._field(x, "x")
        if out is not None:
            self._field(out, "out", like=x)
        need = self.streamed_workspace_size(L, batch)
        with torch.cuda.stream(stream):       # a workspace made here is freed in order with the passes
            if out is None:
                out = torch.empty_like(x)
            if workspace is None and need:
                workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
            ws_ptr, ws_bytes = self._workspace(workspace) if workspace is not None else (None, 0)
            _check(_lib.cbessfm_backpropagate_streamed(
                self._h, x.data_ptr(), out.data_ptr(), ws_ptr, ws_bytes, L, batch,
                _stream_handle(stream)))
        return out

    def set_nlpr_mode(self, per_polarization: bool):
        """Switch between the Manakov NLPR (False) and the per-polarization NLPR (True)."""
        _check(_lib.cbessfm_set_nlpr_mode(self._h, 1 if per_polarization else 0))
        self.per_polarization = bool(per_polarization)

    def set_ratio(self, ratio: float, stream=None):
        _check(_lib.cbessfm_set_ratio(self._h, float(ratio), _stream_handle(stream)))
        self.ratio = float(ratio)

    def set_wait_limit(self, cycles: int):
        """Bound of the staging waits in SM cycles (``cbessfm_set_wait_limit``): > 0 the bound,
        0 one non-blocking test, < 0 the default."""
        _check(_lib.cbessfm_set_wait_limit(self._h, int(cycles)))

    def status(self, stream=None) -> int:
        """Synchronize and return the device status as a cbessfm_status value (0 = OK)."""
        return _lib.cbessfm_get_status(self._h, _stream_handle(stream))

    def close(self):
        if self._h:
            _lib.cbessfm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak(repeats: int = 10, stream=None):
    """Measured FP32 FMA rate of the current device (``cbessfm_measure_fp32_peak``): returns
    ``(flop_per_s, sm_count)``, best of ``repeats`` timed launches.  Synchronous."""
    flops, sms = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(_lib.cbessfm_measure_fp32_peak(int(repeats), ctypes.byref(flops), ctypes.byref(sms),
                                          _stream_handle(stream)))
    return flops.value, sms.value


def version() -> str:
    return _lib.cbessfm_version().decode()


class Batch:
    """Batched form (``cbessfm_batch_*``): independent jobs, each ``(plan, x, y)`` with x, y
    contiguous CUDA tensors in the plan's storage, processed by one persistent launch per group
    of jobs sharing N', subband count and storage.  ``run()`` is graph-capturable."""

    def __init__(self, jobs):
        self._h = ctypes.c_void_p()
        self._jobs = list(jobs)            # keep plans and tensors alive
        arr = (JobStruct * len(self._jobs))()
        for k, (plan, x, y) in enumerate(self._jobs):
            # one realization per job: a (batch, L, ...) field would be cut to its first row
            want = plan._field_dtype()
            last = 2 if plan.storage == STORAGE_C64 else 4
            for name, t in (("x", x), ("y", y)):
                if not (t.is_cuda and t.dtype == want and t.is_contiguous() and t.dim() == 2
                        and t.shape[1] == last and t.shape == x.shape):
                    raise ValueError(f"job {k}: {name} must be a contiguous {want} CUDA tensor "
                                     f"of shape (L, {last}), the same for x and y")
            arr[k] = JobStruct(plan.handle.value, x.data_ptr(), y.data_ptr(), int(x.shape[0]))
        _check(_lib.cbessfm_batch_create(arr, len(self._jobs), ctypes.byref(self._h)))

    def run(self, stream=None):
        _check(_lib.cbessfm_batch_run(self._h, _stream_handle(stream)))

    def info(self):
        g, n = ctypes.c_int(), ctypes.c_longlong()
        _check(_lib.cbessfm_batch_info(self._h, ctypes.byref(g), ctypes.byref(n)))
        return {"groups": g.value, "work_items": n.value}

    def capture(self, warmup: int = 1):
        """Capture ``run()`` into a torch CUDA graph (after ``warmup`` eager runs); returns the
        graph, whose ``replay()`` processes the whole batch."""
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run(s)
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run()
        return graph

    def close(self):
        if self._h:
            _lib.cbessfm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
