"""Python binding of libletkf.so (see include/letkf.h).

Argument marshalling only: every step of the analysis, forecast and residual
runs in the CUDA library. Torch supplies device memory and streams. Importing
this module does not need a GPU; creating a handle does, and fails loudly when
the library is not built or no GPU is present. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_char_p, c_double, c_int32, c_uint64, c_void_p

import numpy as np

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
# LETKF_LIBRARY selects another build of the same library (e.g. the one with
# phase clocks); by default the in-tree libletkf.so.
LIB_PATH = os.environ.get("LETKF_LIBRARY") or os.path.join(PKG_DIR, "libletkf.so")
HEADER = os.path.join(os.path.dirname(PKG_DIR), "include", "letkf.h")

LETKF_OK = 0
STATUS_NAMES = {0: "LETKF_OK", 1: "LETKF_ERR_ARG", 2: "LETKF_ERR_CUDA", 3: "LETKF_ERR_NOCONVERGE",
                4: "LETKF_ERR_TIMEOUT", 5: "LETKF_ERR_NONFINITE", 6: "LETKF_ERR_STATE",
                7: "LETKF_ERR_NOMEM"}


class LetkfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class letkf_config(ctypes.Structure):
    _fields_ = [("nsub", c_int32), ("subap_mask", c_void_p), ("m", c_int32), ("window", c_int32),
                ("taper", c_int32), ("loc_len", c_double), ("rho", c_double), ("sigma2", c_double),
                ("a_ar1", c_double), ("noise_std", c_double), ("precision", c_int32),
                ("fp64_kappa", c_double), ("seed", c_uint64), ("noise_bank", c_void_p),
                ("bank_B", c_int32), ("bank_G", c_int32), ("max_sweeps", c_int32),
                ("partition", c_int32), ("piston", c_int32)]


_SIGS = {
    "letkf_create": [POINTER(letkf_config), c_void_p, POINTER(c_void_p)],
    "letkf_destroy": [c_void_p],
    "letkf_query": [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)],
    "letkf_query_points": [c_void_p, c_void_p, c_void_p],
    "letkf_query_domains": [c_void_p, POINTER(c_int32), c_void_p, c_void_p],
    "letkf_get_state": [c_void_p, c_void_p],
    "letkf_set_state": [c_void_p, c_void_p],
    "letkf_forecast": [c_void_p, c_void_p],
    "letkf_analyze": [c_void_p, c_void_p, c_void_p, c_void_p],
    "letkf_residual": [c_void_p, c_void_p, c_void_p],
    "letkf_run": [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32],
    "letkf_run_graph": [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p],
    "letkf_set_dm": [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                     c_void_p],
    "letkf_get_command": [c_void_p, c_void_p],
    "letkf_run_dm": [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32],
    "letkf_sync": [c_void_p],
    "letkf_stats": [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)],
    "letkf_analyze_noalloc": [POINTER(letkf_config), c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_char_p, ctypes.c_size_t],
    "letkf_noalloc_status": [c_void_p, POINTER(c_int32)],
    "letkf_fma_peaks": [c_void_p],
    "letkf_phase_clocks": [c_void_p],
    "letkf_adjoint_phase_clocks": [c_void_p],
    "letkf_create_batch": [POINTER(letkf_config), c_int32, c_void_p, POINTER(c_void_p)],
    "letkf_query_instance": [c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32),
                             POINTER(c_int32), POINTER(c_int32)],
    "letkf_tile_shape": [c_int32, POINTER(c_int32), POINTER(c_int32)],
    "letkf_set_tile_shape": [c_void_p, c_int32, c_int32],
    "letkf_set_row_split": [c_void_p, c_int32, c_int32],
    "letkf_set_fp64_start": [c_void_p, c_int32],
    "letkf_autotune": [c_void_p, c_void_p, c_int32, POINTER(c_int32), POINTER(ctypes.c_float)],
    "letkf_set_params": [c_void_p, c_int32, c_double, c_double, c_double],
    "letkf_set_frame": [c_void_p, ctypes.c_int64],
    "letkf_set_jacobi": [c_void_p, c_double, c_double],
    "letkf_step": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "letkf_grad": [c_void_p, c_int32, c_void_p, c_void_p, c_int32, POINTER(c_double),
                   POINTER(c_double)],
}

_lib = None


def header_symbols() -> list:
    """Entry points declared in include/letkf.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:letkf_status|const char \*)\s*(letkf_\w+)\s*\(", text,
                                 re.M)))


def lib() -> ctypes.CDLL:
    """Load libletkf.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is not built; run `python -m paper_1408_7069_gb300.build` "
                "(the CUDA library is the only implementation)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = c_int32
        L.letkf_last_error.argtypes = [c_void_p]
        L.letkf_last_error.restype = c_char_p
        _lib = L
    return _lib


def _check(status: int, h) -> None:
    if status != LETKF_OK:
        msg = lib().letkf_last_error(h)
        raise LetkfError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


# ---------------------------------------------------------------------------
# Functions named as the C ABI (handles are ctypes.c_void_p).
# ---------------------------------------------------------------------------
def letkf_create(cfg: letkf_config, stream_ptr: int) -> c_void_p:
    h = c_void_p()
    _check(lib().letkf_create(byref(cfg), c_void_p(stream_ptr), byref(h)), None)
    return h


def letkf_create_batch(cfgs, stream_ptr: int) -> c_void_p:
    arr = (letkf_config * len(cfgs))(*cfgs)
    h = c_void_p()
    _check(lib().letkf_create_batch(arr, len(cfgs), c_void_p(stream_ptr), byref(h)), None)
    return h


def letkf_query_instance(h, i: int):
    """(n_pts, p, m, n_inst) of instance i."""
    n, p, m, k = c_int32(), c_int32(), c_int32(), c_int32()
    _check(lib().letkf_query_instance(h, i, byref(n), byref(p), byref(m), byref(k)), h)
    return n.value, p.value, m.value, k.value


def letkf_tile_shape(shape: int):
    a, b = c_int32(), c_int32()
    _check(lib().letkf_tile_shape(shape, byref(a), byref(b)), None)
    return a.value, b.value


def tile_shapes() -> list:
    """All compiled analysis tile shapes (nodes per CTA side)."""
    out = []
    while True:
        a, b = c_int32(), c_int32()
        if lib().letkf_tile_shape(len(out), byref(a), byref(b)) != LETKF_OK:
            return out
        out.append((a.value, b.value))


def letkf_set_tile_shape(h, width_class: int, shape: int) -> None:
    _check(lib().letkf_set_tile_shape(h, width_class, shape), h)


def letkf_set_row_split(h, width_class: int, split: int) -> None:
    _check(lib().letkf_set_row_split(h, width_class, split), h)


def letkf_set_fp64_start(h, warm: int) -> None:
    _check(lib().letkf_set_fp64_start(h, warm), h)


def letkf_autotune(h, y, reps: int = 3):
    """Times every tile shape per width class; returns ([shape] * 3, [us] * 3)."""
    shapes = (c_int32 * 3)()
    us = (ctypes.c_float * 3)()
    _check(lib().letkf_autotune(h, _ptr(y), reps, shapes, us), h)
    return list(shapes), list(us)


def letkf_destroy(h) -> None:
    _check(lib().letkf_destroy(h), None)


def letkf_query(h):
    n, p, m = c_int32(), c_int32(), c_int32()
    _check(lib().letkf_query(h, byref(n), byref(p), byref(m)), h)
    return n.value, p.value, m.value


def letkf_query_points(h, n_pts: int):
    ij = np.zeros((n_pts, 2), np.int32)
    ws = np.zeros(n_pts, np.int32)
    _check(lib().letkf_query_points(h, ij.ctypes.data, ws.ctypes.data), h)
    return ij, ws


def letkf_get_state(h, X) -> None:
    _check(lib().letkf_get_state(h, _ptr(X)), h)


def letkf_set_state(h, X) -> None:
    _check(lib().letkf_set_state(h, _ptr(X)), h)


def letkf_forecast(h, noise=None) -> None:
    _check(lib().letkf_forecast(h, _ptr(noise)), h)


def letkf_analyze(h, y, mean=None, spread=None) -> None:
    _check(lib().letkf_analyze(h, _ptr(y), _ptr(mean), _ptr(spread)), h)


def letkf_residual(h, truth, resvar) -> None:
    _check(lib().letkf_residual(h, _ptr(truth), _ptr(resvar)), h)


def letkf_run(h, frames: int, y_seq, truth_seq=None, resvar=None, use_graph: bool = True) -> None:
    _check(lib().letkf_run(h, int(frames), _ptr(y_seq), _ptr(truth_seq), _ptr(resvar),
                           1 if use_graph else 0), h)


def letkf_run_graph(h, frames: int, y_seq, truth_seq=None, resvar=None, stamps=None) -> None:
    _check(lib().letkf_run_graph(h, int(frames), _ptr(y_seq), _ptr(truth_seq), _ptr(resvar),
                                 _ptr(stamps)), h)


def letkf_set_params(h, i: int, rho: float, sigma2: float, loc_len: float) -> None:
    _check(lib().letkf_set_params(h, int(i), float(rho), float(sigma2), float(loc_len)), h)


def letkf_step(h, y_host, truth_host=None, mean_host=None, resvar_host=None) -> None:
    """One frame from host (numpy) buffers; see include/letkf.h."""
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    _check(lib().letkf_step(h, ptr(y_host), ptr(truth_host), ptr(mean_host), ptr(resvar_host)),
           h)


def letkf_set_jacobi(h, rotate_tol: float = 4e-6, stop_cos: float = 1e-3) -> None:
    _check(lib().letkf_set_jacobi(h, float(rotate_tol), float(stop_cos)), h)


def letkf_set_frame(h, frame: int) -> None:
    _check(lib().letkf_set_frame(h, int(frame)), h)


def letkf_grad(h, frames: int, y_seq, truth_seq, ckpt_every: int = 0):
    """(J, array([dJ/drho, dJ/dsigma2, dJ/dL])) of the closed loop over `frames` frames."""
    J = c_double()
    g = (c_double * 3)()
    _check(lib().letkf_grad(h, int(frames), _ptr(y_seq), _ptr(truth_seq), int(ckpt_every),
                            byref(J), g), h)
    return J.value, np.array(g[:], dtype=np.float64)


def letkf_sync(h) -> None:
    _check(lib().letkf_sync(h), h)


def letkf_stats(h):
    """(FP64 fallback nodes, max sweeps, total sweeps) of the last analysis."""
    a, b, c = c_int32(), c_int32(), c_int32()
    _check(lib().letkf_stats(h, byref(a), byref(b), byref(c)), h)
    return a.value, b.value, c.value


def letkf_analyze_noalloc(cfg: letkf_config, X, y, mean=None, spread=None, stream_ptr: int = 0):
    """One-frame analysis without a handle and without device allocation (its
    scratch is a static device array inside the library); raises LetkfError."""
    buf = ctypes.create_string_buffer(256)
    st = lib().letkf_analyze_noalloc(byref(cfg), _ptr(X), _ptr(y), _ptr(mean), _ptr(spread),
                                     c_void_p(stream_ptr), buf, 256)
    if st != LETKF_OK:
        raise LetkfError(st, buf.value.decode())


def letkf_noalloc_status(stream_ptr: int = 0) -> tuple:
    """(status, kappa_nodes) of the last allocation-free analysis on the
    current device; synchronises the stream. Returns the status code rather
    than raising, so that a caller can tell the faults apart."""
    n = c_int32(0)
    st = lib().letkf_noalloc_status(c_void_p(stream_ptr), byref(n))
    return int(st), int(n.value)


def letkf_fma_peaks() -> dict:
    """Measured FP32 (scalar and packed FMA) and FP64 peaks of the current
    device in TFLOP/s, each with the SM clock (MHz) it ran at."""
    out = (c_double * 7)()
    _check(lib().letkf_fma_peaks(out), None)
    return {"fp32_tflops": out[0], "fp32_mhz": out[1], "fp32x2_tflops": out[2],
            "fp32x2_mhz": out[3], "fp64_tflops": out[4], "fp64_mhz": out[5], "sms": int(out[6])}


def letkf_phase_clocks():
    """Cycles of the FP32 analysis kernel's phases (staging, Gram, Jacobi,
    apply) and its warp count since the last call, or None when the library
    was built without phase clocks."""
    out = (ctypes.c_uint64 * 5)()
    st = lib().letkf_phase_clocks(out)
    if st == 6:
        return None
    _check(st, None)
    return list(out)


def letkf_adjoint_phase_clocks():
    """Cycles of the reverse-mode node kernel's phases (staging, Gram and
    start, Jacobi, transform adjoint, window slopes) and its node count since
    the last call, FP32 form then FP64 form (12 values), or None without
    phase clocks."""
    out = (ctypes.c_uint64 * 12)()
    st = lib().letkf_adjoint_phase_clocks(out)
    if st == 6:
        return None
    _check(st, None)
    return list(out)


def letkf_last_error(h=None) -> str:
    msg = lib().letkf_last_error(h)
    return msg.decode() if msg else ""


# ---------------------------------------------------------------------------
# Handle object
# ---------------------------------------------------------------------------
def make_config(subap_mask, m: int, window: int, taper: int = 1, loc_len: float = 0.0,
                rho: float = 1.0, sigma2: float = 0.01, a_ar1: float = 1.0,
                noise_std: float = 0.0, precision: int = 0, fp64_kappa: float = 300.0,
                seed: int = 0, bank=None, max_sweeps: int = 0, partition: int = 0,
                piston: int = 0):
    """A letkf_config plus the numpy arrays its pointers refer to (keep both alive)."""
    mask = np.ascontiguousarray(subap_mask, dtype=np.uint8)
    bank = None if bank is None else np.ascontiguousarray(bank, dtype=np.float32)
    cfg = letkf_config()
    cfg.nsub = mask.shape[0]
    cfg.subap_mask = mask.ctypes.data
    cfg.m, cfg.window, cfg.taper, cfg.loc_len = m, window, taper, loc_len
    cfg.rho, cfg.sigma2, cfg.a_ar1, cfg.noise_std = rho, sigma2, a_ar1, noise_std
    cfg.precision, cfg.fp64_kappa, cfg.seed = precision, fp64_kappa, seed
    if bank is not None:
        cfg.noise_bank = bank.ctypes.data
        cfg.bank_B, cfg.bank_G = bank.shape[0], bank.shape[1]
    cfg.max_sweeps = max_sweeps
    cfg.partition, cfg.piston = partition, piston
    return cfg, (mask, bank)


def workload_config(w, bank=None, **kw):
    from .synth import pupil_subap_mask
    args = dict(m=w.m, window=w.window, taper=w.taper, loc_len=w.loc_len, rho=w.rho,
                sigma2=w.sigma2, a_ar1=w.a_ar1, noise_std=w.noise_std, precision=w.precision,
                seed=w.seeds[2], bank=bank, partition=getattr(w, "partition", 0),
                piston=getattr(w, "piston", 0))
    args.update(kw)
    return make_config(pupil_subap_mask(w.nsub, w.obscuration, w.square), **args)


class Letkf:
    """One or more LETKF instances on one GPU, on the handle's own CUDA stream.

    Tensor arguments are contiguous CUDA tensors of the handle's dtype (float32
    when precision = 0, float64 when precision = 1) in the layouts of
    include/letkf.h: the ensemble is [n_pts, 2, m] for one instance and the flat
    concatenation of the instances' blocks for a batch. Calls order the
    handle's stream after torch's current stream on entry and torch's current
    stream after the handle's on exit, so they compose with ordinary torch code.
    """

    def __init__(self, subap_mask=None, m: int = 0, window: int = 0, stream=None,
                 _configs=None, **kw):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("Letkf needs a CUDA GPU; there is no CPU implementation")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if _configs is None:
            _configs = [make_config(subap_mask, m, window, **kw)]
        self._keep = [k for _, k in _configs]
        cfgs = [c for c, _ in _configs]
        if len(cfgs) == 1:
            self.h = letkf_create(cfgs[0], self.stream.cuda_stream)
        else:
            self.h = letkf_create_batch(cfgs, self.stream.cuda_stream)
        self.n_pts, self.p, self.m = letkf_query(self.h)
        self.instances = [letkf_query_instance(self.h, i)[:3] for i in range(len(cfgs))]
        self.n_inst = len(cfgs)
        self.precision = cfgs[0].precision
        self.dtype = torch.float32 if self.precision == 0 else torch.float64
        self.state_numel = sum(2 * n * mm for n, _, mm in self.instances)

    @classmethod
    def from_workload(cls, w, bank=None, stream=None, **kw):
        f = cls(stream=stream, _configs=[workload_config(w, bank, **kw)])
        if getattr(w, "row_split", 1) != 1:
            try:
                f.set_row_split(0 if w.m <= 16 else 1, w.row_split)
            except BaseException:
                f.close()
                raise
        return f

    @classmethod
    def batch(cls, workloads, banks, stream=None, **kw):
        """One handle for many instances (workloads[i] with noise bank banks[i])."""
        return cls(stream=stream,
                   _configs=[workload_config(w, b, **kw) for w, b in zip(workloads, banks)])

    # -- stream ordering ---------------------------------------------------
    def _enter(self):
        self.stream.wait_stream(self._torch.cuda.current_stream())

    def _leave(self):
        self._torch.cuda.current_stream().wait_stream(self.stream)

    def _t(self, t, shape):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor, got {t.dtype} "
                             f"on {t.device} (contiguous={t.is_contiguous()})")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    @property
    def state_shape(self):
        return (self.n_pts, 2, self.m) if self.n_inst == 1 else (self.state_numel,)

    def split_state(self, X):
        """Per-instance [n_pts_i, 2, m_i] views of a (flat) batch ensemble."""
        out, off = [], 0
        flat = X.reshape(-1)
        for n, _, mm in self.instances:
            out.append(flat[off:off + 2 * n * mm].view(n, 2, mm))
            off += 2 * n * mm
        return out

    # -- API -----------------------------------------------------------------
    def points(self):
        return letkf_query_points(self.h, self.n_pts)

    def domains(self):
        """(number of local domains, domain of every node) of a handle with a
        partition; (0, None) for the per-node analysis."""
        n = c_int32(0)
        _check(lib().letkf_query_domains(self.h, byref(n), None, None), self.h)
        if n.value == 0:
            return 0, None
        nd = np.empty(self.n_pts, np.int32)
        _check(lib().letkf_query_domains(self.h, None, nd.ctypes.data, None), self.h)
        return n.value, nd

    def domain_sizes(self):
        """(n_d, p_d) of every local domain: state rows and observed slopes."""
        n, nd = self.domains()
        pd = np.empty(n, np.int32)
        _check(lib().letkf_query_domains(self.h, None, None, pd.ctypes.data), self.h)
        return 2 * np.bincount(nd, minlength=n), pd

    def new(self, *shape):
        return self._torch.zeros(*shape, dtype=self.dtype, device="cuda")

    def set_state(self, X):
        self._enter()
        letkf_set_state(self.h, self._t(X, self.state_shape))
        self._leave()

    def get_state(self):
        X = self.new(*self.state_shape)
        self._enter()
        letkf_get_state(self.h, X)
        self._leave()
        return X

    def forecast(self, noise=None):
        shape = (self.n_pts, self.m) if self.n_inst == 1 else (sum(n * mm for n, _, mm in self.instances),)
        self._enter()
        letkf_forecast(self.h, self._t(noise, shape))
        self._leave()

    def analyze(self, y, mean=None, spread=None, outputs: bool = True):
        if outputs and mean is None:
            mean = self.new(self.n_pts, 2)
        if outputs and spread is None:
            spread = self.new(self.n_pts, 2)
        self._enter()
        letkf_analyze(self.h, self._t(y, (self.p,)), self._t(mean, (self.n_pts, 2)),
                      self._t(spread, (self.n_pts, 2)))
        self._leave()
        return mean, spread

    def residual(self, truth, resvar=None):
        if resvar is None:
            resvar = self._torch.zeros(self.n_inst, dtype=self._torch.float64, device="cuda")
        self._enter()
        letkf_residual(self.h, self._t(truth, (self.n_pts,)), resvar)
        self._leave()
        return resvar

    def run(self, frames: int, y_seq, truth_seq=None, resvar=None, use_graph: bool = True):
        self._t(y_seq, (y_seq.shape[0], self.p))
        if y_seq.shape[0] < frames:
            raise ValueError("y_seq shorter than frames")
        if truth_seq is not None:
            self._t(truth_seq, (truth_seq.shape[0], self.n_pts))
            if truth_seq.shape[0] < frames:
                raise ValueError("truth_seq shorter than frames")
            if resvar is None:
                shape = (frames,) if self.n_inst == 1 else (frames, self.n_inst)
                resvar = self._torch.zeros(*shape, dtype=self._torch.float64, device="cuda")
        self._enter()
        letkf_run(self.h, frames, y_seq, truth_seq, resvar, use_graph)
        self._leave()
        return resvar

    def run_graph(self, frames: int, y_seq, truth_seq=None, resvar=None, stamps: bool = False):
        """All `frames` frames as one CUDA-graph launch (letkf_run_graph).
        Returns (resvar or None, per-frame durations in microseconds from the
        in-graph timer stamps, or None)."""
        self._t(y_seq, (y_seq.shape[0], self.p))
        if y_seq.shape[0] < frames:
            raise ValueError("y_seq shorter than frames")
        if truth_seq is not None:
            self._t(truth_seq, (truth_seq.shape[0], self.n_pts))
            if truth_seq.shape[0] < frames:
                raise ValueError("truth_seq shorter than frames")
            if resvar is None:
                shape = (frames,) if self.n_inst == 1 else (frames, self.n_inst)
                resvar = self._torch.zeros(*shape, dtype=self._torch.float64, device="cuda")
        st = self._torch.zeros(frames + 1, dtype=self._torch.int64, device="cuda") if stamps else None
        self._enter()
        letkf_run_graph(self.h, frames, y_seq, truth_seq, resvar, st)
        self._leave()
        us = None
        if stamps:
            t = st.cpu().numpy().astype(np.float64)
            us = np.diff(t) / 1e3
        return resvar, us

    def set_dm(self, N=None, P=None):
        """Deformable mirror (letkf_set_dm) from scipy CSR matrices N and P
        (n_pts x n_pts); None removes it."""
        if N is None:
            _check(lib().letkf_set_dm(self.h, 0, None, None, None, None, None, None), self.h)
            return
        arrs = []
        for M in (N, P):
            M = M.tocsr()
            arrs += [np.ascontiguousarray(M.indptr, np.int32),
                     np.ascontiguousarray(M.indices, np.int32),
                     np.ascontiguousarray(M.data, np.float64)]
        self._dm_keep = arrs
        _check(lib().letkf_set_dm(self.h, self.n_pts, *[a.ctypes.data for a in arrs]), self.h)

    def command(self):
        """The latest DM command u [n_pts] (device tensor)."""
        u = self.new(self.n_pts)
        self._enter()
        _check(lib().letkf_get_command(self.h, _ptr(u)), self.h)
        self._leave()
        return u

    def run_dm(self, frames: int, truth_seq, wnoise_seq, use_graph: bool = True):
        """The simulated closed loop with the mirror (letkf_run_dm); returns
        the residual variance per frame (device FP64 tensor)."""
        self._t(truth_seq, (truth_seq.shape[0], self.n_pts))
        self._t(wnoise_seq, (wnoise_seq.shape[0], self.p))
        if truth_seq.shape[0] < frames or wnoise_seq.shape[0] < frames:
            raise ValueError("sequences shorter than frames")
        resvar = self._torch.zeros(frames, dtype=self._torch.float64, device="cuda")
        self._enter()
        _check(lib().letkf_run_dm(self.h, int(frames), _ptr(truth_seq), _ptr(wnoise_seq),
                                  _ptr(resvar), 1 if use_graph else 0), self.h)
        self._leave()
        return resvar

    def set_params(self, rho: float, sigma2: float, loc_len: float, instance: int = 0):
        letkf_set_params(self.h, instance, rho, sigma2, loc_len)

    def step(self, y, truth=None, mean=None, resvar=None):
        """One closed-loop frame from host memory (numpy arrays of the handle's
        real type): returns the analysis mean [n_pts, 2] and, with truth, the
        residual variance per instance."""
        rt = np.float32 if self.precision == 0 else np.float64

        def host(a, n):
            if a is None:
                return None
            if not (isinstance(a, np.ndarray) and a.dtype == rt and a.flags.c_contiguous
                    and a.size == n):
                raise ValueError(f"expected a contiguous {np.dtype(rt).name} array of {n} values")
            return a
        y = host(y, self.p)
        truth = host(truth, self.n_pts)
        mean = host(mean, 2 * self.n_pts) if mean is not None else np.empty((self.n_pts, 2), rt)
        if truth is not None and resvar is None:
            resvar = np.empty(self.n_inst, np.float64)
        letkf_step(self.h, y, truth, mean, resvar)
        return mean, resvar

    def set_jacobi(self, rotate_tol: float = 4e-6, stop_cos: float = 1e-3):
        """FP32 eigensolve stopping rule; stop_cos <= rotate_tol: stop after a
        sweep without rotations."""
        letkf_set_jacobi(self.h, rotate_tol, stop_cos)

    def set_frame(self, frame: int):
        letkf_set_frame(self.h, frame)

    def grad(self, frames: int, y_seq, truth_seq, ckpt_every: int = 0):
        """Mean residual variance J over `frames` closed-loop frames from the
        current state and its gradient (dJ/drho, dJ/dsigma2, dJ/dL)."""
        if self.n_inst != 1:
            raise ValueError("grad takes a single-instance handle")
        self._t(y_seq, (y_seq.shape[0], self.p))
        self._t(truth_seq, (truth_seq.shape[0], self.n_pts))
        if y_seq.shape[0] < frames or truth_seq.shape[0] < frames:
            raise ValueError("sequences shorter than frames")
        self._enter()
        out = letkf_grad(self.h, frames, y_seq, truth_seq, ckpt_every)
        self._leave()
        return out

    def autotune(self, y, reps: int = 3):
        self._enter()
        out = letkf_autotune(self.h, self._t(y, (self.p,)), reps)
        self._leave()
        return out

    def set_tile_shape(self, width_class: int, shape: int):
        letkf_set_tile_shape(self.h, width_class, shape)

    def set_fp64_start(self, warm: bool):
        """FP64 handles: start the FP64 eigensolve from an FP32 basis (True,
        the default) or from the identity (False)."""
        letkf_set_fp64_start(self.h, 1 if warm else 0)

    def set_row_split(self, width_class: int, split: int):
        """1: two whole columns per lane; 2: each column's rows on two lanes
        (classes 0 and 1 of FP32 per-node handles; for systems that fill few
        warps per SM)."""
        letkf_set_row_split(self.h, width_class, split)

    def sync(self):
        letkf_sync(self.h)

    def stats(self):
        return letkf_stats(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            letkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Autograd
# ---------------------------------------------------------------------------
def _loss_function():
    import torch

    class LetkfLoss(torch.autograd.Function):
        """J(rho, sigma2, L): mean residual variance of the closed loop over
        `frames` frames on handle `f`, started from ensemble X0 at noise frame
        `frame0` (Section 2.1 Eq. Crit_Opt). rho, sigma2 and L are scalar
        tensors; backward returns dJ/drho, dJ/dsigma2, dJ/dL from the
        library's reverse mode (letkf_grad). The handle's parameters, state
        and frame counter are set by every call."""

        @staticmethod
        def forward(ctx, rho, sigma2, L, f, X0, y_seq, truth_seq, frames, ckpt_every=20,
                    frame0=0):
            f.set_params(float(rho), float(sigma2), float(L))
            f.set_state(X0)
            f.set_frame(frame0)
            J, g = f.grad(frames, y_seq, truth_seq, ckpt_every)
            ctx.save_for_backward(torch.as_tensor(g, dtype=torch.float64))
            ctx.like = (rho, sigma2, L)
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            (g,) = ctx.saved_tensors
            gJ = gJ.detach().to(torch.float64).cpu()
            out = [(gJ * g[i]).to(dtype=t.dtype, device=t.device) if torch.is_tensor(t) else None
                   for i, t in enumerate(ctx.like)]
            return (*out, None, None, None, None, None, None, None)

    return LetkfLoss


_LOSS = None


def letkf_loss(rho, sigma2, L, f, X0, y_seq, truth_seq, frames: int, ckpt_every: int = 20,
               frame0: int = 0):
    """Differentiable J(rho, sigma2, L) (see LetkfLoss)."""
    global _LOSS
    if _LOSS is None:
        _LOSS = _loss_function()
    return _LOSS.apply(rho, sigma2, L, f, X0, y_seq, truth_seq, frames, ckpt_every, frame0)
