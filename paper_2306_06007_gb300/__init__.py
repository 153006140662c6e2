"""Python binding of libhvox (the GB300 HVOX transform library).

Argument marshalling only: every step of a transform runs in the library's CUDA
kernels. The C ABI is declared in ``include/hvox.h``; this module mirrors its names:

    plan = Plan(pix, uvw, eps, isign=-1, weight=None, ...)   # hvox_plan
    V = plan.synthesize(I)    # sky -> vis (alias dirty2vis)  hvox_synthesize
    I = plan.analyze(V)       # vis -> sky (alias vis2dirty)  hvox_analyze
    plan.close()              # hvox_destroy

Inputs may be numpy arrays, CPU tensors or CUDA tensors. Results are torch tensors on
the device of the input (CUDA inputs: asynchronous on the plan's stream).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = ["Plan", "HvoxError", "load", "build", "es_params", "es_ft", "box_dims", "chunk_points", "version",
           "PREC_AUTO", "PREC_FP32", "PREC_FP64", "MODE_AUTO", "MODE_NUFFT", "MODE_DIRECT"]

PREC_AUTO, PREC_FP32, PREC_FP64 = 0, 1, 2
MODE_AUTO, MODE_NUFFT, MODE_DIRECT = 0, 1, 2
_STATUS = {0: "HVOX_OK", 1: "HVOX_EINVAL", 2: "HVOX_ENOMEM", 3: "HVOX_ECUDA", 4: "HVOX_ETIMEOUT",
           5: "HVOX_EUNSUPPORTED", 6: "HVOX_EINTERNAL"}


class HvoxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("mode", ctypes.c_int32), ("upsampfac", ctypes.c_double),
                ("chunk_budget_bytes", ctypes.c_double), ("anisotropy", ctypes.c_double),
                ("direct_threshold", ctypes.c_double), ("search_threshold", ctypes.c_double),
                ("ntrans", ctypes.c_int32), ("plain", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("chunk_order", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("factor", ctypes.c_int32), ("autotune", ctypes.c_int32), ("kernel_width", ctypes.c_int32)]

_FACTOR = {None: 0, "auto": 0, "pixels": 1, "baselines": 2}


class Info(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int64), ("n_vis", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("isign", ctypes.c_int32), ("eps", ctypes.c_double), ("w", ctypes.c_int32),
                ("beta", ctypes.c_double), ("upsampfac", ctypes.c_double), ("budget_bytes", ctypes.c_double),
                ("t", ctypes.c_double), ("h", ctypes.c_double * 3), ("eta", ctypes.c_double * 3),
                ("n_pix_chunks", ctypes.c_int64), ("n_vis_chunks", ctypes.c_int64),
                ("n_nufft_blocks", ctypes.c_int64), ("n_direct_rects", ctypes.c_int64),
                ("direct_pairs", ctypes.c_double), ("nufft_points", ctypes.c_double),
                ("nufft_cells", ctypes.c_double), ("max_grid_bytes", ctypes.c_double),
                ("workspace_bytes", ctypes.c_double), ("plan_seconds", ctypes.c_double),
                ("model_seconds", ctypes.c_double), ("graph_state", ctypes.c_int32),
                ("nufft_pix_points", ctypes.c_double), ("nufft_vis_points", ctypes.c_double),
                ("spread_cells", ctypes.c_double), ("fft_work", ctypes.c_double), ("box_ratio", ctypes.c_double),
                ("spread_bin_pix", ctypes.c_int32), ("spread_bin_vis", ctypes.c_int32),
                ("kernel_width_rule", ctypes.c_int32), ("probe_error", ctypes.c_double),
                ("fft_batches", ctypes.c_int32), ("fft_batches_df", ctypes.c_int32),
                ("direct_vpt", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8), ("transforms", ctypes.c_int64)]


STAGES = ("permute", "direct", "spread", "deconv", "fft", "interp", "zero", "unused")

_lib = None
LIB_PATH = _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load libhvox.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I64, I32, V = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    PI64 = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "hvox_plan": [V, I64, V, I64, V, ctypes.c_double, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(P)],
        "hvox_synthesize": [P, V, V],
        "hvox_analyze": [P, V, V],
        "hvox_dirty2vis": [P, V, V],
        "hvox_vis2dirty": [P, V, V],
        "hvox_destroy": [P],
        "hvox_sync": [P],
        "hvox_plan_info": [P, ctypes.POINTER(Info)],
        "hvox_plan_chunks": [P, PI64, PI64],
        "hvox_plan_order": [P, PI64, PI64],
        "hvox_synthesize_complex": [P, P, P],
        "hvox_analyze_complex": [P, P, P],
        "hvox_profile": [P, ctypes.c_int],
        "hvox_get_stats": [P, ctypes.POINTER(Stats)],
        "hvox_es_params": [ctypes.c_double, ctypes.c_double, ctypes.POINTER(I32), D],
        "hvox_es_ft": [I32, ctypes.c_double, D, I64, D],
        "hvox_box_dims": [D, D, ctypes.c_double, ctypes.c_double, I32, I32, D, D, D],
        "hvox_chunk_points": [D, I64, D, PI64, PI64],
        "hvox_plan_dry": [D, I64, D, I64, ctypes.c_double, ctypes.POINTER(Opts), ctypes.POINTER(Info)],
        "hvox_direct_synthesize_noalloc": [V, I64, V, I64, V, V, ctypes.c_int, V],
        "hvox_cost_model": [I32, I32, D],
        "hvox_synthesize_batch": [ctypes.POINTER(P), ctypes.POINTER(V), ctypes.POINTER(V), I32, V, ctypes.POINTER(I32)],
        "hvox_analyze_batch": [ctypes.POINTER(P), ctypes.POINTER(V), ctypes.POINTER(V), I32, V, ctypes.POINTER(I32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hvox_last_error.restype = ctypes.c_char_p
    lib.hvox_last_error.argtypes = []
    lib.hvox_version.restype = ctypes.c_char_p
    lib.hvox_version.argtypes = []
    lib.hvox_estimate_bytes.restype = ctypes.c_double
    lib.hvox_estimate_bytes.argtypes = [I64, I64, ctypes.c_double, ctypes.POINTER(Opts)]
    _lib = lib
    return lib


def _check(code: int):
    if code != 0:
        raise HvoxError(code, load().hvox_last_error().decode())


def version() -> str:
    return load().hvox_version().decode()


# ------------------------------------------------------------------ host-only planning primitives

def _np():
    import numpy as np
    return np


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def es_params(eps: float, sigma: float = 2.0):
    w, beta = ctypes.c_int32(), ctypes.c_double()
    _check(load().hvox_es_params(eps, sigma, ctypes.byref(w), ctypes.byref(beta)))
    return w.value, beta.value


def es_ft(w: int, beta: float, xi):
    np = _np()
    xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
    out = np.empty_like(xi)
    _check(load().hvox_es_ft(w, beta, _dptr(xi), len(xi), _dptr(out)))
    return out


def box_dims(P, B, budget_bytes: float, sigma: float, w: int, elem_bytes: int):
    np = _np()
    P = np.ascontiguousarray(P, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    eta, h, t = np.zeros(3), np.zeros(3), ctypes.c_double()
    _check(load().hvox_box_dims(_dptr(P), _dptr(B), budget_bytes, sigma, w, elem_bytes, _dptr(eta), _dptr(h),
                                ctypes.byref(t)))
    return eta, h, t.value


def chunk_points(xyz, h):
    np = _np()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    labels = np.zeros(len(xyz), dtype=np.int64)
    nc = ctypes.c_int64()
    _check(load().hvox_chunk_points(_dptr(xyz), len(xyz), _dptr(h),
                                    labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(nc)))
    return labels, nc.value


COST_MODEL_FIELDS = ("direct_pair", "scatter_smem", "scatter_global", "gather_tap", "fft_cell", "grid_cell",
                     "block_fixed", "tile_cells")


def cost_model(precision="fp32", plain: bool = False) -> dict:
    """The planner's stage rates (seconds per unit of work) for plans of this precision."""
    out = (ctypes.c_double * 8)()
    _check(load().hvox_cost_model(_PREC[precision], 1 if plain else 0, out))
    return dict(zip(COST_MODEL_FIELDS, list(out)))


def plan_dry(pix, uvw, eps: float, precision="auto", mode="auto", upsampfac: float = 0.0,
             chunk_budget_bytes: float = 0.0, direct_threshold: float = 0.0, plain: bool = False,
             search_threshold: float = 0.0, factor=None, kernel_width: int = 0) -> dict:
    """Host-only planning (no GPU): partition, block choices and cost-model estimate."""
    np = _np()
    pix = np.ascontiguousarray(pix, dtype=np.float64)
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    o = Opts()
    o.precision = _PREC[precision]
    o.mode = _MODE[mode]
    o.upsampfac = upsampfac
    o.chunk_budget_bytes = chunk_budget_bytes
    o.direct_threshold = direct_threshold
    o.search_threshold = search_threshold
    o.plain = 1 if plain else 0
    o.factor = _FACTOR[factor]
    o.kernel_width = int(kernel_width)
    inf = Info()
    _check(load().hvox_plan_dry(_dptr(pix), len(pix), _dptr(uvw), len(uvw), float(eps), ctypes.byref(o),
                                ctypes.byref(inf)))
    return {name: (list(getattr(inf, name)) if name in ("h", "eta") else getattr(inf, name))
            for name, _ in Info._fields_}


def estimate_bytes(n_pix: int, n_vis: int, eps: float, precision="auto", mode="auto",
                   chunk_budget_bytes: float = 0.0, ntrans: int = 1, plain: bool = False,
                   search_threshold: float = 0.0) -> float:
    """Upper bound of the device memory a plan of these sizes could own (hvox_estimate_bytes)."""
    o = Opts()
    o.precision = _PREC[precision]
    o.mode = _MODE[mode]
    o.chunk_budget_bytes = chunk_budget_bytes
    o.ntrans = ntrans
    o.plain = 1 if plain else 0
    o.search_threshold = search_threshold
    return float(load().hvox_estimate_bytes(int(n_pix), int(n_vis), float(eps), ctypes.byref(o)))


def direct_synthesize_noalloc(pix, uvw, I, V, isign: int = -1, stream=None):
    """sky -> vis by direct FP32 summation without any allocation (hvox_direct_synthesize_noalloc).

    For callers that cannot allocate device memory (a framework owning the device's memory
    pool, or a per-iteration loop where allocation is not allowed). pix (N, 3) and uvw
    (K, 3) float64, I float32 (N,), V complex64 (K,): all CUDA tensors, V overwritten.
    n_pix + n_vis <= 524,288. Calls that overlap on the GPU share one static scratch array
    and race; run them one after another.
    """
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    for t, dt in ((pix, torch.float64), (uvw, torch.float64), (I, torch.float32), (V, torch.complex64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA tensor of {dt}")
    _check(load().hvox_direct_synthesize_noalloc(pix.data_ptr(), pix.shape[0], uvw.data_ptr(), uvw.shape[0],
                                                 I.data_ptr(), V.data_ptr(), int(isign),
                                                 ctypes.c_void_p(stream.cuda_stream)))
    return V


# ------------------------------------------------------------------ plans

def _as_f64_rows(x):
    """(N, 3) float64 contiguous: torch tensor (any device) or numpy. Returns (keepalive, ptr, N)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            t = x.detach().to(torch.float64).contiguous()
            if t.dim() != 2 or t.shape[1] != 3:
                raise ValueError("coordinates must have shape (N, 3)")
            return t, t.data_ptr(), t.shape[0]
    except ImportError:
        pass
    np = _np()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("coordinates must have shape (N, 3)")
    return a, a.ctypes.data, a.shape[0]


def _as_f64_vec(x, n):
    if x is None:
        return None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            t = x.detach().to(torch.float64).contiguous().reshape(-1)
            if t.numel() != n:
                raise ValueError("weights must have n_pix entries")
            return t, t.data_ptr()
    except ImportError:
        pass
    np = _np()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError("weights must have n_pix entries")
    return a, a.ctypes.data


_PREC = {"auto": PREC_AUTO, "fp32": PREC_FP32, "fp64": PREC_FP64, PREC_AUTO: PREC_AUTO, PREC_FP32: PREC_FP32,
         PREC_FP64: PREC_FP64}
_MODE = {"auto": MODE_AUTO, "nufft": MODE_NUFFT, "direct": MODE_DIRECT, MODE_AUTO: MODE_AUTO,
         MODE_NUFFT: MODE_NUFFT, MODE_DIRECT: MODE_DIRECT}


class Plan:
    """A planned HVOX transform pair on one geometry (see include/hvox.h)."""

    def __init__(self, pix, uvw, eps: float, isign: int = -1, weight=None, precision="auto", mode="auto",
                 upsampfac: float = 0.0, chunk_budget_bytes: float = 0.0, anisotropy: float = 0.0,
                 direct_threshold: float = 0.0, ntrans: int = 1, plain: bool = False, graphs: int = 0,
                 search_threshold: float = 0.0, chunk_order: bool = False, stream=None, factor=None,
                 autotune: bool = False, kernel_width: int = 0):
        import torch
        lib = load()
        self._handle = ctypes.c_void_p()
        pk, pp, n_pix = _as_f64_rows(pix)
        uk, up, n_vis = _as_f64_rows(uvw)
        wk, wp = _as_f64_vec(weight, n_pix)
        o = Opts()
        o.precision = _PREC[precision]
        o.mode = _MODE[mode]
        o.upsampfac = upsampfac
        o.chunk_budget_bytes = chunk_budget_bytes
        o.anisotropy = anisotropy
        o.direct_threshold = direct_threshold
        o.search_threshold = search_threshold
        o.ntrans = ntrans
        o.plain = 1 if plain else 0
        o.graphs = int(graphs)
        o.chunk_order = 1 if chunk_order else 0
        o.factor = _FACTOR[factor]
        o.autotune = 1 if autotune else 0
        o.kernel_width = int(kernel_width)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(lib.hvox_plan(pp, n_pix, up, n_vis, wp, float(eps), int(isign), ctypes.byref(o),
                             ctypes.byref(self._handle)))
        del pk, uk, wk
        info = self.info()
        self.n_pix, self.n_vis, self.ntrans = n_pix, n_vis, max(1, ntrans)
        self.precision = info["precision"]
        self.real_dtype = torch.float32 if self.precision == PREC_FP32 else torch.float64
        self.complex_dtype = torch.complex64 if self.precision == PREC_FP32 else torch.complex128

    # -------------------------------------------------------------- transforms
    def _shape(self, n):
        return (n,) if self.ntrans == 1 else (self.ntrans, n)

    def _input(self, x, dtype, n):
        import torch
        if not isinstance(x, torch.Tensor):
            x = torch.as_tensor(x)
        if x.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype} (the plan precision fixes the dtype)")
        if x.numel() != self.ntrans * n:
            raise ValueError(f"expected {self.ntrans * n} elements, got {x.numel()}")
        return x.contiguous()

    def _output(self, out, like, dtype, n):
        import torch
        if out is None:
            return torch.empty(self._shape(n), dtype=dtype, device=like.device)
        if out.dtype != dtype or out.numel() != self.ntrans * n or not out.is_contiguous():
            raise ValueError("output tensor has the wrong dtype, size or layout")
        return out

    def synthesize(self, I, out=None):
        """sky -> vis: V_k = sum_n a_n I_n exp(isign j 2 pi <p_k, r_n>)."""
        I = self._input(I, self.real_dtype, self.n_pix)
        V = self._output(out, I, self.complex_dtype, self.n_vis)
        _check(load().hvox_synthesize(self._handle, ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(V.data_ptr())))
        return V

    def analyze(self, V, out=None):
        """vis -> sky: I_n = a_n Re sum_k V_k exp(-isign j 2 pi <p_k, r_n>)."""
        V = self._input(V, self.complex_dtype, self.n_vis)
        I = self._output(out, V, self.real_dtype, self.n_pix)
        _check(load().hvox_analyze(self._handle, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(I.data_ptr())))
        return I

    def synthesize_complex(self, I):
        """sky -> vis for a complex sky (device tensor, complex dtype of the plan)."""
        import torch
        if self.ntrans != 1:
            raise ValueError("complex-sky transforms take ntrans = 1")
        I = torch.as_tensor(I).to(device="cuda", dtype=self.complex_dtype).contiguous()
        if I.numel() != self.n_pix:
            raise ValueError(f"expected {self.n_pix} elements, got {I.numel()}")
        V = torch.empty(self.n_vis, dtype=self.complex_dtype, device="cuda")
        _check(load().hvox_synthesize_complex(self._handle, ctypes.c_void_p(I.data_ptr()),
                                              ctypes.c_void_p(V.data_ptr())))
        return V

    def analyze_complex(self, V):
        """vis -> sky without taking the real part: a_n sum_k V_k exp(-isign j 2 pi <p_k, r_n>)."""
        import torch
        if self.ntrans != 1:
            raise ValueError("complex-sky transforms take ntrans = 1")
        V = torch.as_tensor(V).to(device="cuda", dtype=self.complex_dtype).contiguous()
        if V.numel() != self.n_vis:
            raise ValueError(f"expected {self.n_vis} elements, got {V.numel()}")
        I = torch.empty(self.n_pix, dtype=self.complex_dtype, device="cuda")
        _check(load().hvox_analyze_complex(self._handle, ctypes.c_void_p(V.data_ptr()),
                                           ctypes.c_void_p(I.data_ptr())))
        return I

    dirty2vis = synthesize
    vis2dirty = analyze

    # -------------------------------------------------------------- introspection
    def info(self) -> dict:
        inf = Info()
        _check(load().hvox_plan_info(self._handle, ctypes.byref(inf)))
        d = {}
        for name, _ in Info._fields_:
            v = getattr(inf, name)
            d[name] = list(v) if name in ("h", "eta") else v
        return d

    def chunks(self):
        np = _np()
        pc = np.zeros(self.n_pix, dtype=np.int64)
        vc = np.zeros(self.n_vis, dtype=np.int64)
        _check(load().hvox_plan_chunks(self._handle, pc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       vc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return pc, vc

    def order(self):
        """(pix_order, vis_order): the caller's index of the point at each chunk position."""
        np = _np()
        po = np.zeros(self.n_pix, dtype=np.int64)
        vo = np.zeros(self.n_vis, dtype=np.int64)
        _check(load().hvox_plan_order(self._handle, po.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      vo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return po, vo

    def sync(self):
        _check(load().hvox_sync(self._handle))

    def profile(self, enable=True):
        """Reset statistics; time every stage with CUDA events while enabled. enable="serial"
        runs every stage alone on the plan's stream (per-kernel device times)."""
        mode = 2 if enable == "serial" else (1 if enable else 0)
        _check(load().hvox_profile(self._handle, mode))

    def stats(self) -> dict:
        """Per-stage device milliseconds and launch counts since the last profile() call."""
        st = Stats()
        _check(load().hvox_get_stats(self._handle, ctypes.byref(st)))
        return {"ms": {n: st.ms[i] for i, n in enumerate(STAGES[:7])},
                "launches": {n: st.launches[i] for i, n in enumerate(STAGES[:7])},
                "transforms": st.transforms}

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            _check(load().hvox_destroy(self._handle))
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _batch(entry, plans, xs, s2v: bool, stream, return_launches: bool):
    import torch
    plans = list(plans)
    xs = list(xs)
    if len(plans) != len(xs):
        raise ValueError("one input per plan")
    cur = torch.cuda.current_stream()
    if stream is None:
        stream = cur
    elif stream != cur:
        stream.wait_stream(cur)  # inputs and fresh outputs are ordered on the current stream
    ins, outs = [], []
    for p, x in zip(plans, xs):
        if p.ntrans != 1:
            raise ValueError("batched transforms take plans with ntrans = 1")
        if s2v:
            x = p._input(x, p.real_dtype, p.n_pix)
            y = torch.empty(p.n_vis, dtype=p.complex_dtype, device=x.device)
        else:
            x = p._input(x, p.complex_dtype, p.n_vis)
            y = torch.empty(p.n_pix, dtype=p.real_dtype, device=x.device)
        if not x.is_cuda:
            raise ValueError("batched transforms take device tensors")
        ins.append(x)
        outs.append(y)
    n = len(plans)
    P = (ctypes.c_void_p * max(n, 1))(*[p._handle.value for p in plans])
    Vin = (ctypes.c_void_p * max(n, 1))(*[x.data_ptr() for x in ins])
    Vout = (ctypes.c_void_p * max(n, 1))(*[y.data_ptr() for y in outs])
    launches = ctypes.c_int32(0)
    _check(entry(P, Vin, Vout, n, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(launches)))
    for t in ins + outs:
        t.record_stream(stream)
    return (outs, launches.value) if return_launches else outs


def synthesize_batch(plans, skies, stream=None, return_launches: bool = False):
    """sky -> vis for several plans in one call (hvox_synthesize_batch): the direct sums of
    plans on the FP32 or double-float kernels share one launch per kernel form. skies: one
    device tensor per plan. Returns the visibilities (and the number of direct launches)."""
    return _batch(load().hvox_synthesize_batch, plans, skies, True, stream, return_launches)


def analyze_batch(plans, vis, stream=None, return_launches: bool = False):
    """vis -> sky for several plans in one call (hvox_analyze_batch); see synthesize_batch."""
    return _batch(load().hvox_analyze_batch, plans, vis, False, stream, return_launches)
