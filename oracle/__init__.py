"""Oracle for the HVOX transform pair (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. It shares no code with the GPU path: the direct sums are plain
C (``direct.c``, FP64, OpenMP over outputs) and the partition steps are plain Python
(``partition.py``).

Direct sums (Sect. 2, Eq. 2 / Eq. 3; 2*pi written out, baselines in wavelengths):
    sky2vis: V_k = sum_n a_n I_n exp(+isign j 2 pi <p_k, r_n>)
    vis2sky: I_n = a_n Re sum_k V_k exp(-isign j 2 pi <p_k, r_n>)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile direct.c with gcc (-O2, OpenMP, strict IEEE: no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            pi64 = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_sky2vis.argtypes = [d, d, d, i64, d, i64, ctypes.c_int, d]
            lib.oracle_sky2vis_sample.argtypes = [d, d, d, i64, d, pi64, i64, ctypes.c_int, d]
            lib.oracle_vis2sky.argtypes = [d, d, i64, d, d, i64, ctypes.c_int, d]
            lib.oracle_vis2sky_sample.argtypes = [d, d, d, d, i64, pi64, i64, ctypes.c_int, d]
            lib.oracle_phase_turns.argtypes = [d, d, i64, d]
            lib.oracle_num_threads.restype = ctypes.c_int
            for f in (lib.oracle_sky2vis, lib.oracle_sky2vis_sample, lib.oracle_vis2sky,
                      lib.oracle_vis2sky_sample, lib.oracle_phase_turns):
                f.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape_last=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_last is not None and (a.ndim != 2 or a.shape[1] != shape_last):
        raise ValueError(f"expected (N, {shape_last}) array, got {a.shape}")
    return a


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def sky2vis(pix, uvw, sky, weight=None, isign: int = -1, sample=None) -> np.ndarray:
    """Visibilities (complex128). With ``sample`` (indices), only those entries."""
    if isign not in (-1, 1):
        raise ValueError("isign must be +1 or -1")
    lib = _load()
    pix, uvw, sky = _f64(pix, 3), _f64(uvw, 3), _f64(sky)
    w = None if weight is None else _f64(weight)
    if sample is None:
        out = np.zeros((len(uvw), 2), dtype=np.float64)
        lib.oracle_sky2vis(_dp(pix), _dp(w), _dp(sky), len(pix), _dp(uvw), len(uvw), isign, _dp(out))
    else:
        idx = np.ascontiguousarray(np.asarray(sample, dtype=np.int64))
        out = np.zeros((len(idx), 2), dtype=np.float64)
        lib.oracle_sky2vis_sample(_dp(pix), _dp(w), _dp(sky), len(pix), _dp(uvw),
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx), isign, _dp(out))
    return out[:, 0] + 1j * out[:, 1]


def vis2sky(pix, uvw, vis, weight=None, isign: int = -1, sample=None) -> np.ndarray:
    """Real dirty image (float64). With ``sample`` (indices), only those pixels."""
    if isign not in (-1, 1):
        raise ValueError("isign must be +1 or -1")
    lib = _load()
    pix, uvw = _f64(pix, 3), _f64(uvw, 3)
    v = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128)).view(np.float64)
    w = None if weight is None else _f64(weight)
    if sample is None:
        out = np.zeros(len(pix), dtype=np.float64)
        lib.oracle_vis2sky(_dp(pix), _dp(w), len(pix), _dp(uvw), _dp(v), len(uvw), isign, _dp(out))
    else:
        idx = np.ascontiguousarray(np.asarray(sample, dtype=np.int64))
        out = np.zeros(len(idx), dtype=np.float64)
        lib.oracle_vis2sky_sample(_dp(pix), _dp(w), _dp(uvw), _dp(v), len(uvw),
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx), isign, _dp(out))
    return out


def phase_turns(uvw, pix) -> np.ndarray:
    """Fraction of <p, r> in turns for paired rows (used to pin the reduction)."""
    lib = _load()
    uvw, pix = _f64(uvw, 3), _f64(pix, 3)
    out = np.zeros(len(uvw), dtype=np.float64)
    lib.oracle_phase_turns(_dp(uvw), _dp(pix), len(uvw), _dp(out))
    return out


def rel_l2(y, y_ref) -> float:
    """Relative l2 error ||y - y_ref|| / ||y_ref|| (the accuracy measure used throughout)."""
    y = np.asarray(y)
    y_ref = np.asarray(y_ref)
    den = np.linalg.norm(y_ref)
    return float(np.linalg.norm(y - y_ref) / (den if den > 0 else 1.0))
