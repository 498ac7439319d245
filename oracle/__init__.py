"""CPU oracle for the dedispersion path -- test infrastructure, not product code.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import this package.  It is written from the paper (eq. p_dedisp, eq. snr,
eq. P_N_dedisp, eq. trial DMs and Sec. 3's delay and smear laws) and shares no code
with the CUDA library.  `dd_oracle.py` is the numpy reference; `dd_oracle.c` is the
same brute-force sum in plain C (int64 / double accumulation, OpenMP over trials)
for the larger parity cases and the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .dd_oracle import *  # noqa: F401,F403
from . import dd_oracle as ref  # noqa: F401

_lib = None


def clib():
    """The compiled C oracle (built on first use)."""
    global _lib
    if _lib is None:
        from .build import build
        path = build()
        lib = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.orc_dedisperse_u8.restype = None
        lib.orc_dedisperse_f32.restype = None
        lib.orc_abs_scale_f32.restype = None
        lib.orc_adjoint_f32.restype = None
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def num_threads() -> int:
    return int(clib().orc_num_threads())


def c_dedisperse(I, delays, taps, w=None, t_offset=0, nsamp=None, rows=None):
    """C brute force of eq. p_dedisp; rows selects trial rows (default all).

    uint8 input without weights -> int64; otherwise float32 input -> float64."""
    I = np.ascontiguousarray(I)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    taps = np.ascontiguousarray(taps, dtype=np.int32)
    D, C = delays.shape
    nsamp = I.shape[1] - t_offset if nsamp is None else nsamp
    t_out = nsamp - int((delays.astype(np.int64) + taps - 1).max())
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nrows = D if rows_a is None else len(rows_a)
    lib = clib()
    if I.dtype == np.uint8 and w is None:
        out = np.zeros((nrows, max(t_out, 0)), dtype=np.int64)
        if t_out > 0:
            lib.orc_dedisperse_u8(_p(I), ctypes.c_int64(I.shape[1]), ctypes.c_int32(C),
                                  ctypes.c_int64(t_offset), _p(delays), _p(taps), ctypes.c_int32(D),
                                  ctypes.c_int64(t_out), _p(rows_a), ctypes.c_int32(nrows), _p(out))
        return out
    If = np.ascontiguousarray(I, dtype=np.float32)
    wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    kmax = 0 if wa is None else wa.shape[2]
    out = np.zeros((nrows, max(t_out, 0)), dtype=np.float64)
    if t_out > 0:
        lib.orc_dedisperse_f32(_p(If), ctypes.c_int64(If.shape[1]), ctypes.c_int32(C),
                               ctypes.c_int64(t_offset), _p(delays), _p(taps), _p(wa),
                               ctypes.c_int32(kmax), ctypes.c_int32(D), ctypes.c_int64(t_out),
                               _p(rows_a), ctypes.c_int32(nrows), _p(out))
    return out


def c_abs_scale(I, delays, taps, w=None, t_offset=0, nsamp=None, rows=None):
    """Σ_c Σ_k |w_dck|·|I[c][t+δ+k]| per output: the scale of the fp32 tolerance."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    taps = np.ascontiguousarray(taps, dtype=np.int32)
    D, C = delays.shape
    nsamp = I.shape[1] - t_offset if nsamp is None else nsamp
    t_out = nsamp - int((delays.astype(np.int64) + taps - 1).max())
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nrows = D if rows_a is None else len(rows_a)
    wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    kmax = 0 if wa is None else wa.shape[2]
    out = np.zeros((nrows, max(t_out, 0)), dtype=np.float64)
    if t_out > 0:
        clib().orc_abs_scale_f32(_p(I), ctypes.c_int64(I.shape[1]), ctypes.c_int32(C),
                                 ctypes.c_int64(t_offset), _p(delays), _p(taps), _p(wa),
                                 ctypes.c_int32(kmax), ctypes.c_int32(D), ctypes.c_int64(t_out),
                                 _p(rows_a), ctypes.c_int32(nrows), _p(out))
    return out


def c_adjoint(I, g, delays, taps, w, t_offset=0):
    """C brute force of the adjoint map: (gw [D][C][K] float64, gI [C][ld] float64)."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    g = np.ascontiguousarray(g, dtype=np.float32)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    taps = np.ascontiguousarray(taps, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    D, C = delays.shape
    K = w.shape[2]
    t_out = g.shape[1]
    gw = np.zeros((D, C, K), dtype=np.float64)
    gI = np.zeros((C, I.shape[1]), dtype=np.float64)
    clib().orc_adjoint_f32(_p(I), ctypes.c_int64(I.shape[1]), ctypes.c_int32(C),
                           ctypes.c_int64(t_offset), _p(delays), _p(taps), _p(w), ctypes.c_int32(K),
                           ctypes.c_int32(D), ctypes.c_int64(t_out), _p(g), _p(gw), _p(gI))
    return gw, gI
