"""Python binding of libdd.so: argument marshalling around the C ABI (include/dd.h).

Every step of the computation runs in the library's CUDA kernels; PyTorch supplies
device memory and the current stream.  There is no CPU fallback: a missing library
raises at import of this module's first call.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import DD_F32, DD_U8, check, dd_band, dd_candidate


@dataclass(frozen=True)
class Band:
    """Filterbank geometry (Sec. 2.1): C channels of width df from f_lo, sampling dt."""
    nchan: int
    f_lo_mhz: float
    df_mhz: float
    dt_ms: float
    nsamp: int = 0
    in_type: str = "u8"          # "u8" or "f32"
    descending: bool = False
    k_dm: float = 4.15           # 1/κ in ms·GHz²

    def c_struct(self) -> dd_band:
        return dd_band(int(self.nchan), float(self.f_lo_mhz), float(self.df_mhz),
                       int(bool(self.descending)), float(self.dt_ms), int(self.nsamp),
                       DD_U8 if self.in_type == "u8" else DD_F32, float(self.k_dm))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _np_ptr(a) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if a is None else a.ctypes.data)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def alu_peak(kind: str = "fma", stream=None) -> float:
    """Measured device throughput: "fma" in flops/s (FP32 FMA), "fma2" in flops/s (packed
    FP32 pairs), "iadd" in additions/s."""
    v = ctypes.c_double()
    check(_lib.load().dd_alu_peak({"fma": 0, "iadd": 1, "fma2": 2}[kind], ctypes.cast(ctypes.byref(v), ctypes.c_void_p),
                                  _stream(stream)), "dd_alu_peak")
    return v.value


def predict_rect(band: Band, dm: float, nt: int, t0_ms: float = 0.0, tau_ms: float = 1.0,
                 tau_prime_ms: float = 1.0, alpha: float = 0.0, nu0_ghz: float = 1.0,
                 p0: float = 1.0) -> np.ndarray:
    """Cell-averaged power [nchan][nt] of the rectangular scattered pulse (eq. Pavg)."""
    out = np.zeros((band.nchan, nt), dtype=np.float64)
    b = band.c_struct()
    check(_lib.load().dd_predict_rect(ctypes.cast(ctypes.byref(b), ctypes.c_void_p), float(dm),
                                      float(t0_ms), float(tau_ms), float(tau_prime_ms), float(alpha),
                                      float(nu0_ghz), float(p0), int(nt), _np_ptr(out)),
          "dd_predict_rect")
    return out


def select_samples(pbar: np.ndarray, kmax: int):
    """Sample selection for maximum S/N (Sec. 2.2) on one trial's predicted powers:
    (delay [C], ntaps [C], weights [C][kmax], samples taken, S/N gain)."""
    pbar = np.ascontiguousarray(pbar, dtype=np.float64)
    C, nt = pbar.shape
    delay = np.zeros(C, np.int32)
    taps = np.zeros(C, np.int32)
    w = np.zeros((C, kmax), np.float32)
    nsel = ctypes.c_int32()
    gain = ctypes.c_double()
    check(_lib.load().dd_select_samples(_np_ptr(pbar), C, nt, int(kmax), _np_ptr(delay), _np_ptr(taps),
                                        _np_ptr(w), ctypes.cast(ctypes.byref(nsel), ctypes.c_void_p),
                                        ctypes.cast(ctypes.byref(gain), ctypes.c_void_p)),
          "dd_select_samples")
    return delay, taps, w, nsel.value, gain.value


DETECTORS = {"dsmf": 0, "ts_mf": 1, "ts_boxcar": 2}


def detector_profile(pbar: np.ndarray, kind: str, kmax: int, align=None):
    """A comparison detector of Sec. 5 as one trial's profile: (delay [C], ntaps [C],
    weights [C][kmax], S/N with unit cell noise).  kind: "dsmf", "ts_mf" or "ts_boxcar";
    the time-series detectors align the channels by `align` (the trial's delays)."""
    pbar = np.ascontiguousarray(pbar, dtype=np.float64)
    C, nt = pbar.shape
    al = None if align is None else np.ascontiguousarray(align, dtype=np.int32)
    delay = np.zeros(C, np.int32)
    taps = np.zeros(C, np.int32)
    w = np.zeros((C, kmax), np.float32)
    snr = ctypes.c_double()
    check(_lib.load().dd_detector_profile(_np_ptr(pbar), C, nt, _np_ptr(al), DETECTORS[kind], int(kmax),
                                          _np_ptr(delay), _np_ptr(taps), _np_ptr(w),
                                          ctypes.cast(ctypes.byref(snr), ctypes.c_void_p)),
          "dd_detector_profile")
    return delay, taps, w, snr.value


def select_profiles(band: Band, dms, tau_ms: float = 1.0, tau_prime_ms: float = 1.0,
                    alpha: float = 0.0, nu0_ghz: float = 1.0, phase: float = 0.0):
    """Selected-sample profiles for every trial (pulse arriving `phase` samples into the
    output sample at the top of the band): delay [D][C], ntaps [D][C], weights [D][C][K]
    and each trial's S/N gain over taking every sample with pulse power
    (dd_select_profiles)."""
    lib = _lib.load()
    plan = Plan(band, dms)
    try:
        D, C = plan.ndm, band.nchan
        delay = np.zeros((D, C), np.int32)
        taps = np.zeros((D, C), np.int32)
        gains = np.zeros(D, np.float64)
        kused = ctypes.c_int32(0)
        args = (float(tau_ms), float(tau_prime_ms), float(alpha), float(nu0_ghz), float(phase))
        check(lib.dd_select_profiles(plan._h, *args, 0, _np_ptr(delay), _np_ptr(taps), None,
                                     None, ctypes.cast(ctypes.byref(kused), ctypes.c_void_p)),
              "dd_select_profiles")
        K = int(kused.value)
        w = np.zeros((D, C, K), np.float32)
        check(lib.dd_select_profiles(plan._h, *args, K, _np_ptr(delay), _np_ptr(taps), _np_ptr(w),
                                     _np_ptr(gains), None), "dd_select_profiles")
    finally:
        plan.close()
    return delay, taps, w, gains


def trial_dms(band: Band, dm0: float, dm_max: float, n: int, tau_av_ms: float | None = None,
              smear_terms: int = 2):
    """Trial DMs of eq. trial DMs (Sec. 6.3) ending exactly at dm_max; returns (dms, ε)."""
    lib = _lib.load()
    out = np.zeros(n, dtype=np.float64)
    eps = ctypes.c_double(0.0)
    b = band.c_struct()
    tau = band.dt_ms if tau_av_ms is None else tau_av_ms
    check(lib.dd_trial_dms(ctypes.byref(b), dm0, dm_max, n, tau, smear_terms, _np_ptr(out),
                           ctypes.cast(ctypes.byref(eps), ctypes.c_void_p)), "dd_trial_dms")
    return out, eps.value


class Plan:
    """A dedispersion plan: trial DMs, per-(trial, channel) delays, taps and weights."""

    def __init__(self, band: Band, dms):
        self._lib = _lib.load()
        self.band = band
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.ndm = len(self.dms)
        self._b = band.c_struct()
        h = ctypes.c_void_p()
        check(self._lib.dd_plan_create(ctypes.byref(h), ctypes.byref(self._b), _np_ptr(self.dms),
                                       self.ndm), "dd_plan_create")
        self._h = h
        self._kw = 0

    # ------------------------------------------------------------------ profiles
    def set_profiles(self, delay=None, taps=None, weights=None) -> None:
        """Host tables: delay/taps int32 [D][C], weights fp32 [D][C][K] (None = unit)."""
        d = None if delay is None else np.ascontiguousarray(delay, dtype=np.int32)
        t = None if taps is None else np.ascontiguousarray(taps, dtype=np.int32)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        for a, shp in ((d, (self.ndm, self.band.nchan)), (t, (self.ndm, self.band.nchan))):
            if a is not None and a.shape != shp:
                raise ValueError(f"table shape {a.shape} != {shp}")
        k = 0
        if w is not None:
            if w.ndim != 3 or w.shape[:2] != (self.ndm, self.band.nchan):
                raise ValueError(f"weights shape {w.shape}")
            k = w.shape[2]
        check(self._lib.dd_set_profiles(self._h, _np_ptr(d), _np_ptr(t), _np_ptr(w), k),
              "dd_set_profiles")
        self._kw = k

    def set_weights(self, w: torch.Tensor, stream=None) -> None:
        """Device weights [D][C][K] fp32 (contiguous), copied in stream order."""
        if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous() and w.dim() == 3):
            raise ValueError("weights must be a contiguous CUDA float32 [D][C][K] tensor")
        check(self._lib.dd_set_weights_device(self._h, _ptr(w), int(w.shape[2]), _stream(stream)),
              "dd_set_weights_device")
        self._kw = int(w.shape[2])

    def info(self) -> dict:
        t_out = ctypes.c_int64()
        d_max = ctypes.c_int32()
        kmax = ctypes.c_int32()
        ns = ctypes.c_int64()
        oi = ctypes.c_int32()
        check(self._lib.dd_plan_info(self._h, *(ctypes.cast(ctypes.byref(v), ctypes.c_void_p)
                                                for v in (t_out, d_max, kmax, ns, oi))),
              "dd_plan_info")
        return dict(t_out=t_out.value, d_max=d_max.value, kmax=kmax.value, ns_total=ns.value,
                    out_is_int=bool(oi.value))

    @property
    def d_max(self) -> int:
        return self.info()["d_max"]

    def tables(self):
        d = np.zeros((self.ndm, self.band.nchan), np.int32)
        t = np.zeros((self.ndm, self.band.nchan), np.int32)
        check(self._lib.dd_get_tables(self._h, _np_ptr(d), _np_ptr(t)), "dd_get_tables")
        return d, t

    # ------------------------------------------------------------------ compute
    def _check_input(self, x: torch.Tensor):
        want = torch.uint8 if self.band.in_type == "u8" else torch.float32
        if not x.is_cuda or x.dtype != want or x.dim() != 2 or x.stride(1) != 1:
            raise ValueError(f"input must be a CUDA {want} [C][ld] tensor with unit column stride")
        if x.shape[0] != self.band.nchan:
            raise ValueError("input rows != nchan")
        return x.stride(0)

    def out_dtype(self):
        return torch.int32 if self.info()["out_is_int"] else torch.float32

    def dedisperse(self, x: torch.Tensor, t_offset: int = 0, nsamp: int | None = None,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """eq. p_dedisp for every trial: returns [D][nsamp - d_max]."""
        ld = self._check_input(x)
        nsamp = (x.shape[1] - t_offset) if nsamp is None else nsamp
        t_out = nsamp - self.d_max
        if out is None:
            out = torch.empty((self.ndm, max(t_out, 0)), dtype=self.out_dtype(), device=x.device)
        check(self._lib.dd_dedisperse(self._h, _ptr(x), ld, t_offset, nsamp, _ptr(out),
                                      out.stride(0), _stream(stream)), "dd_dedisperse")
        return out

    def channel_stats(self, x: torch.Tensor, t_offset: int = 0, nsamp: int | None = None,
                      stream=None):
        ld = self._check_input(x)
        nsamp = (x.shape[1] - t_offset) if nsamp is None else nsamp
        mean = torch.empty(self.band.nchan, dtype=torch.float64, device=x.device)
        sd = torch.empty_like(mean)
        check(self._lib.dd_channel_stats(self._h, _ptr(x), ld, t_offset, nsamp, _ptr(mean),
                                         _ptr(sd), _stream(stream)), "dd_channel_stats")
        return mean, sd

    def boxcar_snr(self, series: torch.Tensor, widths, mean: torch.Tensor, sd: torch.Tensor,
                   t_len: int | None = None, thresh: float | None = None, cap: int = 0,
                   stream=None):
        """Boxcar S/N (eq. snr; Sec. 5): returns (peak_snr [D][W], peak_t [D][W], cands)."""
        wl = np.ascontiguousarray(widths, dtype=np.int32)
        t_len = series.shape[1] if t_len is None else t_len
        dev = series.device
        peak = torch.empty((self.ndm, len(wl)), dtype=torch.float32, device=dev)
        arg = torch.empty((self.ndm, len(wl)), dtype=torch.int32, device=dev)
        cands = ncand = None
        if thresh is not None and cap > 0:
            cands = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
            ncand = torch.zeros(1, dtype=torch.int32, device=dev)
        check(self._lib.dd_boxcar_snr(self._h, _ptr(series), series.stride(0), t_len,
                                      _np_ptr(wl), len(wl), _ptr(mean), _ptr(sd), _ptr(peak),
                                      _ptr(arg), float(thresh if thresh is not None else np.inf),
                                      _ptr(cands), int(cap), _ptr(ncand), _stream(stream)),
              "dd_boxcar_snr")
        if cands is None:
            return peak, arg, None
        return peak, arg, (cands, ncand)

    def boxcar_snr_noalloc(self, series: torch.Tensor, widths, mean: torch.Tensor,
                           sd: torch.Tensor, peak: torch.Tensor, arg: torch.Tensor,
                           t_len: int | None = None, thresh: float | None = None,
                           cands: torch.Tensor | None = None, ncand: torch.Tensor | None = None,
                           stream=None) -> None:
        """Boxcar S/N into caller-provided outputs, with no device allocation by the library
        (scratch in a fixed device array); see dd_boxcar_snr_noalloc in include/dd.h."""
        wl = np.ascontiguousarray(widths, dtype=np.int32)
        t_len = series.shape[1] if t_len is None else t_len
        cap = 0 if cands is None else int(cands.shape[0])
        check(self._lib.dd_boxcar_snr_noalloc(self._h, _ptr(series), series.stride(0), t_len,
                                              _np_ptr(wl), len(wl), _ptr(mean), _ptr(sd), _ptr(peak),
                                              _ptr(arg), float(thresh if thresh is not None else np.inf),
                                              _ptr(cands), cap, _ptr(ncand), _stream(stream)),
              "dd_boxcar_snr_noalloc")

    def dedisperse_boxcar(self, x: torch.Tensor, widths, mean: torch.Tensor, sd: torch.Tensor,
                          t_offset: int = 0, nsamp: int | None = None, thresh: float | None = None,
                          cap: int = 0, stream=None):
        """eq. p_dedisp fused with the boxcar S/N (dd_dedisperse_boxcar): the results of
        dedisperse() followed by boxcar_snr() on its output, without storing the dedispersed
        series.  Returns (peak_snr [D][W], peak_t [D][W], cands)."""
        ld = self._check_input(x)
        nsamp = (x.shape[1] - t_offset) if nsamp is None else nsamp
        wl = np.ascontiguousarray(widths, dtype=np.int32)
        dev = x.device
        peak = torch.empty((self.ndm, len(wl)), dtype=torch.float32, device=dev)
        arg = torch.empty((self.ndm, len(wl)), dtype=torch.int32, device=dev)
        cands = ncand = None
        if thresh is not None and cap > 0:
            cands = torch.zeros((cap, 4), dtype=torch.int32, device=dev)
            ncand = torch.zeros(1, dtype=torch.int32, device=dev)
        check(self._lib.dd_dedisperse_boxcar(self._h, _ptr(x), ld, t_offset, nsamp, _np_ptr(wl), len(wl),
                                             _ptr(mean), _ptr(sd), _ptr(peak), _ptr(arg),
                                             float(thresh if thresh is not None else np.inf),
                                             _ptr(cands), int(cap), _ptr(ncand), _stream(stream)),
              "dd_dedisperse_boxcar")
        if cands is None:
            return peak, arg, None
        return peak, arg, (cands, ncand)

    def test_set_fused_parts(self, nparts: int) -> None:
        """Test hook: CTAs (parts) of the fused launches (0 = automatic)."""
        check(self._lib.dd_test_set_fused_parts(self._h, int(nparts)), "dd_test_set_fused_parts")

    def backward(self, x: torch.Tensor, gout: torch.Tensor, t_offset: int = 0,
                 nsamp: int | None = None, want_gw: bool = True, want_gin: bool = True,
                 stream=None):
        """Adjoint of the weighted map: (gw [D][C][K], gI [C][ld])."""
        ld = self._check_input(x)
        nsamp = (x.shape[1] - t_offset) if nsamp is None else nsamp
        gw = gin = None
        if want_gw:
            gw = torch.empty((self.ndm, self.band.nchan, self._kw), dtype=torch.float32, device=x.device)
        if want_gin:
            gin = torch.zeros_like(x)
        check(self._lib.dd_backward(self._h, _ptr(x), ld, t_offset, nsamp, _ptr(gout),
                                    gout.stride(0), _ptr(gw), _ptr(gin),
                                    gin.stride(0) if gin is not None else 0, _stream(stream)),
              "dd_backward")
        return gw, gin

    def exact_profiles(self, tau_prime_ms: float):
        """Delay and tap tables of eq. num_samples with the pulse width tau' (host)."""
        d = np.zeros((self.ndm, self.band.nchan), np.int32)
        t = np.zeros_like(d)
        check(self._lib.dd_exact_profiles(self._h, float(tau_prime_ms), _np_ptr(d), _np_ptr(t)),
              "dd_exact_profiles")
        return d, t

    def set_schedule(self, nch: int, cs: int) -> None:
        check(self._lib.dd_plan_set_schedule(self._h, int(nch), int(cs)), "dd_plan_set_schedule")

    def schedule(self) -> dict:
        nch, cs, tpc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.dd_plan_get_schedule(self._h, *(ctypes.cast(ctypes.byref(v), ctypes.c_void_p)
                                                        for v in (nch, cs, tpc))), "dd_plan_get_schedule")
        return dict(nch=nch.value, cs=cs.value, trials_per_cta=tpc.value)

    METHODS = {"auto": 0, "direct": 1, "runlength": 2}

    def set_method(self, method: str) -> None:
        """Tap sums as direct multiply-adds or as prefix-sum differences ("runlength",
        uint8 unit-weight plans); "auto" picks by mean tap count."""
        check(self._lib.dd_plan_set_method(self._h, self.METHODS[method]), "dd_plan_set_method")

    @property
    def method(self) -> str:
        m = ctypes.c_int32()
        check(self._lib.dd_plan_get_method(self._h, ctypes.cast(ctypes.byref(m), ctypes.c_void_p)),
              "dd_plan_get_method")
        return {1: "direct", 2: "runlength"}[m.value]

    def autotune(self, x: torch.Tensor, out: torch.Tensor, cache_path: str | None = None,
                 stream=None) -> float:
        """Times the CTA shapes and stage sizes that fit on (x, out) and keeps the fastest;
        returns its time in ms (-1 when taken from the cache)."""
        ld = self._check_input(x)
        best = ctypes.c_float(0.0)
        path = None if cache_path is None else cache_path.encode()
        check(self._lib.dd_plan_autotune(self._h, _ptr(x), ld, _ptr(out), out.stride(0), path,
                                         ctypes.cast(ctypes.byref(best), ctypes.c_void_p),
                                         _stream(stream)), "dd_plan_autotune")
        return best.value

    def device_status(self, stream=None) -> int:
        """Synchronises the stream and returns (and clears) the first device-side error
        code a kernel of this plan recorded (0 = none)."""
        code = ctypes.c_int32(0)
        check(self._lib.dd_get_device_status(self._h, ctypes.cast(ctypes.byref(code), ctypes.c_void_p),
                                             _stream(stream)), "dd_get_device_status")
        return code.value

    def test_set_wait(self, skip_stage: int = -1, wait_ns: int = 0) -> None:
        """Test hook: never issue the copies of one channel stage; bound waits by wait_ns."""
        check(self._lib.dd_test_set_wait(self._h, int(skip_stage), int(wait_ns)), "dd_test_set_wait")

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many beams (one plan each) dedispersed in one launch; optionally the
    beams' boxcar S/N too, and the whole block captured as a CUDA graph."""

    def __init__(self, plans):
        self._lib = _lib.load()
        self.plans = list(plans)
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        check(self._lib.dd_batch_create(ctypes.byref(h), arr, n), "dd_batch_create")
        self._h = h
        self._keep = []

    def bind(self, xs, outs) -> None:
        n = len(self.plans)
        ins = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        ild = (ctypes.c_int64 * n)(*[x.stride(0) for x in xs])
        os_ = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        old = (ctypes.c_int64 * n)(*[o.stride(0) for o in outs])
        check(self._lib.dd_batch_bind(self._h, ins, ild, os_, old), "dd_batch_bind")
        self._keep = [list(xs), list(outs)]

    def bind_boxcar(self, widths, means, sds, peaks, args) -> None:
        n = len(self.plans)
        wl = np.ascontiguousarray(widths, dtype=np.int32)
        arrs = [(ctypes.c_void_p * n)(*[t.data_ptr() for t in ts]) for ts in (means, sds, peaks, args)]
        check(self._lib.dd_batch_bind_boxcar(self._h, _np_ptr(wl), len(wl), *arrs), "dd_batch_bind_boxcar")
        self._keep.append([list(means), list(sds), list(peaks), list(args), wl])

    def dedisperse(self, stream=None) -> None:
        check(self._lib.dd_batch_dedisperse(self._h, _stream(stream)), "dd_batch_dedisperse")

    def run(self, stream=None) -> None:
        check(self._lib.dd_batch_run(self._h, _stream(stream)), "dd_batch_run")

    def capture(self, stream) -> None:
        check(self._lib.dd_batch_capture(self._h, _stream(stream)), "dd_batch_capture")

    def replay(self, stream=None) -> None:
        check(self._lib.dd_batch_replay(self._h, _stream(stream)), "dd_batch_replay")

    def info(self) -> dict:
        ni, g, u = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(self._lib.dd_batch_info(self._h, *(ctypes.cast(ctypes.byref(v), ctypes.c_void_p)
                                                 for v in (ni, g, u))), "dd_batch_info")
        return dict(items=ni.value, grid=g.value, units=u.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def candidates_to_list(cands) -> list[tuple[int, int, int, float]]:
    """Decodes the (cap, 4) int32 candidate buffer into (d, width_index, t, snr) tuples."""
    buf, n = cands
    k = min(int(n.item()), buf.shape[0])
    raw = buf[:k].cpu().numpy()
    snr = raw[:, 3].copy().view(np.float32)
    return [(int(r[0]), int(r[1]), int(r[2]), float(s)) for r, s in zip(raw, snr)]


class DDFunction(torch.autograd.Function):
    """Differentiable profiled dedispersion: out = A(w) I.

    Forward stores only its inputs (I, w); the dedispersed series is not kept, and any
    later use of it is recomputed (checkpointing).  Backward calls the adjoint kernels
    for ∂/∂w and ∂/∂I.
    """

    @staticmethod
    def forward(ctx, x, w, plan, t_offset=0, nsamp=None):
        plan.set_weights(w.detach().contiguous())
        out = plan.dedisperse(x.detach(), t_offset=t_offset, nsamp=nsamp)
        ctx.save_for_backward(x, w)
        ctx.plan = plan
        ctx.t_offset = t_offset
        ctx.nsamp = nsamp
        return out

    @staticmethod
    def backward(ctx, gout):
        x, w = ctx.saved_tensors
        plan = ctx.plan
        plan.set_weights(w.detach().contiguous())
        gw, gin = plan.backward(x.detach(), gout.contiguous(), t_offset=ctx.t_offset,
                                nsamp=ctx.nsamp, want_gw=ctx.needs_input_grad[1],
                                want_gin=ctx.needs_input_grad[0])
        return gin, gw, None, None, None
