"""Synthetic dynamic spectra (filterbanks) with seeded noise and dispersed pulses.

Signal model, restated from the paper:

* A pulse emits power per unit bandwidth P0 (ν/ν0)^-α f(t) (eq. intrinsic_power).
* It arrives at frequency ν delayed by DM/(κ ν²) relative to infinite frequency and is
  convolved in time with a unit-area scattering response (eq. P_obs, Sec. 2.1).
  Here 1/κ is written k_dm in ms·GHz² and the delay is taken relative to the top of
  the band.
* Every filterbank sample holds the average of that power over its Δt×Δν cell
  (eq. Pavg).  `cell_average_pulse` evaluates this average on a sub-grid of
  sub-frequencies × sub-samples; `rect_pulse_cells` integrates the rectangular,
  scatter-broadened profile of eq. profile_sb exactly in time (eq. dispersed pulse)
  and on a fine sub-grid in frequency.
* Noise is Gaussian and constant over frequency (radiometer noise, Sec. 2.1).

Channel c has low edge f_lo + c·Δν (ascending order) unless `descending` is set, in
which case channel 0 is the highest.  Nothing here computes dedispersion delay
tables, tap counts, trial DMs, sums or S/N.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 1301
K_DM = 4.15  # 1/κ in ms·GHz² (κ = 2.41e-16 pc cm^-3 s gives 4.1494)

_SUB = {"plain": 1, "craft": 2, "batched": 3, "diff": 4, "large": 5, "tests": 6}


def sub_seed(name: str, index: int = 0) -> int:
    """Per-config seed derived from the master seed 1301."""
    return MASTER_SEED * 1000 + _SUB.get(name, 99) * 100 + index


@dataclass(frozen=True)
class Band:
    nchan: int
    f_lo_mhz: float
    df_mhz: float
    dt_ms: float
    descending: bool = False

    def chan_lo_mhz(self) -> np.ndarray:
        """Low edge of every channel in MHz, in channel order."""
        idx = np.arange(self.nchan, dtype=np.float64)
        if self.descending:
            idx = (self.nchan - 1) - idx
        return self.f_lo_mhz + idx * self.df_mhz

    def chan_centre_ghz(self) -> np.ndarray:
        return (self.chan_lo_mhz() + 0.5 * self.df_mhz) / 1000.0

    @property
    def f_top_ghz(self) -> float:
        return (self.f_lo_mhz + self.nchan * self.df_mhz) / 1000.0


# ----------------------------------------------------------------------------- profiles


def gaussian_profile(fwhm_ms: float):
    """Unit-peak Gaussian intrinsic profile f(t)."""
    a = 4.0 * math.log(2.0) / (fwhm_ms * fwhm_ms)

    def f(t, nu_ghz):
        return np.exp(-a * t * t)

    return f, 4.0 * fwhm_ms, 4.0 * fwhm_ms


def scattered_boxcar_profile(width_ms: float, tau_1ghz_ms: float, tau_index: float = -4.4):
    """Boxcar of unit height and `width_ms` convolved with a one-sided exponential.

    The exponential has unit area and time constant τ(ν) = τ_1GHz·ν^tau_index, so the
    fluence stays width_ms·1 at every frequency (scattering does not attenuate power,
    Sec. 2.1).
    """
    w = float(width_ms)

    def f(t, nu_ghz):
        tau = np.maximum(tau_1ghz_ms * np.power(nu_ghz, tau_index), 1e-9)
        out = np.zeros(np.broadcast(t, tau).shape)
        tt = np.broadcast_to(t, out.shape)
        ta = np.broadcast_to(tau, out.shape)
        rise = (tt >= 0) & (tt <= w)
        out[rise] = 1.0 - np.exp(-tt[rise] / ta[rise])
        tail = tt > w
        out[tail] = np.exp(-(tt[tail] - w) / ta[tail]) - np.exp(-tt[tail] / ta[tail])
        return out

    max_tau = tau_1ghz_ms * 0.5 ** tau_index  # generous bound for bands above 0.5 GHz
    return f, 0.0, w + 12.0 * max_tau


# ----------------------------------------------------------------------------- pulses


def _arrival_ms(nu_ghz, f_top_ghz, dm, k_dm):
    """Cold-plasma arrival delay relative to the top of the band (Sec. 2.1)."""
    return k_dm * dm * (1.0 / (nu_ghz * nu_ghz) - 1.0 / (f_top_ghz * f_top_ghz))


def cell_average_pulse(band: Band, nsamp: int, dm: float, t0_ms: float, profile,
                       amp: float = 1.0, alpha: float = 0.0, nu0_ghz: float = 1.0,
                       nsub_f: int = 16, nsub_t: int = 16, k_dm: float = K_DM):
    """Cell-averaged dispersed pulse (eq. Pavg divided by Δν, i.e. a mean power).

    `profile` is (f(t, ν), lead_ms, tail_ms).  t0_ms is the arrival time at the top of
    the band.  Returns a list of (channel, first_sample, values[float64]).
    """
    f, lead, tail = profile
    lo = band.chan_lo_mhz() / 1000.0
    dnu = band.df_mhz / 1000.0
    out = []
    sub_f = (np.arange(nsub_f) + 0.5) / nsub_f
    sub_t = (np.arange(nsub_t) + 0.5) / nsub_t
    for c in range(band.nchan):
        nus = lo[c] + sub_f * dnu                                  # [F]
        td = _arrival_ms(nus, band.f_top_ghz, dm, k_dm)           # [F]
        n0 = int(math.floor((t0_ms + td.min() - lead) / band.dt_ms)) - 1
        n1 = int(math.ceil((t0_ms + td.max() + tail) / band.dt_ms)) + 1
        n0 = max(n0, 0)
        n1 = min(n1, nsamp)
        if n1 <= n0:
            continue
        ns = np.arange(n0, n1, dtype=np.float64)
        t = (ns[None, :, None] + sub_t[None, None, :]) * band.dt_ms    # [1,N,S]
        rel = t - t0_ms - td[:, None, None]                            # [F,N,S]
        spec = amp * np.power(nus / nu0_ghz, -alpha)                   # [F]
        val = f(rel, nus[:, None, None]) * spec[:, None, None]
        out.append((c, n0, val.mean(axis=(0, 2))))
    return out


def rect_pulse_cells(band: Band, nsamp: int, dm: float, t0_ms: float, tau_ms: float,
                     tau_prime_ms: float, alpha: float = 0.0, nu0_ghz: float = 1.0,
                     p0: float = 1.0, nsub_f: int = 64, k_dm: float = K_DM) -> np.ndarray:
    """Dense [C][T] array of P̄ for the rectangular scattered pulse (eq. dispersed pulse).

    P̄(t,ν) = (P0/Δt) ∫dν' (ν'/ν0)^-α ∫_t^{t+Δt} dt' [H(t'-t_d) - H(t'-t_d-τ')] τ/τ'.
    The time integral is the exact overlap length.  The frequency integral is a
    midpoint rule on sub-channels, at least `nsub_f` per channel and fine enough that
    one sub-channel's own sweep stays below τ'/16 (ν in GHz, so P̄ carries a GHz
    factor).
    """
    lo = band.chan_lo_mhz() / 1000.0
    dnu = band.df_mhz / 1000.0
    out = np.zeros((band.nchan, nsamp), dtype=np.float64)
    dt = band.dt_ms
    ncell = int(math.ceil(tau_prime_ms / dt)) + 2
    for c in range(band.nchan):
        sweep = k_dm * dm * (1.0 / lo[c] ** 2 - 1.0 / (lo[c] + dnu) ** 2)
        nf = max(nsub_f, int(math.ceil(16.0 * sweep / tau_prime_ms)))
        nus = lo[c] + (np.arange(nf) + 0.5) / nf * dnu
        a = t0_ms + _arrival_ms(nus, band.f_top_ghz, dm, k_dm)    # pulse start [F]
        b = a + tau_prime_ms
        first = np.floor(a / dt).astype(np.int64)
        cells = first[:, None] + np.arange(ncell)[None, :]        # [F, m]
        ts = cells * dt
        overlap = np.clip(np.minimum(ts + dt, b[:, None]) - np.maximum(ts, a[:, None]), 0.0, None)
        wgt = np.power(nus / nu0_ghz, -alpha) * (dnu / nf)       # dν' weights
        val = p0 / dt * wgt[:, None] * overlap * (tau_ms / tau_prime_ms)
        ok = (cells >= 0) & (cells < nsamp) & (val > 0)
        np.add.at(out[c], cells[ok], val[ok])
    return out


def add_cells(arr: np.ndarray, cells, scale: float = 1.0) -> None:
    for c, n0, vals in cells:
        arr[c, n0:n0 + len(vals)] += scale * vals


# ----------------------------------------------------------------------------- noise


def noise_f32(rng: np.random.Generator, nchan: int, nsamp: int, ld: int | None = None) -> np.ndarray:
    """N(0,1) float32 noise, rows padded to `ld` columns (padding is zero)."""
    ld = nsamp if ld is None else ld
    out = np.zeros((nchan, ld), dtype=np.float32)
    out[:, :nsamp] = rng.standard_normal((nchan, nsamp), dtype=np.float32)
    return out


def noise_u8(rng: np.random.Generator, nchan: int, nsamp: int, mean: float = 128.0,
             sigma: float = 16.0, ld: int | None = None, signal=None) -> np.ndarray:
    """clamp(round_half_even(mean + σ·N(0,1) + signal)) as uint8, row by row.

    `signal` is an optional list of (channel, first_sample, values) added before
    quantisation.  Rows are generated one at a time so that 2^30-sample inputs fit.
    """
    ld = nsamp if ld is None else ld
    out = np.zeros((nchan, ld), dtype=np.uint8)
    by_chan: dict[int, list] = {}
    for c, n0, vals in (signal or []):
        by_chan.setdefault(c, []).append((n0, vals))
    for c in range(nchan):
        row = rng.standard_normal(nsamp, dtype=np.float32) * np.float32(sigma) + np.float32(mean)
        for n0, vals in by_chan.get(c, []):
            row[n0:n0 + len(vals)] += vals.astype(np.float32)
        out[c, :nsamp] = np.clip(np.rint(row), 0, 255).astype(np.uint8)
    return out


def spectral_weights(band: Band, index: float = -1.4, nu_ref_ghz: float = 1.298) -> np.ndarray:
    """Per-channel weight factors (ν_centre/ν_ref)^index, float32 [C]."""
    return np.power(band.chan_centre_ghz() / nu_ref_ghz, index).astype(np.float32)


def _pad16(n: int, elem: int) -> int:
    q = 16 // elem
    return (n + q - 1) // q * q


# ----------------------------------------------------------------------------- configs

PLAIN_BAND = Band(64, 1200.0, 4.6875, 1.0)
CRAFT_BAND = Band(336, 1130.0, 1.0, 1.0)
LARGE_BAND = Band(1024, 700.0, 300.0 / 1024.0, 0.064)


def make_plain(seed: int | None = None, nsamp: int = 4096, dm: float = 300.0,
               t0_ms: float = 1000.0, snr_total: float = 8.0):
    """64 ch over 1200–1500 MHz, Δt = 1 ms, uint8 N(128,16²) plus one Gaussian pulse.

    The pulse has FWHM 2 ms and per-channel peak snr_total·σ/√C (= 16 counts for the
    default 8), so the aligned channel sum of the unsmeared pulse has single-sample
    S/N snr_total.
    """
    seed = sub_seed("plain") if seed is None else seed
    rng = np.random.default_rng(seed)
    band = PLAIN_BAND
    amp = snr_total * 16.0 / math.sqrt(band.nchan)
    cells = cell_average_pulse(band, nsamp, dm, t0_ms, gaussian_profile(2.0), amp=amp)
    data = noise_u8(rng, band.nchan, nsamp, ld=_pad16(nsamp, 1), signal=cells)
    dms = np.linspace(0.0, 500.0, 128)
    return dict(band=band, data=data, nsamp=nsamp, dms=dms, pulse=dict(dm=dm, t0_ms=t0_ms))


def _craft_like_pulses(rng, band, nsamp, npulse, dm_lo, dm_hi, alpha_lo, alpha_hi, amp):
    pulses = []
    cells = []
    span = nsamp * band.dt_ms
    for i in range(npulse):
        dm = float(rng.uniform(dm_lo, dm_hi))
        alpha = float(rng.uniform(alpha_lo, alpha_hi))
        tau1 = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        t0 = float(rng.uniform(0.05, 0.85) * span)
        prof = scattered_boxcar_profile(1.0, tau1)
        cells += cell_average_pulse(band, nsamp, dm, t0, prof, amp=amp, alpha=alpha,
                                    nu0_ghz=1.298, nsub_f=8, nsub_t=8)
        pulses.append(dict(dm=dm, alpha=alpha, tau_1ghz_ms=tau1, t0_ms=t0))
    return pulses, cells


def make_craft(seed: int | None = None, nsamp: int = 65536, npulse: int = 16, amp: float = 1.0):
    """336 × 1 MHz over 1130–1466 MHz, Δt = 1 ms, float32 N(0,1) plus scattered pulses."""
    seed = sub_seed("craft") if seed is None else seed
    rng = np.random.default_rng(seed)
    band = CRAFT_BAND
    data = noise_f32(rng, band.nchan, nsamp, ld=_pad16(nsamp, 4))
    pulses, cells = _craft_like_pulses(rng, band, nsamp, npulse, 50.0, 3900.0, 0.0, 3.0, amp)
    for c, n0, vals in cells:
        data[c, n0:n0 + len(vals)] += vals.astype(np.float32)
    return dict(band=band, data=data, nsamp=nsamp, pulses=pulses,
                wchan=spectral_weights(band), widths=np.arange(1, 33, dtype=np.int32),
                dm_max=4000.0, ndm=4096)


def make_diff(seed: int | None = None, nsamp: int = 16384, npulse: int = 64, amp: float = 1.0,
              pulse_dms=None):
    """336 channels, 16384 fp32 samples; pulses with spectral index in [-3, +1].

    `pulse_dms` (the trial DMs the pulses sit on) is supplied by the caller, since the
    trial list belongs to the method.
    """
    seed = sub_seed("diff") if seed is None else seed
    rng = np.random.default_rng(seed)
    band = CRAFT_BAND
    data = noise_f32(rng, band.nchan, nsamp, ld=_pad16(nsamp, 4))
    pulses = []
    span = nsamp * band.dt_ms
    for i in range(npulse):
        dm = float(pulse_dms[i]) if pulse_dms is not None else float(rng.uniform(50, 1900))
        alpha = float(rng.uniform(-3.0, 1.0))
        tau1 = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        t0 = float(rng.uniform(0.02, 0.8) * span)
        prof = scattered_boxcar_profile(1.0, tau1)
        cells = cell_average_pulse(band, nsamp, dm, t0, prof, amp=amp, alpha=alpha,
                                   nu0_ghz=1.298, nsub_f=8, nsub_t=8)
        add_cells(data, cells)
        pulses.append(dict(dm=dm, alpha=alpha, tau_1ghz_ms=tau1, t0_ms=t0))
    return dict(band=band, data=data, nsamp=nsamp, pulses=pulses)


def make_large(seed: int | None = None, nsamp: int = 1 << 20, npulse: int = 8, with_data: bool = True):
    """1024 ch over 700–1000 MHz, Δt = 64 µs, uint8 noise plus Gaussian pulses."""
    seed = sub_seed("large") if seed is None else seed
    rng = np.random.default_rng(seed)
    band = LARGE_BAND
    span = nsamp * band.dt_ms
    cells = []
    pulses = []
    for i in range(npulse):
        dm = float(rng.uniform(100.0, 1900.0))
        t0 = float(rng.uniform(0.05, 0.6) * span)
        amp = 8.0 * 16.0 / math.sqrt(band.nchan) * 2.0
        cells += cell_average_pulse(band, nsamp, dm, t0, gaussian_profile(1.0), amp=amp,
                                    nsub_f=4, nsub_t=4)
        pulses.append(dict(dm=dm, t0_ms=t0))
    data = noise_u8(rng, band.nchan, nsamp, ld=_pad16(nsamp, 1), signal=cells) if with_data else None
    return dict(band=band, data=data, nsamp=nsamp, pulses=pulses,
                dms=np.linspace(0.0, 2000.0, 8192), widths=np.arange(1, 257, dtype=np.int32))


def make_batched_beams(seed: int | None = None, nbeams: int = 36, t_exp=(14, 17), d_exp=(9, 13)):
    """Seeded beam shapes: T_b = round(2^U[14,17]), D_b = round(2^U[9,13]),
    DM_max,b = logU[500, 4000]; every beam uses the CRAFT band and uint8 samples.
    t_exp and d_exp narrow the exponent ranges (e.g. the lower end of both)."""
    seed = sub_seed("batched") if seed is None else seed
    rng = np.random.default_rng(seed)
    beams = []
    for b in range(nbeams):
        T = int(round(2.0 ** rng.uniform(*t_exp)))
        D = int(round(2.0 ** rng.uniform(*d_exp)))
        dmax = float(math.exp(rng.uniform(math.log(500.0), math.log(4000.0))))
        beams.append(dict(nsamp=T, ndm=D, dm_max=dmax, seed=seed * 100 + b))
    return dict(band=CRAFT_BAND, beams=beams)


def make_beam_data(beam: dict, band: Band = CRAFT_BAND, npulse: int = 2):
    """uint8 noise as in the plain config plus `npulse` Gaussian pulses for one beam."""
    rng = np.random.default_rng(beam["seed"])
    T = beam["nsamp"]
    cells = []
    for i in range(npulse):
        dm = float(rng.uniform(0.1, 0.9) * beam["dm_max"])
        t0 = float(rng.uniform(0.05, 0.5) * T * band.dt_ms)
        cells += cell_average_pulse(band, T, dm, t0, gaussian_profile(2.0),
                                    amp=8.0 * 16.0 / math.sqrt(band.nchan), nsub_f=4, nsub_t=4)
    return noise_u8(rng, band.nchan, T, ld=_pad16(T, 1), signal=cells)
