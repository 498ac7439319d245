"""Selected-sample profiles (Sec. 2.2) through the GPU path: on the paper's nominal
resolution point the selected profiles raise the dedispersed S/N of matched noise-free
pulses by the gain the selection predicts (~20 %), against profiles that take every
sample with pulse power, and both agree with the oracle."""
import numpy as np
import pytest

from oracle import ref
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as m
    torch.cuda.set_device(0)
    return m


def test_selected_profiles_gain_on_gpu(dd):
    import torch
    C, dt = 122, 1.0
    b = synth.Band(C, 700.0, 300.0 / C, dt)
    T = 2800
    band = dd.Band(C, b.f_lo_mhz, b.df_mhz, dt, T, "f32")
    dms = np.linspace(26.0, 34.0, 8)
    delay_s, taps_s, w_s, gains = dd.select_profiles(band, dms, tau_ms=1.0, tau_prime_ms=1.0)
    sel = dd.Plan(band, dms)
    sel.set_profiles(delay=delay_s, taps=taps_s, weights=w_s)
    # every cell the model gives pulse power (the set the gain is relative to)
    delay_f = np.zeros((len(dms), C), np.int32)
    taps_f = np.zeros((len(dms), C), np.int32)
    for d, dm in enumerate(dms):
        P = synth.rect_pulse_cells(b, 400, dm, 0.0, 1.0, 1.0)
        for c in range(C):
            nz = np.flatnonzero(P[c] > 0)
            delay_f[d, c], taps_f[d, c] = nz[0], nz[-1] - nz[0] + 1
    full = dd.Plan(band, dms)
    full.set_profiles(delay=delay_f, taps=taps_f)
    # one matched pulse per trial, arriving at the top of the band on a sample boundary
    t_arr = [150 + 320 * i for i in range(len(dms))]
    I = np.zeros((C, T), np.float64)
    for dm, t in zip(dms, t_arr):
        I += synth.rect_pulse_cells(b, T, dm, t * dt, 1.0, 1.0)
    I = I.astype(np.float32)
    x = torch.from_numpy(I).cuda()
    xs = sel.dedisperse(x, nsamp=T).cpu().numpy()
    xf = full.dedisperse(x, nsamp=T).cpu().numpy()
    pts = list(zip(range(len(dms)), t_arr))
    a = np.array([xs[d, t] for d, t in pts], np.float64)
    f = np.array([xf[d, t] for d, t in pts], np.float64)
    np.testing.assert_allclose(a, ref.dedisperse_points(I, delay_s, taps_s, pts, w=w_s), rtol=1e-5)
    wf = np.ones((len(dms), C, int(taps_f.max())), np.float32)
    np.testing.assert_allclose(f, ref.dedisperse_points(I, delay_f, taps_f, pts, w=wf), rtol=1e-5)
    # S/N with unit cell noise: sum / sqrt(sum of squared weights)
    snr_sel = a / np.sqrt((w_s.astype(np.float64) ** 2).sum(axis=(1, 2)))
    snr_all = f / np.sqrt(taps_f.sum(axis=1))
    np.testing.assert_allclose(snr_sel / snr_all, gains, rtol=1e-4)
    assert (gains > 1.15).all() and (gains < 1.25).all()


def test_comparison_detectors_on_gpu(dd):
    """Sec. 5 detectors as profiles on the same kernel: the GPU S/N of a matched noise-free
    pulse equals each detector's closed form, and the dynamic-spectrum matched filter is
    the best of them."""
    import torch
    C, dt, dm = 122, 1.0, 30.0
    b = synth.Band(C, 700.0, 300.0 / C, dt)
    T, t_arr = 1024, 200
    band = dd.Band(C, b.f_lo_mhz, b.df_mhz, dt, T, "f32")
    P = synth.rect_pulse_cells(b, 600, dm, 0.0, 1.0, 1.0)      # predicted cells, arrival at 0
    I = synth.rect_pulse_cells(b, T, dm, t_arr * dt, 1.0, 1.0).astype(np.float32)
    x = torch.from_numpy(I).cuda()
    align = ref.delay_table([dm], C, 700.0, 300.0 / C, dt)[0][0].astype(np.int32)
    snrs = {}
    for kind in ("dsmf", "ts_mf", "ts_boxcar", "selection"):
        if kind == "selection":
            delay, taps, w, _, _ = dd.select_samples(P, 600)
            want = ref.set_snr(P, ref.select_samples(P))
        else:
            delay, taps, w, want = dd.detector_profile(P, kind, 600, align=align)
        K = int(taps.max())
        plan = dd.Plan(band, [dm])
        plan.set_profiles(delay=delay[None, :], taps=taps[None, :], weights=w[None, :, :K])
        out = plan.dedisperse(x, nsamp=T).cpu().numpy()
        snr = float(out[0, t_arr]) / np.sqrt((w.astype(np.float64) ** 2).sum())
        assert snr == pytest.approx(want, rel=1e-5)
        snrs[kind] = snr
    assert snrs["dsmf"] >= max(snrs.values()) * (1 - 1e-6)
    assert snrs["ts_mf"] >= snrs["ts_boxcar"]
