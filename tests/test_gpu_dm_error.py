"""DM-error analysis through the GPU path (Sec. 6, eq. snrb/snri_approx and the trial
spacing of eq. trial DMs): noise-free rectangular pulses (eq. dispersed pulse, cell
averages of eq. Pavg) at true DMs swept across one trial interval are dedispersed and
boxcar-scanned on the GPU with unit-variance channel noise in the normaliser.  The best
S/N over the trials and widths, relative to a pulse on a trial DM, matches the oracle and
bottoms out midway between trials near the drop-out (eps^2 + 1)^(-1/4)."""
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


@pytest.mark.parametrize("ntrials", [300, 150, 80])
def test_dm_error_sweep_dropout(dd, ntrials):
    import torch
    b = synth.CRAFT_BAND
    T = 6144
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    dms_all, eps = dd.trial_dms(band, 0.0, 1000.0, ntrials, tau_av_ms=1.0)
    k = int(np.searchsorted(dms_all, 500.0))
    dms = dms_all[k - 2:k + 4]
    plan = dd.Plan(band, dms)                      # unit weights, fp32 sums
    delay, taps = plan.tables()
    widths = np.arange(1, 33, dtype=np.int32)
    mean = torch.zeros(b.nchan, dtype=torch.float64, device="cuda")
    sd = torch.ones(b.nchan, dtype=torch.float64, device="cuda")
    mu, sdw = ref.boxcar_norm(taps, widths, np.zeros(b.nchan), np.ones(b.nchan))
    w1 = np.ones((len(dms), b.nchan, int(taps.max())), np.float32)
    fracs = np.linspace(0.0, 1.0, 9)
    gpu, orc = [], []
    for f in fracs:
        dm_true = dms_all[k] + f * (dms_all[k + 1] - dms_all[k])
        P = synth.rect_pulse_cells(b, T, dm_true, 3000.0, 1.0, 1.0).astype(np.float32)
        x = plan.dedisperse(torch.from_numpy(P).cuda(), nsamp=T)
        peak, _, _ = plan.boxcar_snr(x, widths, mean, sd)
        gpu.append(float(peak.max()))
        xo = ref.dedisperse(P, delay, taps, w=w1)
        opeak, _, _ = ref.boxcar_snr(xo, widths, mu, sdw)
        orc.append(float(opeak.max()))
    gpu, orc = np.array(gpu), np.array(orc)
    np.testing.assert_allclose(gpu, orc, rtol=1e-5)
    rel = gpu / gpu[0]
    assert abs(rel[-1] - 1.0) < 0.05                 # the next trial recovers the pulse
    assert int(np.argmin(rel)) == 4                  # worst midway between the trials
    floor = ref.dropout(eps)
    assert floor - 0.02 <= rel.min() <= floor + 0.08
