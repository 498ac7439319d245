"""Replicas-only multi-GPU path on one GPU (a plan split into DM ranges reproduces the
one-shot sums), and the measured ALU peaks."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("in_type", ["u8", "f32"])
def test_dm_range_split_concatenates(dd, in_type):
    """Three contiguous DM ranges (as three GPUs would take them) concatenate to the
    one-shot result over the one-shot plan's output span, bit for bit."""
    import torch
    b = synth.CRAFT_BAND
    T = 12288
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, in_type)
    dms, _ = dd.trial_dms(band, 0.0, 2000.0, 96, tau_av_ms=1.0)
    rng = np.random.default_rng(91)
    if in_type == "u8":
        I = rng.integers(0, 256, size=(b.nchan, T)).astype(np.uint8)
    else:
        I = rng.standard_normal((b.nchan, T)).astype(np.float32)
    x = torch.from_numpy(I).cuda()

    def plan_for(sel):
        p = dd.Plan(band, dms[sel])
        if in_type == "f32":
            _, taps = p.tables()
            K = int(taps.max())
            w = np.where(np.arange(K)[None, None, :] < taps[:, :, None],
                         synth.spectral_weights(b)[None, :, None], 0.0).astype(np.float32)
            p.set_profiles(weights=w)
        return p

    full = plan_for(slice(0, 96))
    ref = full.dedisperse(x, nsamp=T).cpu().numpy()
    parts = []
    for lo, hi in ((0, 32), (32, 64), (64, 96)):
        p = plan_for(slice(lo, hi))
        parts.append(p.dedisperse(x, nsamp=T).cpu().numpy()[:, :ref.shape[1]])
    np.testing.assert_array_equal(np.concatenate(parts, axis=0), ref)


def test_measured_alu_peaks_are_plausible(dd):
    import torch
    fma = dd.alu_peak("fma")
    fma2 = dd.alu_peak("fma2")
    iadd = dd.alu_peak("iadd")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.07e9           # FP32 lanes x 2 flops x max SM clock
    assert 0.3 * derived < fma < 1.1 * derived
    # packed pairs: two FMAs per instruction, at most twice the scalar rate
    assert 0.3 * derived < fma2 < 2.2 * derived
    assert 0.1 * derived < iadd < 2.2 * derived    # additions: two per three-input add
