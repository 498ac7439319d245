"""Degenerate and boundary cases through the C ABI on the GPU: zero input, zero DM,
zero weights, the last valid output, the widest boxcar, maximum tap runs, and argument
errors that only the device path can see."""
import numpy as np
import pytest

import oracle
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("in_type,method", [("u8", "direct"), ("u8", "runlength"), ("f32", "direct")])
def test_zero_input_gives_zero_sums(dd, in_type, method):
    C, T, D = 24, 3008, 12
    b = dd.Band(C, 1200.0, 2.0, 1.0, T, in_type)
    plan = dd.Plan(b, np.linspace(0, 400, D))
    if method == "runlength":
        plan.set_method("runlength")
    I = np.zeros((C, T), np.uint8 if in_type == "u8" else np.float32)
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    assert out.shape == (D, T - plan.d_max) and not out.any()


@pytest.mark.parametrize("in_type", ["u8", "f32"])
def test_dm_zero_is_the_channel_sum(dd, in_type):
    """All trials at DM 0: delays 0 and one tap, so every output is the plain channel sum."""
    rng = np.random.default_rng(101)
    C, T, D = 40, 2048, 6
    I = (rng.integers(0, 256, size=(C, T)).astype(np.uint8) if in_type == "u8"
         else rng.standard_normal((C, T)).astype(np.float32))
    plan = dd.Plan(dd.Band(C, 1200.0, 2.0, 1.0, T, in_type), np.zeros(D))
    delay, taps = plan.tables()
    assert not delay.any() and (taps == 1).all() and plan.d_max == 0
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    want = I.astype(np.int64 if in_type == "u8" else np.float64).sum(axis=0)
    if in_type == "u8":
        np.testing.assert_array_equal(out.astype(np.int64), np.tile(want, (D, 1)))
    else:
        scale = np.abs(I).astype(np.float64).sum(axis=0)
        assert (np.abs(out - want) <= 1e-5 * scale).all()


def test_zero_weights_give_zero(dd):
    rng = np.random.default_rng(102)
    C, T, D = 16, 2048, 4
    I = rng.standard_normal((C, T)).astype(np.float32)
    plan = dd.Plan(dd.Band(C, 1200.0, 2.0, 1.0, T, "f32"), np.linspace(0, 300, D))
    _, taps = plan.tables()
    plan.set_profiles(weights=np.zeros((D, C, int(taps.max())), np.float32))
    assert not plan.dedisperse(_dev(I), nsamp=T).cpu().numpy().any()


@pytest.mark.parametrize("method", ["direct", "runlength"])
def test_single_output_sample(dd, method):
    """nsamp = d_max + 1: one output per trial, the last sample of every run included."""
    rng = np.random.default_rng(103)
    C, D = 20, 30
    delay = rng.integers(0, 300, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, 60, size=(D, C)).astype(np.int32)
    T = int((delay + taps - 1).max()) + 1
    ld = (T + 15) // 16 * 16
    I = np.zeros((C, ld), np.uint8)
    I[:, :T] = rng.integers(0, 256, size=(C, T))
    plan = dd.Plan(dd.Band(C, 1200.0, 2.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method(method)
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    assert out.shape == (D, 1)
    np.testing.assert_array_equal(out.astype(np.int64), oracle.c_dedisperse(I, delay, taps, nsamp=T))


def test_widest_boxcar_spans_the_series(dd):
    """Widths up to the whole series length: the widest boxcar has one start time."""
    rng = np.random.default_rng(104)
    C, T, D = 8, 1024, 3
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    plan = dd.Plan(dd.Band(C, 1200.0, 2.0, 1.0, T, "u8"), np.linspace(0, 100, D))
    x = _dev(I)
    out = plan.dedisperse(x, nsamp=T)
    t_len = out.shape[1]
    mean, sd = plan.channel_stats(x, nsamp=T)
    for widths in (np.array([t_len], np.int32), np.arange(t_len - 20, t_len + 1, dtype=np.int32)):
        peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
        _, taps = plan.tables()
        xo = out.cpu().numpy().astype(np.int64)
        mu, sdw = ref.boxcar_norm(taps, widths, *ref.channel_stats(I, nsamp=T))
        opeak, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
        np.testing.assert_array_equal(arg.cpu().numpy(), oarg)
        np.testing.assert_allclose(peak.cpu().numpy(), opeak, rtol=1e-5, atol=1e-5)
        assert (arg.cpu().numpy()[:, -1] == 0).all()


def test_boxcar_widths_longer_than_series_are_refused(dd):
    import torch
    plan = dd.Plan(dd.Band(4, 1200.0, 2.0, 1.0, 256, "u8"), np.zeros(2))
    out = torch.zeros((2, 256), dtype=torch.int32, device="cuda")
    mean = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(dd.DDError):
        plan.boxcar_snr(out, np.array([1, 300], np.int32), mean, mean + 1)
    with pytest.raises(dd.DDError):
        plan.boxcar_snr(out, np.array([3, 2], np.int32), mean, mean + 1)   # not increasing
