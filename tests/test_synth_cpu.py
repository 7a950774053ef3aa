"""The seeded input generators follow their stated recipe.

Both the CUDA path and the oracle consume these frame sets, so a drift in the
generator (a wrong noise level, a missing vignette, cosmic rays that never
land) would leave every parity test green on inputs unlike the paper's data:
16-bit CCD frames of 60 s exposures with a bias, a dark current and a
vignetted flat, a sky background, point sources moved by the dither offsets
and single-pixel cosmic rays (Sec. 2.1, Sec. 2.2).  Each check below measures
a statistic of generated frames against the number the recipe states.
"""
import numpy as np
import torch

from paper_2008_11486_gb300 import synth

W = H = 256
T = 60.0


def _sky_residual(raw, bias, dark, flat):
    """Raw frames with the bias, the dark current and the flat taken out:
    the sky in electrons plus noise (gain 1)."""
    return (raw.astype(np.float64) - bias - dark * T) / flat


def _check_masters(bias, dark, flat):
    assert bias.dtype == dark.dtype == flat.dtype == np.float32
    assert abs(bias.mean() - 1000.0) < 0.5 and abs(bias.std() - 10.0) < 0.3
    assert dark.min() >= 0.0 and abs(dark.mean() - 0.05) < 1e-3
    assert abs(dark.std() - 0.01) < 1e-3
    # vignetting: about 1 at the centre, 5 % down in the corners, with a 2 %
    # pixel-to-pixel pattern on top
    c = flat[H // 2 - 8:H // 2 + 8, W // 2 - 8:W // 2 + 8].mean()
    corners = np.mean([flat[:8, :8].mean(), flat[:8, -8:].mean(),
                       flat[-8:, :8].mean(), flat[-8:, -8:].mean()])
    assert abs(c - 1.0) < 0.01 and abs(corners - 0.95) < 0.01
    assert 0.02 * 0.9 < np.std(flat[H // 2 - 32:H // 2 + 32, W // 2 - 32:W // 2 + 32]) < 0.02 * 1.2


def test_masters_follow_the_recipe():
    _check_masters(*synth.make_masters(W, H, np.random.Generator(np.random.PCG64(5))))


def test_sky_and_read_noise_levels():
    fs = synth.make_set(W, H, 3, 5.0, 7, n_stars=0, n_cr=0)
    assert fs.raw.dtype == np.uint16 and fs.raw.shape == (3, H, W)
    assert np.all(fs.exptime == np.float32(T))
    r = _sky_residual(fs.raw, fs.bias, fs.dark, fs.flat)
    # Poisson sky of 300 e- plus 10 ADU read noise and rounding:
    # variance about 300 + 100 / flat^2 + 1/12
    assert abs(r.mean() - 300.0) < 0.5
    assert 19.5 < r.std() < 21.0


def test_cosmic_rays_are_single_bright_pixels():
    fs = synth.make_set(W, H, 3, 5.0, 7, n_stars=0, n_cr=20)
    # in ADU: cosmic rays land on the detector after the flat
    r = (_sky_residual(fs.raw, fs.bias, fs.dark, fs.flat) - 300.0) * fs.flat
    for k in range(3):
        hit = r[k] > 2000.0  # 100 sigma above the sky noise
        # 20 per frame; two landing on the same pixel would merge
        assert 18 <= hit.sum() <= 20
        assert np.all((r[k][hit] > 5e3 - 200) & (r[k][hit] < 3e4 + 200))
        assert r[k][~hit].max() < 200.0


def test_stars_add_flux_and_offsets_stay_in_range():
    a = synth.make_set(W, H, 4, 5.0, 11, n_cr=0)
    b = synth.make_set(W, H, 4, 5.0, 11, n_stars=0, n_cr=0)
    assert np.all(np.abs(a.dx) <= 5.0) and np.all(np.abs(a.dy) <= 5.0)
    assert np.ptp(a.dx) > 1.0 and np.ptp(a.dy) > 1.0
    # the star flux (lognormal, median 5e3 e-, 200 stars) adds about
    # 200 * 5e3 * exp(1/2) = 1.6e6 e- per frame, mostly inside the frame
    ra = _sky_residual(a.raw, a.bias, a.dark, a.flat)
    rb = _sky_residual(b.raw, b.bias, b.dark, b.flat)
    excess = (ra - rb).reshape(4, -1).sum(axis=1)
    assert np.all((excess > 3e5) & (excess < 1e7))
    # every frame shows the same scene: total flux agrees across frames
    assert np.ptp(excess) < 0.2 * excess.mean()


def test_generator_is_deterministic_in_its_seed():
    a = synth.make_set(64, 48, 3, 4.0, 99)
    b = synth.make_set(64, 48, 3, 4.0, 99)
    c = synth.make_set(64, 48, 3, 4.0, 100)
    for f in ("raw", "bias", "dark", "flat", "dx", "dy"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.raw, c.raw)


def test_named_workload_shapes():
    bands = synth.workload_bands(W=64, H=32, n=3)
    assert len(bands) == 3 and all(fs.raw.shape == (3, 32, 64) for fs in bands)
    # one master set per band
    assert not np.array_equal(bands[0].bias, bands[1].bias)
    shapes = synth.batch_shapes()
    assert shapes == synth.batch_shapes() and len(shapes) == 64
    assert all(3 <= n <= 40 and w == h and w in (512, 1024, 2048, 4096) for n, w, h in shapes)
    assert len({w for _, w, _ in shapes}) == 4


def test_device_generator_follows_the_same_recipe():
    # the large workloads are drawn with torch on the device; the same code
    # runs on the CPU here
    d = synth.make_set_torch(W, H, 2, 5.0, 3, "cpu", n_stars=0, n_cr=20)
    bias, dark, flat = (d[k].numpy() for k in ("bias", "dark", "flat"))
    _check_masters(bias, dark, flat)
    raw = d["raw"].to(torch.int32).numpy()
    r = _sky_residual(raw, bias, dark, flat)
    assert abs(np.median(r) - 300.0) < 1.0
    for k in range(2):
        hit = r[k] - 300.0 > 2000.0
        assert 18 <= hit.sum() <= 20
        assert 19.5 < r[k][~hit].std() < 21.0
    assert np.all(np.abs(d["dx"]) <= 5.0) and np.all(np.abs(d["dy"]) <= 5.0)
