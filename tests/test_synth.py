"""The seeded synthetic inputs follow their stated recipes: reproducible from (recipe, seed),
clean images in [0, 1] on their stated backgrounds, noise with the stated statistics, noisy
images exactly representable in float32, and the batch and serving mixes inside their ranges."""
import numpy as np
import pytest

from paper_2108_10209_gb300 import synth


def test_same_seed_same_image_other_seed_other_image():
    a = synth.image_cells(128, 96, seed=5)[1]
    assert np.array_equal(a, synth.image_cells(128, 96, seed=5)[1])
    assert not np.array_equal(a, synth.image_cells(128, 96, seed=6)[1])


@pytest.mark.parametrize("make", [lambda: synth.image_small(3),
                                  lambda: synth.image_cells(96, 80, seed=3),
                                  lambda: synth.image_cells_pg(96, 80, seed=3)])
def test_noisy_images_are_float32_values(make):
    clean, noisy = make()
    assert clean.min() >= 0.0 and clean.max() <= 1.0
    assert np.array_equal(noisy, noisy.astype(np.float32).astype(np.float64))


def test_backgrounds_and_intensities():
    b = synth.blobs(32, 32, seed=1)
    assert b.min() >= 0.1 - 1e-12                      # blobs add to the 0.1 background
    e = synth.ellipses(256, 256, seed=2, blur=0)
    vals = np.unique(e)
    assert vals[0] == 0.05                             # background, unblurred
    assert np.all((vals[1:] >= 0.2) & (vals[1:] <= 1.0))  # painted intensities U(0.2, 1.0)


def test_gaussian_noise_statistics():
    clean = np.full((512, 512), 0.5)
    sigma = 25.0 / 255.0
    r = synth.gaussian_noise(clean, sigma, seed=11) - clean
    assert abs(r.mean()) < 4 * sigma / 512             # 4 standard errors
    assert abs(r.std() / sigma - 1) < 0.01


def test_poisson_gaussian_statistics():
    # y = Poisson(peak s) / peak + N(0, read^2): mean s, variance s / peak + read^2
    s, peak, read = 0.4, 30.0, 0.02
    y = synth.poisson_gaussian(np.full((512, 512), s), peak, read, seed=12)
    assert abs(y.mean() - s) < 4 * np.sqrt(s / peak + read ** 2) / 512
    assert abs(y.var() / (s / peak + read ** 2) - 1) < 0.02


def test_u16_round_trip_is_within_half_a_step():
    x = np.random.default_rng(0).uniform(-0.1, 1.1, size=1000)
    q = synth.from_u16(synth.to_u16(x))
    inside = (x >= 0) & (x <= 1)
    assert np.all(np.abs(q[inside] - x[inside]) <= 0.5 / 65535 + 1e-15)
    assert np.all(q[x < 0] == 0.0) and np.all(q[x > 1] == 1.0)


def test_psnr():
    ref = np.zeros((4, 4))
    assert synth.psnr(ref, ref) == float("inf")
    assert abs(synth.psnr(ref + 0.1, ref) - 20.0) < 1e-9


def test_batch_and_serving_mixes_stay_in_range():
    jobs = synth.batch_jobs(200, seed=1)
    assert {(j["h"], j["w"]) for j in jobs} <= set(synth.BATCH_SIZES)
    assert all(15 / 255 <= j["sigma"] <= 50 / 255 for j in jobs)
    reqs = synth.serving_stream(300, rate=4.0, seed=2, smin=256, smax=1024)
    t = np.array([q["t"] for q in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] / 4.0 - 1) < 0.2           # Poisson arrivals at the stated rate
    assert all(256 <= q["side"] <= 1024 and q["side"] % 2 == 0 for q in reqs)
