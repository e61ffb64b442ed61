"""The seeded input generators: the fan-beam rays of the synthetic data pass through the
source and their bin, and the analytic data of a disk are its chords along them."""
import numpy as np

from paper_2501_12497_gb300 import synth


def test_fan_rays_pass_through_the_source_and_the_bin():
    rng = np.random.default_rng(0)
    th = rng.uniform(0, 2 * np.pi, 50)
    sig = rng.uniform(-80, 80, 50)
    rs, rd = 120.0, 45.0
    phi, p = synth.fan_rays(th, sig, rs, rd)
    e = np.stack([-np.sin(th), np.cos(th)], 1)
    f = np.stack([np.cos(th), np.sin(th)], 1)
    n = np.stack([np.cos(phi), np.sin(phi)], 1)
    S = -rs * e
    D = rd * e + sig[:, None] * f
    np.testing.assert_allclose(np.sum(S * n, 1), p, atol=1e-10)
    np.testing.assert_allclose(np.sum(D * n, 1), p, atol=1e-10)


def test_fan_data_of_a_centred_disk_are_its_chords():
    """A disk of radius r at the centre: the ray of bin sigma passes at distance
    rs sigma / sqrt(sigma^2 + (rs + rd)^2) from it (similar triangles)."""
    rs, rd, r, rho = 100.0, 50.0, 30.0, 0.7
    sig = np.linspace(-60, 60, 41)
    phi, p = synth.fan_rays(0.3, sig, rs, rd)
    got = synth.ellipse_radon((0.0, 0.0, r, r, 0.0, rho), phi, p)
    d = rs * np.abs(sig) / np.sqrt(sig ** 2 + (rs + rd) ** 2)
    want = np.where(d < r, 2 * rho * np.sqrt(np.maximum(r * r - d * d, 0.0)), 0.0)
    np.testing.assert_allclose(got, want, atol=1e-9)


def test_fan_workloads_keep_the_field_of_view_on_the_detector():
    for w in (synth.fan_form_small(0),):
        bb = w.b_clean.reshape(-1, w.nb)
        assert np.all(bb[:, :2] == 0) and np.all(bb[:, -2:] == 0) and bb.max() > 0
