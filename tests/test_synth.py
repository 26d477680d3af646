"""Host checks of the seeded input generators (no method arithmetic lives there)."""
import numpy as np

from paper_2304_13144_gb300 import synth


def _min_image_dmin(pos, L):
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return r.min()


def test_liquid_rsa_density_and_minimum_distance():
    b = synth.liquid_rsa(seed=5, n_atoms=300)
    L = b["cell"][0, 0, 0]
    assert len(b["type"]) == 300
    assert abs(300 / L ** 3 - 0.085) < 1e-12
    assert np.all((b["pos"] >= 0) & (b["pos"] < L))
    assert _min_image_dmin(b["pos"], L) >= 1.8
    assert set(np.unique(b["type"])) <= {0, 1, 2, 3}


def test_liquid_rsa_tiling_is_seamless():
    b = synth.liquid_rsa(seed=6, n_atoms=8 * 150, tiles=2)
    L = b["cell"][0, 0, 0]
    assert abs(len(b["type"]) / L ** 3 - 0.085) < 1e-12
    assert _min_image_dmin(b["pos"], L) >= 1.8
    # the eight copies are translates of the first
    base = b["pos"][:150]
    for t in range(1, 8):
        shift = b["pos"][150 * t:150 * (t + 1)] - base
        assert np.allclose(shift, shift[0]) and np.allclose(np.abs(shift[0]) % (L / 2), 0, atol=1e-9)


def test_generators_are_seeded():
    a = synth.fcc_ternary(seed=4, n=3)
    b = synth.fcc_ternary(seed=4, n=3)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["type"], b["type"])
    c = synth.liquid_rsa(seed=5, n_atoms=200)
    d = synth.liquid_rsa(seed=5, n_atoms=200)
    assert np.array_equal(c["pos"], d["pos"])
