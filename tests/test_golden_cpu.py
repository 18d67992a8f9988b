"""Golden fixtures (tests/golden/): values the paper prints, with their
citations, checked against the input generators and the readings built on
them.  The Gaussian dome of Section 6.1: the generator's chordal distance
(the paper's x, y, z) against the spherical law of cosines, the centre and
amplitudes as printed, and the coarse level of alpha = 4/5."""
import json
import math
import os

import numpy as np

import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dome():
    with open(os.path.join(GOLDEN, "gaussian_dome_sec6_1.json")) as fh:
        return json.load(fh)


def test_dome_fixture_carries_its_citation_and_the_printed_values():
    g = dome()
    assert "Section 6.1" in g["citation"]
    p = g["printed"]
    assert (p["h_bar_m"], p["A_m"], p["nu_m2_per_s"], p["R_f"], p["dt_s"]) == (29400.0, 6000.0, 1e5, 256, 100.0)
    assert p["pfasst"] == {"n_ts": 16, "fine_nodes": 5, "coarse_nodes": 3, "N_PF": 8, "alpha": [4, 5]}
    assert syn.NU == p["nu_m2_per_s"]


def test_dome_generator_is_the_printed_chordal_distance():
    """(d/a)^2 = 2 - 2 cos(theta), theta the great-circle angle to the
    centre (lambda_c, phi_c) = (pi, pi/4)."""
    g = dome()
    alpha = g["readings"]["dome_sharpness_alpha"]
    A = g["printed"]["A_m"]
    rng = np.random.default_rng(61)
    mu = rng.uniform(-1.0, 1.0, 40)
    lam = rng.uniform(0.0, 2.0 * math.pi, 50)
    got = syn.gaussian_bump(mu, lam, amplitude=A, width=1.0 / math.sqrt(alpha), lam_c=math.pi, phi_c=math.pi / 4)
    phi = np.arcsin(mu)[:, None]
    cos_theta = (np.sin(phi) * math.sin(math.pi / 4)
                 + np.cos(phi) * math.cos(math.pi / 4) * np.cos(lam[None, :] - math.pi))
    ref = A * np.exp(-alpha * (2.0 - 2.0 * cos_theta))
    assert np.max(np.abs(got - ref)) <= 1e-12 * A
    assert got.max() > 0.5 * A     # the sample reaches the dome


def test_coarse_level_of_the_printed_ratio():
    g = dome()
    num, den = g["printed"]["pfasst"]["alpha"]
    R_c = g["printed"]["R_f"] * num // den
    assert R_c - 1 == 203
    assert syn.gaussian_grid_size(R_c - 1) == (306, 612)
    assert syn.gaussian_grid_size(g["printed"]["R_f"] - 1) == (384, 768)
