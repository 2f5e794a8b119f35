"""The k-nearest-neighbour preparation of the halo mixture (input preparation, as an SPH code would do it):
h is the distance to the 32nd nearest neighbour and the value the SPH density estimate over those
neighbours, both against brute force on a small set."""
import math

import numpy as np

from paper_2401_02896_b300 import synthetic as SY


def test_knn_h_and_density_match_brute_force():
    n = 3000
    P = SY.halo_mixture_knn(n, seed=SY.BASE_SEED + 77)
    A = SY.halo_mixture(n, seed=SY.BASE_SEED + 77)
    assert np.array_equal(P["pos"], A["pos"])  # the same positions as the analytic variant
    x = P["pos"].astype(np.float64)
    idx = np.random.default_rng(3).choice(n, 64, replace=False)
    for i in idx:
        d = np.sort(np.linalg.norm(x - x[i], axis=1))  # d[0] = 0: the particle itself
        H = d[32]
        assert abs(P["h"][i] - H) <= 1e-6 * H
        u = d[:33] / H
        w = np.array([1 - 6 * v * v + 6 * v ** 3 if v < 0.5 else (2 * (1 - v) ** 3 if v < 1 else 0.0) for v in u])
        rho = (1.0 / n) * 8.0 / (math.pi * H ** 3) * w.sum()
        assert abs(P["density"][i] - rho) <= 1e-5 * rho
    assert np.array_equal(P["value"], P["density"]) and np.all(P["mass"] == np.float32(1.0 / n))
