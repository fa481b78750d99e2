"""Pins of the oracle's noise: Philox-4x32-10 and Box-Muller.

Philox is pinned by the published known-answer vectors (Salmon et al., SC'11;
tests/golden/philox4x32_10_kat.txt); Box-Muller by closed-form edge values and by
distribution tests against scipy's normal/exponential/uniform laws.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from tests import problems

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", kat_rows())
def test_philox_known_answers(ctr, key, out):
    got = oracle.philox(np.array([ctr], np.uint32), key)[0]
    assert [int(x) for x in got] == out


def test_box_muller_edges():
    # u0 = 1 (top word) -> radius 0 -> both normals exactly 0.
    assert np.all(oracle.box_muller(0xFFFFFFFF, 12345) == 0.0)
    # u0 = 2^-24 (word < 256) -> radius sqrt(48 ln 2); u1 = 1 -> angle 2*pi.
    z = oracle.box_muller(0x000000FF, 0xFFFFFFFF)
    r = math.sqrt(48.0 * math.log(2.0))
    assert z[0] == pytest.approx(r, rel=1e-14)
    assert abs(z[1]) < 1e-14
    # u1 = 1/4 (word = 2^30 - 256 -> (a >> 8) + 1 = 2^22) -> angle pi/2: (0, r).
    z = oracle.box_muller(0x000000FF, (1 << 30) - 256)
    assert abs(z[0]) < 1e-14 and z[1] == pytest.approx(r, rel=1e-14)


@pytest.fixture(scope="module")
def many_normals():
    n = 1 << 20
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 7
    w = oracle.philox(ctr, [0x1234, 0x5678])
    z = np.array([oracle.box_muller(int(a), int(b)) for a, b in w[:20000, :2]])
    return w, z


def test_box_muller_distribution(many_normals):
    _, z = many_normals
    n = z.shape[0]
    for c in range(2):
        assert abs(z[:, c].mean()) < 5.0 / math.sqrt(n)
        assert abs(z[:, c].var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5.0 / math.sqrt(n)
    # radius^2 ~ Exp(mean 2) and the angle is uniform: pins the -2 ln u and 2 pi factors
    assert stats.kstest((z ** 2).sum(1), "expon", args=(0, 2.0)).pvalue > 1e-4
    assert stats.kstest(np.arctan2(z[:, 1], z[:, 0]), "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4


def test_philox_words_uniform(many_normals):
    w, _ = many_normals
    for c in range(4):
        u = (w[:, c].astype(np.float64) + 0.5) / 2.0 ** 32
        assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_noise_scale_and_counter_layout():
    tmap = problems.ellipse_map()
    P = problems.oracle_problem(problems.params_small(K=512, T=40, sigma=(0.3, 0.35)), tmap, problems.network())
    eps = oracle.noise(P, 3)
    assert eps.shape == (512, 40, 2)
    n = eps[..., 0].size
    assert abs(eps[..., 0].std() - 0.3) < 5 * 0.3 / math.sqrt(2 * n)
    assert abs(eps[..., 1].std() - 0.35) < 5 * 0.35 / math.sqrt(2 * n)
    # counter = (k, t, iter_lo, iter_hi & 0xFFFF | instance << 16), key = (seed_lo, seed_hi)
    P2 = P.replace(instance=3)
    for hi in (5, 0xBEEF):  # all 16 kept bits of the iteration's high word reach the counter
        it = (hi << 32) | 9
        for k, t in [(0, 0), (17, 5), (511, 39)]:
            w = oracle.philox(np.array([[k, t, 9, hi | (3 << 16)]], np.uint32),
                              [problems.PHILOX_SEED & 0xFFFFFFFF, problems.PHILOX_SEED >> 32])[0]
            z = oracle.box_muller(int(w[0]), int(w[1]))
            assert np.array_equal(oracle.noise_at(P2, it, k, t), np.array([0.3 * z[0], 0.35 * z[1]]))
    # different iterations, instances and seeds give unrelated streams
    assert not np.allclose(oracle.noise(P, 4)[0, 0], eps[0, 0])
    assert not np.allclose(oracle.noise(P2, 3)[0, 0], eps[0, 0])
