"""The seeded input generators: the generator's test vector, determinism, and the
Plummer model's known properties (mass profile, half-mass radius, virial ratio,
energy in N-body units)."""
import math

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic


def test_splitmix64_test_vector():
    # SplitMix64 seeded with 0: first three outputs of the published generator
    got = ic.u64(np.uint64(0), np.arange(3))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_moments():
    u = ic.uniform(ic.key(1, 2), np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = ic.normal(ic.key(3), 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1) < 1e-2


def test_plummer_deterministic_and_seeded():
    a = ic.plummer(1000, 5)
    b = ic.plummer(1000, 5)
    c = ic.plummer(1000, 6)
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.vel, b.vel)
    assert np.abs(a.pos - c.pos).max() > 0.1


@pytest.fixture(scope="module")
def big():
    return ic.plummer(65536)


def test_plummer_units_and_frame(big):
    assert big.m.sum() == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose((big.m[:, None] * big.pos).sum(0), 0, atol=1e-14)
    np.testing.assert_allclose((big.m[:, None] * big.vel).sum(0), 0, atol=1e-14)


def test_plummer_mass_profile(big):
    """Cumulative mass M(<r) = r^3 / (r^2 + a^2)^(3/2), a = 3 pi / 16 in N-body units,
    truncated at r_cut (Kolmogorov-Smirnov), and half-mass radius ~0.769."""
    stats = pytest.importorskip("scipy.stats")
    a = 3 * math.pi / 16
    r = np.linalg.norm(big.pos, axis=1)
    rc = ic.R_CUT * a
    mcut = rc ** 3 / (rc * rc + a * a) ** 1.5

    def cdf(x):
        x = np.minimum(x, rc)
        return x ** 3 / (x * x + a * a) ** 1.5 / mcut

    assert stats.kstest(r, cdf).pvalue > 1e-3
    assert np.median(r) == pytest.approx(0.769, rel=0.02)


def test_plummer_energy_and_virial():
    p = ic.plummer(4096, 7)
    k, w = oracle.energy(p.m, p.pos, p.vel, 0.0)
    tol = 3 / math.sqrt(4096)
    assert abs(-k / w - 0.5) < tol
    assert abs((k + w) / -0.25 - 1) < tol


def test_lognormal_masses():
    p = ic.plummer(50000, 8, masses="lognormal", sigma=0.5)
    assert p.m.sum() == pytest.approx(1.0, abs=1e-13)
    assert np.log(p.m).std() == pytest.approx(0.5, rel=0.02)


def test_cluster_sizes_and_galaxy():
    n = ic.cluster_sizes(4096, 16, 4096)
    assert n.min() >= 16 and n.max() <= 4096
    assert np.log(n).mean() == pytest.approx((math.log(16) + math.log(4096)) / 2, rel=0.03)
    g = ic.galaxy(300, 3)
    assert g.m[0] == pytest.approx(0.01) and g.m.sum() == pytest.approx(1.0)
    eps = ic.cluster_eps([64, 4096])
    np.testing.assert_allclose(eps, [1 / 16, 1 / 64])


def test_request_stream():
    reqs = ic.request_stream(2000, rate_hz=100.0)
    arr = np.array([r.arrival for r in reqs])
    assert (np.diff(arr) >= 0).all()
    assert np.diff(arr).mean() == pytest.approx(0.01, rel=0.1)
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 256 and ns.max() <= 2 ** 18
    kinds = [r.kind for r in reqs]
    assert 0.45 < kinds.count("force") / len(kinds) < 0.55
    assert {r.galaxy for r in reqs} == set(range(11))
