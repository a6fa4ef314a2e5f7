"""The bridge coupling (nb_kick_ext, nb_bridge_step; Sect. V) against the oracle's kick and
kick-drift-kick run: two systems on the same GPU, FP64 and double-single pairs."""
import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu


def _pair(na=96, nb_=160, sep=1.5):
    a = ic.plummer(na, 80)
    b = ic.plummer(nb_, 81)
    off = np.array([sep / 2, 0.0, 0.0])
    return ((a.m * 0.5, a.pos * 0.2 - off, a.vel * 0.4),
            (b.m * 0.5, b.pos * 0.2 + off, b.vel * 0.4))


def test_kick_matches_oracle(nb):
    (ma, xa, va), (mb, xb, vb) = _pair()
    ea, eb = 0.01, 0.02
    with nb.System(ma, xa, va, variant="f64", eps=ea, device=0) as A, \
            nb.System(mb, xb, vb, variant="f64", eps=eb, device=0) as B:
        nb.nb_init(A.h)
        nb.nb_init(B.h)
        nb.nb_kick_ext(A.h, B.h, 0.03)
        g = A.state()
    sa = oracle.State(ma, xa, va)
    sb = oracle.State(mb, xb, vb)
    oracle.kick(sa, sb, eb * eb, ea * ea, 0.03)
    assert np.abs(g["vel"].T - sa.vel).max() < 1e-14
    assert np.abs(g["acc"].T - sa.acc).max() < 1e-11 * np.abs(sa.acc).max()
    assert np.abs(g["jerk"].T - sa.jerk).max() < 1e-11 * np.abs(sa.jerk).max()
    np.testing.assert_array_equal(g["pos"].T, xa)


@pytest.mark.parametrize("variant,tol", [("f64", 1e-9), ("f32ds", 1e-5)])
def test_bridge_steps_match_oracle(nb, variant, tol):
    """Two clusters, block steps inside (eta = 0.02, dt_max = 1/16), two bridge steps of
    1/16: the oracle's kick-drift-kick run."""
    (ma, xa, va), (mb, xb, vb) = _pair()
    eps = 0.01
    kw = dict(variant=variant, eps=eps, eta=0.02, dt_max=1.0 / 16, device=0)
    with nb.System(ma, xa, va, **kw) as A, nb.System(mb, xb, vb, **kw) as B:
        for _ in range(2):
            nb.nb_bridge_step(A.h, B.h, 1.0 / 16)
        ga, gb = A.state(), B.state()
    sa, sb = oracle.State(ma, xa, va), oracle.State(mb, xb, vb)
    oracle.bridge_run(sa, sb, eps * eps, eps * eps, 1.0 / 16, 2, eta=0.02, dt_max=1.0 / 16)
    np.testing.assert_array_equal(ga["t"], 0.125)
    np.testing.assert_array_equal(gb["t"], 0.125)
    assert np.abs(ga["pos"].T - sa.pos).max() < tol
    assert np.abs(gb["pos"].T - sb.pos).max() < tol
    assert np.abs(ga["vel"].T - sa.vel).max() < 10 * tol
    # total momentum: the oracle's (individual block steps do not keep it exactly)
    p_gpu = (ma[:, None] * ga["vel"].T).sum(0) + (mb[:, None] * gb["vel"].T).sum(0)
    p_orc = (sa.m[:, None] * sa.vel).sum(0) + (sb.m[:, None] * sb.vel).sum(0)
    assert np.abs(p_gpu - p_orc).max() < 10 * tol


def test_bridge_errors(nb):
    (ma, xa, va), (mb, xb, vb) = _pair(32, 40)
    with nb.System(ma, xa, va, variant="f64", eps=0.01, dt_max=1.0 / 16, device=0) as A, \
            nb.System(mb, xb, vb, variant="f64", eps=0.01, dt_max=1.0 / 8, device=0) as B:
        with pytest.raises(nb.NBodyError) as e:
            nb.nb_bridge_step(A.h, B.h, 1.0 / 16)   # not a multiple of B's dt_max
        assert e.value.status == nb.NB_ERR_ARG
        nb.nb_init(A.h)
        nb.nb_init(B.h)
        A.step(1.0 / 32)                            # A's particles are no longer synchronised
        with pytest.raises(nb.NBodyError) as e:
            nb.nb_kick_ext(A.h, B.h, 0.01)
        assert e.value.status == nb.NB_ERR_STATE
        with pytest.raises(nb.NBodyError) as e:
            nb.nb_kick_ext(A.h, A.h, 0.01)
        assert e.value.status == nb.NB_ERR_ARG
