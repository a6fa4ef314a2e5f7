"""nb_force_static: the allocation-free force call, for callers that cannot call
cudaMalloc (a code whose own pool allocator owns the device memory, say).

It is called through the C ABI on buffers the caller allocated, twice in a row
(the shared static scratch keeps the first call's contents), and each result is
compared with the existing entry point nb_force (FP64 pairs) within the FP64
tolerance of the force tests (relative RMS 1e-12). This file is collected last.
"""
import numpy as np
import pytest

from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _rel_rms(got, ref):
    return float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()))


def _reference(nb, p, eps, idx):
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=eps, device=0) as s:
        s.predict(0.0)
        return s.force(idx)


def _static_call(nb, torch, dm, dpos, dvel, ld, idx, eps):
    n_i = idx.size
    d_idx = torch.from_numpy(idx).cuda()
    out = torch.full((7, n_i), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    nb.nb_force_static(dm.numel(), dm.data_ptr(), dpos.data_ptr(), dvel.data_ptr(), ld, n_i,
                       d_idx.data_ptr(), eps, out[0:3].data_ptr(), out[3:6].data_ptr(),
                       out[6].data_ptr(), stream.cuda_stream)
    return out.cpu().numpy()


@pytest.mark.parametrize("pad", [0, 5])
def test_static_force_matches_nb_force_twice(nb, pad):
    torch = pytest.importorskip("torch")
    p = ic.plummer(3001, 77, masses="lognormal")
    eps = 0.01
    n = p.n
    ld = n + pad
    pos = np.zeros((3, ld))
    vel = np.zeros((3, ld))
    pos[:, :n] = p.pos.T
    vel[:, :n] = p.vel.T
    dm = torch.from_numpy(p.m.copy()).cuda()
    dpos = torch.from_numpy(pos).cuda()
    dvel = torch.from_numpy(vel).cuda()
    rng = np.random.default_rng(pad)
    for call, n_i in enumerate((700, 37)):  # two calls in a row on the shared scratch
        idx = np.sort(rng.choice(n, size=n_i, replace=False)).astype(np.int32)
        got = _static_call(nb, torch, dm, dpos, dvel, ld, idx, eps)
        acc, jerk, pot = _reference(nb, p, eps, idx)
        assert _rel_rms(got[0:3], acc) < TOL, call
        assert _rel_rms(got[3:6], jerk) < TOL, call
        assert _rel_rms(got[6], pot) < TOL, call


def test_static_force_rejects_oversized_i_set(nb):
    torch = pytest.importorskip("torch")
    n = 2000
    dm = torch.ones(n, dtype=torch.float64, device="cuda")
    dpos = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    out = torch.empty((7, nb.NB_STATIC_MAX_NI + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NBodyError) as e:
        nb.nb_force_static(n, dm.data_ptr(), dpos.data_ptr(), dpos.data_ptr(), n,
                           nb.NB_STATIC_MAX_NI + 1, 0, 0.1, out[0:3].data_ptr(),
                           out[3:6].data_ptr(), out[6].data_ptr(), 0)
    assert e.value.status == nb.NB_ERR_ARG
