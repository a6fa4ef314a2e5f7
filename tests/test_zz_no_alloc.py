"""nb_force_static: the force call that allocates no device memory.

It serves callers that cannot call cudaMalloc, such as a host code whose own pool
allocator owns the device memory and forbids other allocations. They pass their own
device buffers; the only scratch, the partial sums of the j-split, lives in a fixed
device array inside the library. The tests call it through the C ABI on buffers
allocated here:

- twice in a row (the shared scratch keeps the first call's contents), each result
  against the FP64 oracle and against the existing entry point nb_force (FP64 pairs),
  within the FP64 tolerance of the force tests (relative RMS 1e-12);
- at the largest i-set (NB_STATIC_MAX_NI) against 2^17 j, where the size of the scratch,
  not the SM count, limits the j-split, and with idx = NULL;
- in a fresh process: after the warm-up call (n_i = 0), real calls leave the device's
  free memory unchanged, so nothing was allocated.

This file is collected last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1409_5474_gb300 import ic

pytestmark = pytest.mark.gpu

TOL = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rel_rms(got, ref):
    return float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()))


def _reference(nb, p, eps, idx):
    with nb.System(p.m, p.pos, p.vel, variant="f64", eps=eps, device=0) as s:
        s.predict(0.0)
        return s.force(idx)


def _device_system(torch, p, pad):
    n = p.n
    ld = n + pad
    pos = np.zeros((3, ld))
    vel = np.zeros((3, ld))
    pos[:, :n] = p.pos.T
    vel[:, :n] = p.vel.T
    return (torch.from_numpy(p.m.copy()).cuda(), torch.from_numpy(pos).cuda(),
            torch.from_numpy(vel).cuda(), ld)


def _static_call(nb, torch, dm, dpos, dvel, ld, idx, eps, n_i=None):
    n_i = idx.size if idx is not None else n_i
    d_idx = torch.from_numpy(idx).cuda() if idx is not None else None
    out = torch.full((7, n_i), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    nb.nb_force_static(dm.numel(), dm.data_ptr(), dpos.data_ptr(), dvel.data_ptr(), ld, n_i,
                       d_idx.data_ptr() if d_idx is not None else 0, eps, out[0:3].data_ptr(),
                       out[3:6].data_ptr(), out[6].data_ptr(), stream.cuda_stream)
    return out.cpu().numpy()


def _check(got, ref):
    acc, jerk, pot = ref
    assert _rel_rms(got[0:3], acc) < TOL
    assert _rel_rms(got[3:6], jerk) < TOL
    assert _rel_rms(got[6], pot) < TOL


@pytest.mark.parametrize("pad", [0, 5])
def test_static_force_matches_oracle_and_nb_force_twice(nb, pad):
    torch = pytest.importorskip("torch")
    p = ic.plummer(3001, 77, masses="lognormal")
    eps = 0.01
    dm, dpos, dvel, ld = _device_system(torch, p, pad)
    rng = np.random.default_rng(pad)
    for n_i in (700, 37):  # two calls in a row on the shared scratch
        idx = np.sort(rng.choice(p.n, size=n_i, replace=False)).astype(np.int32)
        got = _static_call(nb, torch, dm, dpos, dvel, ld, idx, eps)
        ra, rj, rp = oracle.force(p.m, p.pos, p.vel, eps * eps, idx=idx)
        _check(got, (ra.T, rj.T, rp))
        _check(got, _reference(nb, p, eps, idx))


def test_static_force_at_the_scratch_limit_and_without_idx(nb):
    """n_i = NB_STATIC_MAX_NI against 2^17 j: the j-split is cut to the splits whose
    partial sums fit the scratch (2^20 / (7 * 1024) = 146 < 256 by the j count). Then the
    identity i-set (idx = NULL) on the same buffers."""
    torch = pytest.importorskip("torch")
    n = 2 ** 17
    p = ic.plummer(n, 78, masses="lognormal")
    eps = 1e-3
    dm, dpos, dvel, ld = _device_system(torch, p, 3)
    idx = np.sort(np.random.default_rng(5).choice(n, size=nb.NB_STATIC_MAX_NI,
                                                  replace=False)).astype(np.int32)
    got = _static_call(nb, torch, dm, dpos, dvel, ld, idx, eps)
    ra, rj, rp = oracle.force(p.m, p.pos, p.vel, eps * eps, idx=idx)
    _check(got, (ra.T, rj.T, rp))
    got0 = _static_call(nb, torch, dm, dpos, dvel, ld, None, eps, n_i=500)
    ra, rj, rp = oracle.force(p.m, p.pos, p.vel, eps * eps, idx=np.arange(500, dtype=np.int32))
    _check(got0, (ra.T, rj.T, rp))


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


_FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
from paper_1409_5474_gb300 import ic, nbody
nbody.load()
p = ic.plummer(4000, 79)
dm = torch.from_numpy(p.m.copy()).cuda()
dpos = torch.from_numpy(np.ascontiguousarray(p.pos.T)).cuda()
dvel = torch.from_numpy(np.ascontiguousarray(p.vel.T)).cuda()
idx = torch.arange(0, 4000, 5, dtype=torch.int32, device="cuda")
out = torch.empty((7, idx.numel()), dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
def call(n_i):
    nbody.nb_force_static(p.n, dm.data_ptr(), dpos.data_ptr(), dvel.data_ptr(), p.n, n_i,
                          idx.data_ptr(), 0.01, out[0:3].data_ptr(), out[3:6].data_ptr(),
                          out[6].data_ptr(), 0)
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]
free = [torch.cuda.mem_get_info()[0], call(0), call(idx.numel()), call(idx.numel())]
print("FREE", *free)
"""


def test_static_force_allocates_nothing_after_the_warm_up():
    """A fresh process: the warm-up call (n_i = 0) takes the scratch and loads the kernels;
    the free device memory is then the same after two real calls."""
    pytest.importorskip("torch")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE")][-1]
    before, warm, first, second = (int(v) for v in line.split()[1:])
    print("free device memory: before %d, after the warm-up %d (-%d), after two calls %d, %d"
          % (before, warm, before - warm, first, second))
    assert warm <= before
    assert first == warm and second == warm, (before, warm, first, second)
