"""Wilson flow on the device (Luscher's RK3, FP64) against the oracle's flow
(oracle/flow.py, pinned in tests/test_oracle_flow.py) on small lattices, and
against the host input generator's flow (checked against the oracle on the CPU)
at the a15m310 workload's full size, where the numpy oracle would take minutes;
the plaquette; unitarity; a pure-gauge field is a fixed point."""
import numpy as np
import pytest

import synth
from oracle import flow as F

pytestmark = pytest.mark.gpu

M = torch = None


def setup_module(module):
    global M, torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf
    import torch as _torch
    M, torch = mdwf, _torch


def _flow_dev(dims, U, eps, n):
    ctx = M.mdwf_create(dims, 0)
    try:
        d = torch.from_numpy(U.copy()).cuda()
        M.mdwf_wilson_flow_dev(ctx, d, eps, n)
        p = M.mdwf_plaquette_dev(ctx, d)
        return d.cpu().numpy(), p
    finally:
        M.mdwf_destroy(ctx)


@pytest.mark.parametrize('dims,seed,eps', [((4, 4, 4, 4), 3, 0.4), ((6, 4, 2, 8), 5, 0.7)])
def test_flow_matches_the_oracle(dims, seed, eps):
    U = synth.random_gauge(dims, seed, eps)
    got, plaq = _flow_dev(dims, U, 0.02, 6)
    ref = F.wilson_flow(U, 0.02, 6)
    assert np.abs(got - ref).max() < 1e-12
    assert abs(plaq - F.plaquette(ref)) < 1e-13
    assert plaq > synth.plaquette(dims, U)               # the flow smooths
    # links stay in SU(3)
    u = got.reshape(-1, 3, 3)
    assert np.abs(np.einsum('kba,kbc->kac', u.conj(), u) - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-12


def _gauge_transform(dims, U, W):
    out = np.empty_like(U)
    for mu in range(4):
        axis = 3 - mu
        Wn = np.roll(W, -1, axis=axis)
        out[..., mu, :, :] = np.einsum('...ab,...bc,...dc->...ad', W, U[..., mu, :, :], Wn.conj())
    return out


def test_pure_gauge_is_a_fixed_point():
    dims = (4, 2, 2, 4)
    U = _gauge_transform(dims, synth.unit_gauge(dims), synth.gauge_rotation(dims, 12))
    got, plaq = _flow_dev(dims, U, 0.05, 4)
    assert np.abs(got - U).max() < 1e-13
    assert abs(plaq - 1.0) < 1e-13


def test_full_size_flow_of_the_workload_links():
    """16^3 x 48, exp(0.4 i H) seed 2, flowed to t = 1 in 100 steps: the links of
    the benchmark workload, device against host."""
    dims = (16, 16, 16, 48)
    ref = synth.flowed_gauge(dims, 2, 0.4, 1.0, 0.01)
    U = synth.random_gauge(dims, 2, 0.4)
    got, plaq = _flow_dev(dims, U, 0.01, 100)
    assert np.abs(got - ref).max() < 1e-11
    assert abs(plaq - synth.plaquette(dims, ref)) < 1e-12
