"""Gauge-covariant Gaussian source smearing on the device against the oracle,
and a propagator solve from a smeared point source."""
import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O

pytestmark = pytest.mark.gpu

M = torch = None


def setup_module(module):
    global M, torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf
    import torch as _torch
    M, torch = mdwf, _torch


@pytest.mark.parametrize('sigma,n', [(2.5, 8), (1.0, 1), (3.0, 15)])
def test_smearing_matches_oracle(sigma, n):
    dims = (6, 4, 4, 8)
    U = synth.random_gauge(dims, 41, 0.5)
    eta = synth.gaussian_spinor((8, 4, 4, 6, 4, 3), 42)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        d = torch.from_numpy(eta.copy()).cuda()
        M.mdwf_smear_source_dev(ctx, 0, d, sigma, n)
        got = d.cpu().numpy()
    finally:
        M.mdwf_destroy(ctx)
    ref = O.gaussian_smear(U, eta, sigma, n)
    assert np.linalg.norm((got - ref).ravel()) <= 1e-13 * np.linalg.norm(ref.ravel())


def test_solve_from_smeared_point_source():
    dims, L5 = (4, 4, 4, 8), 6
    act = (1.3, 1.5, 0.5, 0.05)
    U = synth.flowed_gauge(dims, 43, 0.4, flow_t=0.5, flow_eps=0.02)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        eta = torch.from_numpy(synth.point_source_4d(dims, 1, 2)).cuda()
        M.mdwf_smear_source_dev(ctx, 0, eta, 2.0, 10)
        b = torch.empty((L5, 8, 4, 4, 4, 4, 3), dtype=torch.complex128, device='cuda')
        M.mdwf_make_source_dev(ctx, 0, eta, b)
        x = torch.empty_like(b)
        st = M.mdwf_solve_batch_dev(ctx, 0, [b], [x], 1e-10, opts=M.mdwf_default_opts(precision='half'))
        torch.cuda.synchronize()
        bh, xh = b.cpu().numpy(), x.cpu().numpy()
    finally:
        M.mdwf_destroy(ctx)
    assert st[0]['converged']
    ref_eta = O.gaussian_smear(U, synth.point_source_4d(dims, 1, 2), 2.0, 10)
    assert np.abs(bh - O.make_source(U, ref_eta, act[0], act[2], L5)).max() < 1e-12
    assert O.true_residual(U, bh, xh, *act) <= 1e-10
