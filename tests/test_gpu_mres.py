"""Residual-mass correlators (Sec. III, eq:mres) on the device: the contraction
against the oracle's on the same solutions, and m_res falling with L5 on
flowed links (the wall modes leak less through a longer fifth dimension)."""
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


def _mres(U, dims, L5, act):
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        srcs = [M.mdwf_make_source(ctx, 0, synth.point_source_4d(dims, k // 3, k % 3)) for k in range(12)]
        xs, st = M.mdwf_solve_batch(ctx, 0, srcs, 1e-10, opts=M.mdwf_default_opts(precision='half'))
        assert all(s['converged'] for s in st)
        dev = [torch.from_numpy(x).cuda() for x in xs]
        pp, j5 = M.mdwf_mres_correlators_dev(ctx, 0, dev)
        rpp, rj5 = O.mres_correlators(xs)
        assert np.abs(pp - rpp).max() <= 1e-13 * rpp.max()
        assert np.abs(j5 - rj5).max() <= 1e-13 * rj5.max()
        return pp, j5
    finally:
        M.mdwf_destroy(ctx)


def test_mres_contraction_and_l5_dependence():
    dims = (4, 4, 4, 8)
    U = synth.flowed_gauge(dims, 11, 0.4, flow_t=0.5, flow_eps=0.02)
    act = (1.3, 1.5, 0.5, 0.05)
    mres = {}
    for L5 in (4, 8):
        pp, j5 = _mres(U, dims, L5, act)
        assert np.all(pp > 0) and np.all(j5 > 0)
        mres[L5] = float(np.mean(j5 / pp))
    assert mres[8] < 0.5 * mres[4], mres
