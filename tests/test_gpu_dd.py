"""Domain decomposition along time on the GPU, with virtual sub-domains: P
contexts on one GPU, each holding a slab of Lt / P slices, their faces moved by
device copies (dd.LocalExchange).  The decomposed hop and Moebius operator must
equal the undecomposed library operator bit for bit (the halo path repeats the
local term's operations in the same order) and the oracle to 1e-13; a solve on
the decomposed lattice must be certified by the oracle's D and equal the
oracle's solution.  (Unmeasured on several GPUs: the pool gives one.)"""
import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O

pytestmark = pytest.mark.gpu

M = dd = torch = None
DIMS, L5 = (4, 4, 4, 8), 4
ACT = (1.3, 1.5, 0.5, 0.1)


def setup_module(module):
    global M, dd, torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf, dd as _dd
    import torch as _torch
    M, dd, torch = mdwf, _dd, _torch


def _decomposed(U, parts):
    split = dd.TSplit(DIMS, parts)
    subs = [dd.GPUSubdomain(M, split, k, U, ACT + (L5,)) for k in range(parts)]
    return split, subs, dd.DDOperator(split, range(parts), subs, dd.LocalExchange(split))


@pytest.mark.parametrize('parts', [1, 2, 4])
@pytest.mark.parametrize('kind,dagger', [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_decomposed_operator_equals_undecomposed(parts, kind, dagger):
    U = synth.random_gauge(DIMS, 3, 0.5)
    psi = synth.gaussian_spinor((L5,) + tuple(reversed(DIMS)) + (4, 3), 21)
    ctx = M.mdwf_create(DIMS, 0)
    split, subs, op = _decomposed(U, parts)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *ACT, L5)
        x = torch.from_numpy(psi).cuda()
        ref = torch.empty_like(x)
        if kind == 0:
            M.mdwf_apply_dslash_dev(ctx, 0, x, ref, -1, dagger)
        else:
            M.mdwf_apply_mdwf_dev(ctx, 0, x, ref, dagger)
        outs = op.apply(kind, dagger, [split.field_slab(x, k) for k in range(parts)])
        got = torch.cat(outs, dim=1)
        assert torch.equal(got, ref), 'decomposed operator differs from the undecomposed one'
        if kind == 0:
            want = O.hopping(U, psi, True, bool(dagger))
        else:
            want = (O.mobius_dag if dagger else O.mobius)(U, psi, *ACT)
        g = got.cpu().numpy()
        assert np.linalg.norm((g - want).ravel()) <= 1e-13 * np.linalg.norm(want.ravel())
    finally:
        for s in subs:
            s.close()
        M.mdwf_destroy(ctx)


def test_decomposed_solve_is_certified_and_equals_the_oracle():
    U = synth.random_gauge(DIMS, 1, 0.3)
    split, subs, op = _decomposed(U, 2)
    ctx = M.mdwf_create(DIMS, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *ACT, L5)
        b = M.mdwf_make_source(ctx, 0, synth.point_source_4d(DIMS, 0, 0))
        bd = torch.from_numpy(b).cuda()
        xs, iters, res = dd.solve(op, [split.field_slab(bd, k) for k in range(2)], tol=1e-10)
        x = torch.cat(xs, dim=1).cpu().numpy()
        assert res <= 1e-10 and iters > 0
        assert O.true_residual(U, b, x, *ACT) <= 1e-10
        ref, _ = O.solve_schur(U, b, *ACT, tol=1e-13)
        assert np.linalg.norm((x - ref).ravel()) <= 1e-8 * np.linalg.norm(ref.ravel())
    finally:
        for s in subs:
            s.close()
        M.mdwf_destroy(ctx)


def test_bad_split_and_odd_local_extent_are_rejected():
    with pytest.raises(ValueError):
        dd.TSplit(DIMS, 8)          # slabs of one slice: parities would not match
    ctx = M.mdwf_create((4, 4, 4, 2), 0)
    try:
        M.mdwf_load_gauge(ctx, 0, synth.unit_gauge((4, 4, 4, 2)), 1)
        M.mdwf_set_action(ctx, 0, *ACT, L5)
        x = torch.zeros((L5, 2, 4, 4, 4, 4, 3), dtype=torch.complex128, device='cuda')
        f = torch.zeros(M.dd_face_shape(ctx, 0), dtype=torch.complex128, device='cuda')
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_dd_pack_faces_dev(ctx, 0, 2, 0, x, f, f)
        assert e.value.code == M.MDWF_ERR_ARG
    finally:
        M.mdwf_destroy(ctx)
