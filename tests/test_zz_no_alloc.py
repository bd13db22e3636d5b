"""The Schur operator entry point that allocates no device memory.

Some callers may not call cudaMalloc (their own pool owns the device memory, or
an allocation's implicit synchronisation is not acceptable on their path).
mdwf_apply_schur_batch_dev_noalloc serves them from a fixed scratch array in the
library.  It runs the same kernels, tiling and hop form as the allocating
mdwf_apply_schur_batch_dev with hop variant 1, so the two must give the same
bits.  Each dagger value is applied twice in a row with fresh inputs, so that
scratch left by the previous call would show, and both results are compared
with the oracle's Schur operator.  This file is collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# norm-wise tolerance against the oracle (as tests/test_gpu_parity.py)
TOL = {'double': 1e-13, 'single': 2e-6, 'half': 4e-3, 'bf16': 3e-2}


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize('precision', ['double', 'single', 'half', 'bf16'])
def test_noalloc_schur_matches_allocating_entry_point(precision):
    import torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf as M
    from oracle import mdwf_oracle as O
    dims, L5 = (4, 4, 4, 8), 4
    act = (1.3, 1.5, 0.5, 0.1)
    masses = [0.1, 0.05, 0.02]
    U = synth.random_gauge(dims, 1, 0.3)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        shape = (L5,) + tuple(reversed(dims)) + (4, 3)
        ev = O.parity_mask(dims)
        for call, dagger in enumerate((0, 0, 1, 1)):
            xs = [O.restrict(synth.gaussian_spinor(shape, 300 + 10 * call + i), ev) for i in range(len(masses))]
            ins = [torch.from_numpy(x).cuda() for x in xs]
            ref = [torch.empty_like(t) for t in ins]
            got = [torch.full_like(t, float('nan')) for t in ins]
            M.mdwf_apply_schur_batch_dev(ctx, 0, ins, ref, masses=masses, dagger=dagger, precision=precision,
                                         hop_variant=M.HOP_DIRECT)
            M.mdwf_apply_schur_batch_dev_noalloc(ctx, 0, ins, got, masses=masses, dagger=dagger,
                                                 precision=precision)
            torch.cuda.synchronize()
            f = O.schur_op_dag if dagger else O.schur_op
            for x, r, o, m in zip(xs, ref, got, masses):
                assert torch.equal(o, r), 'no-allocation result differs from the allocating entry point'
                o = o.cpu().numpy()
                assert np.all(o[:, ev == 0] == 0)      # odd sites are zero
                assert _rel(o, f(U, x, act[0], act[1], act[2], m)) <= TOL[precision]
    finally:
        M.mdwf_destroy(ctx)


def test_noalloc_rejects_too_large_problem():
    import torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf as M
    dims, L5 = (16, 16, 16, 16), 8      # four FP64 fields of 16^4/2 x 8 units (50 MB each) exceed the scratch
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, synth.unit_gauge(dims), 1)
        M.mdwf_set_action(ctx, 0, 1.3, 1.5, 0.5, 0.1, L5)
        shape = (L5,) + tuple(reversed(dims)) + (4, 3)
        x = torch.zeros(shape, dtype=torch.complex128, device='cuda')
        y = torch.zeros_like(x)
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_apply_schur_batch_dev_noalloc(ctx, 0, [x], [y], precision='double')
        assert e.value.code == M.MDWF_ERR_ARG
        assert 'scratch' in str(e.value)
    finally:
        M.mdwf_destroy(ctx)
