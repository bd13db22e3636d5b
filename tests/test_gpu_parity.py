"""GPU parity: every step of the hot path, called through the C ABI, against the
FP64 CPU oracle on the same seeded inputs.

Tolerances (norm-wise relative, ||gpu - oracle|| / ||oracle||, and element by
element, max |gpu - oracle| <= C u max |oracle| with u the storage unit roundoff):
  FP64 operator applies                     1e-13
  FP32 storage/arithmetic Schur operator   2e-6   (a few float roundings per term)
  fp16 storage (scaled), FP32 arithmetic   4e-3   (2^-11 rounding of each stored field)
  bf16 storage, FP32 arithmetic            3e-2   (2^-8 rounding of each stored field)
  solves: true FP64 residual ||b - D x||/||b|| <= 1e-10 recomputed by the oracle's D,
          and the error against the oracle's own solution below kappa * 1e-10.
"""
import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O

pytestmark = pytest.mark.gpu

M = None


def setup_module(module):
    global M
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf
    M = mdwf


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# Element-wise bound: max |gpu - oracle| <= C * u * max |oracle|, with u the unit
# roundoff of the storage type (FP64, FP32, fp16, bf16).  C counts the roundings
# that reach one component through the operator: the stored input, the stored
# intermediate odd field, the stored output (each u relative to its unit's
# largest component) and the FP32 products and sums of the 8 hopping terms, of
# A^-1 and of B.  Measured worst cases over every hop form, dagger, L5 and mass
# of these tests: C = 2.7 (FP64), 2.4 (FP32), 1.3 (fp16), 1.3 (bf16); the bound
# C = 16 keeps a margin of at least 6.  A single wrong component
# (a dropped term, a wrong sign) is of the size of max |oracle| itself, 1/u
# times larger than u, so it cannot pass.
UNIT = {'double': 2.0 ** -53, 'single': 2.0 ** -24, 'half': 2.0 ** -11, 'bf16': 2.0 ** -8}
CELEM = {'double': 16.0, 'single': 16.0, 'half': 16.0, 'bf16': 16.0}


def _check_elementwise(out, ref, precision):
    err = np.abs(out - ref).max()
    bound = CELEM[precision] * UNIT[precision] * np.abs(ref).max()
    assert err <= bound, 'max |gpu - oracle| = %.3g > %.3g (%s)' % (err, bound, precision)


# (dims, L5, action, gauge seed/eps): several tiles, ragged tails (Vh*L5 not a
# multiple of the tile), anisotropic extents and L5 from 2 to 12.
CASES = [
    ((4, 4, 4, 8), 4, (1.3, 1.5, 0.5, 0.1), (1, 0.3)),          # the oracle-sized workload
    ((6, 4, 2, 4), 5, (1.2, 1.25, 0.25, 0.05), (2, 0.5)),
    ((2, 2, 2, 2), 2, (1.1, 1.7, 0.3, 0.2), (3, 0.8)),
    ((8, 6, 4, 10), 12, (1.3, 1.5, 0.5, 0.0158), (4, 0.4)),
]


class Lat:
    def __init__(self, dims, L5, act, gseed):
        self.dims, self.L5, self.act = dims, L5, act
        self.U = synth.random_gauge(dims, gseed[0], gseed[1])
        self.ctx = M.mdwf_create(dims, 0)
        M.mdwf_load_gauge(self.ctx, 0, self.U, 1)
        M.mdwf_set_action(self.ctx, 0, *act, L5)
        self.shape = (L5,) + tuple(reversed(dims)) + (4, 3)

    def close(self):
        M.mdwf_destroy(self.ctx)


@pytest.fixture(scope='module', params=range(len(CASES)))
def lat(request):
    L = Lat(*CASES[request.param])
    yield L
    L.close()


@pytest.mark.parametrize('out_parity', [-1, 0, 1])
@pytest.mark.parametrize('dagger', [0, 1])
def test_dslash_fp64(lat, out_parity, dagger):
    psi = synth.gaussian_spinor(lat.shape, 11)
    out = M.mdwf_apply_dslash(lat.ctx, 0, psi, out_parity, dagger)
    ref = O.hopping(lat.U, psi, True, bool(dagger))
    if out_parity >= 0:
        mask = O.parity_mask(lat.dims)
        ref = O.restrict(ref, mask if out_parity == 0 else 1 - mask)
    assert _rel(out, ref) < 1e-13
    _check_elementwise(out, ref, 'double')


@pytest.mark.parametrize('dagger', [0, 1])
def test_mdwf_fp64(lat, dagger):
    psi = synth.gaussian_spinor(lat.shape, 12)
    out = M.mdwf_apply_mdwf(lat.ctx, 0, psi, dagger)
    f = O.mobius_dag if dagger else O.mobius
    ref = f(lat.U, psi, *lat.act)
    assert _rel(out, ref) < 1e-13
    _check_elementwise(out, ref, 'double')


@pytest.mark.parametrize('op', ['A', 'B', 'Ainv'])
@pytest.mark.parametrize('dagger', [0, 1])
def test_fifth_dimension_ops(lat, op, dagger):
    psi = synth.gaussian_spinor(lat.shape, 13)
    out = M.mdwf_apply_5d(lat.ctx, 0, op, psi, dagger)
    M5, b5, c5, mf = lat.act
    ref = {'A': lambda v: O.op_A(v, M5, b5, c5, mf, bool(dagger)),
           'B': lambda v: O.op_B(v, b5, c5, mf, bool(dagger)),
           'Ainv': lambda v: O.op_A_inv(v, M5, b5, c5, mf, bool(dagger))}[op](psi)
    assert _rel(out, ref) < 1e-13
    _check_elementwise(out, ref, 'double')


@pytest.mark.parametrize('precision,tol', [('double', 1e-13), ('single', 2e-6), ('half', 4e-3), ('bf16', 3e-2)])
@pytest.mark.parametrize('dagger', [0, 1])
def test_schur_operator(lat, precision, tol, dagger):
    ev = O.parity_mask(lat.dims)
    psi = O.restrict(synth.gaussian_spinor(lat.shape, 14), ev)
    out = M.mdwf_apply_schur(lat.ctx, 0, psi, dagger, precision)
    f = O.schur_op_dag if dagger else O.schur_op
    ref = f(lat.U, psi, *lat.act)
    assert _rel(out, ref) < tol
    _check_elementwise(out, ref, precision)


def test_make_source(lat):
    eta = synth.gaussian_spinor(tuple(reversed(lat.dims)) + (4, 3), 15)
    out = M.mdwf_make_source(lat.ctx, 0, eta)
    M5, b5, c5, mf = lat.act
    ref = O.make_source(lat.U, eta, M5, c5, lat.L5)
    assert _rel(out, ref) < 1e-13
    _check_elementwise(out, ref, 'double')


def test_time_boundary_periodic_option():
    dims, L5 = (4, 2, 2, 4), 3
    U = synth.random_gauge(dims, 5, 0.5)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 0)
        M.mdwf_set_action(ctx, 0, 1.3, 1.5, 0.5, 0.1, L5)
        psi = synth.gaussian_spinor((L5, 4, 2, 2, 4, 4, 3), 16)
        out = M.mdwf_apply_dslash(ctx, 0, psi, -1, 0)
        ref = O.hopping(U, psi, False)
        assert _rel(out, ref) < 1e-13
        _check_elementwise(out, ref, 'double')
    finally:
        M.mdwf_destroy(ctx)


# ---------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------
def _check_solution(lat, b, x, st, tol=1e-10, mf=None):
    M5, b5, c5, mf0 = lat.act
    mf = mf0 if mf is None else mf
    res = O.true_residual(lat.U, b, x, M5, b5, c5, mf)
    assert st['converged'] and st['rel_true_resid'] <= tol
    assert res <= tol, res
    assert abs(res - st['rel_true_resid']) <= 0.05 * tol + 1e-3 * res
    return res


@pytest.mark.parametrize('precision', ['double', 'single', 'half', 'bf16'])
def test_solve_point_source_oracle_workload(precision):
    """4^3 x 8, L5 = 4, M5 = 1.3, b5 = 1.5, c5 = 0.5, mf = 0.1, exp(0.3 i H) links,
    point source (spin 0, colour 0, origin) as a 5D unit vector on the s = 0 slice."""
    L = Lat(*CASES[0])
    try:
        b = np.zeros(L.shape, dtype=np.complex128)
        b[0, 0, 0, 0, 0, 0, 0] = 1.0
        x, st = M.mdwf_solve(L.ctx, 0, b, 1e-10, M.mdwf_default_opts(precision=precision))
        _check_solution(L, b, x, st)
        ref, _ = O.solve_schur(L.U, b, *L.act, tol=1e-13)
        assert _rel(x, ref) < 1e-8
    finally:
        L.close()


@pytest.mark.parametrize('precision', ['single', 'half', 'bf16'])
def test_solve_batch_spin_colour_and_masses(precision):
    """12 spin-colour wall sources with three masses in one batch (flowed links)."""
    dims, L5 = (4, 4, 4, 8), 6
    act = (1.2, 1.25, 0.25, 0.02)
    U = synth.flowed_gauge(dims, 7, 0.4, flow_t=0.2, flow_eps=0.02)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        srcs, masses = [], []
        for k in range(12):
            srcs.append(M.mdwf_make_source(ctx, 0, synth.point_source_4d(dims, k // 3, k % 3)))
            masses.append((0.02, 0.05, 0.1)[k % 3])
        xs, stats = M.mdwf_solve_batch(ctx, 0, srcs, 1e-10, masses=masses,
                                       opts=M.mdwf_default_opts(precision=precision))
        for b, x, st, m in zip(srcs, xs, stats, masses):
            res = O.true_residual(U, b, x, act[0], act[1], act[2], m)
            assert st['converged'] and res <= 1e-10, (st, res)
        # one system against the oracle's own solution
        ref, _ = O.solve_schur(U, srcs[4], act[0], act[1], act[2], masses[4], tol=1e-13)
        assert _rel(xs[4], ref) < 1e-7
    finally:
        M.mdwf_destroy(ctx)


def test_batch_result_same_alone_and_in_mix():
    """A system solved alone and inside a batch of other systems gives the same x
    (the reductions of one slot do not depend on the other slots)."""
    dims, L5 = (4, 4, 4, 8), 4
    act = (1.3, 1.5, 0.5, 0.1)
    U = synth.random_gauge(dims, 9, 0.3)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        shape = (L5, 8, 4, 4, 4, 4, 3)
        target = synth.gaussian_spinor(shape, 100)
        others = [synth.gaussian_spinor(shape, 101 + k) for k in range(5)]
        opts = M.mdwf_default_opts(precision='half')
        alone, st_a = M.mdwf_solve_batch(ctx, 0, [target], 1e-10, masses=[0.1], opts=opts)
        mix, st_m = M.mdwf_solve_batch(ctx, 0, others[:3] + [target] + others[3:], 1e-10,
                                       masses=[0.05, 0.2, 0.1, 0.1, 0.3, 0.1], opts=opts)
        assert st_a[0]['iters'] == st_m[3]['iters']
        assert np.array_equal(alone[0], mix[3])
    finally:
        M.mdwf_destroy(ctx)


def test_solve_errors():
    dims = (4, 4, 4, 4)
    ctx = M.mdwf_create(dims, 0)
    try:
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_set_action(ctx, 0, 1.3, 1.5, 0.5, 0.1, 1)
        assert e.value.code == M.MDWF_ERR_ARG
        U = synth.random_gauge(dims, 1, 0.3)
        U[0, 0, 0, 0, 0, 0, 0] = np.nan
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_load_gauge(ctx, 0, U, 1)
        assert e.value.code == M.MDWF_ERR_NONFINITE
        M.mdwf_load_gauge(ctx, 0, synth.random_gauge(dims, 1, 0.3), 1)
        M.mdwf_set_action(ctx, 0, 1.3, 1.5, 0.5, 0.1, 4)
        b = synth.gaussian_spinor((4, 4, 4, 4, 4, 4, 3), 1)
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_solve(ctx, 0, b, 1e-10, M.mdwf_default_opts(max_iter=3))
        assert e.value.code == M.MDWF_ERR_NOT_CONVERGED
        b[0, 0, 0, 0, 0, 0, 0] = np.inf
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_solve(ctx, 0, b, 1e-10)
        assert e.value.code == M.MDWF_ERR_NONFINITE
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_apply_mdwf(ctx, 5, b, 0)
        assert e.value.code == M.MDWF_ERR_STATE
    finally:
        M.mdwf_destroy(ctx)


@pytest.mark.parametrize('variant', [2, 5])
def test_bounded_wait_reports_timeout_and_context_survives(variant):
    """A bulk-copy wait that runs out (the test knob makes each barrier expect bytes
    that never arrive) ends the solve with MDWF_ERR_TIMEOUT; the same context then
    solves normally.  Variant 2: the staged CUDA-core hop; 5: the pipelined
    tensor-core hop (two right-hand sides, so that its 8-unit tiles are whole)."""
    L = Lat(*CASES[0])
    try:
        bs = [synth.gaussian_spinor(L.shape, 17 + k) for k in range(2)]
        bad = M.mdwf_default_opts(precision='half', timeout_test=1, wait_timeout_s=0.05, hop_variant=variant)
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_solve_batch(L.ctx, 0, bs, 1e-10, opts=bad)
        assert e.value.code == M.MDWF_ERR_TIMEOUT
        xs, st = M.mdwf_solve_batch(L.ctx, 0, bs, 1e-10, opts=M.mdwf_default_opts(precision='half',
                                                                                     hop_variant=variant))
        for b, x, s in zip(bs, xs, st):
            _check_solution(L, b, x, s)
    finally:
        L.close()


# the production tiling: N = 12, two sites per block (what the autotuner picks for
# the 16^3 x 48, L5 = 12 workload), at the L5 of every workload (8, 12) and 16
MASSES12 = [0.0022, 0.0102, 0.0126, 0.0158, 0.0216, 0.05, 0.1, 0.2, 0.3, 0.01, 0.02, 0.07]


@pytest.mark.parametrize('precision,tol', [('double', 1e-13), ('single', 2e-6), ('half', 4e-3), ('bf16', 3e-2)])
@pytest.mark.parametrize('dagger', [0, 1])
@pytest.mark.parametrize('variant', [0, 1, 2, 3, 5, 6, 7, 1 | (2 << 8), 6 | (2 << 8), 7 | (2 << 8), 1 | (1 << 16)])
@pytest.mark.parametrize('L5,masses', [(5, [0.05, 0.01, 0.2, 0.0022, 0.1]),            # L5 N = 25
                                       (4, [0.05, 0.01, 0.2, 0.0022]),                 # L5 N = 16: tensor-core tiles
                                       (6, [0.05, 0.01, 0.2, 0.0022, 0.1, 0.3, 0.02, 0.07]),   # L5 N = 48
                                       (8, MASSES12), (12, MASSES12), (16, MASSES12)])
def test_schur_batch_multi_rhs(precision, tol, dagger, variant, L5, masses):
    """The batched Schur operator (the solver's kernels, N RHS with different masses,
    every hop variant; bits 8..15 of the variant fix the sites per block, bit 16
    selects 12-real links) against the oracle, slot by slot, norm-wise and element
    by element."""
    import torch
    dims = (6, 4, 4, 6)
    act = (1.2, 1.25, 0.25, 0.05)
    U = synth.random_gauge(dims, 19, 0.5)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        shape = (L5,) + tuple(reversed(dims)) + (4, 3)
        ev = O.parity_mask(dims)
        xs = [O.restrict(synth.gaussian_spinor(shape, 200 + i), ev) for i in range(len(masses))]
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.empty_like(t) for t in ins]
        M.mdwf_apply_schur_batch_dev(ctx, 0, ins, outs, masses=masses, dagger=dagger, precision=precision,
                                     hop_variant=variant)
        f = O.schur_op_dag if dagger else O.schur_op
        for x, o, m in zip(xs, outs, masses):
            ref = f(U, x, act[0], act[1], act[2], m)
            o = o.cpu().numpy()
            assert _rel(o, ref) < tol
            _check_elementwise(o, ref, precision)
    finally:
        M.mdwf_destroy(ctx)


@pytest.mark.parametrize('dims,L5,n', [((6, 4, 4, 6), 12, 12), ((6, 4, 4, 6), 7, 5), ((4, 4, 2, 6), 3, 13),
                                       ((4, 4, 2, 6), 12, 25), ((8, 6, 4, 10), 8, 12)])
@pytest.mark.parametrize('nsb', [1, 2, 4])
def test_prefetching_pair_hop_gives_the_same_bits(dims, L5, n, nsb):
    """fp16: the prefetching form of the paired hop (links in shared memory, the
    neighbour loads two directions ahead) against the plain form at the same block
    shape, for odd L5 (a thread with one slice) and an RHS count that leaves a
    partial block (25 RHS at L5 = 12 and four sites per block: 21 + 4): every
    output bit is the same for Mhat and Mhat^+ (their four epilogues), and the
    result matches the oracle element by element."""
    import torch
    act = (1.3, 1.5, 0.5, 0.05)
    U = synth.random_gauge(dims, 23, 0.6)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        shape = (L5,) + tuple(reversed(dims)) + (4, 3)
        ev = O.parity_mask(dims)
        masses = [0.01 * (k + 1) for k in range(n)]
        xs = [O.restrict(synth.gaussian_spinor(shape, 300 + i), ev) for i in range(n)]
        ins = [torch.from_numpy(x).cuda() for x in xs]
        for dagger in (0, 1):
            a = [torch.empty_like(t) for t in ins]
            b = [torch.empty_like(t) for t in ins]
            M.mdwf_apply_schur_batch_dev(ctx, 0, ins, a, masses=masses, dagger=dagger, precision='half',
                                         hop_variant=M.HOP_DIRECT | (nsb << 8))
            M.mdwf_apply_schur_batch_dev(ctx, 0, ins, b, masses=masses, dagger=dagger, precision='half',
                                         hop_variant=M.HOP_PAIR_PF | (nsb << 8))
            for x, y in zip(a, b):
                assert torch.equal(x, y)
            f = O.schur_op_dag if dagger else O.schur_op
            k = n - 1
            _check_elementwise(b[k].cpu().numpy(), f(U, xs[k], act[0], act[1], act[2], masses[k]), 'half')
    finally:
        M.mdwf_destroy(ctx)


def test_autotuner_choice_is_cached_and_keeps_results():
    """The autotuner picks a hop form per (L5, N, precision); its default candidate
    set shares one arithmetic, so a solve gives the same bits with the tuned form
    as with a fixed one."""
    L = Lat(*CASES[3])
    try:
        t1 = M.mdwf_autotune(L.ctx, 0, 3, 'half')
        t2 = M.mdwf_autotune(L.ctx, 0, 3, 'half')
        assert t1 == t2 and t1['hop_variant'] in (M.HOP_DIRECT, M.HOP_PAIR_PF) and t1['ms_per_pair'] > 0
        ta = M.mdwf_autotune(L.ctx, 0, 3, 'half', include_tensor_core=True)
        assert ta['hop_variant'] in (M.HOP_DIRECT, M.HOP_PAIR_PF, M.HOP_STAGED, M.HOP_MMA)
        bs = [synth.gaussian_spinor(L.shape, 40 + k) for k in range(3)]
        xa, sa = M.mdwf_solve_batch(L.ctx, 0, bs, 1e-10, opts=M.mdwf_default_opts(precision='half'))
        xd, sd = M.mdwf_solve_batch(L.ctx, 0, bs, 1e-10, opts=M.mdwf_default_opts(precision='half', hop_variant=1,
                                                                                      nsb=1))
        for x, y in zip(xa, xd):
            assert np.array_equal(x, y)
        for b, x, s in zip(bs, xa, sa):
            _check_solution(L, b, x, s)
    finally:
        L.close()


@pytest.mark.parametrize('precision', ['single', 'half', 'bf16'])
def test_solve_with_12_real_links(precision):
    """Inner hops on 12-real links (the third row rebuilt in the kernel) on a flowed
    field with the antiperiodic time boundary: the solve is certified by the
    oracle's D and equals the oracle's solution."""
    dims, L5 = (4, 4, 4, 8), 6
    act = (1.2, 1.25, 0.25, 0.05)
    U = synth.flowed_gauge(dims, 7, 0.4, flow_t=0.2, flow_eps=0.02)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        b = M.mdwf_make_source(ctx, 0, synth.point_source_4d(dims, 1, 2))
        x, st = M.mdwf_solve(ctx, 0, b, 1e-10, M.mdwf_default_opts(precision=precision, link_recon=12))
        assert st['converged'] and O.true_residual(U, b, x, *act) <= 1e-10
        ref, _ = O.solve_schur(U, b, *act, tol=1e-13)
        assert _rel(x, ref) < 1e-8
    finally:
        M.mdwf_destroy(ctx)


@pytest.mark.parametrize('precision', ['double', 'half'])
def test_restart_after_missed_certificate(precision):
    """Reading 7: a solve whose FP64 full-lattice certificate misses tol resumes from
    its x.  The testing knob makes the Schur stopping norm 100 times too loose, so
    the first certificate misses 1e-10; with restarts the solve still returns a
    certified x equal to the oracle's solution, without them it reports
    NOT_CONVERGED."""
    L = Lat(*CASES[0])
    try:
        b = np.zeros(L.shape, dtype=np.complex128)
        b[0, 0, 0, 0, 0, 0, 0] = 1.0
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_solve(L.ctx, 0, b, 1e-10, M.mdwf_default_opts(precision=precision, stop_scale_test=100.0,
                                                                 max_restarts=0))
        assert e.value.code == M.MDWF_ERR_NOT_CONVERGED
        x, st = M.mdwf_solve(L.ctx, 0, b, 1e-10, M.mdwf_default_opts(precision=precision, stop_scale_test=100.0))
        assert st['restarts'] >= 1
        _check_solution(L, b, x, st)
        ref, _ = O.solve_schur(L.U, b, *L.act, tol=1e-13)
        assert _rel(x, ref) < 1e-8
    finally:
        L.close()


@pytest.mark.parametrize('precision', ['double', 'single', 'half'])
def test_symmetric_schur_solve(precision):
    """The symmetric Schur form (opts.schur = 1) reaches the same solution."""
    L = Lat(*CASES[0])
    try:
        b = np.zeros(L.shape, dtype=np.complex128)
        b[0, 0, 0, 0, 0, 0, 0] = 1.0
        x, st = M.mdwf_solve(L.ctx, 0, b, 1e-10, M.mdwf_default_opts(precision=precision, schur=1))
        _check_solution(L, b, x, st)
        ref, _ = O.solve_schur(L.U, b, *L.act, tol=1e-13)
        assert _rel(x, ref) < 1e-8
    finally:
        L.close()


def test_symmetric_schur_batch_masses_and_session():
    import torch
    dims, L5 = (4, 4, 4, 8), 6
    act = (1.2, 1.25, 0.25, 0.02)
    U = synth.flowed_gauge(dims, 7, 0.4, flow_t=0.2, flow_eps=0.02)
    ctx = M.mdwf_create(dims, 0)
    try:
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, *act, L5)
        srcs = [M.mdwf_make_source(ctx, 0, synth.point_source_4d(dims, k // 3, k % 3)) for k in range(6)]
        masses = [0.02, 0.05, 0.1] * 2
        opts = M.mdwf_default_opts(precision='half', schur=1)
        xs, stats = M.mdwf_solve_batch(ctx, 0, srcs, 1e-10, masses=masses, opts=opts)
        for b, x, st, m in zip(srcs, xs, stats, masses):
            assert st['converged'] and O.true_residual(U, b, x, act[0], act[1], act[2], m) <= 1e-10
        sess = M.mdwf_session_create(ctx, 0, 2, 1e-10, opts=opts)
        try:
            db = torch.from_numpy(srcs[1]).cuda()
            dx = torch.empty_like(db)
            M.mdwf_session_submit(sess, db, 0.05, dx, 1)
            done = {}
            for _ in range(500):
                if M.mdwf_session_occupied(sess) == 0:
                    break
                M.mdwf_session_launch(sess)
                done.update(dict(M.mdwf_session_poll(sess)))
            assert done[1]['converged']
            assert O.true_residual(U, srcs[1], dx.cpu().numpy(), act[0], act[1], act[2], 0.05) <= 1e-10
        finally:
            M.mdwf_session_destroy(sess)
    finally:
        M.mdwf_destroy(ctx)
