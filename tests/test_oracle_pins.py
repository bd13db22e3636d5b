"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own formulas: closed forms in
momentum space, dense linear algebra, the paper's Moebius kernel equation
(Sec. II), symmetry identities and invariants.  ``test_planted_mistakes``
shows that plausible slips in the oracle (a sign, a projector, a transposed
matrix, a boundary phase) are each caught by at least one of these pins.
"""
import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O

TINY = (2, 2, 2, 2)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# ---------------------------------------------------------------------------
# gamma matrices
# ---------------------------------------------------------------------------
def test_gamma_clifford_hermitian_chiral():
    G = O.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T, atol=0)
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2.0 * (m == n) * np.eye(4), atol=0)
    # chiral basis: gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 is diag(1, 1, -1, -1)
    assert np.allclose(O.GAMMA5, np.diag([1, 1, -1, -1]), atol=0)
    for m in range(4):
        assert np.allclose(O.GAMMA5 @ G[m] + G[m] @ O.GAMMA5, 0, atol=0)


# ---------------------------------------------------------------------------
# free field: momentum-space closed forms
# ---------------------------------------------------------------------------
def _plane_wave(dims, p, u):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing='ij')
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * u[None, None, None, None]


@pytest.mark.parametrize("nvec", [(0, 0, 0, 0), (1, 2, 3, 1), (3, 1, 0, 6), (2, 2, 2, 7)])
def test_free_wilson_plane_wave(nvec):
    """D_W on e^{ipx} u equals [sum(1 - cos p) - M5 + i sum g sin p] u (antiperiodic p_t)."""
    dims = (4, 4, 4, 8)
    M5 = 1.3
    p = tuple(2 * np.pi * nvec[i] / dims[i] for i in range(3)) + (2 * np.pi * (nvec[3] + 0.5) / dims[3],)
    u = synth.gaussian_spinor((4, 3), 5)
    psi = _plane_wave(dims, p, u)
    out = O.wilson(synth.unit_gauge(dims), psi, M5)
    expect = _plane_wave(dims, p, np.einsum('st,tc->sc', O.wilson_momentum(p, M5), u))
    assert _rel(out, expect) < 1e-14


def test_free_field_point_propagator():
    """Point-source solve on unit links vs the Fourier sum of dense D(p)^-1 (4^3 x 8, L5 = 4)."""
    dims, L5 = (4, 4, 4, 8), 4
    M5, b5, c5, mf = 1.3, 1.5, 0.5, 0.1
    U = synth.unit_gauge(dims)
    for spin, colour, s0 in [(0, 0, 0), (3, 2, L5 - 1)]:
        b = np.zeros((L5,) + tuple(reversed(dims)) + (4, 3), dtype=np.complex128)
        b[s0, 0, 0, 0, 0, spin, colour] = 1.0
        expect = O.free_propagator_point(dims, L5, M5, b5, c5, mf, spin, colour, s0)
        x_full, _ = O.solve_full(U, b, M5, b5, c5, mf, tol=1e-12)
        x_schur, _ = O.solve_schur(U, b, M5, b5, c5, mf, tol=1e-12)
        assert _rel(x_full, expect) < 1e-9
        assert _rel(x_schur, expect) < 1e-9


# ---------------------------------------------------------------------------
# the 5D operator against the paper's Moebius kernel (Sec. II)
# ---------------------------------------------------------------------------
def _dense_ops(U, dims, M5, b5, c5, mf, L5):
    shape4 = tuple(reversed(dims)) + (4, 3)
    shape5 = (L5,) + shape4
    D = O.dense_matrix(lambda v: O.mobius(U, v, M5, b5, c5, mf), shape5)
    DW = O.dense_matrix(lambda v: O.wilson(U, v, M5), shape4)
    return D, DW, shape4, shape5


def _eps_L5(H, L5):
    I = np.eye(H.shape[0])
    a = np.linalg.matrix_power(I + H, L5)
    b = np.linalg.matrix_power(I - H, L5)
    return (a - b) @ np.linalg.inv(a + b)


def _kernel(DW, b5, c5):
    """The paper's Moebius kernel, times gamma_5: g5 (b5+c5) D_W (2 + (b5-c5) D_W)^-1."""
    n = DW.shape[0]
    g5 = np.kron(np.eye(n // 12), np.kron(O.GAMMA5, np.eye(3)))
    return g5 @ ((b5 + c5) * DW) @ np.linalg.inv(2 * np.eye(n) + (b5 - c5) * DW), g5


def _q_matrix(U, D, shape4, shape5, M5, c5, L5):
    """Columns: q = P_- x_0 + P_+ x_{L5-1} with x = D^-1 (wall source of each 4D unit vector)."""
    n4 = int(np.prod(shape4))
    Q = np.zeros((n4, n4), dtype=np.complex128)
    lu = np.linalg.inv(D)
    for j in range(n4):
        eta = np.zeros(n4, dtype=np.complex128)
        eta[j] = 1.0
        b = O.make_source(U, eta.reshape(shape4), M5, c5, L5)
        x = (lu @ b.ravel()).reshape(shape5)
        Q[:, j] = O.extract_prop4d(x).ravel()
    return Q


@pytest.mark.parametrize("M5,b5,c5,mf,L5", [(1.3, 1.5, 0.5, 0.1, 4),      # a15m310-like Moebius
                                            (1.2, 1.25, 0.25, 0.05, 6),   # a12m310-like Moebius
                                            (1.3, 1.0, 0.0, 0.1, 4),      # Shamir
                                            (1.1, 1.7, 0.3, 0.2, 4)])     # b5 - c5 != 1
def test_effective_operator_matches_paper_kernel(M5, b5, c5, mf, L5):
    """(D_eff^-1 - 1)/(1 - mf) from 5D solves equals the overlap-type operator built
    from the paper's kernel D^Moeb = (b5+c5) D_W / (2 + (b5-c5) D_W):
    D_eff = (1+mf)/2 + (1-mf)/2 g5 eps_L5(g5 D^Moeb), eps_L5 the polar (tanh) approximation."""
    U = synth.random_gauge(TINY, 21, 0.6)
    D, DW, shape4, shape5 = _dense_ops(U, TINY, M5, b5, c5, mf, L5)
    HM, g5 = _kernel(DW, b5, c5)
    I = np.eye(DW.shape[0])
    Deff = 0.5 * (1 + mf) * I + 0.5 * (1 - mf) * g5 @ _eps_L5(HM, L5)
    Q = _q_matrix(U, D, shape4, shape5, M5, c5, L5)
    expect = (np.linalg.inv(Deff) - I) / (1 - mf)
    assert np.abs(Q - expect).max() / np.abs(expect).max() < 1e-12


def test_moebius_is_rescaled_shamir_when_b5_minus_c5_is_one():
    """Sec. II: with b5 - c5 = 1 the Moebius kernel is alpha times the Shamir kernel,
    alpha = b5 + c5.  The 5D Moebius operator's D_eff must equal the one built from
    alpha * (Shamir kernel)."""
    M5, mf, L5, alpha = 1.2, 0.08, 4, 2.0
    b5, c5 = (alpha + 1) / 2, (alpha - 1) / 2
    U = synth.random_gauge(TINY, 22, 0.6)
    D, DW, shape4, shape5 = _dense_ops(U, TINY, M5, b5, c5, mf, L5)
    H_shamir, g5 = _kernel(DW, 1.0, 0.0)
    I = np.eye(DW.shape[0])
    Deff = 0.5 * (1 + mf) * I + 0.5 * (1 - mf) * g5 @ _eps_L5(alpha * H_shamir, L5)
    Q = _q_matrix(U, D, shape4, shape5, M5, c5, L5)
    expect = (np.linalg.inv(Deff) - I) / (1 - mf)
    assert np.abs(Q - expect).max() / np.abs(expect).max() < 1e-12


def test_ginsparg_wilson_defect_falls_with_L5():
    """At mf = 0 the 4D operator from the 5D solve approaches a Ginsparg-Wilson
    operator ({g5, D} = 2 D g5 D in this normalisation) as L5 grows (Sec. I)."""
    M5, b5, c5 = 1.3, 1.5, 0.5
    U = synth.random_gauge(TINY, 23, 0.4)
    defects = []
    for L5 in (2, 4, 8):
        D, DW, shape4, shape5 = _dense_ops(U, TINY, M5, b5, c5, 0.0, L5)
        Q = _q_matrix(U, D, shape4, shape5, M5, c5, L5)
        I = np.eye(Q.shape[0])
        D0 = np.linalg.inv(I + Q)
        g5 = np.kron(np.eye(Q.shape[0] // 12), np.kron(O.GAMMA5, np.eye(3)))
        defects.append(np.linalg.norm(g5 @ D0 + D0 @ g5 - 2 * D0 @ g5 @ D0))
    assert defects[0] > defects[1] > defects[2]
    assert defects[2] < 0.05 * defects[0]


# ---------------------------------------------------------------------------
# symmetries
# ---------------------------------------------------------------------------
def test_gamma5_hermiticity_of_wilson():
    dims = (4, 2, 2, 4)
    U = synth.random_gauge(dims, 31, 0.7)
    x = synth.gaussian_spinor(tuple(reversed(dims)) + (4, 3), 1)
    y = synth.gaussian_spinor(tuple(reversed(dims)) + (4, 3), 2)
    lhs = O.vdot(y, O.wilson(U, x, 1.3))
    rhs = O.vdot(O.spin_mul(O.GAMMA5, O.wilson(U, O.spin_mul(O.GAMMA5, y), 1.3)), x)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("which", ["mobius", "schur", "wilson", "A", "B", "Ainv"])
def test_adjoints(which):
    """<y, K x> = <K^+ y, x> with each K^+ coded separately from K."""
    dims, L5 = (4, 2, 2, 4), 4
    M5, b5, c5, mf = 1.2, 1.25, 0.25, 0.05
    U = synth.random_gauge(dims, 32, 0.7)
    shape = (L5,) + tuple(reversed(dims)) + (4, 3)
    x = synth.gaussian_spinor(shape, 3)
    y = synth.gaussian_spinor(shape, 4)
    if which == "schur":
        ev = O.parity_mask(dims)
        x, y = O.restrict(x, ev), O.restrict(y, ev)
    f = {
        "mobius": (lambda v: O.mobius(U, v, M5, b5, c5, mf), lambda v: O.mobius_dag(U, v, M5, b5, c5, mf)),
        "schur": (lambda v: O.schur_op(U, v, M5, b5, c5, mf), lambda v: O.schur_op_dag(U, v, M5, b5, c5, mf)),
        "wilson": (lambda v: O.wilson(U, v, M5), lambda v: O.wilson(U, v, M5, dagger=True)),
        "A": (lambda v: O.op_A(v, M5, b5, c5, mf), lambda v: O.op_A(v, M5, b5, c5, mf, dagger=True)),
        "B": (lambda v: O.op_B(v, b5, c5, mf), lambda v: O.op_B(v, b5, c5, mf, dagger=True)),
        "Ainv": (lambda v: O.op_A_inv(v, M5, b5, c5, mf), lambda v: O.op_A_inv(v, M5, b5, c5, mf, dagger=True)),
    }[which]
    lhs = O.vdot(y, f[0](x))
    rhs = O.vdot(f[1](y), x)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_gauge_covariance():
    """D[U^W](W psi) = W (D[U] psi) and x[U^W] = W x[U], U^W_mu(x) = W(x) U_mu(x) W(x+mu)^+."""
    dims, L5 = (4, 2, 2, 4), 4
    M5, b5, c5, mf = 1.3, 1.5, 0.5, 0.1
    U = synth.random_gauge(dims, 33, 0.7)
    W = synth.gauge_rotation(dims, 34)
    UW = np.empty_like(U)
    for mu, ax in enumerate((3, 2, 1, 0)):
        Wf = np.roll(W, -1, axis=ax)
        UW[..., mu, :, :] = W @ U[..., mu, :, :] @ np.conj(np.swapaxes(Wf, -1, -2))
    psi = synth.gaussian_spinor((L5,) + tuple(reversed(dims)) + (4, 3), 5)
    rot = lambda f: np.einsum('tzyxab,...tzyxsb->...tzyxsa', W, f)
    assert _rel(O.mobius(UW, rot(psi), M5, b5, c5, mf), rot(O.mobius(U, psi, M5, b5, c5, mf))) < 1e-13
    x, _ = O.solve_schur(U, psi, M5, b5, c5, mf, tol=1e-12)
    xW, _ = O.solve_schur(UW, rot(psi), M5, b5, c5, mf, tol=1e-12)
    assert _rel(xW, rot(x)) < 1e-9


# ---------------------------------------------------------------------------
# fifth-dimension operators
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("M5,b5,c5,mf,L5", [(1.3, 1.5, 0.5, 0.0158, 12), (1.2, 1.25, 0.25, 0.0022, 8),
                                            (1.3, 1.5, 0.5, 0.1, 4), (1.8, 2.25, 1.25, 0.3, 5)])
def test_a_inverse_closed_form(M5, b5, c5, mf, L5):
    """The closed-form A^-1 against a dense inverse of A built from the P operator."""
    shape = (L5, 1, 1, 1, 2, 4, 3)
    A = O.dense_matrix(lambda v: O.op_A(v, M5, b5, c5, mf), shape)
    Ainv = O.dense_matrix(lambda v: O.op_A_inv(v, M5, b5, c5, mf), shape)
    assert np.abs(Ainv @ A - np.eye(A.shape[0])).max() < 1e-13
    assert np.abs(Ainv - np.linalg.inv(A)).max() < 1e-13 * np.abs(Ainv).max()


def test_p5_structure():
    """P maps the P_+ half down one slice and the P_- half up one, with -mf at the walls."""
    L5, mf = 5, 0.3
    psi = synth.gaussian_spinor((L5, 1, 1, 1, 2, 4, 3), 6)
    out = O.p5(psi, mf)
    for s in range(L5):
        up = psi[s - 1] if s > 0 else -mf * psi[L5 - 1]
        dn = psi[s + 1] if s < L5 - 1 else -mf * psi[0]
        assert np.allclose(out[s][..., :2, :], up[..., :2, :], atol=1e-15)   # P_+ = upper spins
        assert np.allclose(out[s][..., 2:, :], dn[..., 2:, :], atol=1e-15)   # P_- = lower spins


def test_shamir_limit_is_textbook_dwf():
    """b5 = 1, c5 = 0: D = D_W + 1 - P, i.e. the 4D Wilson term on every slice plus the
    fifth-dimension hop (1 - P)."""
    dims, L5, M5, mf = (2, 2, 2, 4), 4, 1.3, 0.1
    U = synth.random_gauge(dims, 35, 0.6)
    psi = synth.gaussian_spinor((L5,) + tuple(reversed(dims)) + (4, 3), 7)
    expect = O.wilson(U, psi, M5) + psi - O.p5(psi, mf)
    assert _rel(O.mobius(U, psi, M5, 1.0, 0.0, mf), expect) < 1e-15


# ---------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------
def test_dense_lu_solve():
    """CG solutions (full and Schur) against a dense LU solve on 2^4 x L5 = 4."""
    M5, b5, c5, mf, L5 = 1.3, 1.5, 0.5, 0.1, 4
    U = synth.random_gauge(TINY, 41, 0.8)
    shape = (L5,) + TINY + (4, 3)
    D = O.dense_matrix(lambda v: O.mobius(U, v, M5, b5, c5, mf), shape)
    b = synth.gaussian_spinor(shape, 8)
    x_lu = np.linalg.solve(D, b.ravel()).reshape(shape)
    x_full, _ = O.solve_full(U, b, M5, b5, c5, mf, tol=1e-12)
    x_schur, _ = O.solve_schur(U, b, M5, b5, c5, mf, tol=1e-12)
    assert _rel(x_full, x_lu) < 1e-10
    assert _rel(x_schur, x_lu) < 1e-10
    assert O.true_residual(U, b, x_schur, M5, b5, c5, mf) < 1e-12


def test_schur_operator_is_dense_schur_complement():
    """Mhat restricted to even sites equals D_ee - D_eo D_oo^-1 D_oe of the dense D."""
    M5, b5, c5, mf, L5 = 1.2, 1.25, 0.25, 0.05, 4
    U = synth.random_gauge(TINY, 42, 0.8)
    shape = (L5,) + TINY + (4, 3)
    D = O.dense_matrix(lambda v: O.mobius(U, v, M5, b5, c5, mf), shape)
    Mhat = O.dense_matrix(lambda v: O.schur_op(U, O.restrict(v, O.parity_mask(TINY)), M5, b5, c5, mf), shape)
    ev = np.broadcast_to(O.parity_mask(TINY)[None, ..., None, None], shape).ravel() > 0.5
    od = ~ev
    S = D[np.ix_(ev, ev)] - D[np.ix_(ev, od)] @ np.linalg.inv(D[np.ix_(od, od)]) @ D[np.ix_(od, ev)]
    assert np.abs(Mhat[np.ix_(ev, ev)] - S).max() < 1e-13 * np.abs(S).max()


def test_schur_prepare_and_reconstruct():
    """With x_e the exact solution of Mhat x_e = bhat_e, reconstruct gives D x = b."""
    M5, b5, c5, mf, L5 = 1.2, 1.25, 0.25, 0.05, 4
    U = synth.random_gauge(TINY, 43, 0.8)
    shape = (L5,) + TINY + (4, 3)
    b = synth.gaussian_spinor(shape, 9)
    ev = O.parity_mask(TINY)
    Mhat = O.dense_matrix(lambda v: O.schur_op(U, O.restrict(v, ev), M5, b5, c5, mf), shape)
    mask = np.broadcast_to(ev[None, ..., None, None], shape).ravel() > 0.5
    bhat = O.schur_prepare(U, b, M5, b5, c5, mf).ravel()
    x_e = np.zeros(Mhat.shape[0], dtype=np.complex128)
    x_e[mask] = np.linalg.solve(Mhat[np.ix_(mask, mask)], bhat[mask])
    x = O.schur_reconstruct(U, b, x_e.reshape(shape), M5, b5, c5, mf)
    assert O.true_residual(U, b, x, M5, b5, c5, mf) < 1e-13


def test_source_and_prop4d_roundtrip():
    """make_source/extract_prop4d: the 4D propagator of a point source solves D_eff q' = eta
    with q' = (1-mf) q + eta, on a small random lattice (dense check)."""
    M5, b5, c5, mf, L5 = 1.3, 1.5, 0.5, 0.1, 4
    U = synth.random_gauge(TINY, 44, 0.6)
    D, DW, shape4, shape5 = _dense_ops(U, TINY, M5, b5, c5, mf, L5)
    HM, g5 = _kernel(DW, b5, c5)
    I = np.eye(DW.shape[0])
    Deff = 0.5 * (1 + mf) * I + 0.5 * (1 - mf) * g5 @ _eps_L5(HM, L5)
    eta = synth.point_source_4d(TINY, 1, 2)
    b = O.make_source(U, eta, M5, c5, L5)
    x, _ = O.solve_schur(U, b, M5, b5, c5, mf, tol=1e-12)
    q = O.extract_prop4d(x)
    assert _rel(Deff @ ((1 - mf) * q + eta).ravel(), eta.ravel()) < 1e-9


# ---------------------------------------------------------------------------
# planted mistakes: each plausible slip must fail at least one pin
# ---------------------------------------------------------------------------
def _pins_pass(module):
    """A fast subset of the pins above, run against a (possibly patched) module."""
    ok = True
    # free field plane wave (gamma basis, hop direction, boundary phase)
    dims = (2, 2, 2, 4)
    p = (np.pi, 0.0, np.pi, 2 * np.pi * 1.5 / 4)
    u = synth.gaussian_spinor((4, 3), 5)
    psi = _plane_wave(dims, p, u)
    out = module.wilson(synth.unit_gauge(dims), psi, 1.3)
    ok &= _rel(out, _plane_wave(dims, p, np.einsum('st,tc->sc', O.wilson_momentum(p, 1.3), u))) < 1e-12
    # effective operator vs the paper's kernel (5D structure, walls, A)
    M5, b5, c5, mf, L5 = 1.3, 1.5, 0.5, 0.1, 4
    U = synth.random_gauge(TINY, 21, 0.6)
    shape4 = TINY + (4, 3)
    shape5 = (L5,) + shape4
    D = O.dense_matrix(lambda v: module.mobius(U, v, M5, b5, c5, mf), shape5)
    DW = O.dense_matrix(lambda v: O.wilson(U, v, M5), shape4)
    HM, g5 = _kernel(DW, b5, c5)
    I = np.eye(DW.shape[0])
    Deff = 0.5 * (1 + mf) * I + 0.5 * (1 - mf) * g5 @ _eps_L5(HM, L5)
    Q = _q_matrix(U, D, shape4, shape5, M5, c5, L5)
    ok &= np.abs(Q - (np.linalg.inv(Deff) - I) / (1 - mf)).max() < 1e-8
    # closed-form A^-1
    shape = (L5, 1, 1, 1, 2, 4, 3)
    A = O.dense_matrix(lambda v: O.op_A(v, M5, b5, c5, mf), shape)
    Ainv = O.dense_matrix(lambda v: module.op_A_inv(v, M5, b5, c5, mf), shape)
    ok &= np.abs(Ainv @ A - np.eye(A.shape[0])).max() < 1e-12
    # Schur complement
    Dd = O.dense_matrix(lambda v: module.mobius(U, v, M5, b5, c5, mf), shape5)
    Mh = O.dense_matrix(lambda v: module.schur_op(U, O.restrict(v, O.parity_mask(TINY)), M5, b5, c5, mf), shape5)
    ev = np.broadcast_to(O.parity_mask(TINY)[None, ..., None, None], shape5).ravel() > 0.5
    od = ~ev
    S = Dd[np.ix_(ev, ev)] - Dd[np.ix_(ev, od)] @ np.linalg.inv(Dd[np.ix_(od, od)]) @ Dd[np.ix_(od, ev)]
    ok &= np.abs(Mh[np.ix_(ev, ev)] - S).max() < 1e-10
    return bool(ok)


class _Patched:
    """The oracle module with selected functions replaced."""

    def __init__(self, **over):
        self._over = over

    def __getattr__(self, name):
        return self._over.get(name, getattr(O, name))


def test_planted_mistakes():
    assert _pins_pass(O), "the unmodified oracle must pass the planted-mistake harness"

    def p5_wrong_sign(psi, mf):          # +mf instead of -mf at the walls
        return O.p5(psi, -mf)

    def p5_swapped(psi, mf):             # P_+ and P_- exchanged
        return O.p5_dag(psi, mf)

    def hop_no_antiperiodic(U, psi, antiperiodic_t=True, dagger=False):
        return O.hopping(U, psi, False, dagger)

    def hop_wrong_projector(U, psi, antiperiodic_t=True, dagger=False):
        return O.hopping(U, psi, antiperiodic_t, not dagger)

    def ainv_transposed(psi, M5, b5, c5, mf, dagger=False):
        return O.op_A_inv(psi, M5, b5, c5, mf, not dagger)

    def mobius_wrong_order(U, psi, M5, b5, c5, mf, antiperiodic_t=True):   # (b5 + c5 P) D_W
        w = O.wilson(U, psi, M5, antiperiodic_t)
        return b5 * w + c5 * O.p5(w, mf) + psi - O.p5(psi, mf)

    def mobius_from_p5(p5fn):
        def f(U, psi, M5, b5, c5, mf, antiperiodic_t=True):
            P = p5fn(psi, mf)
            return O.wilson(U, b5 * psi + c5 * P, M5, antiperiodic_t) + psi - P
        return f

    def wilson_from_hop(hop):
        def w(U, psi, M5, antiperiodic_t=True, dagger=False):
            return (4.0 - M5) * psi - 0.5 * hop(U, psi, antiperiodic_t, dagger)
        return w

    def schur_bad_coupling(U, psi_e, M5, b5, c5, mf, antiperiodic_t=True):   # 1/2 instead of 1/4
        return 2 * O.schur_op(U, psi_e, M5, b5, c5, mf) - O.op_A(psi_e, M5, b5, c5, mf)

    planted = {
        "wall sign": dict(p5=p5_wrong_sign, mobius=mobius_from_p5(p5_wrong_sign)),
        "chirality swap": dict(p5=p5_swapped, mobius=mobius_from_p5(p5_swapped)),
        "periodic time": dict(wilson=wilson_from_hop(hop_no_antiperiodic)),
        "projector sign": dict(wilson=wilson_from_hop(hop_wrong_projector)),
        "A^-1 transposed": dict(op_A_inv=ainv_transposed),
        "operator order": dict(mobius=mobius_wrong_order),
        "Schur coupling": dict(schur_op=schur_bad_coupling),
    }
    for name, over in planted.items():
        assert not _pins_pass(_Patched(**over)), "planted mistake not caught: " + name


def test_sampled_site_operator_equals_full_operator():
    """The single-site D x used for sampled checks of full-size results equals the
    full-lattice D x at those sites (every boundary case of the window)."""
    from oracle import sampled
    dims, L5 = (4, 3, 2, 5), 4
    U = synth.random_gauge(dims, 21, 0.6)
    x = synth.gaussian_spinor((L5, 5, 2, 3, 4, 4, 3), 22)
    act = (1.3, 1.5, 0.5, 0.07)
    full = O.mobius(U, x, *act)
    for site in [(0, 0, 0, 0), (3, 2, 1, 4), (1, 1, 0, 2), (2, 0, 1, 0), (0, 2, 1, 4)]:
        got = sampled.dx_at_site(U, x, site, *act)
        xs, ys, zs, ts = site
        assert np.abs(got - full[:, ts, zs, ys, xs]).max() < 1e-13


def test_mres_correlators_l5_two_identity_and_hand_example():
    """L5 = 2: the wall field q and the midpoint field Q take complementary
    chiral halves of the same two slices, so c_pp + c_j5q is the full norm of
    the solution per time slice; a single component lands in exactly one."""
    dims, L5 = (2, 2, 2, 4), 2
    xs = [synth.gaussian_spinor((L5, 4, 2, 2, 2, 4, 3), 60 + k) for k in range(3)]
    pp, j5 = O.mres_correlators(xs)
    full = sum(np.sum(np.abs(x) ** 2, axis=(0, 2, 3, 4, 5, 6)) for x in xs)
    assert np.allclose(pp + j5, full, rtol=1e-14)
    L5 = 6
    x = np.zeros((L5, 3, 2, 2, 2, 4, 3), dtype=np.complex128)
    x[0, 1, 0, 0, 0, 2, 1] = 2.0            # s = 0, spin 2: P_- keeps it -> q
    x[2, 2, 0, 1, 0, 0, 0] = 3.0            # s = L5/2 - 1, spin 0: P_+ keeps it -> Q
    x[3, 2, 0, 1, 0, 1, 0] = 5.0            # s = L5/2, spin 1: P_- drops it
    pp, j5 = O.mres_correlators([x])
    assert np.array_equal(pp, [0.0, 4.0, 0.0]) and np.array_equal(j5, [0.0, 0.0, 9.0])


def test_mres_falls_with_l5_free_shamir():
    """Free field, Shamir (b5 = 1, c5 = 0): the midpoint correlator, relative to
    the pseudoscalar one, falls geometrically with L5 (the leakage of the wall
    modes through the bulk), from the momentum-space solutions."""
    dims, M5, mf = (2, 2, 2, 6), 1.3, 0.05
    ratios = []
    for L5 in (4, 6, 8):
        xs = []
        for spin in range(4):
            for colour in range(3):
                s0 = 0 if spin < 2 else L5 - 1      # the wall-injected source (c5 = 0): P_+ at s=0, P_- at L5-1
                xs.append(O.free_propagator_point(dims, L5, M5, 1.0, 0.0, mf, spin, colour, s0))
        pp, j5 = O.mres_correlators(xs)
        assert np.all(pp > 0) and np.all(j5 > 0)
        ratios.append(np.sum(j5) / np.sum(pp))
    assert ratios[1] < 0.5 * ratios[0] and ratios[2] < 0.5 * ratios[1]


def test_gaussian_smearing_free_field_plane_wave():
    """Free field: a plane wave is an eigenvector of the smearing with eigenvalue
    (1 + k sum_i (2 cos p_i - 2))^n, k = sigma^2 / (4 n); time is not smeared."""
    dims = (4, 6, 2, 5)
    Lx, Ly, Lz, Lt = dims
    U = synth.unit_gauge(dims)
    p = (2 * np.pi * 1 / Lx, 2 * np.pi * 2 / Ly, 2 * np.pi * 1 / Lz, 2 * np.pi * 3 / Lt)
    t, z, y, x = np.meshgrid(range(Lt), range(Lz), range(Ly), range(Lx), indexing='ij')
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    chi = synth.gaussian_spinor((4, 3), 5)
    eta = phase[..., None, None] * chi
    sigma, n = 2.0, 7
    k = sigma ** 2 / (4 * n)
    lam = (1 + k * sum(2 * np.cos(p[i]) - 2 for i in range(3))) ** n
    assert np.abs(O.gaussian_smear(U, eta, sigma, n) - lam * eta).max() < 1e-13


def test_gaussian_smearing_covariance_and_width():
    dims = (4, 4, 2, 3)
    U = synth.random_gauge(dims, 31, 0.7)
    eta = synth.gaussian_spinor((3, 2, 4, 4, 4, 3), 32)
    W = synth.gauge_rotation(dims, 33)
    UW = np.empty_like(U)
    for mu, ax in enumerate((3, 2, 1, 0)):
        UW[..., mu, :, :] = W @ U[..., mu, :, :] @ np.conj(np.swapaxes(np.roll(W, -1, axis=ax), -1, -2))
    a = O.gaussian_smear(UW, np.einsum('tzyxab,tzyxsb->tzyxsa', W, eta), 1.5, 4)
    b = np.einsum('tzyxab,tzyxsb->tzyxsa', W, O.gaussian_smear(U, eta, 1.5, 4))
    assert np.abs(a - b).max() < 1e-13
    # free field: each step spreads a point by variance 2k per direction, so n steps give 2 k n = sigma^2 / 2
    # (24 sites per direction: the support of 10 steps stays clear of the wrap-around)
    big = (24, 24, 24, 1)
    eta = np.zeros((1, 24, 24, 24, 4, 3), dtype=np.complex128)
    eta[0, 12, 12, 12, 0, 0] = 1.0
    sigma, n = 2.0, 10
    sm = O.gaussian_smear(synth.unit_gauge(big), eta, sigma, n)[0, ..., 0, 0].real
    c = np.arange(24) - 12
    for axis in range(3):
        w = sm.sum(axis=tuple(a for a in range(3) if a != axis))
        assert abs(w.sum() - 1.0) < 1e-13
        assert abs((w * c ** 2).sum() - sigma ** 2 / 2) < 1e-12


def test_symmetric_schur_form():
    """The symmetric Schur operator: its adjoint (coded separately) and its
    solution, which must equal the asymmetric one and the full-lattice one."""
    dims, L5 = (4, 2, 2, 4), 4
    act = (1.3, 1.5, 0.5, 0.1)
    U = synth.random_gauge(dims, 51, 0.5)
    ev = O.parity_mask(dims)
    shape = (L5, 4, 2, 2, 4, 4, 3)
    x = O.restrict(synth.gaussian_spinor(shape, 52), ev)
    y = O.restrict(synth.gaussian_spinor(shape, 53), ev)
    lhs = O.vdot(y, O.schur_op_sym(U, x, *act))
    rhs = O.vdot(O.schur_op_sym_dag(U, y, *act), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    b = synth.gaussian_spinor(shape, 54)
    xs, _ = O.solve_schur_sym(U, b, *act, tol=1e-12)
    xa, _ = O.solve_schur(U, b, *act, tol=1e-12)
    xf, _ = O.solve_full(U, b, *act, tol=1e-12)
    assert np.linalg.norm((xs - xa).ravel()) <= 1e-9 * np.linalg.norm(xa.ravel())
    assert np.linalg.norm((xs - xf).ravel()) <= 1e-9 * np.linalg.norm(xf.ravel())
    assert O.true_residual(U, b, xs, *act) <= 1e-12
