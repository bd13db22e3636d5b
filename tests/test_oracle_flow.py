"""Pins of the oracle's gradient flow (oracle/flow.py, Sec. III), and the host
input generator's flow (synth/, plain C) checked against it.

The pins come from outside the oracle's flow code: the generator is the
steepest-descent direction of the plain Wilson action (finite differences),
pure gauge fields are fixed points, the flow is gauge covariant, the
Runge-Kutta scheme converges at third order, the weak-field limit is the
lattice heat equation with coefficient one, and the matrix exponential agrees
with scipy's."""
import numpy as np
import pytest

import synth
from oracle import flow as F


def _random_links(dims, seed, eps):
    """exp(i eps H) links, H a Gaussian Hermitian traceless matrix per link."""
    Lx, Ly, Lz, Lt = dims
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((Lt, Lz, Ly, Lx, 4, 3, 3)) + 1j * rng.standard_normal((Lt, Lz, Ly, Lx, 4, 3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    H -= (np.trace(H, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
    return F.expm_antihermitian(-1j * eps * H)


def _random_ta(rng):
    A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    X = 0.5 * (A - A.conj().T)
    return X - np.trace(X) / 3.0 * np.eye(3)


def _gauge_transform(U, W):
    out = np.empty_like(U)
    for mu in range(4):
        Wn = np.roll(W, -1, axis=3 - mu)
        out[..., mu, :, :] = np.einsum('...ab,...bc,...dc->...ad', W, U[..., mu, :, :], Wn.conj())
    return out


def test_exponential_matches_scipy_and_is_special_unitary():
    scipy_linalg = pytest.importorskip('scipy.linalg')
    rng = np.random.default_rng(1)
    for scale in (1e-3, 0.7, 3.0):
        X = scale * _random_ta(rng)
        E = F.expm_antihermitian(X)
        assert np.abs(E - scipy_linalg.expm(X)).max() < 1e-13
        assert np.abs(E @ E.conj().T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(E) - 1.0) < 1e-13


def test_generator_is_steepest_descent_of_the_plain_action():
    """d/ds S(e^{sX} V) = Re tr(X Z) at every probed link, for S the plain sum of
    Re tr(1 - plaquette); a wrong staple, orientation or sign fails it."""
    dims = (4, 2, 2, 4)
    U = _random_links(dims, 4, 0.6)
    Z = F.flow_generator(U)
    rng = np.random.default_rng(5)
    h = 1e-5
    for site, mu in (((0, 0, 0, 0), 0), ((3, 1, 0, 2), 1), ((1, 1, 1, 1), 2), ((2, 0, 1, 3), 3)):
        X = _random_ta(rng)
        Up, Um = U.copy(), U.copy()
        Up[site + (mu,)] = F.expm_antihermitian(h * X) @ U[site + (mu,)]
        Um[site + (mu,)] = F.expm_antihermitian(-h * X) @ U[site + (mu,)]
        fd = (F.wilson_action(Up) - F.wilson_action(Um)) / (2 * h)
        want = np.real(np.trace(X @ Z[site + (mu,)]))
        assert abs(fd - want) < 1e-7 * max(1.0, abs(want)), (site, mu, fd, want)
    # anti-Hermitian and traceless
    assert np.abs(Z + np.conj(np.swapaxes(Z, -1, -2))).max() < 1e-14
    assert np.abs(np.trace(Z, axis1=-2, axis2=-1)).max() < 1e-14


def test_action_falls_and_plaquette_of_unit_links_is_one():
    dims = (4, 4, 2, 4)
    U = _random_links(dims, 6, 0.8)
    s = [F.wilson_action(U)]
    for _ in range(4):
        U = F.wilson_flow(U, 0.02, 3)
        s.append(F.wilson_action(U))
    assert all(b < a for a, b in zip(s, s[1:]))
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (2, 2, 2, 2, 4, 3, 3)).copy()
    assert F.plaquette(one) == 1.0 and F.wilson_action(one) == 0.0


def test_pure_gauge_is_a_fixed_point():
    dims = (4, 2, 2, 4)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, 2, 2, 4, 4, 3, 3)).copy()
    W = _random_links(dims, 7, 2.0)[..., 0, :, :]
    U = _gauge_transform(one, W)
    assert np.abs(F.wilson_flow(U, 0.05, 3) - U).max() < 1e-13


def test_flow_is_gauge_covariant():
    dims = (4, 2, 2, 4)
    U = _random_links(dims, 8, 0.6)
    W = _random_links(dims, 9, 2.0)[..., 0, :, :]
    a = F.wilson_flow(_gauge_transform(U, W), 0.02, 4)
    b = _gauge_transform(F.wilson_flow(U, 0.02, 4), W)
    assert np.abs(a - b).max() < 1e-12


def test_runge_kutta_is_third_order():
    dims = (4, 2, 2, 4)
    U = _random_links(dims, 10, 0.6)
    t = 0.2
    ref = F.wilson_flow(U, t / 64, 64)
    errs = [np.abs(F.wilson_flow(U, t / n, n) - ref).max() for n in (4, 8, 16)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.0 < r1 < 10.0 and 6.0 < r2 < 10.0, (errs, r1, r2)


def test_weak_field_is_the_heat_equation():
    """Diagonal links exp(i theta T3), theta tiny: d theta_mu/dt equals
    -sum_nu [F_mu nu(x) - F_mu nu(x - nu)] (the lattice D_nu F_nu mu)."""
    dims = (4, 4, 2, 2)
    Lx, Ly, Lz, Lt = dims
    theta = 1e-4 * np.random.default_rng(11).standard_normal((Lt, Lz, Ly, Lx, 4))
    d3 = (1.0, -1.0, 0.0)
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
    for i in range(3):
        U[..., i, i] = np.exp(1j * theta * d3[i])
    eps = 1e-5
    dtheta = (np.angle(F.wilson_flow(U, eps, 1)[..., 0, 0]) - theta) / eps
    ax = (3, 2, 1, 0)
    expect = np.zeros_like(theta)
    for mu in range(4):
        for nu in range(4):
            if nu != mu:
                Fmn = (theta[..., mu] + np.roll(theta[..., nu], -1, axis=ax[mu])
                       - np.roll(theta[..., mu], -1, axis=ax[nu]) - theta[..., nu])
                expect[..., mu] -= Fmn - np.roll(Fmn, 1, axis=ax[nu])
    assert np.abs(dtheta - expect).max() < 1e-3 * np.abs(expect).max()


@pytest.mark.parametrize('dims,seed,eps,n', [((4, 4, 4, 4), 3, 0.4, 6), ((6, 4, 2, 8), 5, 0.7, 4)])
def test_host_generator_flow_equals_the_oracle(dims, seed, eps, n):
    """The input generator's C flow (which makes the benchmark's flowed links)
    against the oracle: same links in, same links out."""
    U = synth.random_gauge(dims, seed, eps)
    ref = F.wilson_flow(U, 0.02, n)
    assert np.abs(synth.wilson_flow(dims, U, 0.02, n) - ref).max() < 1e-12
    assert abs(synth.plaquette(dims, ref) - F.plaquette(ref)) < 1e-14
