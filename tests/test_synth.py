"""Pins of the synthetic-input generator: SU(3) links and the Wilson flow (Sec. III).

The flow is input preparation, not the solve; it is pinned by invariants
(unitarity, plaquette monotone, pure gauge fixed point, gauge covariance) and
by the third-order convergence of the Runge-Kutta integrator.
"""
import numpy as np

import synth


def test_links_are_special_unitary():
    U = synth.random_su3(2000, 7, 1, 0.9)
    I = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13


def test_links_are_counter_based():
    a = synth.random_su3(100, 7, 1, 0.4)
    b = synth.random_su3(300, 7, 1, 0.4)
    assert np.array_equal(a, b[:100])            # prefix independent of n
    c = synth.random_su3(100, 8, 1, 0.4)
    d = synth.random_su3(100, 7, 2, 0.4)
    assert np.abs(a - c).max() > 1e-3 and np.abs(a - d).max() > 1e-3


def test_generator_statistics():
    """exp(i eps H) with H = sum w_a lambda_a/2: for small eps, -i log U / eps has
    Gell-Mann weights with unit variance, i.e. <|H|^2_F> = 8 * 1/2 = 4."""
    eps = 1e-4
    U = synth.random_su3(20000, 3, 1, eps)
    H = (U - np.eye(3)) / (1j * eps)
    fro2 = np.mean(np.sum(np.abs(H) ** 2, axis=(1, 2)))
    assert abs(fro2 - 4.0) < 0.15
    assert np.abs(np.trace(H, axis1=1, axis2=2)).max() < 1e-3


def test_plaquette_rises_under_flow():
    dims = (4, 4, 4, 4)
    U = synth.random_gauge(dims, 11, 0.8)
    plaq = [synth.plaquette(dims, U)]
    for _ in range(5):
        U = synth.wilson_flow(dims, U, 0.02, 5)
        plaq.append(synth.plaquette(dims, U))
    assert all(b > a for a, b in zip(plaq, plaq[1:]))
    assert plaq[-1] < 1.0


def test_unit_field_plaquette_is_one():
    dims = (2, 2, 2, 4)
    assert abs(synth.plaquette(dims, synth.unit_gauge(dims)) - 1.0) < 1e-15


def _gauge_transform(dims, U, W):
    UW = np.empty_like(U)
    for mu, ax in enumerate((3, 2, 1, 0)):
        Wf = np.roll(W, -1, axis=ax)
        UW[..., mu, :, :] = W @ U[..., mu, :, :] @ np.conj(np.swapaxes(Wf, -1, -2))
    return UW


def test_pure_gauge_is_a_fixed_point():
    dims = (4, 2, 2, 4)
    W = synth.gauge_rotation(dims, 12)
    U = _gauge_transform(dims, synth.unit_gauge(dims), W)
    V = synth.wilson_flow(dims, U, 0.05, 4)
    assert np.abs(V - U).max() < 1e-13


def test_flow_is_gauge_covariant():
    dims = (4, 2, 2, 4)
    U = synth.random_gauge(dims, 13, 0.6)
    W = synth.gauge_rotation(dims, 14)
    a = synth.wilson_flow(dims, _gauge_transform(dims, U, W), 0.02, 5)
    b = _gauge_transform(dims, synth.wilson_flow(dims, U, 0.02, 5), W)
    assert np.abs(a - b).max() < 1e-12


def test_runge_kutta_is_third_order():
    """Global error at fixed flow time scales as eps^3."""
    dims = (4, 2, 2, 4)
    U = synth.random_gauge(dims, 15, 0.6)
    t = 0.2
    ref = synth.wilson_flow(dims, U, t / 64, 64)
    errs = [np.abs(synth.wilson_flow(dims, U, t / n, n) - ref).max() for n in (4, 8, 16)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.0 < r1 < 10.0 and 6.0 < r2 < 10.0, (errs, r1, r2)


def test_flow_weak_field_is_heat_equation():
    """Abelian weak-field limit: for links exp(i theta T3) with tiny theta, the flow
    evolves theta by d theta_mu/dt = -sum_nu [F_mu_nu(x) - F_mu_nu(x - nu)] (the
    lattice form of dA_mu/dt = D_nu F_nu_mu, coefficient one)."""
    dims = (4, 4, 2, 2)
    Lx, Ly, Lz, Lt = dims
    rng = np.random.default_rng(3)
    theta = 1e-4 * rng.standard_normal((Lt, Lz, Ly, Lx, 4))
    T3 = np.diag([1.0, -1.0, 0.0])
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
    for i in range(3):
        U[..., i, i] = np.exp(1j * theta * T3[i, i])
    eps = 1e-5
    V = synth.wilson_flow(dims, U, eps, 1)
    dtheta = (np.angle(V[..., 0, 0]) - theta) / eps
    ax = (3, 2, 1, 0)
    expect = np.zeros_like(theta)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            F = (theta[..., mu] + np.roll(theta[..., nu], -1, axis=ax[mu])
                 - np.roll(theta[..., mu], -1, axis=ax[nu]) - theta[..., nu])
            expect[..., mu] -= F - np.roll(F, 1, axis=ax[nu])
    assert np.abs(dtheta - expect).max() < 1e-3 * np.abs(expect).max()


def test_z2_counter_source():
    dims = (4, 2, 2, 6)
    eta = synth.z2_source_4d_counter(dims, 77)
    assert eta.shape == (6, 2, 2, 4, 4, 3)
    assert np.all(eta.imag == 0) and np.all(np.abs(eta.real) == 1)
    # element k from the k-th generator output alone
    z = synth.splitmix64(77, eta.size)
    k = 123
    assert eta.ravel()[k].real == (-1.0 if int(z[k]) >> 63 else 1.0)
    big = synth.z2_source_4d_counter((8, 8, 8, 8), 5)
    assert abs(big.real.mean()) < 4.0 / np.sqrt(big.size)
    assert not np.array_equal(big, synth.z2_source_4d_counter((8, 8, 8, 8), 6))
