"""Plain FP64 CPU oracle of the gradient-flow smearing of the links (Sec. III).

TEST INFRASTRUCTURE, as the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's oracle legs use it.  It shares no code
with the CUDA library or with the host input generator (synth/), and imports
neither.

Sec. III smears the gauge links with the gradient (Wilson) flow to flow time
t_gf = 1 in lattice units, following Luscher's definition (JHEP 08 (2010) 071,
cited there).  Written out:

* Wilson plaquette action  S(V) = sum_x sum_{mu<nu} Re tr(1 - V_mu nu(x)).
* The flow  dV_mu(x)/dt = Z_mu(x) V_mu(x),  Z = -P_TA(Omega),  where Omega_mu(x)
  is the sum of the six plaquettes that start with the link V_mu(x) and
  P_TA(M) = (M - M^+)/2 - tr(M - M^+)/6 is the traceless anti-Hermitian part.
  This is steepest descent of S: for any traceless anti-Hermitian X at the link,
  d/ds S(e^{sX} V) at s = 0 equals Re tr(X Z) (pinned by finite differences of
  the plain action in tests/test_oracle_flow.py).
* Integration: Luscher's third-order Runge-Kutta scheme for the flow (App. C of
  the cited paper): with Z_i = eps Z(W_i),
      W_1 = exp(Z_0 / 4) W_0,
      W_2 = exp(8 Z_1 / 9 - 17 Z_0 / 36) W_1,
      V(t + eps) = exp(3 Z_2 / 4 - 8 Z_1 / 9 + 17 Z_0 / 36) W_2.
* The exponential of a traceless anti-Hermitian matrix X = -i H is taken from
  the eigen-decomposition of the Hermitian H:  exp(X) = Q diag(e^{-i lambda}) Q^+.

Layout: U[t, z, y, x, mu, a, b] complex128, mu = 0..3 for x, y, z, t; periodic
in every direction (the links are periodic; the fermion's antiperiodic time
boundary does not enter the flow).
"""
import numpy as np

# lattice axis of direction mu in U[t, z, y, x, ...]
_AX = (3, 2, 1, 0)


def _shift(F, mu, step):
    """F(x + step * mu_hat) as a field on x."""
    return np.roll(F, -step, axis=_AX[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum('...ab,...bc->...ac', out, m)
    return out


def plaquette_field(U, mu, nu):
    """U_mu(x) U_nu(x + mu) U_mu(x + nu)^+ U_nu(x)^+ at every x."""
    return _mm(U[..., mu, :, :], _shift(U[..., nu, :, :], mu, 1),
               _dag(_shift(U[..., mu, :, :], nu, 1)), _dag(U[..., nu, :, :]))


def wilson_action(U):
    """S(V) = sum over sites and the six planes mu < nu of Re tr(1 - U_mu nu)."""
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = plaquette_field(U, mu, nu)
            s += float(np.sum(3.0 - np.real(np.trace(P, axis1=-2, axis2=-1))))
    return s


def plaquette(U):
    """Average of Re tr(U_mu nu) / 3 over sites and the six planes."""
    n = U[..., 0, 0, 0].size * 6
    return 1.0 - wilson_action(U) / (3.0 * n)


def omega(U):
    """Omega_mu(x): the six plaquettes that begin with the link U_mu(x) (for each
    nu != mu one forward, through x + nu, and one backward, through x - nu)."""
    Om = np.zeros_like(U)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        for nu in range(4):
            if nu == mu:
                continue
            Unu = U[..., nu, :, :]
            # U_mu(x) U_nu(x + mu) U_mu(x + nu)^+ U_nu(x)^+
            fwd = _mm(Umu, _shift(Unu, mu, 1), _dag(_shift(Umu, nu, 1)), _dag(Unu))
            # U_mu(x) U_nu(x + mu - nu)^+ U_mu(x - nu)^+ U_nu(x - nu)
            bwd = _mm(Umu, _dag(_shift(_shift(Unu, mu, 1), nu, -1)),
                      _dag(_shift(Umu, nu, -1)), _shift(Unu, nu, -1))
            Om[..., mu, :, :] += fwd + bwd
    return Om


def project_ta(M):
    """Traceless anti-Hermitian part (M - M^+)/2 - tr(M - M^+)/6."""
    A = 0.5 * (M - _dag(M))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


def flow_generator(U):
    """Z = -P_TA(Omega): the right-hand side of dV/dt = Z V."""
    return -project_ta(omega(U))


def expm_antihermitian(X):
    """exp(X) for anti-Hermitian X, from the eigenvectors of H = i X."""
    H = 1j * X
    H = 0.5 * (H + _dag(H))
    lam, Q = np.linalg.eigh(H)
    return _mm(Q, np.exp(-1j * lam)[..., :, None] * _dag(Q))


def flow_step(V, eps):
    """One step of the third-order Runge-Kutta scheme."""
    Z0 = eps * flow_generator(V)
    W1 = _mm(expm_antihermitian(0.25 * Z0), V)
    Z1 = eps * flow_generator(W1)
    W2 = _mm(expm_antihermitian((8.0 / 9.0) * Z1 - (17.0 / 36.0) * Z0), W1)
    Z2 = eps * flow_generator(W2)
    return _mm(expm_antihermitian(0.75 * Z2 - (8.0 / 9.0) * Z1 + (17.0 / 36.0) * Z0), W2)


def wilson_flow(U, eps, nsteps):
    """The links flowed by nsteps steps of size eps (flow time eps * nsteps)."""
    V = np.array(U, dtype=np.complex128, copy=True)
    for _ in range(int(nsteps)):
        V = flow_step(V, eps)
    return V
