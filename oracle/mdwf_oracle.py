"""Plain FP64 CPU oracle for the even-odd preconditioned Moebius domain-wall solve.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
oracle legs of ``bench.py`` (``cpu_baseline`` with its sampled residual check,
``--impl reference``) may import this module.  It shares no code with the CUDA library and never imports it.

Everything is written out in the most direct form: full-lattice complex128
arrays, ``np.roll`` for the nearest-neighbour shifts and ``np.einsum`` for the
spin and colour contractions.  No blocking, fusion or reordering.

What is computed, and where it comes from (arXiv:1701.07559):

* The Moebius kernel  D^Moeb = (b5+c5) D_W / (2 + (b5-c5) D_W)  (Sec. II, first
  displayed equation) and its Shamir special case b5-c5=1 (Sec. II, second
  equation).  The paper gives only this 4D kernel; the 5D operator that
  realises it is the Brower-Neff-Orginos form, read here as

      D = D_W (b5 + c5 P) + (1 - P),
      (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
      psi_{L5} = -m_f psi_0,  psi_{-1} = -m_f psi_{L5-1},

  with  D_W = (4 - M5) - 1/2 H  the Wilson operator at negative mass -M5
  ("domain-wall height" M5, Sec. II) and H the nearest-neighbour hopping term.
  The test suite pins this reading to the paper's kernel equation through the
  4D effective operator identity (tests/test_oracle_pins.py).
* The even-odd ("red-black") Schur complement named in Sec. VII (asymmetric
  form, the one Chroma used):  Mhat = A_ee - D_eo A_oo^-1 D_oe  with
  A = (b5 d + 1) + (c5 d - 1) P, B = b5 + c5 P, d = 4 - M5, D_eo = -1/2 H_eo B.
* Conjugate gradient on the normal equations (Sec. VII: the solver QUDA runs).
* The residual-mass correlators of Sec. III (midpoint and wall pseudoscalar
  densities, equation eq:mres).
* Gauge-covariant Gaussian smearing of 4D sources (Sec. VII's propagators).

Gamma matrices: DeGrand-Rossi chiral basis (gamma_5 = diag(1,1,-1,-1)).
Boundary conditions: periodic in x, y, z; antiperiodic in t.

Array layouts (identical to the C ABI's host layout):
  gauge  U[t, z, y, x, mu, a, b]      complex128, mu = 0..3 for x, y, z, t
  4D     psi[t, z, y, x, spin, colour]
  5D     psi[s, t, z, y, x, spin, colour]
"""
import numpy as np

# ---------------------------------------------------------------------------
# Gamma matrices (DeGrand-Rossi basis, Euclidean, Hermitian)
# ---------------------------------------------------------------------------
GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
GAMMA[0] = [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]]
GAMMA[1] = [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]
GAMMA[2] = [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]]
GAMMA[3] = [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (ID4 + GAMMA5)
P_MINUS = 0.5 * (ID4 - GAMMA5)

# Lattice axis of direction mu in a 4D field [t, z, y, x, ...]:
# x -> 3, y -> 2, z -> 1, t -> 0.
_AX4 = (3, 2, 1, 0)


def spin_mul(M, psi):
    """Apply a 4x4 spin matrix to every site of a 4D or 5D spinor field."""
    return np.einsum('st,...tc->...sc', M, psi)


def colour_mul(U, psi):
    """Apply a field of 3x3 colour matrices U[t,z,y,x,a,b] to psi[..., spin, b]."""
    return np.einsum('tzyxab,...tzyxsb->...tzyxsa', U, psi)


def _shift(psi, mu, sign, antiperiodic_t, ndim_lead):
    """Return psi(x + sign*mu_hat) with the time boundary phase applied.

    ``ndim_lead`` is the number of leading (non-lattice) axes, 1 for a 5D
    field [s, t, z, y, x, ...], 0 for a 4D field.
    """
    ax = ndim_lead + _AX4[mu]
    out = np.roll(psi, -sign, axis=ax)
    if mu == 3 and antiperiodic_t:
        Lt = psi.shape[ax]
        idx = [slice(None)] * psi.ndim
        # the slice that wrapped around the time boundary picks up a -1
        idx[ax] = Lt - 1 if sign > 0 else 0
        out[tuple(idx)] *= -1.0
    return out


def hopping(U, psi, antiperiodic_t=True, dagger=False):
    """Wilson hopping term on every slice of a 4D or 5D field.

    (H psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) ]

    With ``dagger`` the projectors are exchanged, which is H^+ (= g5 H g5).
    """
    lead = psi.ndim - 6
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        Umu_back = np.conj(np.swapaxes(np.roll(Umu, 1, axis=_AX4[mu]), -1, -2))
        fwd = colour_mul(Umu, _shift(psi, mu, +1, antiperiodic_t, lead))
        bwd = colour_mul(Umu_back, _shift(psi, mu, -1, antiperiodic_t, lead))
        s = 1.0 if dagger else -1.0
        out += spin_mul(ID4 + s * GAMMA[mu], fwd) + spin_mul(ID4 - s * GAMMA[mu], bwd)
    return out


def wilson(U, psi, M5, antiperiodic_t=True, dagger=False):
    """D_W psi = (4 - M5) psi - 1/2 H psi   (Wilson operator at mass -M5)."""
    return (4.0 - M5) * psi - 0.5 * hopping(U, psi, antiperiodic_t, dagger)


# ---------------------------------------------------------------------------
# Fifth-dimension operators
# ---------------------------------------------------------------------------
def p5(psi, mf):
    """(P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}; psi_{L5} = -mf psi_0, psi_{-1} = -mf psi_{L5-1}."""
    up = np.roll(psi, -1, axis=0)           # psi_{s+1}
    up[-1] *= -mf
    dn = np.roll(psi, 1, axis=0)            # psi_{s-1}
    dn[0] *= -mf
    return spin_mul(P_MINUS, up) + spin_mul(P_PLUS, dn)


def p5_dag(psi, mf):
    """Adjoint of p5: (P^+ psi)_s = P_+ psi_{s+1} + P_- psi_{s-1}, same wall factors."""
    up = np.roll(psi, -1, axis=0)
    up[-1] *= -mf
    dn = np.roll(psi, 1, axis=0)
    dn[0] *= -mf
    return spin_mul(P_PLUS, up) + spin_mul(P_MINUS, dn)


def op_B(psi, b5, c5, mf, dagger=False):
    """B = b5 + c5 P (or its adjoint)."""
    P = p5_dag(psi, mf) if dagger else p5(psi, mf)
    return b5 * psi + c5 * P


def op_A(psi, M5, b5, c5, mf, dagger=False):
    """A = (b5 d + 1) + (c5 d - 1) P with d = 4 - M5 (or its adjoint)."""
    d = 4.0 - M5
    P = p5_dag(psi, mf) if dagger else p5(psi, mf)
    return (b5 * d + 1.0) * psi + (c5 * d - 1.0) * P


def a_inverse_matrices(M5, b5, c5, mf, L5):
    """Closed-form inverse of A on each chirality, as two real L5 x L5 matrices.

    On the P_+ half A acts as  alpha x_s + beta x_{s-1}  (x_{-1} = -mf x_{L5-1}),
    on the P_- half as         alpha x_s + beta x_{s+1}  (x_{L5} = -mf x_0),
    alpha = b5 d + 1, beta = c5 d - 1.  With kappa = beta/alpha the inverse is
    (-kappa)^k sigma / (alpha (1 + mf (-kappa)^L5)), k the number of steps from
    s' to s along the shift direction (mod L5), sigma = -mf when the path
    crosses the wall, else 1.  Returns (Ainv_plus, Ainv_minus).
    """
    d = 4.0 - M5
    alpha = b5 * d + 1.0
    beta = c5 * d - 1.0
    kappa = beta / alpha
    norm = 1.0 / (alpha * (1.0 + mf * (-kappa) ** L5))
    plus = np.zeros((L5, L5))
    minus = np.zeros((L5, L5))
    for s in range(L5):
        for sp in range(L5):
            k = (s - sp) % L5
            sigma = 1.0 if s >= sp else -mf
            plus[s, sp] = (-kappa) ** k * sigma * norm
            k = (sp - s) % L5
            sigma = 1.0 if s <= sp else -mf
            minus[s, sp] = (-kappa) ** k * sigma * norm
    return plus, minus


def op_A_inv(psi, M5, b5, c5, mf, dagger=False):
    """A^-1 (or its adjoint, the transposed real matrices) on a 5D field."""
    L5 = psi.shape[0]
    plus, minus = a_inverse_matrices(M5, b5, c5, mf, L5)
    if dagger:
        plus, minus = plus.T, minus.T
    yp = np.einsum('ij,j...->i...', plus, spin_mul(P_PLUS, psi))
    ym = np.einsum('ij,j...->i...', minus, spin_mul(P_MINUS, psi))
    return yp + ym


# ---------------------------------------------------------------------------
# The 5D Moebius domain-wall operator
# ---------------------------------------------------------------------------
def mobius(U, psi, M5, b5, c5, mf, antiperiodic_t=True):
    """D psi = D_W (b5 + c5 P) psi + (1 - P) psi."""
    P = p5(psi, mf)
    return wilson(U, b5 * psi + c5 * P, M5, antiperiodic_t) + psi - P


def mobius_dag(U, psi, M5, b5, c5, mf, antiperiodic_t=True):
    """D^+ psi = (b5 + c5 P^+) D_W^+ psi + (1 - P^+) psi, coded separately from D."""
    w = wilson(U, psi, M5, antiperiodic_t, dagger=True)
    return b5 * w + c5 * p5_dag(w, mf) + psi - p5_dag(psi, mf)


# ---------------------------------------------------------------------------
# Even-odd decomposition (4D checkerboard) and the Schur complement
# ---------------------------------------------------------------------------
def parity_mask(dims):
    """1.0 on sites with (x+y+z+t) even, shape [t, z, y, x]; dims = (Lx, Ly, Lz, Lt)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing='ij')
    return ((x + y + z + t) % 2 == 0).astype(np.float64)


def restrict(psi, mask):
    """Zero the sites where mask is 0 (mask has shape [t, z, y, x])."""
    return psi * mask[..., None, None]


def schur_op(U, psi_e, M5, b5, c5, mf, antiperiodic_t=True):
    """Mhat psi_e = A psi_e - D_eo A^-1 D_oe psi_e,  D_eo = D_oe = -1/2 H B (restricted).

    Fields are full-lattice arrays that vanish on odd sites.
    """
    dims = (psi_e.shape[4], psi_e.shape[3], psi_e.shape[2], psi_e.shape[1])
    even = parity_mask(dims)
    odd = 1.0 - even
    d_oe = restrict(-0.5 * hopping(U, op_B(psi_e, b5, c5, mf), antiperiodic_t), odd)
    t = op_A_inv(d_oe, M5, b5, c5, mf)
    d_eo = restrict(-0.5 * hopping(U, op_B(t, b5, c5, mf), antiperiodic_t), even)
    return op_A(psi_e, M5, b5, c5, mf) - d_eo


def schur_op_dag(U, psi_e, M5, b5, c5, mf, antiperiodic_t=True):
    """Mhat^+ = A^+ - D_oe^+ A^-+ D_eo^+, with D_eo^+ = -1/2 B^+ H^+ (restricted)."""
    dims = (psi_e.shape[4], psi_e.shape[3], psi_e.shape[2], psi_e.shape[1])
    even = parity_mask(dims)
    odd = 1.0 - even
    w = restrict(-0.5 * op_B(hopping(U, psi_e, antiperiodic_t, dagger=True), b5, c5, mf, dagger=True), odd)
    t = op_A_inv(w, M5, b5, c5, mf, dagger=True)
    v = restrict(-0.5 * op_B(hopping(U, t, antiperiodic_t, dagger=True), b5, c5, mf, dagger=True), even)
    return op_A(psi_e, M5, b5, c5, mf, dagger=True) - v


def schur_prepare(U, b, M5, b5, c5, mf, antiperiodic_t=True):
    """bhat_e = b_e - D_eo A^-1 b_o."""
    dims = (b.shape[4], b.shape[3], b.shape[2], b.shape[1])
    even = parity_mask(dims)
    b_e = restrict(b, even)
    b_o = restrict(b, 1.0 - even)
    t = op_A_inv(b_o, M5, b5, c5, mf)
    return b_e - restrict(-0.5 * hopping(U, op_B(t, b5, c5, mf), antiperiodic_t), even)


def schur_reconstruct(U, b, x_e, M5, b5, c5, mf, antiperiodic_t=True):
    """x_o = A^-1 (b_o - D_oe x_e); returns the full x = x_e + x_o."""
    dims = (b.shape[4], b.shape[3], b.shape[2], b.shape[1])
    even = parity_mask(dims)
    odd = 1.0 - even
    b_o = restrict(b, odd)
    d_oe = restrict(-0.5 * hopping(U, op_B(x_e, b5, c5, mf), antiperiodic_t), odd)
    return x_e + op_A_inv(b_o - d_oe, M5, b5, c5, mf)


# ---------------------------------------------------------------------------
# Conjugate gradient on the normal equations
# ---------------------------------------------------------------------------
def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.vdot(a.ravel(), a.ravel()).real)


def cgnr(apply, apply_dag, b, tol, max_iter=100000, x0=None, target_norm=None):
    """Textbook CG on  A^+ A x = A^+ b.

    Stops when the recursively updated residual ||b - A x|| falls below
    tol * target_norm (default ||b||), then confirms it with a true residual;
    if the check fails it restarts from the current x.  Returns (x, iterations).
    """
    bnorm = np.sqrt(norm2(b)) if target_norm is None else target_norm
    x = np.zeros_like(b) if x0 is None else x0.copy()
    total = 0
    while True:
        rho = b - apply(x)                 # residual of A x = b
        if np.sqrt(norm2(rho)) <= tol * bnorm or total >= max_iter:
            return x, total
        r = apply_dag(rho)                 # residual of the normal equations
        p = r.copy()
        gamma = norm2(r)
        while total < max_iter:
            q = apply(p)
            alpha = gamma / norm2(q)
            x += alpha * p
            rho -= alpha * q
            r -= alpha * apply_dag(q)
            total += 1
            if np.sqrt(norm2(rho)) <= 0.5 * tol * bnorm:
                break
            gamma_new = norm2(r)
            p = r + (gamma_new / gamma) * p
            gamma = gamma_new


def solve_full(U, b, M5, b5, c5, mf, tol=1e-10, antiperiodic_t=True, max_iter=100000):
    """x = D^-1 b by CG on D^+ D over the full (unpreconditioned) lattice."""
    return cgnr(lambda v: mobius(U, v, M5, b5, c5, mf, antiperiodic_t),
                lambda v: mobius_dag(U, v, M5, b5, c5, mf, antiperiodic_t),
                b, tol, max_iter)


def solve_schur(U, b, M5, b5, c5, mf, tol=1e-10, antiperiodic_t=True, max_iter=100000):
    """x = D^-1 b through the asymmetric even-odd Schur complement and CGNR.

    The inner stopping rule is on ||bhat - Mhat x_e|| <= tol ||b||, which equals
    the full residual ||b - D x|| after reconstruction (the odd rows vanish).
    """
    bhat = schur_prepare(U, b, M5, b5, c5, mf, antiperiodic_t)
    x_e, iters = cgnr(lambda v: schur_op(U, v, M5, b5, c5, mf, antiperiodic_t),
                      lambda v: schur_op_dag(U, v, M5, b5, c5, mf, antiperiodic_t),
                      bhat, tol, max_iter, target_norm=np.sqrt(norm2(b)))
    return schur_reconstruct(U, b, x_e, M5, b5, c5, mf, antiperiodic_t), iters


def schur_op_sym(U, psi_e, M5, b5, c5, mf, antiperiodic_t=True):
    """Symmetric form Mhat_s = A_ee^-1 Mhat = 1 - A^-1 D_eo A^-1 D_oe (Sec. VII names it as the
    better-conditioned alternative to the asymmetric form)."""
    return op_A_inv(schur_op(U, psi_e, M5, b5, c5, mf, antiperiodic_t), M5, b5, c5, mf)


def schur_op_sym_dag(U, psi_e, M5, b5, c5, mf, antiperiodic_t=True):
    """Mhat_s^+ = Mhat^+ A^-+."""
    return schur_op_dag(U, op_A_inv(psi_e, M5, b5, c5, mf, dagger=True), M5, b5, c5, mf, antiperiodic_t)


def solve_schur_sym(U, b, M5, b5, c5, mf, tol=1e-10, antiperiodic_t=True, max_iter=100000):
    """x = D^-1 b through the symmetric Schur form: CGNR on Mhat_s x_e = A^-1 bhat_e."""
    bhat = op_A_inv(schur_prepare(U, b, M5, b5, c5, mf, antiperiodic_t), M5, b5, c5, mf)
    d = 4.0 - M5
    na = abs(b5 * d + 1.0) + abs(c5 * d - 1.0)
    x_e, iters = cgnr(lambda v: schur_op_sym(U, v, M5, b5, c5, mf, antiperiodic_t),
                      lambda v: schur_op_sym_dag(U, v, M5, b5, c5, mf, antiperiodic_t),
                      bhat, tol / na, max_iter, target_norm=np.sqrt(norm2(b)))
    return schur_reconstruct(U, b, x_e, M5, b5, c5, mf, antiperiodic_t), iters


def true_residual(U, b, x, M5, b5, c5, mf, antiperiodic_t=True):
    """||b - D x|| / ||b|| in FP64."""
    r = b - mobius(U, x, M5, b5, c5, mf, antiperiodic_t)
    return np.sqrt(norm2(r) / norm2(b))


# ---------------------------------------------------------------------------
# Sources and the 4D propagator
# ---------------------------------------------------------------------------
def make_source(U, eta, M5, c5, L5, antiperiodic_t=True):
    """5D source from a 4D field: b = (1 - c5 D_W)(P_+ eta delta_{s,0} + P_- eta delta_{s,L5-1})."""
    walls = np.zeros((L5,) + eta.shape, dtype=np.complex128)
    walls[0] = spin_mul(P_PLUS, eta)
    walls[L5 - 1] = spin_mul(P_MINUS, eta)
    return walls - c5 * wilson(U, walls, M5, antiperiodic_t)


def extract_prop4d(x):
    """4D quark field from a 5D solution: q = P_- x_0 + P_+ x_{L5-1}."""
    return spin_mul(P_MINUS, x[0]) + spin_mul(P_PLUS, x[-1])


def point_source_4d(dims, spin, colour, site=(0, 0, 0, 0)):
    """Unit point source eta at site = (x, y, z, t)."""
    Lx, Ly, Lz, Lt = dims
    eta = np.zeros((Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    eta[t, z, y, x, spin, colour] = 1.0
    return eta


def point_source_5d(dims, L5, spin, colour, s=0, site=(0, 0, 0, 0)):
    """5D unit vector: 1 at (s, site, spin, colour)."""
    Lx, Ly, Lz, Lt = dims
    b = np.zeros((L5, Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[s, t, z, y, x, spin, colour] = 1.0
    return b


# ---------------------------------------------------------------------------
# Single-site evaluation (for sampled checks on lattices too large for a
# full-field pass)
# ---------------------------------------------------------------------------
def hopping_at_site(U, psi, site, antiperiodic_t=True, dagger=False):
    """(H psi)(x) at one site x = (x, y, z, t), for all leading (s) indices.

    psi is a 5D field [s, t, z, y, x, spin, colour]; returns [s, spin, colour].
    Plain loops over the eight neighbours.
    """
    Lt, Lz, Ly, Lx = psi.shape[1:5]
    L = (Lx, Ly, Lz, Lt)
    out = np.zeros((psi.shape[0], 4, 3), dtype=np.complex128)
    sgn = 1.0 if dagger else -1.0
    for mu in range(4):
        fwd = list(site)
        fwd[mu] += 1
        phase_f = 1.0
        if fwd[mu] == L[mu]:
            fwd[mu] = 0
            if mu == 3 and antiperiodic_t:
                phase_f = -1.0
        bwd = list(site)
        bwd[mu] -= 1
        phase_b = 1.0
        if bwd[mu] < 0:
            bwd[mu] = L[mu] - 1
            if mu == 3 and antiperiodic_t:
                phase_b = -1.0
        x, y, z, t = site
        Uf = U[t, z, y, x, mu]
        xb, yb, zb, tb = bwd
        Ub = np.conj(U[tb, zb, yb, xb, mu]).T
        xf, yf, zf, tf = fwd
        pf = psi[:, tf, zf, yf, xf]          # [s, spin, colour]
        pb = psi[:, tb, zb, yb, xb]
        out += phase_f * np.einsum('st,ab,ntb->nsa', ID4 + sgn * GAMMA[mu], Uf, pf)
        out += phase_b * np.einsum('st,ab,ntb->nsa', ID4 - sgn * GAMMA[mu], Ub, pb)
    return out


# ---------------------------------------------------------------------------
# Gauge-covariant Gaussian source smearing
# ---------------------------------------------------------------------------
def covariant_laplacian_3d(U, eta):
    """(Delta eta)(x) = sum_{i=x,y,z} [U_i(x) eta(x+i) + U_i(x-i)^+ eta(x-i) - 2 eta(x)], on a 4D
    field [t, z, y, x, spin, colour] (spin-diagonal; no hop in time)."""
    out = -6.0 * eta
    for mu in range(3):
        out = out + colour_mul(U[..., mu, :, :], _shift(eta, mu, +1, False, 0))
        Ub = np.conj(np.swapaxes(U[..., mu, :, :], -1, -2))
        out = out + _shift(colour_mul(Ub, eta), mu, -1, False, 0)
    return out


def gaussian_smear(U, eta, sigma, n_iter):
    """Gauge-covariant Gaussian smearing of a 4D source (the sources of Sec. VII's propagators):
    eta <- (1 + sigma^2 / (4 n) Delta)^n eta, which tends to exp(sigma^2 Delta / 4) eta."""
    k = sigma * sigma / (4.0 * n_iter)
    for _ in range(n_iter):
        eta = eta + k * covariant_laplacian_3d(U, eta)
    return eta


# ---------------------------------------------------------------------------
# Residual mass
# ---------------------------------------------------------------------------
def mres_correlators(xs):
    """Correlators of the residual-mass ratio (Sec. III, equation eq:mres).

    xs: the 5D solutions of the point-source solves (one per source spin and
    colour), each [s, t, z, y, x, spin, colour].  The wall quark field is
    q = P_- x_0 + P_+ x_{L5-1} and the midpoint field Q = P_+ x_{L5/2-1} +
    P_- x_{L5/2}; summed over the spatial sites of each time slice and over
    the sources, the pseudoscalar correlators are the squared norms of q and
    of Q (gamma_5-hermiticity of the sources' propagator).  Returns
    (c_pp[t], c_j5q[t]); m_res(t) = c_j5q / c_pp.
    """
    L5 = xs[0].shape[0]
    Lt = xs[0].shape[1]
    c_pp = np.zeros(Lt)
    c_j5q = np.zeros(Lt)
    for x in xs:
        q = spin_mul(P_MINUS, x[0]) + spin_mul(P_PLUS, x[L5 - 1])
        Q = spin_mul(P_PLUS, x[L5 // 2 - 1]) + spin_mul(P_MINUS, x[L5 // 2])
        c_pp += np.sum(np.abs(q) ** 2, axis=(1, 2, 3, 4, 5))
        c_j5q += np.sum(np.abs(Q) ** 2, axis=(1, 2, 3, 4, 5))
    return c_pp, c_j5q


# ---------------------------------------------------------------------------
# Free field (unit links) in momentum space
# ---------------------------------------------------------------------------
def momenta(dims, antiperiodic_t=True):
    """All lattice momenta (p_x, p_y, p_z, p_t); p_t = 2 pi (n + 1/2)/Lt when antiperiodic."""
    Lx, Ly, Lz, Lt = dims
    out = []
    for nt in range(Lt):
        for nz in range(Lz):
            for ny in range(Ly):
                for nx in range(Lx):
                    pt = 2 * np.pi * (nt + (0.5 if antiperiodic_t else 0.0)) / Lt
                    out.append((2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly, 2 * np.pi * nz / Lz, pt))
    return out


def wilson_momentum(p, M5):
    """Free Wilson operator D_W(p) = sum_mu (1 - cos p_mu) - M5 + i sum_mu g_mu sin p_mu."""
    D = (sum(1.0 - np.cos(pm) for pm in p) - M5) * ID4
    for mu in range(4):
        D = D + 1j * np.sin(p[mu]) * GAMMA[mu]
    return D


def mobius_momentum(p, M5, b5, c5, mf, L5):
    """Free 5D operator D(p) as a (4 L5) x (4 L5) matrix, index (s, spin)."""
    Dw = wilson_momentum(p, M5)
    P = np.zeros((4 * L5, 4 * L5), dtype=np.complex128)
    for s in range(L5):
        # P_- psi_{s+1}
        sp = (s + 1) % L5
        f = -mf if s == L5 - 1 else 1.0
        P[4 * s:4 * s + 4, 4 * sp:4 * sp + 4] += f * P_MINUS
        # P_+ psi_{s-1}
        sm = (s - 1) % L5
        f = -mf if s == 0 else 1.0
        P[4 * s:4 * s + 4, 4 * sm:4 * sm + 4] += f * P_PLUS
    DW5 = np.kron(np.eye(L5), Dw)
    I = np.eye(4 * L5)
    return DW5 @ (b5 * I + c5 * P) + (I - P)


def free_propagator_point(dims, L5, M5, b5, c5, mf, spin, colour, s0=0, antiperiodic_t=True):
    """Free-field D^-1 applied to the 5D unit source at the origin, by Fourier sum.

    x(y) = (1/V) sum_p e^{i p.y} D(p)^-1 b(0).
    """
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    rhs = np.zeros(4 * L5, dtype=np.complex128)
    rhs[4 * s0 + spin] = 1.0
    coords = np.stack(np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                                  indexing='ij'), axis=-1)   # [t,z,y,x,(t,z,y,x)]
    x = np.zeros((L5, Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    for p in momenta(dims, antiperiodic_t):
        sol = np.linalg.solve(mobius_momentum(p, M5, b5, c5, mf, L5), rhs).reshape(L5, 4)
        phase = np.exp(1j * (p[0] * coords[..., 3] + p[1] * coords[..., 2]
                             + p[2] * coords[..., 1] + p[3] * coords[..., 0]))
        x[..., colour] += np.einsum('tzyx,sd->stzyxd', phase, sol) / V
    return x


# ---------------------------------------------------------------------------
# Dense matrices on tiny lattices
# ---------------------------------------------------------------------------
def dense_matrix(apply, shape):
    """Dense matrix of a linear map on fields of the given shape (column by column)."""
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).ravel()
    return M
