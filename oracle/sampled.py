"""The oracle's D x at single sites of a large lattice, for sampled checks of
full-size results: D = A - 1/2 H B evaluated on the 3^4 window of sites around
the sampled site (time-boundary phases folded into the window), with the
oracle's own A, B and single-site hop (Sec. II operator, as in mdwf_oracle).

TEST INFRASTRUCTURE, as the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's oracle legs use it."""
import numpy as np

from . import mdwf_oracle as O


def _window(field, site, dims, antiperiodic_t, links=False):
    Lx, Ly, Lz, Lt = dims
    x, y, z, t = site
    if links:
        w = np.empty((3, 3, 3, 3) + field.shape[4:], dtype=field.dtype)
    else:
        w = np.empty((field.shape[0], 3, 3, 3, 3) + field.shape[5:], dtype=field.dtype)
    for dt in (-1, 0, 1):
        tt = t + dt
        phase = -1.0 if antiperiodic_t and (tt < 0 or tt >= Lt) else 1.0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    src = (tt % Lt, (z + dz) % Lz, (y + dy) % Ly, (x + dx) % Lx)
                    idx = (1 + dt, 1 + dz, 1 + dy, 1 + dx)
                    if links:
                        w[idx] = field[src]
                    else:
                        w[(slice(None),) + idx] = phase * field[(slice(None),) + src]
    return w


def dx_at_site(U, x, site, M5, b5, c5, mf, antiperiodic_t=True):
    """(D x)(site) for all slices: array [L5, spin, colour]."""
    dims = (x.shape[4], x.shape[3], x.shape[2], x.shape[1])
    xw = _window(x, site, dims, antiperiodic_t)
    Uw = _window(U, site, dims, antiperiodic_t, links=True)
    hop = O.hopping_at_site(Uw, O.op_B(xw, b5, c5, mf), (1, 1, 1, 1), antiperiodic_t=False)
    ax = O.op_A(xw[:, 1:2, 1:2, 1:2, 1:2], M5, b5, c5, mf)[:, 0, 0, 0, 0]
    return ax - 0.5 * hop


def residual_at_site(U, b, x, site, M5, b5, c5, mf, antiperiodic_t=True):
    xs, ys, zs, ts = site
    return b[:, ts, zs, ys, xs] - dx_at_site(U, x, site, M5, b5, c5, mf, antiperiodic_t)
