"""The larger workloads at full size, in the solver's production configuration
(fp16 storage, FP32 arithmetic, FP64 reliable updates, CUDA graphs, autotuned
hop).  No oracle solve is feasible at these sizes, so each result is checked by
what holds at any size and by oracle values at sampled sites:

  * every solve reports a true FP64 residual |b - D x| / |b| <= 1e-10;
  * at sampled sites the residual b - D x, with D x computed by the oracle's
    own operators on the returned x, is small against |b| (it is a part of the
    global residual);
  * the FP64 operator D applied by the library agrees with the oracle's at
    those sites to 1e-13.

24^3 x 64, L5 = 8, M5 = 1.2, b5 = 1.25, c5 = 0.25, m_f in {0.0126, 0.0102}: the
12 spin-colour point sources of both masses in one 24-RHS batch.
48^3 x 64, L5 = 8, m_f = 0.0022 (light quark): two of the spin-colour sources
(the full set of 12 is the same solve repeated; its fields do not fit at once).
"""
import numpy as np
import pytest

import synth
from oracle import sampled

pytestmark = pytest.mark.gpu

M = torch = None


def setup_module(module):
    global M, torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf
    import torch as _torch
    M, torch = mdwf, _torch


def _sites(dims, rng, n=3):
    out = [(0, 0, 0, 0), (dims[0] - 1, 0, dims[2] - 1, dims[3] - 1)]
    while len(out) < n:
        out.append(tuple(int(rng.integers(d)) for d in dims))
    return out


def _run(dims, L5, act, masses, sources, seed, n_check):
    M5, b5, c5 = act
    ctx = M.mdwf_create(dims, 0)
    try:
        U = M.flowed_gauge_dev(ctx, synth.random_gauge(dims, seed, 0.4), 1.0, 0.01)
        M.mdwf_load_gauge(ctx, 0, U, 1)
        M.mdwf_set_action(ctx, 0, M5, b5, c5, masses[0], L5)
        shape5 = (L5,) + tuple(reversed(dims)) + (4, 3)
        shape4 = tuple(reversed(dims)) + (4, 3)
        srcs = {}
        for spin, colour in sources:
            eta = torch.zeros(shape4, dtype=torch.complex128, device='cuda')
            eta[0, 0, 0, 0, spin, colour] = 1.0
            b = torch.empty(shape5, dtype=torch.complex128, device='cuda')
            M.mdwf_make_source_dev(ctx, 0, eta, b)
            srcs[(spin, colour)] = b
        rhs = [(m, sc) for m in masses for sc in sources]
        xs = [torch.empty(shape5, dtype=torch.complex128, device='cuda') for _ in rhs]
        stats = M.mdwf_solve_batch_dev(ctx, 0, [srcs[sc] for _, sc in rhs], xs, 1e-10,
                                       masses=[m for m, _ in rhs], opts=M.mdwf_default_opts(precision='half'))
        torch.cuda.synchronize()
        for st in stats:
            assert st['converged'] and st['rel_true_resid'] <= 1e-10, st
        rng = np.random.default_rng(seed)
        sites = _sites(dims, rng)
        # sampled checks on the first RHS of each mass (host copies of x and b)
        for k in [i * len(sources) for i in range(len(masses))][:n_check]:
            m, sc = rhs[k]
            x = xs[k].cpu().numpy()
            b = srcs[sc].cpu().numpy()
            bn = np.linalg.norm(b.ravel())
            # the library's FP64 D x against the oracle's at the sampled sites
            dx = torch.empty_like(xs[k])
            M.mdwf_set_action(ctx, 0, M5, b5, c5, m, L5)
            M.mdwf_apply_mdwf_dev(ctx, 0, xs[k], dx)
            dxh = dx.cpu().numpy()
            del dx
            for site in sites:
                xs_, ys_, zs_, ts_ = site
                ref = sampled.dx_at_site(U, x, site, M5, b5, c5, m)
                got = dxh[:, ts_, zs_, ys_, xs_]
                assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
                r = sampled.residual_at_site(U, b, x, site, M5, b5, c5, m)
                assert np.linalg.norm(r.ravel()) <= 1e-10 * bn
        return stats
    finally:
        M.mdwf_destroy(ctx)


def test_a12m310_shaped_24cubed_two_masses_24_rhs():
    sources = [(s, c) for s in range(4) for c in range(3)]
    stats = _run((24, 24, 24, 64), 8, (1.2, 1.25, 0.25), [0.0126, 0.0102], sources, 3, 2)
    assert len(stats) == 24


def test_a12m130_shaped_48cubed_light_mass():
    stats = _run((48, 48, 48, 64), 8, (1.2, 1.25, 0.25), [0.0022], [(0, 0), (2, 1)], 4, 1)
    assert len(stats) == 2
