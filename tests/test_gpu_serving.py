"""Serving path on the device: request sources made on the device, solver
sessions with continuous batching, and the server over several resident
configurations.  Each result must be the same alone and in a mix (bitwise: a
slot's arithmetic and reductions never involve another slot), and every solve
must reach the FP64 true residual 1e-10 recomputed by the oracle's own D."""
import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O

pytestmark = pytest.mark.gpu

M = S = torch = None


def setup_module(module):
    global M, S, torch
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf, serving
    import torch as _torch
    M, S, torch = mdwf, serving, _torch


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


DIMS, L5, ACT = (4, 4, 4, 8), 4, (1.3, 1.5, 0.5, 0.1)


class Ctx:
    def __init__(self, dims=DIMS, L5=L5, act=ACT, seed=9, eps=0.3):
        self.dims, self.L5, self.act = dims, L5, act
        self.U = synth.random_gauge(dims, seed, eps)
        self.ctx = M.mdwf_create(dims, 0)
        M.mdwf_load_gauge(self.ctx, 0, self.U, 1)
        M.mdwf_set_action(self.ctx, 0, *act, L5)
        self.shape = (L5,) + tuple(reversed(dims)) + (4, 3)

    def close(self):
        M.mdwf_destroy(self.ctx)


@pytest.fixture(scope='module')
def lat():
    c = Ctx()
    yield c
    c.close()


def test_z2_source_on_device_matches_counter_generator(lat):
    eta = torch.empty(tuple(reversed(lat.dims)) + (4, 3), dtype=torch.complex128, device='cuda')
    for seed in (0, 12345, 2 ** 63 + 7):
        M.mdwf_z2_source_dev(lat.ctx, seed, eta)
        torch.cuda.synchronize()
        assert np.array_equal(eta.cpu().numpy(), synth.z2_source_4d_counter(lat.dims, seed))


def test_make_source_on_device(lat):
    eta = synth.gaussian_spinor(tuple(reversed(lat.dims)) + (4, 3), 15)
    out = torch.full(lat.shape, float('nan'), dtype=torch.complex128, device='cuda')
    M.mdwf_make_source_dev(lat.ctx, 0, torch.from_numpy(eta).cuda(), out)
    torch.cuda.synchronize()
    M5, b5, c5, mf = lat.act
    assert _rel(out.cpu().numpy(), O.make_source(lat.U, eta, M5, c5, lat.L5)) < 1e-13


def _drain(sess, limit=2000):
    done = {}
    for _ in range(limit):
        if M.mdwf_session_occupied(sess) == 0:
            return done
        M.mdwf_session_launch(sess)
        for tag, st in M.mdwf_session_poll(sess):
            done[tag] = st
    raise AssertionError('session did not drain')


@pytest.mark.parametrize('precision', ['half', 'single', 'double'])
def test_session_same_alone_and_in_mix(lat, precision):
    """Request T alone in a session, and T entering a session where other
    requests are already part-way through their solves: bitwise the same x."""
    torch.cuda.synchronize()
    opts = M.mdwf_default_opts(precision=precision)
    srcs = [torch.from_numpy(synth.gaussian_spinor(lat.shape, 200 + k)).cuda() for k in range(5)]
    masses = [0.1, 0.05, 0.2, 0.1, 0.3]
    xs_alone = torch.empty((5,) + lat.shape, dtype=torch.complex128, device='cuda')
    xs_mix = torch.empty_like(xs_alone)
    sess = M.mdwf_session_create(lat.ctx, 0, 3, 1e-10, opts=opts)
    try:
        st_alone = {}
        for k in range(5):
            M.mdwf_session_submit(sess, srcs[k], masses[k], xs_alone[k], k)
            st_alone.update(_drain(sess))
        # the mix: 0 and 1 start; after two chunks 2 joins; each later request
        # takes the first slot that frees
        M.mdwf_session_submit(sess, srcs[0], masses[0], xs_mix[0], 0)
        M.mdwf_session_submit(sess, srcs[1], masses[1], xs_mix[1], 1)
        st_mix = {}
        for _ in range(2):
            M.mdwf_session_launch(sess)
            for tag, st in M.mdwf_session_poll(sess):
                st_mix[tag] = st
        M.mdwf_session_submit(sess, srcs[2], masses[2], xs_mix[2], 2)
        nxt = 3
        for _ in range(2000):
            while nxt < 5 and M.mdwf_session_occupied(sess) < 3:
                M.mdwf_session_submit(sess, srcs[nxt], masses[nxt], xs_mix[nxt], nxt)
                nxt += 1
            if nxt == 5 and M.mdwf_session_occupied(sess) == 0:
                break
            M.mdwf_session_launch(sess)
            for tag, st in M.mdwf_session_poll(sess):
                st_mix[tag] = st
        with pytest.raises(M.MdwfError) as e:
            for k in range(4):
                M.mdwf_session_submit(sess, srcs[k], masses[k], xs_mix[k], 10 + k)
        assert e.value.code == M.MDWF_ERR_FULL
        _drain(sess)
    finally:
        M.mdwf_session_destroy(sess)
    torch.cuda.synchronize()
    a, m = xs_alone.cpu().numpy(), xs_mix.cpu().numpy()
    M5, b5, c5, _ = lat.act
    for k in range(5):
        assert st_alone[k]['converged'] and st_mix[k]['converged']
        assert st_alone[k]['iters'] == st_mix[k]['iters']
        assert np.array_equal(a[k], m[k]), k
        res = O.true_residual(lat.U, srcs[k].cpu().numpy(), a[k], M5, b5, c5, masses[k])
        assert res <= 1e-10, (k, res)
    ref, _ = O.solve_schur(lat.U, srcs[1].cpu().numpy(), M5, b5, c5, masses[1], tol=1e-13)
    assert _rel(a[1], ref) < 1e-8


def test_session_max_iter_reports_not_converged(lat):
    opts = M.mdwf_default_opts(precision='half', max_iter=20)
    src = torch.from_numpy(synth.gaussian_spinor(lat.shape, 300)).cuda()
    x = torch.empty_like(src)
    sess = M.mdwf_session_create(lat.ctx, 0, 2, 1e-10, opts=opts)
    try:
        M.mdwf_session_submit(sess, src, 0.05, x, 7)
        done = _drain(sess)
    finally:
        M.mdwf_session_destroy(sess)
    assert list(done) == [7]
    assert not done[7]['converged'] and done[7]['iters'] <= 32
    assert np.all(np.isfinite(x.cpu().numpy()))


def test_session_rejects_bad_arguments(lat):
    with pytest.raises(M.MdwfError):
        M.mdwf_session_create(lat.ctx, 0, 0, 1e-10)
    with pytest.raises(M.MdwfError):
        M.mdwf_session_create(lat.ctx, 0, 2, -1.0)
    sess = M.mdwf_session_create(lat.ctx, 0, 2, 1e-10)
    try:
        bad = torch.from_numpy(synth.gaussian_spinor(lat.shape, 301)).cuda()
        bad[0, 0, 0, 0, 0, 0, 0] = float('nan')
        with pytest.raises(M.MdwfError) as e:
            M.mdwf_session_submit(sess, bad, 0.1, torch.empty_like(bad), 1)
        assert e.value.code == M.MDWF_ERR_NONFINITE
        assert M.mdwf_session_occupied(sess) == 0
    finally:
        M.mdwf_session_destroy(sess)


def test_server_poisson_mix_over_two_configs():
    """Poisson arrivals over two resident configurations with different L5 and
    masses, Z2 and point sources; every result equals the one the same request
    gets when served alone."""
    cfgs = {'a': ((4, 4, 4, 8), 4, (1.3, 1.5, 0.5, 0.1), 21), 'b': ((4, 4, 2, 6), 6, (1.2, 1.25, 0.25, 0.05), 22)}
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(14):
        name = 'a' if rng.random() < 0.5 else 'b'
        dims = cfgs[name][0]
        mass = float(rng.choice([0.0102, 0.0158, 0.0216]) * 5)
        if rng.random() < 0.5:
            src = ('z2', int(rng.integers(1 << 40)))
        else:
            src = ('point', int(rng.integers(4)), int(rng.integers(3)),
                   tuple(int(rng.integers(d)) for d in dims))
        reqs.append((name, mass, src))
    arrivals = S.poisson_arrivals(len(reqs), 40.0, 8)
    Us = {n: synth.random_gauge(c[0], c[3], 0.3) for n, c in cfgs.items()}

    def serve(items, arr, max_slots):
        srv = S.Server(device=0, hbm_budget=2 << 30, tol=1e-10, precision='half', max_slots=max_slots,
                       keep_solutions=True)
        try:
            for n, (dims, l5, act, _) in cfgs.items():
                srv.add_config(n, dims, Us[n], *act[:3], act[3], l5)
            done = srv.run([S.Request(n, m, s) for n, m, s in items], arr, deadline=600)
            torch.cuda.synchronize()
            return sorted(done, key=lambda r: r.tag), srv
        finally:
            srv.close()

    done, srv = serve(reqs, arrivals, 3)
    assert len(done) == len(reqs)
    m = S.Server.metrics(done)
    assert m['all_converged'] and m['max_true_resid'] <= 1e-10 and m['p99_s'] >= m['p50_s'] > 0
    assert max(s[2] for s in srv.samples) >= 2          # requests overlapped on the device
    for r, (n, mass, src) in zip(done, reqs):
        dims, l5, act, _ = cfgs[n]
        x = r.x.cpu().numpy()
        # the source this request was served with, rebuilt on the host
        eta = synth.z2_source_4d_counter(dims, src[1]) if src[0] == 'z2' else \
            synth.point_source_4d(dims, src[1], src[2], src[3])
        b = O.make_source(Us[n], eta, act[0], act[2], l5)
        assert O.true_residual(Us[n], b, x, act[0], act[1], act[2], mass) <= 1e-10
    # alone: one request at a time through a fresh server
    for i in (0, 5, 11):
        alone, _ = serve([reqs[i]], None, 3)
        assert np.array_equal(alone[0].x.cpu().numpy(), done[i].x.cpu().numpy()), i
