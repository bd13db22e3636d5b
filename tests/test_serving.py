"""Host logic of the serving loop (queueing, admission by HBM footprint,
no starvation, latency metrics), driven by a stand-in for the library's session
functions: no device needed.  The device path is tested in test_gpu_serving.py."""
import numpy as np
import pytest

from paper_1701_07559_gb300 import build


@pytest.fixture(scope='module')
def serving():
    build.build()
    from paper_1701_07559_gb300 import serving
    return serving


class FakeLib:
    """Sessions whose requests finish after a number of launches set by the mass."""

    def __init__(self, bytes_per_slot):
        self.bytes_per_slot = bytes_per_slot
        self.created, self.destroyed, self.launches = [], [], 0
        self.live = 0
        self.max_live = 0

    class Ctx:
        def __init__(self, dims):
            self.dims = dims

    class Sess:
        def __init__(self, ctx, slots):
            self.ctx, self.slots, self.reqs = ctx, slots, {}

    def mdwf_create(self, dims, device):
        return self.Ctx(dims)

    def mdwf_load_gauge(self, ctx, cfg, U, anti):
        pass

    def mdwf_set_action(self, ctx, cfg, M5, b5, c5, mf, L5):
        ctx.L5 = L5

    def mdwf_destroy(self, ctx):
        pass

    def mdwf_session_bytes(self, ctx, cfg, slots, precision):
        return self.bytes_per_slot[ctx.dims] * slots

    def mdwf_session_create(self, ctx, cfg, slots, tol, opts=None, stream=None):
        s = self.Sess(ctx, slots)
        self.created.append((ctx.dims, slots))
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return s

    def mdwf_session_destroy(self, s):
        self.destroyed.append(s.ctx.dims)
        self.live -= 1

    def mdwf_z2_source_dev(self, ctx, seed, eta, stream=None):
        eta.fill_(1.0)

    def mdwf_make_source_dev(self, ctx, cfg, eta, src, stream=None):
        src.zero_()

    def mdwf_session_submit(self, s, src, mass, x, tag):
        assert len(s.reqs) < s.slots
        s.reqs[tag] = int(round(mass * 100))

    def mdwf_session_launch(self, s, iters=0):
        self.launches += 1
        for t in s.reqs:
            s.reqs[t] -= 1

    def mdwf_session_poll(self, s, max_done=None):
        out = [(t, {'iters': 16, 'rel_true_resid': 1e-11, 'converged': True}) for t, n in s.reqs.items() if n <= 0]
        for t, _ in out:
            del s.reqs[t]
        return out


def _server(serving, fake, budget, max_slots=4):
    return serving.Server(device=0, hbm_budget=budget, max_slots=max_slots, lib=fake)


def _add(srv, name, dims, L5=4):
    srv.add_config(name, dims, None, 1.3, 1.5, 0.5, 0.1, L5)


def test_poisson_arrivals(serving):
    t = serving.poisson_arrivals(20000, 5.0, 8)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 5.0) < 0.15
    assert serving.percentile([1, 2, 3, 4], 50) == 2.5


def test_every_request_completes_in_fifo_order_per_config(serving):
    fake = FakeLib({(2, 2, 2, 2): 1000})
    srv = _server(serving, fake, budget=10 ** 9)
    _add(srv, 'a', (2, 2, 2, 2))
    reqs = [serving.Request('a', 0.03, ('z2', i)) for i in range(10)]
    done = srv.run(reqs)
    assert sorted(r.tag for r in done) == list(range(10))
    # all requests take the same number of chunks: completion follows admission order
    assert [r.tag for r in done] == list(range(10))
    assert all(r.t_admit >= r.t_arrival and r.t_done >= r.t_admit for r in done)
    assert fake.created == [((2, 2, 2, 2), 4)]       # slot count capped by max_slots
    m = serving.Server.metrics(done)
    assert m['requests'] == 10 and m['all_converged'] and m['p99_s'] >= m['p50_s'] >= 0


def test_continuous_batching_admits_into_freed_slots(serving):
    fake = FakeLib({(2, 2, 2, 2): 1000})
    srv = _server(serving, fake, budget=10 ** 9, max_slots=2)
    _add(srv, 'a', (2, 2, 2, 2))
    long_req = serving.Request('a', 0.10, ('z2', 0))       # 10 chunks
    short = [serving.Request('a', 0.02, ('point', 0, 0, (0, 0, 0, 0))) for _ in range(4)]   # 2 chunks each
    done = srv.run([long_req] + short)
    # the short requests pass through the second slot while the long one runs
    assert [r.tag for r in done][-1] == long_req.tag
    assert fake.launches == 10


def test_admission_by_memory_and_no_starvation(serving):
    # each config's session (one slot) fits alone, not both together
    fa, fb = (2, 2, 2, 2), (4, 2, 2, 2)
    field = lambda dims, L5: L5 * int(np.prod(dims)) * 12 * 16
    slot = {fa: 10 ** 6, fb: 10 ** 6}
    fake = FakeLib(slot)
    srv = _server(serving, fake, budget=10 ** 12, max_slots=1)
    _add(srv, 'a', fa)
    _add(srv, 'b', fb)
    gauges = sum(c.gauge_bytes for c in srv.configs.values())
    # room for one session (with its scratch and one solution field) at a time
    srv.budget = gauges + 10 ** 6 + 3 * field(fb, 4) + field(fb, 4) + 10 ** 5
    reqs = [serving.Request('a' if i % 2 == 0 else 'b', 0.03, ('z2', i)) for i in range(8)]
    done = srv.run(reqs)
    assert len(done) == 8
    assert fake.max_live == 1                          # never both sessions at once
    assert len(fake.created) >= 2 and {d for d, _ in fake.created} == {fa, fb}
    assert srv.samples and max(s[3] for s in srv.samples) <= srv.budget


def test_configuration_too_large_for_budget(serving):
    fake = FakeLib({(2, 2, 2, 2): 10 ** 12})
    srv = _server(serving, fake, budget=10 ** 8)
    _add(srv, 'a', (2, 2, 2, 2))
    with pytest.raises(MemoryError):
        srv.run([serving.Request('a', 0.03, ('z2', 1))])


def test_unknown_configuration(serving):
    srv = _server(serving, FakeLib({}), budget=10 ** 8)
    with pytest.raises(KeyError):
        srv.submit(serving.Request('nope', 0.1, ('z2', 1)))
