"""Serving loop: propagator solves as requests, continuously batched on one GPU.

A request asks for the 5D solution of D_MDWF x = b on one of the resident gauge
configurations, for one quark mass and one 4D source (Z2 noise or a point
source), to a fixed tolerance: one propagator column of Sec. VII's
propagators, arriving at a time of its own.

Each configuration has its own library context (its gauge links stay resident
in HBM), its own CUDA stream and, while it has work, one solver session: a
fixed number of slots whose CG state lives on the device.  Requests wait in a
queue and are admitted into free slots between CG chunks; converged slots are
finalised and freed at the next poll.  Each configuration's session is driven
by a host thread of its own on its own stream, so sessions progress at their own
pace and their chunks overlap on the device (the library calls release the
Python interpreter lock).

Admission is by HBM footprint: a session is created only when its device bytes
(as the library reports them), plus the solution fields of its slots, fit in
the budget beside the gauge fields and the other sessions; its slot count is
capped at a fair share of the budget per resident configuration.  When a
configuration cannot get a session, the others stop taking new requests until
one of them is idle and can be released (so no configuration starves).

All arithmetic runs in libmdwf; this module moves requests, allocates device
tensors through PyTorch and keeps the clock.
"""
import collections
import dataclasses
import threading
import time

import numpy as np

from . import mdwf as M


@dataclasses.dataclass
class Request:
    """One solve.  source: ('z2', seed) or ('point', spin, colour, (x, y, z, t))."""
    config: str
    mass: float
    source: tuple
    t_arrival: float = None
    tag: int = -1
    t_admit: float = None
    t_done: float = None
    stats: dict = None
    x: object = None            # device solution (kept only with keep_solutions)

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


class _Config:
    def __init__(self, name, ctx, dims, L5, stream, gauge_bytes):
        self.name, self.ctx, self.dims, self.L5, self.stream = name, ctx, tuple(dims), L5, stream
        self.gauge_bytes = gauge_bytes
        self.session = None
        self.slots = 0
        self.queue = collections.deque()
        self.running = {}
        self.eta = None
        self.src = None

    @property
    def V(self):
        d = self.dims
        return d[0] * d[1] * d[2] * d[3]

    @property
    def shape5(self):
        d = self.dims
        return (self.L5, d[3], d[2], d[1], d[0], 4, 3)

    @property
    def field_bytes(self):
        return self.L5 * self.V * 12 * 16

    @property
    def scratch_bytes(self):
        return self.V * 12 * 16 + self.field_bytes


def poisson_arrivals(n, rate, seed):
    """Arrival times (seconds from 0) of n requests of a Poisson stream of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def percentile(values, q):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return None
    return float(np.percentile(v, q))


class Server:
    """Continuous-batching server over resident gauge configurations (one device)."""

    def __init__(self, device=0, hbm_budget=None, tol=1e-10, precision='half', chunk=16, max_slots=12,
                 keep_solutions=False, opts=None, clock=time.perf_counter, lib=None, priorities=False):
        """lib: the binding module (default: the libmdwf binding); a stand-in with the
        same session functions drives the host logic without a device (tests).
        priorities: rank the configurations' streams by request cost (see _prioritise)."""
        import torch
        self.torch = torch
        self.lib = lib if lib is not None else M
        self.device = int(device)
        self.on_gpu = lib is None
        self.dev = torch.device('cuda', self.device) if self.on_gpu else torch.device('cpu')
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.85 * free)
        self.budget = int(hbm_budget)
        self.tol = float(tol)
        self.precision = M.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.opts = opts if opts is not None else M.mdwf_default_opts(precision=self.precision, chunk=int(chunk))
        self.opts.precision = self.precision
        self.max_slots = int(max_slots)
        self.keep = bool(keep_solutions)
        self.clock = clock
        self.configs = collections.OrderedDict()
        self.next_tag = 0
        self.blocked = None          # name of a configuration waiting for room
        self.samples = []            # (time, queued, running, bytes in use)
        self.done = []
        self.cv = threading.Condition(threading.RLock())
        self.priorities = bool(priorities)

    # --- configurations -------------------------------------------------------
    def add_config(self, name, dims, U, M5, b5, c5, mf, L5, t_antiperiodic=1):
        """Make a gauge configuration resident (links copied to the device now)."""
        L = self.lib
        ctx = L.mdwf_create(dims, self.device)
        L.mdwf_load_gauge(ctx, 0, U, t_antiperiodic)
        L.mdwf_set_action(ctx, 0, M5, b5, c5, mf, L5)
        V = int(np.prod(dims))
        # FP64, padded FP32 and fp16-fragment link copies, and the library's workspace
        # of six FP64 half-lattice fields for the device source construction
        gauge_bytes = V * 4 * (144 + 80 + 256) + 3 * int(L5) * V * 12 * 16
        self.configs[name] = _Config(name, ctx, dims, int(L5), None, gauge_bytes)
        self._prioritise()

    def _prioritise(self):
        """Give every configuration its own stream.  With priorities, the stream
        priority ranks the configuration by the cost of one request (smallest
        lattice first): the device then schedules the blocks of cheap requests
        ahead of queued blocks of expensive ones (shortest job first)."""
        if not self.on_gpu:
            return
        order = sorted(self.configs.values(), key=lambda c: c.field_bytes)
        for rank, c in enumerate(order):
            if c.session is None:
                prio = -(len(order) - 1 - rank) if self.priorities else 0
                c.stream = self.torch.cuda.Stream(self.dev, priority=prio)

    def close(self):
        for c in self.configs.values():
            self._release(c)
            self.lib.mdwf_destroy(c.ctx)
        self.configs.clear()

    # --- memory ---------------------------------------------------------------
    def bytes_in_use(self):
        b = 0
        for c in self.configs.values():
            b += c.gauge_bytes
            if c.session is not None:
                b += self.lib.mdwf_session_bytes(c.ctx, 0, c.slots, self.precision) + c.scratch_bytes
            b += len(c.running) * c.field_bytes
        return b

    def _slot_bytes(self, c, slots):
        return self.lib.mdwf_session_bytes(c.ctx, 0, slots, self.precision) + slots * c.field_bytes + c.scratch_bytes

    def _release(self, c):
        if c.session is not None:
            self.lib.mdwf_session_destroy(c.session)
            c.session = None
            c.slots = 0
            c.eta = c.src = None

    def _open_session(self, c):
        free = self.budget - self.bytes_in_use()
        if free < self._slot_bytes(c, 1):
            # release sessions of other configurations that have nothing in flight
            for o in self.configs.values():
                if o is not c and o.session is not None and not o.running:
                    self._release(o)
            if self.on_gpu:
                self.torch.cuda.empty_cache()
            free = self.budget - self.bytes_in_use()
        # at most a fair share of the budget per resident configuration (at least one slot)
        share = (self.budget - sum(o.gauge_bytes for o in self.configs.values())) // max(1, len(self.configs))
        slots = self.max_slots
        while slots > 1 and self._slot_bytes(c, slots) > min(free, share):
            slots -= 1
        if self._slot_bytes(c, slots) > free:
            slots = 0
        if slots == 0:
            if not any(o.session is not None or o.running for o in self.configs.values() if o is not c):
                raise MemoryError('configuration %r does not fit in the HBM budget (%d bytes)' % (c.name, self.budget))
            return False
        c.session = self.lib.mdwf_session_create(c.ctx, 0, slots, self.tol, opts=self.opts, stream=c.stream)
        c.slots = slots
        c.eta = self.torch.empty((c.dims[3], c.dims[2], c.dims[1], c.dims[0], 4, 3), dtype=self.torch.complex128,
                                 device=self.dev)
        c.src = self.torch.empty(c.shape5, dtype=self.torch.complex128, device=self.dev)
        return True

    # --- requests -------------------------------------------------------------
    def submit(self, req):
        """Queue a request (t_arrival defaults to now).  Returns its tag."""
        if req.config not in self.configs:
            raise KeyError('unknown configuration %r' % (req.config,))
        if req.t_arrival is None:
            req.t_arrival = self.clock()
        req.tag = self.next_tag
        self.next_tag += 1
        self.configs[req.config].queue.append(req)
        return req.tag

    def _source(self, c, req):
        kind = req.source[0]
        L = self.lib
        if kind == 'z2':
            L.mdwf_z2_source_dev(c.ctx, int(req.source[1]), c.eta, stream=c.stream)
        elif kind == 'point':
            _, spin, colour, site = req.source
            x, y, z, t = site
            if self.on_gpu:
                with self.torch.cuda.stream(c.stream):
                    c.eta.zero_()
                    c.eta[t, z, y, x, spin, colour] = 1.0
            else:
                c.eta.zero_()
                c.eta[t, z, y, x, spin, colour] = 1.0
        else:
            raise ValueError('unknown source kind %r' % (kind,))
        L.mdwf_make_source_dev(c.ctx, 0, c.eta, c.src, stream=c.stream)

    def _admit_config(self, c, now):
        """Admit queued requests of configuration c into free slots (lock held)."""
        if not c.queue or (self.blocked is not None and self.blocked != c.name):
            return
        if c.session is None:
            if not self._open_session(c):
                if self.blocked is None:
                    self.blocked = c.name
                return
            if self.blocked == c.name:
                self.blocked = None
        while c.queue and len(c.running) < c.slots:
            if self.bytes_in_use() + c.field_bytes > self.budget:
                break
            req = c.queue.popleft()
            x = self.torch.empty(c.shape5, dtype=self.torch.complex128, device=self.dev)
            self._source(c, req)
            self.lib.mdwf_session_submit(c.session, c.src, req.mass, x, req.tag)
            req.t_admit = now
            req.x = x
            c.running[req.tag] = req

    def _admit(self):
        now = self.clock()
        order = sorted((c for c in self.configs.values() if c.queue), key=lambda c: c.queue[0].t_arrival)
        for c in order:
            self._admit_config(c, now)

    def _collect(self, c, done):
        out = []
        for tag, st in done:
            req = c.running.pop(tag)
            req.t_done = self.clock()
            req.stats = st
            if not self.keep:
                req.x = None
            out.append(req)
        self.done.extend(out)
        self.samples.append((self.clock(), sum(len(o.queue) for o in self.configs.values()),
                             sum(len(o.running) for o in self.configs.values()), self.bytes_in_use()))
        return out

    def step(self):
        """Single-threaded driving: admit what fits, run one CG chunk on every busy
        session, then collect completed requests.  Returns them."""
        with self.cv:
            self._admit()
            busy = [c for c in self.configs.values() if c.running]
        for c in busy:
            self.lib.mdwf_session_launch(c.session)
        out = []
        for c in busy:
            done = self.lib.mdwf_session_poll(c.session)
            with self.cv:
                out.extend(self._collect(c, done))
        with self.cv:
            for c in self.configs.values():
                if c.session is not None and not c.running and self.blocked not in (None, c.name):
                    self._release(c)
        return out

    def _worker(self, c, stop, errors):
        """Drive configuration c's session until stop is set and c has no work."""
        try:
            while True:
                with self.cv:
                    if errors or (stop.is_set() and not c.queue and not c.running):
                        return
                    self._admit_config(c, self.clock())
                    if not c.running:
                        if c.session is not None and self.blocked not in (None, c.name):
                            self._release(c)
                            self.cv.notify_all()
                        self.cv.wait(timeout=0.01)
                        continue
                    sess = c.session
                self.lib.mdwf_session_launch(sess)
                done = self.lib.mdwf_session_poll(sess)
                with self.cv:
                    self._collect(c, done)
                    self.cv.notify_all()
        except BaseException as e:      # reported by run()
            errors.append(e)
            stop.set()
            with self.cv:
                self.cv.notify_all()

    def idle(self):
        return not any(c.queue or c.running for c in self.configs.values())

    def run(self, requests, arrivals=None, deadline=None):
        """Serve `requests` arriving at the given times (seconds after the start;
        None: all at once), one driving thread per configuration.  Returns them
        completed, in completion order."""
        pending = list(requests)
        if arrivals is None:
            arrivals = np.zeros(len(pending))
        order = np.argsort(arrivals, kind='stable')
        pending = [pending[i] for i in order]
        times = [float(arrivals[i]) for i in order]
        n0 = len(self.done)
        stop, errors = threading.Event(), []
        workers = [threading.Thread(target=self._worker, args=(c, stop, errors), daemon=True)
                   for c in self.configs.values()]
        t0 = self.clock()
        for w in workers:
            w.start()
        try:
            for req, t in zip(pending, times):
                while not errors:
                    wait = t - (self.clock() - t0)
                    if wait <= 0:
                        break
                    time.sleep(min(wait, 0.05))
                if errors:
                    break
                with self.cv:
                    req.t_arrival = t0 + t
                    self.submit(req)
                    self.cv.notify_all()
        finally:
            stop.set()
            with self.cv:
                self.cv.notify_all()
            for w in workers:
                left = None if deadline is None else max(0.0, deadline - (self.clock() - t0))
                w.join(left)
        if errors:
            raise errors[0]
        if any(w.is_alive() for w in workers):
            raise TimeoutError('serving run exceeded its deadline')
        return self.done[n0:]

    @staticmethod
    def metrics(reqs):
        """p50/p99 latency, solves/s and solve statistics of completed requests."""
        lat = [r.latency for r in reqs]
        t_first = min(r.t_arrival for r in reqs)
        t_last = max(r.t_done for r in reqs)
        span = t_last - t_first
        return {
            'requests': len(reqs),
            'solves_per_s': len(reqs) / span if span > 0 else None,
            'p50_s': percentile(lat, 50),
            'p99_s': percentile(lat, 99),
            'wait_p50_s': percentile([r.t_admit - r.t_arrival for r in reqs], 50),
            'max_true_resid': max(r.stats['rel_true_resid'] for r in reqs),
            'all_converged': all(r.stats['converged'] for r in reqs),
            'iters_mean': float(np.mean([r.stats['iters'] for r in reqs])),
        }
