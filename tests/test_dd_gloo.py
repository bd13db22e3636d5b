"""Host logic of the time-split domain decomposition (paper_1701_07559_gb300/dd.py)
with two gloo ranks on the CPU: slab geometry, the face routing of DistExchange
(both neighbours are one rank when P = 2), the signs of the global antiperiodic
boundary and the CG with one fused all-reduce per iteration.

Each rank's sub-domain operator here is a CPU stand-in written from the oracle:
its faces are the hop input's first slice (for the previous rank) and the last
slice together with its time links (for the next rank); it applies the oracle's
hop to its slab extended by the two received ghost slices, each multiplied by
its boundary sign.  The decomposed operator and solve must equal the oracle on
the whole lattice."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import mdwf_oracle as O
from paper_1701_07559_gb300 import dd

DIMS, L5 = (4, 4, 2, 8), 4
ACT = (1.3, 1.5, 0.5, 0.1)


class CPUSubdomain:
    def __init__(self, split, k, U):
        self.U = split.gauge_slab(U, k)
        self.lt = split.lt

    def _hop_input(self, kind, dagger, x):
        return O.op_B(x, ACT[1], ACT[2], ACT[3]) if (kind == 1 and not dagger) else x

    def pack(self, kind, dagger, x):
        import torch
        h = self._hop_input(kind, dagger, x.numpy())
        prev = np.ascontiguousarray(h[:, 0])
        nxt = np.concatenate([h[:, -1].ravel(), self.U[-1, ..., 3, :, :].ravel()])
        return torch.from_numpy(prev), torch.from_numpy(nxt)

    def apply(self, kind, dagger, x, halo_next, halo_prev, sign_next, sign_prev):
        import torch
        x = x.numpy()
        h = self._hop_input(kind, dagger, x)
        L5_, lt = h.shape[0], h.shape[1]
        ns = h[:, 0].size
        gp = sign_prev * halo_prev.numpy()[:ns].reshape(h[:, 0].shape)
        gn = sign_next * halo_next.numpy().reshape(h[:, 0].shape)
        ext = np.concatenate([gp[:, None], h, gn[:, None]], axis=1)
        eye = np.broadcast_to(np.eye(3, dtype=complex), self.U.shape[1:4] + (4, 3, 3)).copy()
        ghost_links = eye.copy()
        ghost_links[..., 3, :, :] = halo_prev.numpy()[ns:].reshape(self.U.shape[1:4] + (3, 3))
        Uext = np.concatenate([ghost_links[None], self.U, eye[None]], axis=0)
        hop = O.hopping(Uext, ext, antiperiodic_t=False, dagger=bool(dagger))[:, 1:lt + 1]
        if kind == 0:
            out = hop
        elif not dagger:
            out = O.op_A(x, *ACT) - 0.5 * hop
        else:
            out = O.op_A(x, *ACT, dagger=True) - 0.5 * O.op_B(hop, ACT[1], ACT[2], ACT[3], dagger=True)
        return torch.from_numpy(np.ascontiguousarray(out))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        U = synth.random_gauge(DIMS, 5, 0.5)
        split = dd.TSplit(DIMS, world)
        op = dd.DDOperator(split, [rank], [CPUSubdomain(split, rank, U)], dd.DistExchange(split))
        psi = synth.gaussian_spinor((L5,) + tuple(reversed(DIMS)) + (4, 3), 9)
        mine = torch.from_numpy(split.field_slab(psi, rank))
        errs = {}
        for kind, dagger in ((0, 0), (0, 1), (1, 0), (1, 1)):
            got = op.apply(kind, dagger, [mine])[0].numpy()
            want = O.hopping(U, psi, True, bool(dagger)) if kind == 0 else \
                (O.mobius_dag if dagger else O.mobius)(U, psi, *ACT)
            want = split.field_slab(want, rank)
            errs[(kind, dagger)] = float(np.abs(got - want).max() / np.abs(want).max())
        # a solve of D x = b on the decomposed lattice
        b = np.zeros_like(psi)
        b[0, 0, 0, 0, 0, 0, 0] = 1.0
        xs, iters, res = dd.solve(op, [torch.from_numpy(split.field_slab(b, rank))], tol=1e-10)
        ref, _ = O.solve_schur(U, b, *ACT, tol=1e-13)
        ref = split.field_slab(ref, rank)
        xerr = float(np.linalg.norm((xs[0].numpy() - ref).ravel()))
        q.put((rank, errs, iters, res, xerr, float(np.linalg.norm(ref.ravel()))))
    finally:
        dist.destroy_process_group()


def test_tsplit_geometry():
    s = dd.TSplit((4, 4, 4, 16), 4)
    assert s.local_dims == (4, 4, 4, 4) and [s.t0(k) for k in range(4)] == [0, 4, 8, 12]
    assert [s.next(k) for k in range(4)] == [1, 2, 3, 0] and [s.prev(k) for k in range(4)] == [3, 0, 1, 2]
    # the antiperiodic boundary sits between the last slab and the first
    assert [s.sign_next(k) for k in range(4)] == [1, 1, 1, -1]
    assert [s.sign_prev(k) for k in range(4)] == [-1, 1, 1, 1]
    assert dd.TSplit((4, 4, 4, 16), 4, antiperiodic=False).sign_prev(0) == 1
    x = np.arange(2 * 16 * 4 * 4 * 4 * 4 * 3).reshape(2, 16, 4, 4, 4, 4, 3)
    assert np.array_equal(s.assemble([s.field_slab(x, k) for k in range(4)]), x)
    for bad in (3, 16, 0):
        with pytest.raises(ValueError):
            dd.TSplit((4, 4, 4, 16), bad)


def test_two_gloo_ranks_decomposed_operator_and_solve():
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    xerr2 = ref2 = 0.0
    for rank, errs, iters, res, xerr, refn in out:
        for key, e in errs.items():
            assert e <= 1e-13, (rank, key, e)
        assert res <= 1e-10 and iters > 0
        xerr2 += xerr ** 2
        ref2 += refn ** 2
    assert out[0][2] == out[1][2]          # both ranks took the same CG path
    assert np.sqrt(xerr2) <= 1e-8 * np.sqrt(ref2)
