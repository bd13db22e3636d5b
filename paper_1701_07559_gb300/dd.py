"""Domain decomposition of the Moebius operator and solve along time.

The lattice Lx x Ly x Lz x Lt is cut along t into P slabs of Lt / P slices
(even, so a site keeps its parity); sub-domain k holds t in [k Lt/P, (k+1) Lt/P)
with every L5 slice and right-hand side of its sites, as the paper's multi-GPU
runs split the lattice (Sec. VII, Table VII: geometries 1.1.1.P and up).  Per hop
every sub-domain packs two faces, 12 reals per (3D site, slice) (the library's
mdwf_dd_pack_faces_dev), they travel to the neighbours' own halo buffers, and
the library applies the sub-domain's operator with them (mdwf_dd_apply_dev).
The global antiperiodic time boundary is a sign on the two faces that cross it
(between the last and the first sub-domain).

The CG on the normal equations runs in the Chronopoulos-Gear form: both
scalars of an iteration, <r, r> and <A r, r>, come from one fused FP64
all-reduce, and each iteration applies the operator once.

Exchanges: LocalExchange for virtual sub-domains held by one process (device
copies), DistExchange for one sub-domain per rank over torch.distributed (NCCL
between GPUs, gloo on the CPU): the sends deliver each face into the receiving
rank's own buffer, in the same order on every rank.
"""
import math

import numpy as np


class TSplit:
    """Geometry of a time split of `dims` = (Lx, Ly, Lz, Lt) into `parts` slabs."""

    def __init__(self, dims, parts, antiperiodic=True):
        dims = tuple(int(d) for d in dims)
        if parts < 1 or dims[3] % parts or (dims[3] // parts) % 2:
            raise ValueError('Lt = %d does not split into %d slabs of an even number of slices' % (dims[3], parts))
        self.dims, self.parts, self.antiperiodic = dims, int(parts), bool(antiperiodic)
        self.lt = dims[3] // parts
        self.local_dims = dims[:3] + (self.lt,)

    def t0(self, k):
        return k * self.lt

    def next(self, k):
        return (k + 1) % self.parts

    def prev(self, k):
        return (k - 1) % self.parts

    def sign_next(self, k):
        """Factor of the face sub-domain k receives from its next neighbour."""
        return -1.0 if (self.antiperiodic and k == self.parts - 1) else 1.0

    def sign_prev(self, k):
        """Factor of the face sub-domain k receives from its previous neighbour."""
        return -1.0 if (self.antiperiodic and k == 0) else 1.0

    def gauge_slab(self, U, k):
        """Links of slab k from a global field [t][z][y][x][mu][3][3]."""
        return np.ascontiguousarray(U[self.t0(k):self.t0(k) + self.lt])

    def field_slab(self, x, k):
        """Slab k of a 5D field [s][t][z][y][x][4][3] (numpy or torch)."""
        return x[:, self.t0(k):self.t0(k) + self.lt].contiguous() if hasattr(x, 'contiguous') \
            else np.ascontiguousarray(x[:, self.t0(k):self.t0(k) + self.lt])

    def assemble(self, slabs):
        """Global 5D field from the slabs (numpy)."""
        return np.concatenate([np.asarray(s) for s in slabs], axis=1)


class LocalExchange:
    """Virtual sub-domains held by one process: every halo is a copy of the
    neighbour's face (device to device)."""

    def __init__(self, split):
        self.split = split

    def __call__(self, ks, faces):
        # faces[i] = (face_prev, face_next) of sub-domain ks[i]; all sub-domains are here
        by_k = dict(zip(ks, faces))
        out = []
        for k in ks:
            out.append((by_k[self.split.next(k)][0].clone(), by_k[self.split.prev(k)][1].clone()))
        return out

    def allreduce(self, partials):
        """Sum of the sub-domains' partial sums, in the order of the sub-domains."""
        tot = np.zeros_like(np.asarray(partials[0], dtype=np.float64))
        for p in partials:
            tot = tot + np.asarray(p, dtype=np.float64)
        return tot


class DistExchange:
    """One sub-domain per rank of a torch.distributed group (NCCL or gloo).  Rank
    k sends face_prev to k - 1 and face_next to k + 1 and receives the matching
    faces into its own halo buffers; the four operations are issued in the same
    order on every rank, so they pair up even when both neighbours are one rank."""

    def __init__(self, split, group=None):
        import torch.distributed as dist
        self.dist, self.split, self.group = dist, split, group
        self.rank = dist.get_rank(group)

    def __call__(self, ks, faces):
        import torch
        assert len(ks) == 1 and ks[0] == self.rank
        k = self.rank
        face_prev, face_next = faces[0]
        halo_next = torch.empty_like(face_prev)
        halo_prev = torch.empty_like(face_next)
        if self.split.parts == 1:
            halo_next.copy_(face_prev)
            halo_prev.copy_(face_next)
            return [(halo_next, halo_prev)]
        d = self.dist
        gp = (lambda r: d.get_global_rank(self.group, r)) if self.group is not None else (lambda r: r)
        nxt, prv = gp(self.split.next(k)), gp(self.split.prev(k))
        real = torch.view_as_real if face_prev.is_complex() else (lambda t: t)
        ops = [d.P2POp(d.isend, real(face_prev), prv, self.group, 0),
               d.P2POp(d.isend, real(face_next), nxt, self.group, 1),
               d.P2POp(d.irecv, real(halo_next), nxt, self.group, 0),
               d.P2POp(d.irecv, real(halo_prev), prv, self.group, 1)]
        for req in d.batch_isend_irecv(ops):
            req.wait()
        return [(halo_next, halo_prev)]

    def allreduce(self, partials):
        """One all-reduce of the local partial sums (a small FP64 vector)."""
        import torch
        dev = 'cuda' if self.dist.get_backend(self.group) == 'nccl' else 'cpu'
        t = torch.tensor(np.asarray(partials[0], dtype=np.float64), dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()


class DDOperator:
    """The operator of the decomposed lattice on the sub-domains this process
    holds.  subdomains: objects with pack(kind, dagger, x) -> (face_prev,
    face_next) and apply(kind, dagger, x, halo_next, halo_prev, sign_next,
    sign_prev) -> out (GPUSubdomain, or a CPU stand-in in the tests);
    kind 0 is the hop H, kind 1 the Moebius operator D."""

    def __init__(self, split, ks, subdomains, exchange):
        self.split, self.ks, self.subs, self.exchange = split, list(ks), list(subdomains), exchange

    def apply(self, kind, dagger, xs):
        faces = [s.pack(kind, dagger, x) for s, x in zip(self.subs, xs)]
        halos = self.exchange(self.ks, faces)
        return [s.apply(kind, dagger, x, hn, hp, self.split.sign_next(k), self.split.sign_prev(k))
                for s, x, (hn, hp), k in zip(self.subs, xs, halos, self.ks)]

    def normal(self, xs):
        """D^+ D x."""
        return self.apply(1, 1, self.apply(1, 0, xs))

    def dots(self, pairs):
        """Fused real parts of <a, b> for each (a_list, b_list) in pairs: one all-reduce."""
        part = np.array([sum(float(_vdot(a, b)) for a, b in zip(al, bl)) for al, bl in pairs], dtype=np.float64)
        return self.exchange.allreduce([part])


def _vdot(a, b):
    if hasattr(a, 'conj'):
        try:
            import torch
            if isinstance(a, torch.Tensor):
                return torch.sum((a.conj() * b).real).item()
        except ImportError:
            pass
    return float(np.real(np.vdot(np.asarray(a), np.asarray(b))))


def fused_cg(op, bs, tol=1e-10, max_iter=100000):
    """CG on the Hermitian positive operator A = op.normal for the right-hand
    sides bs (the local parts), Chronopoulos-Gear form: per iteration one
    application of A and one all-reduce of (<r, r>, <A r, r>).
    Returns (x, iterations, |r| / |b| of the recursion)."""
    xs = [b * 0 for b in bs]
    rs = [b.clone() if hasattr(b, 'clone') else b.copy() for b in bs]
    bnorm = math.sqrt(op.dots([(bs, bs)])[0])
    if bnorm == 0.0:
        return xs, 0, 0.0
    ws = op.normal(rs)
    ps = ss = None
    gamma_old = alpha_old = None
    it = 0
    rel = 1.0
    while it < max_iter:
        gamma, delta = op.dots([(rs, rs), (ws, rs)])
        rel = math.sqrt(max(gamma, 0.0)) / bnorm
        if rel <= tol:
            break
        if ps is None:
            beta, alpha = 0.0, gamma / delta
            ps = [r.clone() if hasattr(r, 'clone') else r.copy() for r in rs]
            ss = [w.clone() if hasattr(w, 'clone') else w.copy() for w in ws]
        else:
            beta = gamma / gamma_old
            alpha = gamma / (delta - beta * gamma / alpha_old)
            ps = [r + beta * p for r, p in zip(rs, ps)]
            ss = [w + beta * s for w, s in zip(ws, ss)]
        xs = [x + alpha * p for x, p in zip(xs, ps)]
        rs = [r - alpha * s for r, s in zip(rs, ss)]
        ws = op.normal(rs)
        gamma_old, alpha_old = gamma, alpha
        it += 1
    return xs, it, rel


def solve(op, bs, tol=1e-10, max_iter=100000, passes=5):
    """D x = b on the decomposed lattice: CG on D^+ D dx = D^+ r for the current
    true residual r = b - D x, repeated until |b - D x| / |b| <= tol (each pass
    asks the normal equations for 0.1 tol / |r| of their right-hand side).
    Returns (x, CG iterations, |b - D x| / |b|)."""
    bnorm = math.sqrt(op.dots([(bs, bs)])[0])
    xs = [b * 0 for b in bs]
    total = 0
    res = 1.0
    for _ in range(passes):
        rs = [b - d for b, d in zip(bs, op.apply(1, 0, xs))]
        res = math.sqrt(op.dots([(rs, rs)])[0]) / bnorm if bnorm > 0 else 0.0
        if res <= tol:
            break
        dx, it, _ = fused_cg(op, op.apply(1, 1, rs), tol=0.1 * tol / res, max_iter=max_iter)
        total += it
        xs = [x + d for x, d in zip(xs, dx)]
    else:
        rs = [b - d for b, d in zip(bs, op.apply(1, 0, xs))]
        res = math.sqrt(op.dots([(rs, rs)])[0]) / bnorm
    return xs, total, res


class GPUSubdomain:
    """A sub-domain on the GPU: a context of the local dims with the slab's links
    and the action; its faces and halos are torch CUDA tensors (FP64)."""

    def __init__(self, M, split, k, U_global, action, device=0, cfg_id=0):
        import torch
        self.M, self.cfg_id = M, cfg_id
        self.ctx = M.mdwf_create(split.local_dims, device)
        M.mdwf_load_gauge(self.ctx, cfg_id, split.gauge_slab(U_global, k), 1)
        M.mdwf_set_action(self.ctx, cfg_id, *action)
        self.fshape = M.dd_face_shape(self.ctx, cfg_id)
        self.device = torch.device('cuda', device)

    def pack(self, kind, dagger, x):
        import torch
        fp = torch.empty(self.fshape, dtype=torch.complex128, device=self.device)
        fn = torch.empty_like(fp)
        self.M.mdwf_dd_pack_faces_dev(self.ctx, self.cfg_id, kind, dagger, x, fp, fn)
        return fp, fn

    def apply(self, kind, dagger, x, halo_next, halo_prev, sign_next, sign_prev):
        import torch
        out = torch.empty_like(x)
        self.M.mdwf_dd_apply_dev(self.ctx, self.cfg_id, kind, dagger, x, out, halo_next, halo_prev,
                                 sign_next, sign_prev)
        return out

    def close(self):
        self.M.mdwf_destroy(self.ctx)
