"""Thin ctypes binding of libmdwf (include/mdwf.h), same function names.

Argument marshalling only: every operator and solver step runs in the CUDA
library.  There is no CPU fallback; if libmdwf.so has not been built the
import of this module fails.

Host fields are numpy complex128 arrays in the C ABI's layouts:
  gauge  [t, z, y, x, mu, 3, 3]      4D spinor [t, z, y, x, spin, colour]
  5D spinor [s, t, z, y, x, spin, colour]
Device fields (``*_dev`` functions) are torch CUDA tensors of the same shapes,
dtype complex128 (or float64 with a trailing axis of 2).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, 'libmdwf.so')
if not os.path.exists(_LIB_PATH):
    raise ImportError('libmdwf.so is not built; run paper_1701_07559_gb300.build.build() '
                      '(or __graft_entry__.build()) first')
_lib = ctypes.CDLL(_LIB_PATH)

MDWF_OK = 0
MDWF_ERR_ARG = -1
MDWF_ERR_NOMEM = -2
MDWF_ERR_NONFINITE = -3
MDWF_ERR_NOT_CONVERGED = -4
MDWF_ERR_TIMEOUT = -5
MDWF_ERR_CUDA = -6
MDWF_ERR_STATE = -7
MDWF_ERR_FULL = -8

MDWF_PREC_DOUBLE = 0
MDWF_PREC_SINGLE = 1
MDWF_PREC_HALF = 2
MDWF_PREC_BF16 = 3
PRECISIONS = {'double': 0, 'single': 1, 'half': 2, 'bf16': 3}

_ERRNAMES = {v: k for k, v in globals().items() if k.startswith('MDWF_ERR_')}


class mdwf_solver_opts(ctypes.Structure):
    _fields_ = [('precision', ctypes.c_int), ('max_iter', ctypes.c_int), ('delta', ctypes.c_double),
                ('chunk', ctypes.c_int), ('use_graph', ctypes.c_int), ('nsb', ctypes.c_int),
                ('profile', ctypes.c_int), ('wait_timeout_s', ctypes.c_double), ('timeout_test', ctypes.c_int),
                ('hop_variant', ctypes.c_int), ('schur', ctypes.c_int), ('max_restarts', ctypes.c_int),
                ('stop_scale_test', ctypes.c_double), ('link_recon', ctypes.c_int)]


# the phases of mdwf_solve_stats.phase_ms
PHASES = ('prep', 'cg', 'fp32_update', 'fp64_reref', 'final')


class mdwf_solve_stats(ctypes.Structure):
    _fields_ = [('iters', ctypes.c_int), ('reliable_updates', ctypes.c_int), ('converged', ctypes.c_int),
                ('hop_launches', ctypes.c_int), ('rel_true_resid', ctypes.c_double), ('time_s', ctypes.c_double),
                ('hop_ms', ctypes.c_double), ('kernel_launches', ctypes.c_longlong),
                ('hop_units', ctypes.c_longlong), ('phase_ms', ctypes.c_double * 5),
                ('fp32_updates', ctypes.c_int), ('fp64_rerefs', ctypes.c_int), ('restarts', ctypes.c_int)]

    def as_dict(self):
        return {'iters': self.iters, 'reliable_updates': self.reliable_updates, 'converged': bool(self.converged),
                'rel_true_resid': self.rel_true_resid, 'time_s': self.time_s, 'hop_launches': self.hop_launches,
                'hop_ms': self.hop_ms, 'kernel_launches': self.kernel_launches, 'hop_units': self.hop_units,
                'phase_ms': dict(zip(PHASES, list(self.phase_ms))), 'fp32_updates': self.fp32_updates,
                'fp64_rerefs': self.fp64_rerefs, 'restarts': self.restarts}


class MdwfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s (%d): %s' % (_ERRNAMES.get(code, 'MDWF_ERR'), code, msg))
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_sig = {
    'mdwf_default_opts': (None, [ctypes.POINTER(mdwf_solver_opts)]),
    'mdwf_create': (_I, [ctypes.POINTER(_I), _I, ctypes.POINTER(_P)]),
    'mdwf_destroy': (_I, [_P]),
    'mdwf_last_error': (ctypes.c_char_p, [_P]),
    'mdwf_load_gauge': (_I, [_P, _I, _P, _I]),
    'mdwf_set_action': (_I, [_P, _I, _D, _D, _D, _D, _I]),
    'mdwf_apply_dslash': (_I, [_P, _I, _P, _P, _I, _I]),
    'mdwf_apply_mdwf': (_I, [_P, _I, _P, _P, _I]),
    'mdwf_apply_schur': (_I, [_P, _I, _P, _P, _I, _I]),
    'mdwf_apply_5d': (_I, [_P, _I, _I, _P, _P, _I]),
    'mdwf_make_source': (_I, [_P, _I, _P, _P]),
    'mdwf_solve': (_I, [_P, _I, _P, _P, _D, ctypes.POINTER(mdwf_solver_opts), ctypes.POINTER(mdwf_solve_stats)]),
    'mdwf_solve_batch': (_I, [_P, _I, _I, ctypes.POINTER(_P), _P, ctypes.POINTER(_P), _D,
                              ctypes.POINTER(mdwf_solver_opts), ctypes.POINTER(mdwf_solve_stats)]),
    'mdwf_solve_batch_dev': (_I, [_P, _I, _I, ctypes.POINTER(_P), _P, ctypes.POINTER(_P), _D,
                                  ctypes.POINTER(mdwf_solver_opts), ctypes.POINTER(mdwf_solve_stats), _P]),
    'mdwf_apply_schur_batch_dev': (_I, [_P, _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _I, _I, _I, _P]),
    'mdwf_apply_schur_batch_dev_noalloc': (_I, [_P, _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _I, _I, _P]),
    'mdwf_apply_dslash_dev': (_I, [_P, _I, _P, _P, _I, _I, _P]),
    'mdwf_apply_mdwf_dev': (_I, [_P, _I, _P, _P, _I, _P]),
    'mdwf_dd_pack_faces_dev': (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    'mdwf_dd_apply_dev': (_I, [_P, _I, _I, _I, _P, _P, _P, _P, _D, _D, _P]),
    'mdwf_extract_prop4d': (_I, [_P, ctypes.POINTER(_I), _I, _P]),
    'mdwf_session_bytes': (ctypes.c_longlong, [_P, _I, _I, _I]),
    'mdwf_session_create': (_I, [_P, _I, _I, ctypes.POINTER(mdwf_solver_opts), _D, _P, ctypes.POINTER(_P)]),
    'mdwf_session_destroy': (_I, [_P]),
    'mdwf_session_submit': (_I, [_P, _P, _D, _P, ctypes.c_longlong, ctypes.POINTER(_I)]),
    'mdwf_session_launch': (_I, [_P, _I]),
    'mdwf_session_poll': (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(mdwf_solve_stats),
                               ctypes.POINTER(_I)]),
    'mdwf_session_occupied': (_I, [_P]),
    'mdwf_make_source_dev': (_I, [_P, _I, _P, _P, _P]),
    'mdwf_z2_source_dev': (_I, [_P, ctypes.c_ulonglong, _P, _P]),
    'mdwf_wilson_flow_dev': (_I, [_P, _P, _D, _I, _P]),
    'mdwf_plaquette_dev': (_I, [_P, _P, ctypes.POINTER(_D)]),
    'mdwf_smear_source_dev': (_I, [_P, _I, _P, _D, _I, _P]),
    'mdwf_mres_correlators_dev': (_I, [_P, _I, _I, ctypes.POINTER(_P), _P, _P, _P]),
    'mdwf_autotune': (_I, [_P, _I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class Context:
    """Opaque handle of an mdwf_ctx (one lattice geometry on one device)."""

    def __init__(self, handle, dims):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.L5 = {}

    @property
    def V(self):
        d = self.dims
        return d[0] * d[1] * d[2] * d[3]


def _check(ctx, rc):
    if rc != MDWF_OK:
        msg = _lib.mdwf_last_error(ctx.handle if ctx is not None else None)
        raise MdwfError(rc, msg.decode() if msg else '')


def _host(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != tuple(shape):
        raise ValueError('expected shape %s, got %s' % (tuple(shape), a.shape))
    return a


def _shape5(ctx, cfg_id):
    d = ctx.dims
    if cfg_id not in ctx.L5:
        raise MdwfError(MDWF_ERR_STATE, 'no action set for cfg_id %r' % (cfg_id,))
    return (ctx.L5[cfg_id], d[3], d[2], d[1], d[0], 4, 3)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def mdwf_default_opts(**over):
    o = mdwf_solver_opts()
    _lib.mdwf_default_opts(ctypes.byref(o))
    for k, v in over.items():
        if k == 'precision' and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


def mdwf_create(dims, device=0):
    d = (_I * 4)(*[int(x) for x in dims])
    h = _P()
    rc = _lib.mdwf_create(d, int(device), ctypes.byref(h))
    if rc != MDWF_OK:
        raise MdwfError(rc, 'mdwf_create failed (dims must be even and >= 2; device must exist)')
    return Context(h, dims)


def mdwf_destroy(ctx):
    if ctx is not None and ctx.handle:
        _lib.mdwf_destroy(ctx.handle)
        ctx.handle = None


def mdwf_last_error(ctx):
    return _lib.mdwf_last_error(ctx.handle).decode()


def mdwf_load_gauge(ctx, cfg_id, U, t_antiperiodic=1):
    d = ctx.dims
    U = _host(U, (d[3], d[2], d[1], d[0], 4, 3, 3))
    _check(ctx, _lib.mdwf_load_gauge(ctx.handle, int(cfg_id), _ptr(U), int(t_antiperiodic)))


def mdwf_set_action(ctx, cfg_id, M5, b5, c5, mf, L5):
    _check(ctx, _lib.mdwf_set_action(ctx.handle, int(cfg_id), float(M5), float(b5), float(c5), float(mf), int(L5)))
    ctx.L5[cfg_id] = int(L5)


def mdwf_apply_dslash(ctx, cfg_id, psi, out_parity=-1, dagger=0):
    shape = _shape5(ctx, cfg_id)
    psi = _host(psi, shape)
    out = np.empty(shape, dtype=np.complex128)
    _check(ctx, _lib.mdwf_apply_dslash(ctx.handle, int(cfg_id), _ptr(psi), _ptr(out), int(out_parity), int(dagger)))
    return out


def mdwf_apply_mdwf(ctx, cfg_id, psi, dagger=0):
    shape = _shape5(ctx, cfg_id)
    psi = _host(psi, shape)
    out = np.empty(shape, dtype=np.complex128)
    _check(ctx, _lib.mdwf_apply_mdwf(ctx.handle, int(cfg_id), _ptr(psi), _ptr(out), int(dagger)))
    return out


def mdwf_apply_schur(ctx, cfg_id, psi, dagger=0, precision=MDWF_PREC_DOUBLE):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    shape = _shape5(ctx, cfg_id)
    psi = _host(psi, shape)
    out = np.empty(shape, dtype=np.complex128)
    _check(ctx, _lib.mdwf_apply_schur(ctx.handle, int(cfg_id), _ptr(psi), _ptr(out), int(dagger), int(precision)))
    return out


def mdwf_apply_5d(ctx, cfg_id, op, psi, dagger=0):
    """op: 0 = A, 1 = B, 2 = A^-1 (or 'A', 'B', 'Ainv')."""
    if isinstance(op, str):
        op = {'A': 0, 'B': 1, 'Ainv': 2}[op]
    shape = _shape5(ctx, cfg_id)
    psi = _host(psi, shape)
    out = np.empty(shape, dtype=np.complex128)
    _check(ctx, _lib.mdwf_apply_5d(ctx.handle, int(cfg_id), int(op), _ptr(psi), _ptr(out), int(dagger)))
    return out


def mdwf_make_source(ctx, cfg_id, eta):
    d = ctx.dims
    eta = _host(eta, (d[3], d[2], d[1], d[0], 4, 3))
    out = np.empty(_shape5(ctx, cfg_id), dtype=np.complex128)
    _check(ctx, _lib.mdwf_make_source(ctx.handle, int(cfg_id), _ptr(eta), _ptr(out)))
    return out


def mdwf_solve(ctx, cfg_id, src, tol, opts=None):
    """Returns (x, stats dict).  Raises MdwfError on failure (including not converged)."""
    shape = _shape5(ctx, cfg_id)
    src = _host(src, shape)
    x = np.empty(shape, dtype=np.complex128)
    st = mdwf_solve_stats()
    o = opts if opts is not None else mdwf_default_opts()
    _check(ctx, _lib.mdwf_solve(ctx.handle, int(cfg_id), _ptr(src), _ptr(x), float(tol), ctypes.byref(o),
                                ctypes.byref(st)))
    return x, st.as_dict()


def mdwf_solve_batch(ctx, cfg_id, srcs, tol, masses=None, opts=None, raise_on_nonconv=True, out=None):
    """Solve len(srcs) systems in one batch.  Returns (list of x, list of stats dicts).

    ``out``: optional list of preallocated contiguous complex128 host arrays (for
    example views of pinned memory) that receive the solutions."""
    shape = _shape5(ctx, cfg_id)
    n = len(srcs)
    hs = [_host(s, shape) for s in srcs]
    if out is not None:
        xs = list(out)
        if len(xs) != n:
            raise ValueError('mdwf_solve_batch: %d sources but %d output arrays' % (n, len(xs)))
        for x in xs:
            if x.dtype != np.complex128 or x.shape != shape or not x.flags['C_CONTIGUOUS']:
                raise ValueError('out arrays must be contiguous complex128 of shape %s' % (shape,))
    else:
        xs = [np.empty(shape, dtype=np.complex128) for _ in range(n)]
    sp = (_P * n)(*[s.ctypes.data for s in hs])
    xp = (_P * n)(*[x.ctypes.data for x in xs])
    m = None
    if masses is not None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
        if m.shape != (n,):
            raise ValueError('masses must have one entry per source')
    st = (mdwf_solve_stats * n)()
    o = opts if opts is not None else mdwf_default_opts()
    rc = _lib.mdwf_solve_batch(ctx.handle, int(cfg_id), n, sp, _ptr(m) if m is not None else None, xp, float(tol),
                               ctypes.byref(o), st)
    if rc != MDWF_OK and (raise_on_nonconv or rc != MDWF_ERR_NOT_CONVERGED):
        _check(ctx, rc)
    return xs, [s.as_dict() for s in st]


def _dev_ptr(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError('expected a contiguous CUDA tensor')
    if t.dtype == torch.complex128:
        ok = tuple(t.shape) == tuple(shape)
    elif t.dtype == torch.float64:
        ok = tuple(t.shape) == tuple(shape) + (2,)
    else:
        ok = False
    if not ok:
        raise ValueError('expected complex128 %s (or float64 with a trailing 2), got %s %s'
                         % (tuple(shape), t.dtype, tuple(t.shape)))
    return t.data_ptr()


def mdwf_solve_batch_dev(ctx, cfg_id, srcs, xs, tol, masses=None, opts=None, stream=None, raise_on_nonconv=True):
    """Batched solve on torch CUDA tensors (srcs read, xs written).  stream: torch.cuda.Stream or None."""
    shape = _shape5(ctx, cfg_id)
    n = len(srcs)
    if len(xs) != n:
        raise ValueError('mdwf_solve_batch_dev: %d sources but %d solutions' % (n, len(xs)))
    sp = (_P * n)(*[_dev_ptr(s, shape) for s in srcs])
    xp = (_P * n)(*[_dev_ptr(x, shape) for x in xs])
    m = None
    if masses is not None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
        if m.shape != (n,):
            raise ValueError('mdwf_solve_batch_dev: masses must have one entry per source')
    st = (mdwf_solve_stats * n)()
    o = opts if opts is not None else mdwf_default_opts()
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = _lib.mdwf_solve_batch_dev(ctx.handle, int(cfg_id), n, sp, _ptr(m) if m is not None else None, xp,
                                   float(tol), ctypes.byref(o), st, sh)
    if rc != MDWF_OK and (raise_on_nonconv or rc != MDWF_ERR_NOT_CONVERGED):
        _check(ctx, rc)
    return [s.as_dict() for s in st]


HOP_AUTO, HOP_DIRECT, HOP_STAGED, HOP_MMA, HOP_TUNE_ALL, HOP_MMA_PIPE, HOP_UNIT, HOP_PAIR_PF = 0, 1, 2, 3, 4, 5, 6, 7


def mdwf_apply_schur_batch_dev(ctx, cfg_id, ins, outs, masses=None, dagger=0, precision=MDWF_PREC_HALF,
                               hop_variant=HOP_AUTO, stream=None):
    """Batched Schur operator (the solver's hot kernels) on torch CUDA tensors."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    shape = _shape5(ctx, cfg_id)
    n = len(ins)
    if len(outs) != n:
        raise ValueError('mdwf_apply_schur_batch_dev: %d inputs but %d outputs' % (n, len(outs)))
    if masses is not None and len(masses) != n:
        raise ValueError('mdwf_apply_schur_batch_dev: %d inputs but %d masses' % (n, len(masses)))
    ip = (_P * n)(*[_dev_ptr(t, shape) for t in ins])
    op = (_P * n)(*[_dev_ptr(t, shape) for t in outs])
    m = None
    if masses is not None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_apply_schur_batch_dev(ctx.handle, int(cfg_id), n, ip, op, _ptr(m) if m is not None else None,
                                                int(dagger), int(precision), int(hop_variant), sh))


MDWF_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


def mdwf_apply_schur_batch_dev_noalloc(ctx, cfg_id, ins, outs, masses=None, dagger=0, precision=MDWF_PREC_HALF,
                                       stream=None):
    """The batched Schur operator without any device allocation (scratch in a fixed
    library array of MDWF_NOALLOC_SCRATCH_BYTES; see include/mdwf.h for the limit and
    the rule that overlapping calls race)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    shape = _shape5(ctx, cfg_id)
    n = len(ins)
    if len(outs) != n:
        raise ValueError('mdwf_apply_schur_batch_dev_noalloc: %d inputs but %d outputs' % (n, len(outs)))
    if masses is not None and len(masses) != n:
        raise ValueError('mdwf_apply_schur_batch_dev_noalloc: %d inputs but %d masses' % (n, len(masses)))
    ip = (_P * n)(*[_dev_ptr(t, shape) for t in ins])
    op = (_P * n)(*[_dev_ptr(t, shape) for t in outs])
    m = None
    if masses is not None:
        m = np.ascontiguousarray(masses, dtype=np.float64)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_apply_schur_batch_dev_noalloc(ctx.handle, int(cfg_id), n, ip, op,
                                                        _ptr(m) if m is not None else None, int(dagger),
                                                        int(precision), sh))


def mdwf_apply_dslash_dev(ctx, cfg_id, psi, out, out_parity=-1, dagger=0, stream=None):
    shape = _shape5(ctx, cfg_id)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_apply_dslash_dev(ctx.handle, int(cfg_id), _dev_ptr(psi, shape), _dev_ptr(out, shape),
                                           int(out_parity), int(dagger), sh))


def mdwf_apply_mdwf_dev(ctx, cfg_id, psi, out, dagger=0, stream=None):
    shape = _shape5(ctx, cfg_id)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_apply_mdwf_dev(ctx.handle, int(cfg_id), _dev_ptr(psi, shape), _dev_ptr(out, shape),
                                         int(dagger), sh))


def dd_face_shape(ctx, cfg_id):
    """Shape of one time face of a sub-domain: (Lz, Ly, Lx, L5, 2 spins, 3 colours), complex."""
    L5 = _shape5(ctx, cfg_id)[0]
    Lx, Ly, Lz, _ = ctx.dims
    return (Lz, Ly, Lx, L5, 2, 3)


def mdwf_dd_pack_faces_dev(ctx, cfg_id, kind, dagger, psi, face_prev, face_next, stream=None):
    """Faces of a time-split sub-domain (see include/mdwf.h); torch CUDA tensors."""
    shape = _shape5(ctx, cfg_id)
    fs = dd_face_shape(ctx, cfg_id)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_dd_pack_faces_dev(ctx.handle, int(cfg_id), int(kind), int(dagger), _dev_ptr(psi, shape),
                                            _dev_ptr(face_prev, fs), _dev_ptr(face_next, fs), sh))


def mdwf_dd_apply_dev(ctx, cfg_id, kind, dagger, psi, out, halo_next, halo_prev, sign_next=1.0, sign_prev=1.0,
                      stream=None):
    """The operator of a time-split sub-domain with its halos (see include/mdwf.h)."""
    shape = _shape5(ctx, cfg_id)
    fs = dd_face_shape(ctx, cfg_id)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_dd_apply_dev(ctx.handle, int(cfg_id), int(kind), int(dagger), _dev_ptr(psi, shape),
                                       _dev_ptr(out, shape), _dev_ptr(halo_next, fs), _dev_ptr(halo_prev, fs),
                                       float(sign_next), float(sign_prev), sh))


def mdwf_extract_prop4d(x5d, dims, L5):
    Lx, Ly, Lz, Lt = dims
    x5d = _host(x5d, (L5, Lt, Lz, Ly, Lx, 4, 3))
    q = np.empty((Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    d = (_I * 4)(*[int(v) for v in dims])
    rc = _lib.mdwf_extract_prop4d(_ptr(x5d), d, int(L5), _ptr(q))
    if rc != MDWF_OK:
        raise MdwfError(rc, 'mdwf_extract_prop4d: bad arguments')
    return q


def mdwf_make_source_dev(ctx, cfg_id, eta, out, stream=None):
    """5D domain-wall source from a 4D source, on torch CUDA tensors."""
    d = ctx.dims
    shape4 = (d[3], d[2], d[1], d[0], 4, 3)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_make_source_dev(ctx.handle, int(cfg_id), _dev_ptr(eta, shape4),
                                          _dev_ptr(out, _shape5(ctx, cfg_id)), sh))


def _gauge_dev(ctx, U):
    d = ctx.dims
    return _dev_ptr(U, (d[3], d[2], d[1], d[0], 4, 3, 3))


def mdwf_wilson_flow_dev(ctx, U, eps, nsteps, stream=None):
    """Wilson flow (Luscher RK3, FP64) of a device gauge field (torch complex128
    [t, z, y, x, mu, 3, 3]) in place: nsteps steps of size eps."""
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_wilson_flow_dev(ctx.handle, _gauge_dev(ctx, U), float(eps), int(nsteps), sh))


def mdwf_plaquette_dev(ctx, U):
    p = _D()
    _check(ctx, _lib.mdwf_plaquette_dev(ctx.handle, _gauge_dev(ctx, U), ctypes.byref(p)))
    return p.value


def flowed_gauge_dev(ctx, U_host, flow_t=1.0, flow_eps=0.01):
    """Flow a host gauge field on the device to flow time flow_t; returns the host
    result (numpy complex128, the layout mdwf_load_gauge takes)."""
    import torch
    U = torch.from_numpy(np.ascontiguousarray(U_host, dtype=np.complex128)).to('cuda')
    mdwf_wilson_flow_dev(ctx, U, flow_eps, int(round(flow_t / flow_eps)))
    return U.cpu().numpy()


def mdwf_smear_source_dev(ctx, cfg_id, eta, sigma, n_iter, stream=None):
    """Gauge-covariant Gaussian smearing of a 4D source (torch CUDA tensor) in place."""
    d = ctx.dims
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_smear_source_dev(ctx.handle, int(cfg_id), _dev_ptr(eta, (d[3], d[2], d[1], d[0], 4, 3)),
                                           float(sigma), int(n_iter), sh))


def mdwf_mres_correlators_dev(ctx, cfg_id, xs, stream=None):
    """Residual-mass correlators of the solutions xs (torch CUDA 5D fields):
    returns (c_pp, c_j5q) as numpy arrays over the time slices."""
    shape = _shape5(ctx, cfg_id)
    n = len(xs)
    xp = (_P * n)(*[_dev_ptr(x, shape) for x in xs])
    Lt = ctx.dims[3]
    pp = np.empty(Lt)
    j5 = np.empty(Lt)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_mres_correlators_dev(ctx.handle, int(cfg_id), n, xp, _ptr(pp), _ptr(j5), sh))
    return pp, j5


def mdwf_autotune(ctx, cfg_id, n, precision=MDWF_PREC_HALF, include_tensor_core=False):
    """The inner hop form the solver picks for n right-hand sides: returns
    {'hop_variant', 'nsb', 'ms_per_pair'} (ms for one Mhat + Mhat^+ application)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    v, nsb, ms = _I(), _I(), _D()
    _check(ctx, _lib.mdwf_autotune(ctx.handle, int(cfg_id), int(n), int(precision), int(bool(include_tensor_core)),
                                   ctypes.byref(v), ctypes.byref(nsb), ctypes.byref(ms)))
    return {'hop_variant': v.value, 'nsb': nsb.value, 'ms_per_pair': ms.value}


def mdwf_z2_source_dev(ctx, seed, eta, stream=None):
    """Z2 noise 4D source (counter-based SplitMix64 of seed) into a torch CUDA tensor."""
    d = ctx.dims
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_z2_source_dev(ctx.handle, ctypes.c_ulonglong(int(seed) & (2 ** 64 - 1)),
                                        _dev_ptr(eta, (d[3], d[2], d[1], d[0], 4, 3)), sh))


class Session:
    """Opaque handle of an mdwf_session (continuous batching of solves on one config)."""

    def __init__(self, ctx, cfg_id, handle, slots):
        self.ctx, self.cfg_id, self.handle, self.slots = ctx, cfg_id, handle, slots
        self.keep = {}      # tag -> output tensor, kept alive until the request completes


def mdwf_session_bytes(ctx, cfg_id, slots, precision=MDWF_PREC_HALF):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return int(_lib.mdwf_session_bytes(ctx.handle, int(cfg_id), int(slots), int(precision)))


def mdwf_session_create(ctx, cfg_id, slots, tol, opts=None, stream=None):
    o = opts if opts is not None else mdwf_default_opts()
    h = _P()
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(ctx, _lib.mdwf_session_create(ctx.handle, int(cfg_id), int(slots), ctypes.byref(o), float(tol), sh,
                                         ctypes.byref(h)))
    return Session(ctx, cfg_id, h, int(slots))


def mdwf_session_destroy(sess):
    if sess is not None and sess.handle:
        _lib.mdwf_session_destroy(sess.handle)
        sess.handle = None
        sess.keep.clear()


def mdwf_session_submit(sess, src, mass, x, tag):
    """Put a request (device source src, mass, device output x, integer tag) into a
    free slot; returns the slot.  Raises MdwfError(MDWF_ERR_FULL) when none is free."""
    shape = _shape5(sess.ctx, sess.cfg_id)
    slot = _I(-1)
    _check(sess.ctx, _lib.mdwf_session_submit(sess.handle, _dev_ptr(src, shape), float(mass), _dev_ptr(x, shape),
                                              int(tag), ctypes.byref(slot)))
    sess.keep[int(tag)] = x
    return slot.value


def mdwf_session_launch(sess, iters=0):
    _check(sess.ctx, _lib.mdwf_session_launch(sess.handle, int(iters)))


def mdwf_session_poll(sess, max_done=None):
    """Returns [(tag, stats dict), ...] of the requests completed by this call."""
    n = sess.slots if max_done is None else int(max_done)
    tags = (ctypes.c_longlong * max(n, 1))()
    st = (mdwf_solve_stats * max(n, 1))()
    nd = _I(0)
    _check(sess.ctx, _lib.mdwf_session_poll(sess.handle, n, tags, st, ctypes.byref(nd)))
    out = []
    for i in range(nd.value):
        sess.keep.pop(int(tags[i]), None)
        out.append((int(tags[i]), st[i].as_dict()))
    return out


def mdwf_session_occupied(sess):
    return int(_lib.mdwf_session_occupied(sess.handle))
