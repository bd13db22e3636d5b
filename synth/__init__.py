"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

Holds none of the solver's arithmetic: random SU(3) gauge links, their Wilson
(gradient) flow smoothing (Sec. III of arXiv:1701.07559, t_gf = 1), random
gauge rotations, and spinor sources (random Gaussian fields, point sources,
Z2 noise).  Gauge work runs in the small C library ``gauge_gen.c`` (built on
first use with gcc, OpenMP); spinor fields come from numpy's PCG64 generator,
which is platform independent.

Layouts: gauge U[t, z, y, x, mu, a, b]; 4D spinor [t, z, y, x, spin, colour];
5D spinor [s, t, z, y, x, spin, colour]; all complex128.  dims = (Lx, Ly, Lz, Lt).
"""
import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'gauge_gen.c')
_LIB_PATH = os.path.join(_HERE, 'libsynth.so')
_lib = None
_lock = threading.Lock()

# Streams of the counter-based generator, one per kind of field.
STREAM_LINKS = 1
STREAM_ROTATION = 2


def build(force=False):
    """Compile gauge_gen.c into libsynth.so (no -march flags: same code on x86 and Arm)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + '.%d.tmp' % os.getpid()
        subprocess.check_call(['gcc', '-O2', '-fPIC', '-shared', '-fopenmp', '-ffp-contract=off',
                               '-std=c11', '-D_DEFAULT_SOURCE', '-o', tmp, _SRC, '-lm'])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.synth_random_su3.argtypes = [ctypes.c_long, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_double, ctypes.c_void_p]
            lib.synth_random_su3.restype = None
            lib.synth_wilson_flow.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
            lib.synth_wilson_flow.restype = ctypes.c_int
            lib.synth_plaquette.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_plaquette.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dims_arr(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def random_su3(n, seed, stream, eps):
    """n matrices exp(i eps H), H = sum_a w_a lambda_a / 2 with w_a ~ N(0, 1); shape (n, 3, 3)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    _load().synth_random_su3(n, seed, stream, eps, out.ctypes.data)
    return out


def random_gauge(dims, seed, eps):
    """Unflowed random links U = exp(i eps H), shape [t, z, y, x, mu, 3, 3]."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    return random_su3(4 * V, seed, STREAM_LINKS, eps).reshape(Lt, Lz, Ly, Lx, 4, 3, 3)


def wilson_flow(dims, U, eps, nsteps):
    """Flow U (copied) by nsteps Runge-Kutta steps of size eps; returns the new field."""
    out = np.ascontiguousarray(U, dtype=np.complex128).copy()
    rc = _load().synth_wilson_flow(_dims_arr(dims), out.ctypes.data, eps, nsteps)
    if rc != 0:
        raise MemoryError('wilson_flow: allocation failed')
    return out


def plaquette(dims, U):
    """Average plaquette Re tr P / 3."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    return _load().synth_plaquette(_dims_arr(dims), U.ctypes.data)


def gauge_rotation(dims, seed, eps=1.0):
    """Random SU(3) gauge transformation Omega(x), shape [t, z, y, x, 3, 3]."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    return random_su3(V, seed, STREAM_ROTATION, eps).reshape(Lt, Lz, Ly, Lx, 3, 3)


def _cache_dir():
    d = os.environ.get('MDWF_SYNTH_CACHE', '/tmp/mdwf_synth_cache')
    os.makedirs(d, exist_ok=True)
    return d


def flowed_gauge(dims, seed, eps, flow_t=1.0, flow_eps=0.01, cache=True):
    """Random links exp(i eps H) flowed to time flow_t with step flow_eps (FP64).

    The result is cached on disk (MDWF_SYNTH_CACHE, default /tmp/mdwf_synth_cache)
    keyed by all parameters, since the flow of a large lattice takes seconds.
    """
    nsteps = int(round(flow_t / flow_eps)) if flow_t > 0 else 0
    key = hashlib.sha256(repr((tuple(int(d) for d in dims), int(seed), float(eps), nsteps,
                               float(flow_eps), 'v1')).encode()).hexdigest()[:24]
    path = os.path.join(_cache_dir(), 'gauge_%s.npy' % key) if cache else None
    if path is not None and os.path.exists(path):
        return np.load(path)
    U = random_gauge(dims, seed, eps)
    if nsteps > 0:
        U = wilson_flow(dims, U, flow_eps, nsteps)
    if path is not None:
        tmp = path + '.%d.tmp.npy' % os.getpid()
        np.save(tmp, U)
        os.replace(tmp, path)
    return U


def unit_gauge(dims):
    """Free field: every link the identity."""
    Lx, Ly, Lz, Lt = dims
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_spinor(shape, seed):
    """Complex Gaussian field (re, im ~ N(0, 1/2)) of the given shape."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(tuple(shape) + (2,))
    return (a[..., 0] + 1j * a[..., 1]) * np.sqrt(0.5)


def z2_source_4d(dims, seed):
    """Real Z2 noise (+-1) on every 4D site, spin and colour."""
    Lx, Ly, Lz, Lt = dims
    rng = np.random.default_rng(seed)
    return (2.0 * rng.integers(0, 2, size=(Lt, Lz, Ly, Lx, 4, 3)) - 1.0).astype(np.complex128)


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed, n):
    """First n outputs of SplitMix64 from state `seed` (Steele, Lea and Flood,
    OOPSLA 2014): state += golden-ratio increment, output = mix(state)."""
    with np.errstate(over='ignore'):
        z = np.uint64(seed & (2 ** 64 - 1)) + np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def z2_source_4d_counter(dims, seed):
    """Real Z2 noise (+-1) on every 4D site, spin and colour: element k in
    [t, z, y, x, spin, colour] order takes its sign from the top bit of the k-th
    SplitMix64 output of `seed` (counter based: any element is computable alone)."""
    Lx, Ly, Lz, Lt = dims
    z = splitmix64(seed, Lx * Ly * Lz * Lt * 12)
    sign = 1.0 - 2.0 * (z >> np.uint64(63)).astype(np.float64)
    return sign.reshape(Lt, Lz, Ly, Lx, 4, 3).astype(np.complex128)


def point_source_4d(dims, spin, colour, site=(0, 0, 0, 0)):
    """Unit point source at site = (x, y, z, t)."""
    Lx, Ly, Lz, Lt = dims
    eta = np.zeros((Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    eta[t, z, y, x, spin, colour] = 1.0
    return eta
