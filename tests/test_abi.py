"""The C-ABI library builds, loads and exports every entry point of include/mdwf.h
(no GPU needed: nothing here launches a kernel)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def lib():
    from paper_1701_07559_gb300 import build
    build.build()
    from paper_1701_07559_gb300 import mdwf
    return mdwf


def _declared():
    hdr = open(os.path.join(ROOT, 'include', 'mdwf.h')).read()
    hdr = re.sub(r'/\*.*?\*/', '', hdr, flags=re.S)
    return sorted(set(re.findall(r'\b(mdwf_[a-z0-9_]+)\s*\(', hdr)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ('mdwf_create', 'mdwf_destroy', 'mdwf_load_gauge', 'mdwf_set_action', 'mdwf_apply_dslash',
                     'mdwf_apply_mdwf', 'mdwf_make_source', 'mdwf_solve', 'mdwf_solve_batch',
                     'mdwf_extract_prop4d'):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib._LIB_PATH)
    for name in _declared():
        assert hasattr(so, name), name


def test_binding_covers_every_symbol(lib):
    for name in _declared():
        assert name in lib.EXPORTED or name == 'mdwf_default_opts'
        assert hasattr(lib, name), name


def test_default_opts(lib):
    o = lib.mdwf_default_opts()
    assert o.precision == lib.MDWF_PREC_HALF and o.max_iter == 100000 and o.delta == 0.1 and o.chunk == 16


def test_extract_prop4d_host(lib):
    """q = P_- x_0 + P_+ x_{L5-1} (host code of the library) against the oracle."""
    import synth
    from oracle import mdwf_oracle as O
    dims, L5 = (4, 2, 2, 6), 5
    x = synth.gaussian_spinor((L5, 6, 2, 2, 4, 4, 3), 3)
    q = lib.mdwf_extract_prop4d(x, dims, L5)
    assert np.array_equal(q, O.extract_prop4d(x))


def test_create_rejects_bad_dims(lib):
    with pytest.raises(lib.MdwfError):
        lib.mdwf_create((3, 4, 4, 4), 0)
