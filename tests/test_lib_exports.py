"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/sq.h (no compute calls: this runs on CPU-only hosts)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, 'include', 'sq.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    names = re.findall(r'^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*([a-z_0-9]+)\s*\(', src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope='module')
def lib():
    if shutil.which('nvcc') is None and not os.path.exists('/usr/local/cuda/bin/nvcc'):
        pytest.skip('nvcc not available')
    from paper_1411_2223_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ('gauge_load', 'dslash_apply', 'cg_solve', 'serve_submit', 'serve_poll'):
        assert n in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib):
    from paper_1411_2223_gb300 import sq
    assert set(_declared()) == set(sq.SIGNATURES)


def test_host_only_calls_without_gpu(lib):
    from paper_1411_2223_gb300 import sq
    l = sq.load_library()
    assert l.sq_strerror(sq.ERR_NOTFOUND) == b'not found'
    o = sq.CgOpts()
    l.sq_cg_opts_default(ctypes.byref(o))
    assert (o.precision, o.long_recon, o.max_iter, o.block_iters) == (1, 18, 100000, 16)
    assert o.delta < 0  # precision-dependent default
    # argument checks fail before touching a device
    assert l.gauge_load(None, None, None, None, 0, None) == sq.ERR_ARG
    assert l.sq_destroy(None) == sq.ERR_ARG
    assert l.sq_kernel_launches(None) == 0


def test_spin_taste_host_rule_matches_oracle_traces(lib):
    """The library's sign rule for (gamma_S x xi_F) (host code, used to build
    the GPU's operator tables) against the oracle's explicit Dirac-matrix
    traces, for all 256 (S, F)."""
    import numpy as np

    import oracle
    from paper_1411_2223_gb300 import sq as sqmod
    for s in range(16):
        for f in range(16):
            partner, sign = sqmod.spin_taste(s, f)
            m = np.zeros((16, 16))
            m[np.arange(16), partner] = sign
            ref = oracle.spin_taste(s, f)
            assert np.abs(ref.imag).max() < 1e-15
            assert np.array_equal(m, np.rint(ref.real)), (s, f)
    with pytest.raises(sqmod.SqError):
        sqmod.spin_taste(16, 0)
