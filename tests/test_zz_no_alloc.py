"""mdagm_apply_static: the allocation-free form of the CG operator.

Some callers cannot let the library allocate device memory when they call
it (an application that owns all of HBM through its own memory pool, a
latency-critical loop that cannot take a first-use cudaMalloc), so this
entry point keeps its temporary in a fixed device array.  Through the
C ABI, two calls in a row must reproduce mdagm_apply (same kernels: the
results are compared within the Dslash tolerances and are expected to agree
bit for bit), and a lattice whose temporary does not fit the array must be
refused.  Collected last on purpose; passes alone and after the other tests.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL_DSLASH, gauge, pack, packed_buffer, rel, unpack

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('prec,recon', [('f32', 18), ('f64', 18), ('i16', 12)])
def test_static_matches_mdagm_apply_twice(sq, prec, recon):
    dims = (8, 8, 8, 16)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    gid = sq.gauge_load(dims, fat, lng)
    try:
        for call, seed in enumerate((1, 2)):  # two calls in a row, new input each
            v = synth.gaussian_source(vh, seed)
            src = pack(sq, gid, prec, v)
            ref_buf = packed_buffer(sq, gid, prec)
            sq.mdagm_apply(gid, prec, recon, 0.03, src, ref_buf)
            ref = unpack(sq, gid, prec, ref_buf, vh)
            out_buf = packed_buffer(sq, gid, prec)
            sq.mdagm_apply_static(gid, prec, recon, 0.03, src, out_buf)
            got = unpack(sq, gid, prec, out_buf, vh)
            assert rel(got, ref) <= 2 * TOL_DSLASH[prec], (call, rel(got, ref))
            assert np.array_equal(got, ref)
            # and against the oracle on the unquantised input
            want = oracle.mdagm(dims, fat, lng, 0.03, v)
            assert rel(got, want) <= 2 * TOL_DSLASH[prec]
    finally:
        sq.gauge_free(gid)


def test_static_rejects_too_large_lattice(sq):
    from paper_1411_2223_gb300 import sq as sqm
    # FP64: 48 B per site and parity; 66 x 64 x 64 x 2 has 270336 > 262144 sites
    dims = (66, 64, 64, 2)
    vol = oracle.volume(dims)
    eye = np.eye(3, dtype=np.complex128)
    fat = np.broadcast_to(synth.C1 * eye, (vol, 4, 3, 3)).copy()
    lng = np.broadcast_to(synth.C3 * eye, (vol, 4, 3, 3)).copy()
    gid = sq.gauge_load(dims, fat, lng, flags=sqm.GAUGE_NO_F32 | sqm.GAUGE_NO_I16
                        | sqm.GAUGE_NO_LONG12)
    try:
        nbytes, _ = sq.spinor_bytes(gid, 'f64')
        assert nbytes > sqm.STATIC_SCRATCH_BYTES
        a = packed_buffer(sq, gid, 'f64')
        b = packed_buffer(sq, gid, 'f64')
        with pytest.raises(sqm.SqError) as e:
            sq.mdagm_apply_static(gid, 'f64', 18, 0.1, a, b)
        assert e.value.status == sqm.ERR_ARG
    finally:
        sq.gauge_free(gid)
