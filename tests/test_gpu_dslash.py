"""GPU Dslash and CG operator vs the FP64 oracle, element by element.

Relative 2-norm tolerances: 1e-13 (FP64), 1e-5 (FP32), 5e-3 (16-bit storage
with per-site norms, FP32 accumulation).  The oracle always sees the
unquantised FP64 fields.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL_DSLASH, gauge, gpu_dslash, gpu_mdagm, pack, rel, site_rel, unpack

pytestmark = pytest.mark.gpu

SMALL = [(4, 4, 4, 4), (4, 6, 8, 10), (8, 8, 8, 8), (2, 4, 2, 6), (6, 4, 4, 4)]


@pytest.mark.parametrize('dims', SMALL)
@pytest.mark.parametrize('prec', ['f64', 'f32', 'i16'])
@pytest.mark.parametrize('recon', [18, 12])
def test_dslash_matches_oracle(sq, dims, prec, recon):
    fat, lng = gauge(dims)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        vh = oracle.volume(dims) // 2
        for out_parity in (0, 1):
            v = synth.gaussian_source(vh, 11 + out_parity)
            got = gpu_dslash(sq, gid, prec, recon, v, out_parity, vh)
            want = oracle.dslash_half(dims, fat, lng, v, out_parity)
            assert rel(got, want) <= TOL_DSLASH[prec], (prec, recon, out_parity, rel(got, want))
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f64', 'f32', 'i16'])
def test_dslash_antiperiodic_t(sq, prec):
    dims = (4, 4, 6, 8)
    fat, lng = gauge(dims)
    gid = sq.gauge_load(dims, fat, lng, antiperiodic_t=True)
    try:
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 3)
        got = gpu_dslash(sq, gid, prec, 18, v, 1, vh)
        want = oracle.dslash_half(dims, fat, lng, v, 1, t_sign=-1)
        assert rel(got, want) <= TOL_DSLASH[prec]
        # and it differs from the periodic operator
        assert rel(oracle.dslash_half(dims, fat, lng, v, 1), want) > 1e-2
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f64', 'f32', 'i16'])
@pytest.mark.parametrize('recon', [18, 12])
def test_mdagm_matches_oracle(sq, prec, recon):
    dims = (4, 6, 4, 8)
    fat, lng = gauge(dims)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 5)
        got = gpu_mdagm(sq, gid, prec, recon, 0.05, v, vh)
        want = oracle.mdagm(dims, fat, lng, 0.05, v)
        # A = m^2 - D_eo D_oe has two Dslash roundings
        assert rel(got, want) <= 2 * TOL_DSLASH[prec]
    finally:
        sq.gauge_free(gid)


def test_free_field_plane_wave_eigenvector(sq):
    """Unit links: an even-site plane wave is an eigenvector of A on the GPU."""
    dims = (8, 4, 4, 8)
    vol = oracle.volume(dims)
    u = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 4, 3, 3)).copy()
    fat, lng = synth.fat_long_links(u, dims)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        lex = oracle.half_sites(dims, 0)
        lx, ly, lz, lt = dims
        c = np.stack([lex % lx, (lex // lx) % ly, (lex // (lx * ly)) % lz,
                      lex // (lx * ly * lz)], 1)
        p = 2 * np.pi * np.array([1, 1, 0, 3]) / np.array(dims)
        pw = np.exp(1j * c @ p)[:, None] * np.array([1.0, 0.5j, -0.25])[None, :]
        s = sum((synth.C1 * np.sin(q) + synth.C3 * np.sin(3 * q)) ** 2 for q in p)
        got = gpu_mdagm(sq, gid, 'f64', 18, 0.05, pw, vol // 2)
        assert rel(got, (0.05 ** 2 + s) * pw) <= 1e-13
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f64', 'f32', 'i16'])
def test_pack_roundtrip(sq, prec):
    dims = (4, 6, 8, 10)
    fat, lng = gauge(dims)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 8)
        v[7] = 0  # a zero site
        back = unpack(sq, gid, prec, pack(sq, gid, prec, v), vh)
        if prec == 'f64':
            assert np.array_equal(back, v)
        elif prec == 'f32':
            assert np.array_equal(back, v.astype(np.complex64).astype(np.complex128))
        else:
            re = np.stack([v.real, v.imag], -1).reshape(vh, 6)
            bk = np.stack([back.real, back.imag], -1).reshape(vh, 6)
            n = np.abs(re).max(axis=1, keepdims=True)
            assert np.all(np.abs(bk - re) <= n / 65534 * (1 + 1e-4) + 1e-7 * np.abs(re))
            assert np.all(back[7] == 0)
    finally:
        sq.gauge_free(gid)


def test_i16_codes_bit_exact(sq):
    """The GPU's 16-bit spinor codes equal the oracle's, bit for bit."""
    import torch
    dims = (4, 6, 8, 10)
    fat, lng = gauge(dims)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 21) * np.exp(np.random.default_rng(1).uniform(-8, 8, (vh, 1)))
        v[3] = [1.0 + 0.5j, -1.0j, 0.25 - 0.5j]   # ties to even
        v[4] = 0
        buf = pack(sq, gid, 'i16', v)
        torch.cuda.synchronize()
        raw = buf.cpu().numpy()[: vh * 16].view(np.uint32).reshape(vh, 4)
        words = raw[:, :3]
        lo = (words & 0xFFFF).astype(np.int64) - 32768
        hi = (words >> 16).astype(np.int64) - 32768
        codes = np.stack([lo, hi], -1).reshape(vh, 6)
        norms = raw[:, 3].view(np.float32)
        q, n = oracle.quantize_spinor_i16(v)
        assert np.array_equal(codes, q.astype(np.int64))
        assert np.array_equal(norms, n)
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f64', 'f32', 'i16'])
def test_dslash_full_size_20x64(sq, prec):
    """The benchmark lattice 20^3 x 64 at full size, both link formats."""
    dims = (20, 20, 20, 64)
    fat, lng = gauge(dims, eps=0.25, seed=0)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 0)
        want = oracle.dslash_half(dims, fat, lng, v, 1)
        for recon in (18, 12):
            got = gpu_dslash(sq, gid, prec, recon, v, 1, vh)
            assert rel(got, want) <= TOL_DSLASH[prec], (recon, rel(got, want))
            # and site by site: one wrong site among the 256000 fails this
            assert site_rel(got, want) <= TOL_DSLASH[prec], (recon, site_rel(got, want))
    finally:
        sq.gauge_free(gid)


def test_gauge_load_rejects_bad_input(sq):
    from paper_1411_2223_gb300 import sq as sqm
    dims = (4, 4, 4, 4)
    fat, lng = gauge(dims)
    with pytest.raises(sqm.SqError) as e:
        sq.gauge_load((4, 4, 3, 4), fat, lng)
    assert e.value.status == sqm.ERR_ARG
    bad = fat.copy()
    bad[5, 1, 0, 0] = np.nan
    with pytest.raises(sqm.SqError) as e:
        sq.gauge_load(dims, bad, lng)
    assert e.value.status == sqm.ERR_NONFINITE
    # long links that are not c * SU(3): the 12-real form is refused
    gid = sq.gauge_load(dims, fat, fat)
    try:
        with pytest.raises(sqm.SqError) as e:
            gpu_dslash(sq, gid, 'f32', 12, synth.gaussian_source(128, 0), 0, 128)
        assert e.value.status == sqm.ERR_UNSUPPORTED
    finally:
        sq.gauge_free(gid)


def test_null_stream_is_the_legacy_default_stream(sq):
    """The asynchronous calls run on the stream they are given, and NULL is
    the legacy default stream (torch's default stream).  Work queued before
    them -- here the copy of the input, held back by a spin of about 50 ms
    on the GPU -- is therefore done before they read, on the default stream
    and on a torch side stream alike."""
    import contextlib
    import torch
    dims = (8, 8, 8, 8)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    v = synth.gaussian_source(vh, 3)
    want = oracle.dslash_half(dims, fat, lng, v, 1)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        src = pack(sq, gid, 'f32', v)
        torch.cuda.synchronize()
        for side in (False, True):
            stream = torch.cuda.Stream() if side else None
            with torch.cuda.stream(stream) if side else contextlib.nullcontext():
                inp = torch.zeros_like(src)
                out = torch.zeros_like(src)
                canon = torch.zeros((vh, 3), dtype=torch.complex128, device='cuda')
                torch.cuda._sleep(100_000_000)
                inp.copy_(src)
                sq.dslash_apply(gid, 1, 'f32', 18, inp, out, stream=stream)
                sq.unpack_spinor(gid, 'f32', out, canon, stream=stream)
                got = canon.cpu().numpy()
            assert rel(got, want) <= TOL_DSLASH['f32'], (side, rel(got, want))
    finally:
        sq.gauge_free(gid)
