"""Fat and long links built on the GPU from thin links (gauge_fatten,
gauge_load_thin) vs the FP64 oracle's construction of the same recipe."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def _fatten_gpu(sq, dims, thin, **kw):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(thin)).cuda()
    fat = torch.zeros_like(u)
    lng = torch.zeros_like(u)
    sq.gauge_fatten(dims, u, fat, lng, **kw)
    torch.cuda.synchronize()
    return fat.cpu().numpy(), lng.cpu().numpy()


@pytest.mark.parametrize('dims', [(4, 6, 8, 10), (2, 4, 6, 4), (4, 4, 4, 4)])
def test_fatten_matches_oracle(sq, dims):
    thin = synth.thin_links(dims, 0.8, seed=2)
    fat, lng = _fatten_gpu(sq, dims, thin)
    f0, l0 = oracle.fat_long(dims, thin)
    assert np.abs(fat - f0).max() <= 1e-14
    assert np.abs(lng - l0).max() <= 1e-15
    # other coefficients reach the kernel
    fat2, lng2 = _fatten_gpu(sq, dims, thin, c1=1.0, c3=0.5, staple_weight=0.25)
    f2, l2 = oracle.fat_long(dims, thin, c1=1.0, c3=0.5, w=0.25)
    assert np.abs(fat2 - f2).max() <= 1e-14 and np.abs(lng2 - l2).max() <= 1e-14


def test_load_thin_then_dslash_and_solve(sq):
    dims = (4, 6, 8, 10)
    thin = synth.thin_links(dims, 0.25, seed=0)
    fat, lng = oracle.fat_long(dims, thin)
    gid = sq.gauge_load_thin(dims, thin)
    try:
        from gpu_helpers import gpu_dslash
        vh = oracle.volume(dims) // 2
        v = synth.gaussian_source(vh, 1)
        got = gpu_dslash(sq, gid, 'f64', 18, v, 1, vh)
        want = oracle.dslash_half(dims, fat, lng, v, 1)
        assert rel(got, want) <= 1e-13
        x, st = sq.cg_solve(gid, v, 0.05, 1e-9, long_recon=12)
        assert st['status'] == 0
        assert oracle.true_residual(dims, fat, lng, 0.05, v, x) <= 1e-9
    finally:
        sq.gauge_free(gid)


def test_fatten_rejects_bad_arguments(sq):
    import torch
    from paper_1411_2223_gb300 import sq as sqm
    u = torch.zeros((16 * 4, 4, 3, 3), dtype=torch.complex128, device='cuda')
    with pytest.raises(sqm.SqError):
        sq.gauge_fatten((4, 4, 4, 3), u, u.clone(), u.clone())   # odd extent
    with pytest.raises(sqm.SqError):
        sq.gauge_fatten((4, 4, 2, 2), u, u.clone(), u.clone(), staple_weight=float('inf'))
    thin = np.full((16 * 4, 4, 3, 3), np.nan, dtype=np.complex128)
    with pytest.raises(sqm.SqError) as e:
        sq.gauge_load_thin((4, 4, 2, 2), thin)
    assert e.value.status == sqm.ERR_NONFINITE


def test_fatten_full_size_20x64(sq):
    """The benchmark lattice 20^3 x 64 (eps 0.25): every link against the oracle."""
    dims = (20, 20, 20, 64)
    thin = synth.thin_links(dims, 0.25, seed=0)
    fat, lng = _fatten_gpu(sq, dims, thin)
    f0, l0 = oracle.fat_long(dims, thin)
    assert np.abs(fat - f0).max() <= 1e-14
    assert np.abs(lng - l0).max() <= 1e-15


def _asqtad_gpu(sq, dims, thin):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(thin)).cuda()
    fat = torch.zeros_like(u)
    lng = torch.zeros_like(u)
    sq.gauge_fatten_asqtad(dims, u, fat, lng)
    torch.cuda.synchronize()
    return fat, lng


@pytest.mark.parametrize('dims', [(4, 6, 8, 10), (2, 4, 6, 4)])
def test_asqtad_links_match_oracle(sq, dims):
    thin = synth.thin_links(dims, 0.6, seed=4)
    fat, lng = _asqtad_gpu(sq, dims, thin)
    f0, l0 = oracle.asqtad_links(dims, thin)
    assert np.abs(fat.cpu().numpy() - f0).max() <= 1e-14
    assert np.abs(lng.cpu().numpy() - l0).max() <= 1e-15


def test_asqtad_links_solve(sq):
    """A CG solve on the GPU-built asqtad links (12-real Naik links) meets the
    oracle's residual computed on the oracle's own asqtad links."""
    dims = (4, 6, 8, 10)
    thin = synth.thin_links(dims, 0.25, seed=0)
    fat_d, lng_d = _asqtad_gpu(sq, dims, thin)
    f0, l0 = oracle.asqtad_links(dims, thin)
    gid = sq.gauge_load(dims, fat_d, lng_d)
    try:
        b = synth.gaussian_source(oracle.volume(dims) // 2, 2)
        for prec, recon in (('f32', 12), ('i16', 12), ('f64', 18)):
            x, st = sq.cg_solve(gid, b, 0.03, 1e-9, precision=prec, long_recon=recon)
            assert st['status'] == 0
            assert oracle.true_residual(dims, f0, l0, 0.03, b, x) <= 1e-9
    finally:
        sq.gauge_free(gid)


def test_asqtad_full_size_20x64(sq):
    """The benchmark lattice 20^3 x 64: every asqtad link against the oracle."""
    dims = (20, 20, 20, 64)
    thin = synth.thin_links(dims, 0.25, seed=0)
    fat, lng = _asqtad_gpu(sq, dims, thin)
    f0, l0 = oracle.asqtad_links(dims, thin)
    assert np.abs(fat.cpu().numpy() - f0).max() <= 1e-14
    assert np.abs(lng.cpu().numpy() - l0).max() <= 1e-15
