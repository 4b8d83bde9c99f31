"""The NPR one-colour four-fermion operator (Eq. 1) on the GPU vs the FP64
oracle, hypercube by hypercube.

Tolerance: both sides are FP64.  One output is a sum of 256 products of two
sandwiches, each a sum of 9 products with averaged links (sums of up to 24
path products), so the rounding differs by a few hundred ulps of the terms'
size at most; the tests allow 1e-12 of the largest output of the tensor.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import npr as snpr

pytestmark = pytest.mark.gpu

TOL = 1e-12
OPS16 = snpr.bk_ops() + [(0, 0, 0, 0), (15, 15, 15, 15), (3, 5, 12, 9), (1, 3, 12, 9),
                         (6, 0, 0, 10), (9, 9, 6, 6), (7, 8, 11, 4), (14, 1, 2, 13)]


def _inputs(dims, eps=0.5, seed=3):
    return synth.thin_links(dims, eps, seed), snpr.propagators(dims, seed + 10)


def _gpu(sq, dims, links, props, ops, per_hc=True):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(links)).cuda()
    ps = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in props]
    nops = len(ops)
    out = torch.full((max(nops, 1), 3, 3, 3, 3), float('nan'), dtype=torch.complex128,
                     device='cuda')
    hc = None
    if per_hc:
        hc = torch.full((oracle.hypercube_count(dims), max(nops, 1), 3, 3, 3, 3), float('nan'),
                        dtype=torch.complex128, device='cuda')
    sq.npr_four_fermion(dims, u, ps, ops, out, hc)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:nops], None if hc is None else hc.cpu().numpy()[:, :nops]


def _close(got, want, tol=TOL):
    scale = np.abs(want).max()
    assert scale > 0
    err = np.abs(got - want).max()
    assert err <= tol * scale, (err, scale)


@pytest.mark.parametrize('dims,nops', [((4, 4, 4, 4), 16), ((6, 2, 10, 4), 1),
                                       ((2, 2, 2, 2), 3), ((4, 6, 4, 8), 8)])
def test_npr_matches_oracle(sq, dims, nops):
    links, props = _inputs(dims)
    ops = OPS16[:nops]
    out, hc = _gpu(sq, dims, links, props, ops)
    want = oracle.npr_four_fermion(dims, links, props, ops)
    _close(hc, want)
    _close(out, want.sum(axis=0))


def test_npr_ragged_grid(sq):
    # 384 hypercubes: more than one resident CTA per hypercube slot, some
    # CTAs take two hypercubes and the rest one
    dims = (8, 8, 8, 12)
    links, props = _inputs(dims, 0.25, 7)
    ops = snpr.bk_ops()
    out, hc = _gpu(sq, dims, links, props, ops)
    want = oracle.npr_four_fermion(dims, links, props, ops)
    _close(hc, want)
    _close(out, want.sum(axis=0))
    # without the per-hypercube output (the kernel's other form: running
    # sums across hypercubes), the same sums to rounding
    out2, _ = _gpu(sq, dims, links, props, ops, per_hc=False)
    _close(out2, want.sum(axis=0))


def test_npr_full_size_sampled(sq):
    """The 20^3 x 64 workload of the benchmark: sampled hypercubes against the
    oracle, and the sum over all 32000 against the per-hypercube outputs."""
    dims = (20, 20, 20, 64)
    links, props = synth.thin_links(dims, 0.25, 0), snpr.propagators(dims, 1)
    ops = snpr.bk_ops()
    out, hc = _gpu(sq, dims, links, props, ops)
    nhc = oracle.hypercube_count(dims)
    pick = [0, 1, 9, 10, 99, 100, nhc // 2, nhc - 101, nhc - 1]
    pick += list(np.random.default_rng(5).choice(nhc, 16, replace=False))
    want = oracle.npr_four_fermion(dims, links, props, ops, hypercubes=pick)
    _close(hc[pick], want)
    _close(out, hc.sum(axis=0), 1e-12)


def test_npr_gauge_invariant_on_gpu(sq):
    dims = (8, 8, 8, 8)
    links, props = _inputs(dims, 0.4, 2)
    ops = snpr.bk_ops()[:4]
    g = synth.random_su3(oracle.volume(dims), 2.0, np.random.default_rng(21))
    out, hc = _gpu(sq, dims, links, props, ops)
    outg, hcg = _gpu(sq, dims, synth.gauge_transform_links(links, g, dims),
                     [g @ p for p in props], ops)
    _close(hcg, hc)
    _close(outg, out)


def test_npr_more_operators_than_one_launch(sq):
    # 37 operators: three groups of at most 16, each a launch pair; outputs
    # land at their operator's place in both tensors
    dims = (4, 4, 6, 4)
    links, props = _inputs(dims, 0.4, 9)
    rng = np.random.default_rng(3)
    ops = [tuple(int(v) for v in rng.integers(0, 16, 4)) for _ in range(37)]
    out, hc = _gpu(sq, dims, links, props, ops)
    want = oracle.npr_four_fermion(dims, links, props, ops)
    _close(hc, want)
    _close(out, want.sum(axis=0))


@pytest.mark.parametrize('nops', [16, 8, 5])
def test_npr_deterministic(sq, nops):
    dims = (8, 8, 8, 12)
    links, props = _inputs(dims, 0.3, 4)
    a, _ = _gpu(sq, dims, links, props, OPS16[:nops], per_hc=False)
    b, _ = _gpu(sq, dims, links, props, OPS16[:nops], per_hc=False)
    assert np.array_equal(a, b)
    want = oracle.npr_four_fermion(dims, links, props, OPS16[:nops]).sum(axis=0)
    _close(a, want)


def test_npr_arguments(sq):
    import torch
    from paper_1411_2223_gb300.sq import SqError
    dims = (4, 4, 4, 4)
    links, props = _inputs(dims)
    u = torch.from_numpy(links).cuda()
    ps = [torch.from_numpy(p).cuda() for p in props]
    out = torch.zeros((SQ_MAX + 1, 3, 3, 3, 3), dtype=torch.complex128, device='cuda')
    # no operators: nothing to do, nothing written
    sq.npr_four_fermion(dims, u, ps, [], out)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    with pytest.raises(SqError):
        sq.npr_four_fermion(dims, u, ps, [(16, 0, 0, 0)], out)          # mask out of range
    with pytest.raises(SqError):
        sq.npr_four_fermion((4, 4, 4, 5), u, ps, [(0, 0, 0, 0)], out)   # odd extent
    with pytest.raises(SqError):                                        # misaligned output
        sq.npr_four_fermion(dims, u, ps, [(0, 0, 0, 0)], out.data_ptr() + 8)


SQ_MAX = 16
