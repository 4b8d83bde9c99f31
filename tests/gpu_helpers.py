"""Helpers shared by the GPU parity tests (device buffers via torch)."""
import numpy as np

import oracle
import synth

TOL_DSLASH = {'f64': 1e-13, 'f32': 1e-5, 'i16': 5e-3}

_FIELDS = {}


def gauge(dims, eps=0.3, seed=0):
    key = (tuple(dims), eps, seed)
    if key not in _FIELDS:
        _FIELDS.clear() if len(_FIELDS) > 4 else None
        _FIELDS[key] = synth.gauge_field(dims, eps, seed)
    return _FIELDS[key]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def site_rel(a, b):
    """Largest error of one site's colour vector, relative to the RMS site
    norm of b: unlike rel(), one wrong site among 10^5 fails it."""
    a = np.asarray(a).reshape(-1, 3)
    b = np.asarray(b).reshape(-1, 3)
    err = np.linalg.norm(a - b, axis=1).max()
    return float(err / np.sqrt(np.mean(np.sum(np.abs(b) ** 2, axis=1))))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def packed_buffer(ctx, gid, prec):
    import torch
    nbytes, _ = ctx.spinor_bytes(gid, prec)
    # the library's asynchronous calls without a stream run on the legacy
    # default stream, which is torch's default stream too: they are ordered
    # after this fill
    return torch.zeros(nbytes, dtype=torch.uint8, device='cuda')


def pack(ctx, gid, prec, v_half):
    buf = packed_buffer(ctx, gid, prec)
    ctx.pack_spinor(gid, prec, to_dev(v_half), buf)
    return buf


def unpack(ctx, gid, prec, buf, vh):
    import torch
    out = torch.zeros((vh, 3), dtype=torch.complex128, device='cuda')
    ctx.unpack_spinor(gid, prec, buf, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def gpu_dslash(ctx, gid, prec, recon, v_half, out_parity, vh):
    src = pack(ctx, gid, prec, v_half)
    dst = packed_buffer(ctx, gid, prec)
    ctx.dslash_apply(gid, out_parity, prec, recon, src, dst)
    return unpack(ctx, gid, prec, dst, vh)


def gpu_mdagm(ctx, gid, prec, recon, mass, v_half, vh):
    src = pack(ctx, gid, prec, v_half)
    dst = packed_buffer(ctx, gid, prec)
    ctx.mdagm_apply(gid, prec, recon, mass, src, dst)
    return unpack(ctx, gid, prec, dst, vh)


def o9_check(dims, fat, lng, mass, b, x, x_ref, tol):
    """Solve acceptance: the oracle's FP64 residual of x is <= tol; the
    residual of x - x_ref is <= 10 tol; |x - x_ref| <= (|r| + |r_ref|)/m^2."""
    r = oracle.true_residual(dims, fat, lng, mass, b, x)
    assert r <= tol, r
    bn = np.linalg.norm(b)
    d = oracle.mdagm(dims, fat, lng, mass, x - x_ref)
    assert np.linalg.norm(d) / bn <= 10 * tol
    r_ref = oracle.true_residual(dims, fat, lng, mass, b, x_ref)
    assert np.linalg.norm(x - x_ref) <= (r + r_ref) * bn / mass ** 2 * (1 + 1e-9)
    return r, float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref))
