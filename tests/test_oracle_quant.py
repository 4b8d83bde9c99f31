"""Pins of the oracle's 16-bit storage codes.

Spinor sites: q_k = rint(v_k * 32767 / n) with n the site's max |v_k| (FP32);
links: one global scale.  Checked on hand-computed sites (including a
round-half-to-even tie), the zero site, the error bound |q n / 32767 - v| <=
n / 65534 (+ FP32 rounding) and saturation.
"""
import numpy as np

import oracle


def test_hand_computed_site():
    v = np.array([[1.0 + 0.5j, 0.0 - 1.0j, 0.25 - 0.5j]])
    q, n = oracle.quantize_spinor_i16(v)
    assert n[0] == np.float32(1.0)
    # 32767*0.5 = 16383.5 ties to the even 16384; 32767*0.25 = 8191.75 -> 8192
    assert q.tolist() == [[32767, 16384, 0, -32767, 8192, -16384]]


def test_zero_site_and_scale_invariance():
    v = np.zeros((2, 3), dtype=np.complex128)
    v[1] = [3.0, -1.5j, 0.75]
    q, n = oracle.quantize_spinor_i16(v)
    assert n[0] == 0 and np.all(q[0] == 0)
    q2, n2 = oracle.quantize_spinor_i16(v * 4.0)   # power-of-two scaling is exact
    assert np.array_equal(q, q2) and n2[1] == 4 * n[1]


def test_error_bound_random():
    rng = np.random.default_rng(0)
    v = rng.standard_normal((5000, 3)) + 1j * rng.standard_normal((5000, 3))
    q, n = oracle.quantize_spinor_i16(v)
    re = np.stack([v.real, v.imag], -1).reshape(5000, 6)
    deq = q.astype(np.float64) * n[:, None].astype(np.float64) / 32767
    err = np.abs(deq - re)
    bound = n[:, None] / 65534 * (1 + 1e-5) + np.abs(re) * 2 ** -23
    assert np.all(err <= bound)
    # the largest element of every site maps to +-32767
    assert np.all(np.abs(q).max(axis=1) == 32767)


def test_links_global_scale():
    vals = np.array([0.0, 1.125, -1.125, 0.5625, 1e-9, -0.3])
    q = oracle.quantize_links_i16(vals, 1.125)
    assert q.tolist()[:4] == [0, 32767, -32767, 16384]   # 16383.5 -> 16384
    assert q[4] == 0
    assert abs(q[5] * 1.125 / 32767 + 0.3) <= 1.125 / 65534
    # saturation for values beyond the scale
    assert oracle.quantize_links_i16(np.array([2.0, -2.0]), 1.0).tolist() == [32767, -32767]
