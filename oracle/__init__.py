"""FP64 CPU oracle for the asqtad even-odd CG and the NPR four-fermion
operator (Eq. 1) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The GPU library neither imports nor links
it, and the two share no code: the oracle is plain C (``oracle.c``) written
site by site from the operator definitions, driven through ctypes.

The NPR part builds the hypercube spin-taste matrices here, from explicit
Dirac matrices and traces, and evaluates Eq. 1 term by term in C.

Vectors here are numpy complex128 arrays.  Full-lattice vectors have shape
``(V, 3)`` indexed by ``site_lex``; parity-half vectors have shape
``(V/2, 3)`` indexed by ``i = site_lex // 2`` within the parity.
``embed_half``/``extract_half`` convert between the two.

Parity: every function is pinned by the CPU tests (``tests/test_oracle_*``)
against closed forms, invariants and dense linear algebra; see the header of
``oracle.c`` for the definitions it follows.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'oracle.c')
_LIB = os.path.join(_HERE, 'liboracle.so')
_lock = threading.Lock()
_lib = None

CFLAGS = ['-O2', '-std=c11', '-fopenmp', '-ffp-contract=off', '-fPIC', '-shared']


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + '.%d.tmp' % os.getpid()
    subprocess.check_call(['gcc'] + CFLAGS + ['-o', tmp, _SRC, '-lm'])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            Lg = ctypes.c_long
            D = ctypes.c_double
            lib.oracle_dslash.argtypes = [P, P, P, I, I, P, P]
            lib.oracle_dslash_site.argtypes = [P, P, P, I, Lg, P, P]
            lib.oracle_mdagm.argtypes = [P, P, P, I, D, P, P, P]
            lib.oracle_true_residual.argtypes = [P, P, P, I, D, P, P]
            lib.oracle_true_residual.restype = D
            lib.oracle_cg.argtypes = [P, P, P, I, D, P, D, I, P, P]
            lib.oracle_cg.restype = I
            lib.oracle_cg_multishift.argtypes = [P, P, P, I, I, P, P, D, I, P, P]
            lib.oracle_cg_multishift.restype = I
            lib.oracle_neighbor.argtypes = [P, Lg, I, I, I, P]
            lib.oracle_neighbor.restype = Lg
            lib.oracle_eta.argtypes = [P, Lg, I]
            lib.oracle_eta.restype = I
            lib.oracle_parity.argtypes = [P, Lg]
            lib.oracle_parity.restype = I
            lib.oracle_quantize_spinor_i16.argtypes = [Lg, P, P, P]
            lib.oracle_quantize_links_i16.argtypes = [Lg, P, D, P]
            lib.oracle_fat_long.argtypes = [P, P, D, D, D, P, P]
            lib.oracle_asqtad_links.argtypes = [P, P, P, P, P]
            lib.oracle_npr_avg_link.argtypes = [P, P, P, I, I, P]
            lib.oracle_npr.argtypes = [P, P, P, P, P, P, I, P, P, Lg, P, P]
            _lib = lib
    return _lib


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(dims):
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def half_sites(dims, parity):
    """site_lex of the parity's sites in half-lattice order."""
    lx, ly, lz, lt = (int(d) for d in dims)
    lex = np.arange(volume(dims))
    x = lex % lx
    y = (lex // lx) % ly
    z = (lex // (lx * ly)) % lz
    t = lex // (lx * ly * lz)
    return lex[((x + y + z + t) & 1) == parity]


def embed_half(dims, parity, v):
    full = np.zeros((volume(dims), 3), dtype=np.complex128)
    full[half_sites(dims, parity)] = v
    return full


def extract_half(dims, parity, full):
    return np.ascontiguousarray(full[half_sites(dims, parity)])


# ----------------------------------------------------------------- lattice

def neighbor(dims, s, mu, d, t_sign=1):
    """(site_lex of x + d*mu_hat, boundary sign)."""
    lib = _load()
    sg = ctypes.c_int(0)
    n = lib.oracle_neighbor(_ptr(_dims(dims)), int(s), int(mu), int(d), int(t_sign),
                            ctypes.byref(sg))
    return n, sg.value


def eta(dims, s, mu):
    return _load().oracle_eta(_ptr(_dims(dims)), int(s), int(mu))


def parity(dims, s):
    return _load().oracle_parity(_ptr(_dims(dims)), int(s))


# ----------------------------------------------------------------- operators

def dslash(dims, fat, lng, v, out_parity=-1, t_sign=1):
    """Full-lattice D applied to v (V, 3); rows of parity out_parity (or all)."""
    lib = _load()
    fat, lng, v = _c128(fat), _c128(lng), _c128(v)
    out = np.zeros((volume(dims), 3), dtype=np.complex128)
    lib.oracle_dslash(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign), int(out_parity),
                      _ptr(v), _ptr(out))
    return out


def dslash_half(dims, fat, lng, v_half, out_parity, t_sign=1):
    """D_{p,1-p}: parity-half input of parity 1-p to parity-half output p."""
    full = embed_half(dims, 1 - out_parity, v_half)
    return extract_half(dims, out_parity, dslash(dims, fat, lng, full, out_parity, t_sign))


def dslash_site(dims, fat, lng, v, site_lex, t_sign=1):
    """One output site (3,) of D applied to the full-lattice vector v."""
    lib = _load()
    fat, lng, v = _c128(fat), _c128(lng), _c128(v)
    out = np.zeros(3, dtype=np.complex128)
    lib.oracle_dslash_site(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign), int(site_lex),
                           _ptr(v), _ptr(out))
    return out


def mdagm(dims, fat, lng, mass, p_even, t_sign=1):
    """A p = m^2 p - D_eo D_oe p on the even half (input and output (V/2, 3))."""
    lib = _load()
    fat, lng = _c128(fat), _c128(lng)
    p = embed_half(dims, 0, p_even)
    out = np.zeros_like(p)
    tmp = np.zeros_like(p)
    lib.oracle_mdagm(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign), float(mass),
                     _ptr(p), _ptr(out), _ptr(tmp))
    return extract_half(dims, 0, out)


def true_residual(dims, fat, lng, mass, b_even, x_even, t_sign=1):
    """|b - A x| / |b| in FP64 (even half vectors)."""
    lib = _load()
    fat, lng = _c128(fat), _c128(lng)
    b = embed_half(dims, 0, b_even)
    x = embed_half(dims, 0, x_even)
    return lib.oracle_true_residual(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign),
                                    float(mass), _ptr(b), _ptr(x))


def cg(dims, fat, lng, mass, b_even, tol, max_iter=100000, t_sign=1):
    """FP64 CG on A x = b.  Returns (x_even, iterations or -1, true residual)."""
    lib = _load()
    fat, lng = _c128(fat), _c128(lng)
    b = embed_half(dims, 0, b_even)
    x = np.zeros_like(b)
    tr = ctypes.c_double(0)
    it = lib.oracle_cg(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign), float(mass),
                       _ptr(b), float(tol), int(max_iter), _ptr(x), ctypes.byref(tr))
    return extract_half(dims, 0, x), it, tr.value


C1 = 9.0 / 8.0
C3 = -1.0 / 24.0
STAPLE_WEIGHT = 0.1


def fat_long(dims, thin, c1=C1, c3=C3, w=STAPLE_WEIGHT):
    """Fat and long links (V, 4, 3, 3) from thin links by the workloads'
    recipe: F = c1 [U + w * (6 staples)] / (1 + 6w), L = c3 U U U (see
    oracle.c; the paper's links are MILC asqtad links, Sec. 2)."""
    lib = _load()
    u = _c128(thin)
    fat = np.zeros_like(u)
    lng = np.zeros_like(u)
    lib.oracle_fat_long(_ptr(_dims(dims)), _ptr(u), float(c1), float(c3), float(w), _ptr(fat),
                        _ptr(lng))
    return fat, lng


# Tree-level asqtad path coefficients with the orientation of oracle.c:
# one-link, 3-staple, 5-staple, 7-staple, Lepage, Naik.
ASQTAD_COEFFS = (5.0 / 8.0, 1.0 / 16.0, 1.0 / 64.0, 1.0 / 384.0, -1.0 / 16.0, -1.0 / 24.0)


def asqtad_links(dims, thin, coeffs=ASQTAD_COEFFS):
    """Fat and Naik links of the asqtad action (MILC's path set: one-link,
    3-, 5- and 7-link staples, Lepage term) from thin links -- the kind of
    links the paper's MILC lattices carry (Sec. 2).  See oracle.c."""
    lib = _load()
    u = _c128(thin)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    assert c.shape == (6,)
    fat = np.zeros_like(u)
    lng = np.zeros_like(u)
    lib.oracle_asqtad_links(_ptr(_dims(dims)), _ptr(u), _ptr(c), _ptr(fat), _ptr(lng))
    return fat, lng


def dirac(dims, fat, lng, mass, v, t_sign=1):
    """(m + D) v on the whole lattice: the staggered matrix M = m + D, with D
    the asqtad operator above (the equation the paper's CG inverter solves,
    Sec. 2).  v and the result are full-lattice (V, 3) arrays."""
    v = _c128(v)
    return mass * v + dslash(dims, fat, lng, v, -1, t_sign)


def full_residual(dims, fat, lng, mass, b, x, t_sign=1):
    """|b - (m + D) x| / |b| in FP64 on the whole lattice."""
    r = _c128(b) - dirac(dims, fat, lng, mass, x, t_sign)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def solve_full(dims, fat, lng, mass, b, tol, max_iter=100000, t_sign=1):
    """Solve (m + D) x = b on the whole lattice by even-odd reduction.

    D joins only opposite parities, so with b = (b_e, b_o):
      (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o   (the oracle CG above),
      x_o = (b_o - D_oe x_e) / m.
    The even system is solved to tol * m |b| / |m b_e - D_eo b_o|, which
    bounds the full relative residual by tol (b - M x = (r_e / m, 0)).
    Returns (x (V, 3), iterations of the even CG)."""
    b = _c128(b)
    b_e = extract_half(dims, 0, b)
    b_o_full = embed_half(dims, 1, extract_half(dims, 1, b))
    bt = mass * b_e - extract_half(dims, 0, dslash(dims, fat, lng, b_o_full, 0, t_sign))
    bn, btn = np.linalg.norm(b), np.linalg.norm(bt)
    it = 0
    if bn == 0 or btn == 0:
        x_e = np.zeros_like(b_e)
    else:
        x_e, it, _ = cg(dims, fat, lng, mass, bt, tol * mass * bn / btn, max_iter, t_sign)
    x_e_full = embed_half(dims, 0, x_e)
    d_oe = extract_half(dims, 1, dslash(dims, fat, lng, x_e_full, 1, t_sign))
    x_o = (extract_half(dims, 1, b) - d_oe) / mass
    return x_e_full + embed_half(dims, 1, x_o), it


def bicgstab_full(dims, fat, lng, mass, b, tol, max_iter=100000, t_sign=1):
    """Solve (m + D) x = b on the whole lattice by BiCGstab (van der Vorst,
    SIAM J. Sci. Stat. Comput. 13 (1992) 631), the BiCG-family solver the
    paper names among QUDA's inverters (Sec. 3), applied to the
    non-Hermitian staggered matrix itself.  Textbook recurrences, x0 = 0,
    shadow residual r^ = r0, complex scalars:
      rho = <r^, r>; beta = (rho / rho_old)(alpha / omega);
      p = r + beta (p - omega v); v = M p; alpha = rho / <r^, v>;
      s = r - alpha v; t = M s; omega = <t, s> / <t, t>;
      x += alpha p + omega s; r = s - omega t.
    Stops when |r| / |b| <= tol and the recomputed |b - M x| / |b| <= tol;
    if the recomputed residual is larger, restarts from it.
    Returns (x (V, 3), iterations, true relative residual)."""
    b = _c128(b)
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bn == 0:
        return x, 0, 0.0

    def matvec(v):
        return dirac(dims, fat, lng, mass, v, t_sign)

    def vdot(a, c):
        return complex(np.vdot(a.reshape(-1), c.reshape(-1)))

    r = b.copy()
    it = 0
    while it < max_iter:
        rhat = r.copy()
        rho_old = alpha = omega = 1.0 + 0j
        p = np.zeros_like(b)
        v = np.zeros_like(b)
        while it < max_iter:
            rho = vdot(rhat, r)
            if rho == 0:
                break
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = matvec(p)
            alpha = rho / vdot(rhat, v)
            s = r - alpha * v
            it += 1
            if np.linalg.norm(s) <= tol * bn:
                x = x + alpha * p
                r = s
                break
            t = matvec(s)
            tt = vdot(t, t).real
            if tt == 0:
                x = x + alpha * p
                r = s
                break
            omega = vdot(t, s) / tt
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho_old = rho
            if np.linalg.norm(r) <= tol * bn or omega == 0:
                break
        r = b - matvec(x)
        res = float(np.linalg.norm(r) / bn)
        if res <= tol:
            return x, it, res
    return x, it, float(np.linalg.norm(b - matvec(x)) / bn)


def cg_multishift(dims, fat, lng, masses, b_even, tol, max_iter=100000, t_sign=1):
    """Multi-shift CG.  Returns (x (nshift, V/2, 3), iterations, true residuals)."""
    lib = _load()
    fat, lng = _c128(fat), _c128(lng)
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    ns = len(masses)
    b = embed_half(dims, 0, b_even)
    x = np.zeros((ns,) + b.shape, dtype=np.complex128)
    tr = np.zeros(ns)
    it = lib.oracle_cg_multishift(_ptr(_dims(dims)), _ptr(fat), _ptr(lng), int(t_sign), ns,
                                  _ptr(masses), _ptr(b), float(tol), int(max_iter), _ptr(x),
                                  _ptr(tr))
    return np.stack([extract_half(dims, 0, x[i]) for i in range(ns)]), it, tr


# ----------------------------------------------------------------- int16 codes

def quantize_spinor_i16(v_half):
    """int16 codes (n, 6) and FP32 site norms (n,) of an (n, 3) complex field."""
    lib = _load()
    v = _c128(v_half)
    n = v.shape[0]
    q = np.zeros((n, 6), dtype=np.int16)
    norm = np.zeros(n, dtype=np.float32)
    lib.oracle_quantize_spinor_i16(n, _ptr(v), _ptr(q), _ptr(norm))
    return q, norm


def quantize_links_i16(values, scale):
    """int16 codes of real link elements with one global scale."""
    lib = _load()
    v = np.ascontiguousarray(values, dtype=np.float64).ravel()
    q = np.zeros(v.shape[0], dtype=np.int16)
    lib.oracle_quantize_links_i16(v.shape[0], _ptr(v), float(scale), _ptr(q))
    return q.reshape(np.shape(values))


# ------------------------------------------- NPR four-fermion operator (Eq. 1)

def gammas():
    """Euclidean Dirac matrices gamma_1..gamma_4 (Hermitian, {g_mu, g_nu} =
    2 delta), chiral basis: g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1],
    [1, 0]].  Shape (4, 4, 4); index mu = 0..3 is gamma_{mu+1}."""
    s = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
         np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
         np.array([[1, 0], [0, -1]], dtype=np.complex128)]
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in s]
    g.append(np.block([[z, one], [one, z]]))
    return np.stack(g)


def gamma_of(x, g=None):
    """gamma_X = g_1^{X_0} g_2^{X_1} g_3^{X_2} g_4^{X_3} for a hypercube vector
    X given as a 4-bit mask (bit mu = X_mu)."""
    g = gammas() if g is None else g
    m = np.eye(4, dtype=np.complex128)
    for mu in range(4):
        if (x >> mu) & 1:
            m = m @ g[mu]
    return m


def spin_taste(s, f, g=None):
    """The hypercube spin-taste matrix of Eq. 1, (gamma_S x xi_F)_{AB} =
    Tr(gamma_A^dag gamma_S gamma_B gamma_F^dag) / 4, A, B = 0..15 (16 x 16
    complex).  S and F are 4-bit masks."""
    g = gammas() if g is None else g
    gs, gf = gamma_of(s, g), gamma_of(f, g)
    m = np.zeros((16, 16), dtype=np.complex128)
    for a in range(16):
        ga = gamma_of(a, g)
        for b in range(16):
            m[a, b] = np.trace(ga.conj().T @ gs @ gamma_of(b, g) @ gf.conj().T) / 4
    return m


def hypercube_count(dims):
    return volume(dims) // 16


def hypercube_index(dims, z):
    """Index of hypercube z = (z_x, z_y, z_z, z_t), 0 <= z_mu < L_mu / 2."""
    h = [int(d) // 2 for d in dims]
    return int(z[0] + h[0] * (z[1] + h[1] * (z[2] + h[2] * z[3])))


def npr_avg_link(dims, links, z, a, d):
    """U_AD(z): the mean of the links' products over all shortest paths from
    corner A to corner D of hypercube z (Eq. 1).  3 x 3 complex."""
    lib = _load()
    u = _c128(links)
    out = np.zeros((3, 3), dtype=np.complex128)
    zz = np.ascontiguousarray(z, dtype=np.int32)
    lib.oracle_npr_avg_link(_ptr(_dims(dims)), _ptr(u), _ptr(zz), int(a), int(d), _ptr(out))
    return out


def npr_four_fermion(dims, links, props, ops, hypercubes=None, g=None):
    """The one-colour four-fermion operator of Eq. 1 on every hypercube (or
    the listed hypercube indices), for each operator (S1, F1, S2, F2) of ops.

    props: four propagators (V, 3, 3) complex, [site][colour][source colour];
    flavours 1 and 3 enter as chibar (conjugated columns), 2 and 4 as chi.
    Returns (nz, nops, 3, 3, 3, 3) complex, axes [z][op][a1][a2][a3][a4]."""
    lib = _load()
    u = _c128(links)
    gs = [_c128(p) for p in props]
    assert len(gs) == 4 and all(p.shape == (volume(dims), 3, 3) for p in gs)
    nops = len(ops)
    m1 = np.ascontiguousarray(np.stack([spin_taste(o[0], o[1], g) for o in ops]))
    m2 = np.ascontiguousarray(np.stack([spin_taste(o[2], o[3], g) for o in ops]))
    if hypercubes is None:
        nz, zl = hypercube_count(dims), None
    else:
        zl = np.ascontiguousarray(hypercubes, dtype=np.int64)
        nz = len(zl)
    out = np.zeros((nz, nops, 3, 3, 3, 3), dtype=np.complex128)
    lib.oracle_npr(_ptr(_dims(dims)), _ptr(u), _ptr(gs[0]), _ptr(gs[1]), _ptr(gs[2]),
                   _ptr(gs[3]), nops, _ptr(m1), _ptr(m2), nz,
                   None if zl is None else _ptr(zl), _ptr(out))
    return out
