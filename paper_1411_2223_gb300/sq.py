"""Python binding of libsq.so (the C ABI in include/sq.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  There is no CPU fallback -- importing this module without a built
libsq.so raises, and every call that fails returns its status as an
``SqError``.  Device buffers are torch CUDA tensors (PyTorch supplies device
memory and streams); host buffers are numpy arrays.

Method names follow the C entry points: ``gauge_load``, ``dslash_apply``,
``mdagm_apply``, ``cg_solve``, ``cg_solve_multi``, ``cg_solve_multishift``,
``serve_submit``, ``serve_poll`` ...; module-level functions of the same
names take the context as first argument.
"""

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, 'libsq.so')

OK, PENDING, NOT_CONVERGED = 0, 1, 2
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE = -1, -2, -3, -4
ERR_TIMEOUT, ERR_BUSY, ERR_NOTFOUND, ERR_UNSUPPORTED = -5, -6, -7, -8
PREC = {'f64': 0, 'f32': 1, 'i16': 2}

GAUGE_DEVICE_PTRS = 0x1
GAUGE_ANTIPERIODIC_T = 0x2
GAUGE_NO_F32 = 0x10
GAUGE_NO_I16 = 0x20
GAUGE_NO_LONG12 = 0x40
GAUGE_NO_F64 = 0x80
CG_DEVICE_PTRS = 0x1
CG_INITIAL_GUESS = 0x2
CG_NO_GRAPH = 0x4
STATIC_SCRATCH_BYTES = 12 << 20   # SQ_STATIC_SCRATCH_BYTES of include/sq.h


class SqError(RuntimeError):
    def __init__(self, status, what=''):
        self.status = status
        super().__init__('%s: %s (status %d)' % (what, _strerror(status), status))


class CgOpts(ctypes.Structure):
    _fields_ = [('precision', ctypes.c_int), ('long_recon', ctypes.c_int),
                ('delta', ctypes.c_double), ('max_iter', ctypes.c_int),
                ('block_iters', ctypes.c_int), ('flags', ctypes.c_uint),
                ('stream', ctypes.c_void_p)]


class CgStats(ctypes.Structure):
    _fields_ = [('status', ctypes.c_int), ('iterations', ctypes.c_int),
                ('reliable_updates', ctypes.c_int), ('true_residual', ctypes.c_double),
                ('seconds', ctypes.c_double), ('gflops', ctypes.c_double),
                ('oe_block', ctypes.c_int), ('oe_rhs_tile', ctypes.c_int),
                ('eo_block', ctypes.c_int), ('eo_rhs_tile', ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeStats(ctypes.Structure):
    _fields_ = [('submitted', ctypes.c_uint64), ('completed', ctypes.c_uint64),
                ('rejected', ctypes.c_uint64), ('queued', ctypes.c_int),
                ('running', ctypes.c_int), ('p50_ms', ctypes.c_double),
                ('p99_ms', ctypes.c_double), ('mean_ms', ctypes.c_double),
                ('solves_per_s', ctypes.c_double), ('hbm_in_use', ctypes.c_size_t),
                ('hbm_budget', ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# symbol -> (restype, argtypes)
_P, _I, _U, _D, _SZ, _U64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                             ctypes.c_size_t, ctypes.c_uint64)
SIGNATURES = {
    'sq_create': (_I, [ctypes.POINTER(_P), _I, _SZ]),
    'sq_destroy': (_I, [_P]),
    'sq_strerror': (ctypes.c_char_p, [_I]),
    'sq_cg_opts_default': (None, [ctypes.POINTER(CgOpts)]),
    'sq_kernel_launches': (_U64, [_P]),
    'gauge_load': (_I, [_P, _P, _P, _P, _U, ctypes.POINTER(_I)]),
    'gauge_free': (_I, [_P, _I]),
    'gauge_fatten': (_I, [_P, _P, _P, _D, _D, _D, _P, _P, _P]),
    'gauge_load_thin': (_I, [_P, _P, _P, _D, _D, _D, _U, ctypes.POINTER(_I)]),
    'gauge_fatten_asqtad': (_I, [_P, _P, _P, _P, _P, _P, _P]),
    'sq_spinor_bytes': (_I, [_P, _I, _I, ctypes.POINTER(_SZ), ctypes.POINTER(_I)]),
    'sq_pack_spinor': (_I, [_P, _I, _I, _P, _P, _P]),
    'sq_unpack_spinor': (_I, [_P, _I, _I, _P, _P, _P]),
    'dslash_apply': (_I, [_P, _I, _I, _I, _I, _P, _P, _P]),
    'dslash_apply_multi': (_I, [_P, _I, _I, _I, _I, _I, _P, _P, _P]),
    'sq_tuned_launch': (_I, [_P, _I, _I, _I, _I, _I, _P, ctypes.POINTER(_I),
                             ctypes.POINTER(_I)]),
    'sq_time_dslash': (_I, [_P, _I, _I, _I, _I, _I, _I, _P, ctypes.POINTER(ctypes.c_float)]),
    'mdagm_apply': (_I, [_P, _I, _I, _I, _D, _P, _P, _P]),
    'mdagm_apply_static': (_I, [_P, _I, _I, _I, _D, _P, _P, _P]),
    'cg_solve': (_I, [_P, _I, _P, _D, _D, ctypes.POINTER(CgOpts), _P, ctypes.POINTER(CgStats)]),
    'cg_solve_multi': (_I, [_P, _I, _I, _P, _P, _D, ctypes.POINTER(CgOpts), _P,
                            ctypes.POINTER(CgStats)]),
    'cg_solve_multishift': (_I, [_P, _I, _P, _I, _P, _D, ctypes.POINTER(CgOpts), _P,
                                 ctypes.POINTER(CgStats)]),
    'cg_solve_full': (_I, [_P, _I, _P, _D, _D, ctypes.POINTER(CgOpts), _P,
                           ctypes.POINTER(CgStats)]),
    'bicgstab_solve_full': (_I, [_P, _I, _P, _D, _D, ctypes.POINTER(CgOpts), _P,
                                 ctypes.POINTER(CgStats)]),
    'dirac_apply': (_I, [_P, _I, _D, _P, _P, _P]),
    'serve_submit': (_I, [_P, _I, _P, _D, _D, ctypes.POINTER(_U64)]),
    'serve_poll': (_I, [_P, _U64, _P, ctypes.POINTER(CgStats), _I]),
    'serve_cancel': (_I, [_P, _U64]),
    'serve_stats': (_I, [_P, ctypes.POINTER(ServeStats), _I]),
    'serve_configure': (_I, [_P, _I, _I]),
    'sq_spin_taste': (_I, [_I, _I, _P, _P]),
    'npr_four_fermion': (_I, [_P, _P, _P, _P, _I, _P, _P, _P, _P]),
}

_lib = None


def load_library(path=LIB_PATH):
    """Load libsq.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError('libsq.so not built at %s: run `python -c "import __graft_entry__ '
                              'as g; g.build()"`' % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _strerror(status):
    try:
        return load_library().sq_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return 'status %d' % status


def _check(status, what, allow=(OK,)):
    if status not in allow:
        raise SqError(status, what)
    return status


def _ptr(x):
    """Address of a numpy array or torch tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags['C_CONTIGUOUS']:
            raise ValueError('array must be C-contiguous')
        return x.ctypes.data
    if hasattr(x, 'data_ptr'):
        if not x.is_contiguous():
            raise ValueError('tensor must be contiguous')
        return x.data_ptr()
    raise TypeError('expected numpy array, torch tensor or address')


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _is_device(x):
    return hasattr(x, 'is_cuda') and x.is_cuda


class Context:
    """A library context on one CUDA device (owns gauge fields and workspaces)."""

    def __init__(self, device=0, hbm_budget=0):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.sq_create(ctypes.byref(h), int(device), int(hbm_budget)), 'sq_create')
        self.handle = h
        self.device = device
        self._dims = {}

    def close(self):
        if self.handle:
            self._lib.sq_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def kernel_launches(self):
        return int(self._lib.sq_kernel_launches(self.handle))

    # ---------------------------------------------------------------- gauge
    def gauge_load(self, dims, fat, lng, antiperiodic_t=False, flags=0):
        dims_a = (ctypes.c_int * 4)(*[int(d) for d in dims])
        if _is_device(fat):
            flags |= GAUGE_DEVICE_PTRS
        else:
            fat = np.ascontiguousarray(fat, dtype=np.complex128)
            lng = np.ascontiguousarray(lng, dtype=np.complex128)
        if antiperiodic_t:
            flags |= GAUGE_ANTIPERIODIC_T
        gid = ctypes.c_int(0)
        _check(self._lib.gauge_load(self.handle, dims_a, _ptr(fat), _ptr(lng), flags,
                                    ctypes.byref(gid)), 'gauge_load')
        self._dims[gid.value] = tuple(int(d) for d in dims)
        return gid.value

    def gauge_fatten(self, dims, thin_dev, fat_dev, lng_dev, c1=9.0 / 8.0, c3=-1.0 / 24.0,
                     staple_weight=0.1, stream=None):
        """Fat and long links from thin links on the device (torch CUDA tensors
        of shape (V, 4, 3, 3) complex128)."""
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        _check(self._lib.gauge_fatten(self.handle, d, _ptr(thin_dev), float(c1), float(c3),
                                      float(staple_weight), _ptr(fat_dev), _ptr(lng_dev),
                                      _stream(stream)), 'gauge_fatten')

    ASQTAD_COEFFS = (5.0 / 8.0, 1.0 / 16.0, 1.0 / 64.0, 1.0 / 384.0, -1.0 / 16.0, -1.0 / 24.0)

    def gauge_fatten_asqtad(self, dims, thin_dev, fat_dev, lng_dev, coeffs=ASQTAD_COEFFS,
                            stream=None):
        """asqtad fat (MILC path set) and Naik links from thin links on the
        device (torch CUDA tensors of shape (V, 4, 3, 3) complex128)."""
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        c = (ctypes.c_double * 6)(*[float(v) for v in coeffs])
        _check(self._lib.gauge_fatten_asqtad(self.handle, d, _ptr(thin_dev), c, _ptr(fat_dev),
                                             _ptr(lng_dev), _stream(stream)),
               'gauge_fatten_asqtad')

    def gauge_load_thin(self, dims, thin, c1=9.0 / 8.0, c3=-1.0 / 24.0, staple_weight=0.1,
                        antiperiodic_t=False, flags=0):
        """Fatten thin links on the GPU and load the result; returns a gauge id."""
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        if _is_device(thin):
            flags |= GAUGE_DEVICE_PTRS
            t = thin.contiguous()
        else:
            t = np.ascontiguousarray(thin, dtype=np.complex128)
        if antiperiodic_t:
            flags |= GAUGE_ANTIPERIODIC_T
        gid = ctypes.c_int(0)
        _check(self._lib.gauge_load_thin(self.handle, d, _ptr(t), float(c1), float(c3),
                                         float(staple_weight), flags, ctypes.byref(gid)),
               'gauge_load_thin')
        return gid.value

    def gauge_free(self, gauge_id):
        _check(self._lib.gauge_free(self.handle, gauge_id), 'gauge_free')
        self._dims.pop(gauge_id, None)

    def vh(self, gauge_id):
        return int(np.prod(self._dims[gauge_id])) // 2

    def spinor_bytes(self, gauge_id, prec):
        b, s = ctypes.c_size_t(0), ctypes.c_int(0)
        _check(self._lib.sq_spinor_bytes(self.handle, gauge_id, PREC[prec], ctypes.byref(b),
                                         ctypes.byref(s)), 'sq_spinor_bytes')
        return b.value, s.value

    def pack_spinor(self, gauge_id, prec, canon_dev, packed_dev, stream=None):
        _check(self._lib.sq_pack_spinor(self.handle, gauge_id, PREC[prec], _ptr(canon_dev),
                                        _ptr(packed_dev), _stream(stream)), 'sq_pack_spinor')

    def unpack_spinor(self, gauge_id, prec, packed_dev, canon_dev, stream=None):
        _check(self._lib.sq_unpack_spinor(self.handle, gauge_id, PREC[prec], _ptr(packed_dev),
                                          _ptr(canon_dev), _stream(stream)), 'sq_unpack_spinor')

    # ------------------------------------------------------------ operators
    def dslash_apply(self, gauge_id, out_parity, prec, long_recon, in_dev, out_dev, stream=None):
        _check(self._lib.dslash_apply(self.handle, gauge_id, int(out_parity), PREC[prec],
                                      int(long_recon), _ptr(in_dev), _ptr(out_dev),
                                      _stream(stream)), 'dslash_apply')

    def dslash_apply_multi(self, gauge_id, out_parity, prec, long_recon, nrhs, in_dev, out_dev,
                           stream=None):
        """out_j = D in_j for nrhs packed vectors back to back (device)."""
        _check(self._lib.dslash_apply_multi(self.handle, gauge_id, int(out_parity), PREC[prec],
                                            int(long_recon), int(nrhs), _ptr(in_dev),
                                            _ptr(out_dev), _stream(stream)),
               'dslash_apply_multi')

    MODES = {'plain': 0, 'mdagm': 1, 'cg_oe': 3, 'cg_eo': 4}

    def tuned_launch(self, gauge_id, prec, long_recon, nrhs, mode, stream=None):
        """(threads per block, right-hand sides per thread) the library
        launches a Dslash kernel with; mode in MODES (or its number)."""
        b, t = ctypes.c_int(0), ctypes.c_int(0)
        m = self.MODES.get(mode, mode)
        _check(self._lib.sq_tuned_launch(self.handle, gauge_id, PREC[prec], int(long_recon),
                                         int(nrhs), int(m), _stream(stream), ctypes.byref(b),
                                         ctypes.byref(t)), 'sq_tuned_launch')
        return b.value, t.value

    def time_dslash(self, gauge_id, prec, long_recon, nrhs, mode, reps=50, stream=None):
        """Microseconds per launch of a Dslash kernel at the library's launch
        shape (CUDA events, back-to-back launches on synthetic vectors)."""
        us = ctypes.c_float(0)
        m = self.MODES.get(mode, mode)
        _check(self._lib.sq_time_dslash(self.handle, gauge_id, PREC[prec], int(long_recon),
                                        int(nrhs), int(m), int(reps), _stream(stream),
                                        ctypes.byref(us)), 'sq_time_dslash')
        return float(us.value)

    def mdagm_apply(self, gauge_id, prec, long_recon, mass, in_dev, out_dev, stream=None):
        _check(self._lib.mdagm_apply(self.handle, gauge_id, PREC[prec], int(long_recon),
                                     float(mass), _ptr(in_dev), _ptr(out_dev), _stream(stream)),
               'mdagm_apply')

    def mdagm_apply_static(self, gauge_id, prec, long_recon, mass, in_dev, out_dev,
                           stream=None):
        """mdagm_apply with the temporary in the library's fixed device array
        (no allocation; for callers that cannot allocate at call time)."""
        _check(self._lib.mdagm_apply_static(self.handle, gauge_id, PREC[prec], int(long_recon),
                                            float(mass), _ptr(in_dev), _ptr(out_dev),
                                            _stream(stream)), 'mdagm_apply_static')

    # --------------------------------------------------------------- solvers
    def _opts(self, precision, long_recon, delta, max_iter, block_iters, flags, stream):
        o = CgOpts()
        self._lib.sq_cg_opts_default(ctypes.byref(o))
        o.precision = PREC[precision]
        o.long_recon = int(long_recon)
        o.delta = float(delta)
        o.max_iter = int(max_iter)
        o.block_iters = int(block_iters)
        o.flags = flags
        o.stream = _stream(stream)
        return o

    def cg_solve(self, gauge_id, src, mass, tol, precision='f32', long_recon=18, delta=-1.0,
                 max_iter=100000, block_iters=16, x0=None, graph=True, stream=None,
                 check=True, out=None):
        """Solve (m^2 - D_eo D_oe) x = src.  Returns (x, stats dict).

        src: numpy (Vh, 3) complex128 (host) or a torch complex128 CUDA tensor
        (device; x is then a device tensor).  out: optional buffer for x of the
        same kind (e.g. pinned host memory or a preallocated device tensor).
        """
        xs, st, status = self.cg_solve_multi(
            gauge_id, src[None], [mass], tol, precision, long_recon, delta, max_iter,
            block_iters, None if x0 is None else x0[None], graph, stream, check,
            out=None if out is None else out[None])
        return xs[0], st[0]

    def cg_solve_multi(self, gauge_id, srcs, masses, tol, precision='f32', long_recon=18,
                       delta=-1.0, max_iter=100000, block_iters=16, x0=None, graph=True,
                       stream=None, check=True, out=None):
        """Batched solve; returns (x (nrhs, Vh, 3), [stats dicts], status).

        srcs: (nrhs, Vh, 3) numpy array / list of arrays, or a torch CUDA tensor.
        """
        dev = _is_device(srcs)
        if dev:
            src = srcs.contiguous()
            x = out if out is not None else src.new_zeros(src.shape)
            if x0 is not None:
                x.copy_(x0)
        else:
            if isinstance(srcs, np.ndarray):
                src = np.ascontiguousarray(srcs, dtype=np.complex128)
            else:
                src = np.ascontiguousarray(np.stack([np.asarray(v) for v in srcs]),
                                           dtype=np.complex128)
            x = out if out is not None else np.zeros_like(src)
            if x0 is not None:
                x[...] = np.asarray(x0)
        nrhs = src.shape[0]
        flags = (CG_DEVICE_PTRS if dev else 0) | (CG_INITIAL_GUESS if x0 is not None else 0)
        if not graph:
            flags |= CG_NO_GRAPH
        o = self._opts(precision, long_recon, delta, max_iter, block_iters, flags, stream)
        m = np.ascontiguousarray(masses, dtype=np.float64)
        if m.shape != (nrhs,):
            raise ValueError('one mass per right-hand side')
        stats = (CgStats * nrhs)()
        status = self._lib.cg_solve_multi(self.handle, gauge_id, nrhs, _ptr(src), _ptr(m),
                                          float(tol), ctypes.byref(o), _ptr(x), stats)
        if check:
            _check(status, 'cg_solve', allow=(OK,))
        return x, [s.as_dict() for s in stats], status

    def cg_solve_multishift(self, gauge_id, src, masses, tol, precision='f32', long_recon=18,
                            delta=-1.0, max_iter=100000, block_iters=16, stream=None, check=True):
        """Multi-shift solve; returns (x (nshift, Vh, 3), [stats dicts], status)."""
        dev = _is_device(src)
        ns = len(masses)
        if dev:
            import torch
            s = src.contiguous()
            x = torch.empty((ns,) + tuple(s.shape), dtype=s.dtype, device=s.device)
        else:
            s = np.ascontiguousarray(src, dtype=np.complex128)
            x = np.zeros((ns,) + s.shape, dtype=np.complex128)
        o = self._opts(precision, long_recon, delta, max_iter, block_iters,
                       CG_DEVICE_PTRS if dev else 0, stream)
        m = np.ascontiguousarray(masses, dtype=np.float64)
        stats = (CgStats * ns)()
        status = self._lib.cg_solve_multishift(self.handle, gauge_id, _ptr(s), ns, _ptr(m),
                                               float(tol), ctypes.byref(o), _ptr(x), stats)
        if check:
            _check(status, 'cg_solve_multishift')
        return x, [st.as_dict() for st in stats], status

    def cg_solve_full(self, gauge_id, src, mass, tol, precision='f32', long_recon=18,
                      delta=-1.0, max_iter=100000, block_iters=16, x0=None, graph=True,
                      stream=None, check=True):
        """Solve (m + D) x = src on the whole lattice.  Returns (x, stats dict).

        src: numpy (V, 3) complex128 in site_lex order (host) or a torch
        complex128 CUDA tensor (x is then a device tensor).
        """
        dev = _is_device(src)
        if dev:
            s = src.contiguous()
            x = s.new_zeros(s.shape)
        else:
            s = np.ascontiguousarray(src, dtype=np.complex128)
            x = np.zeros_like(s)
        flags = CG_DEVICE_PTRS if dev else 0
        if x0 is not None:
            flags |= CG_INITIAL_GUESS
            if dev:
                x.copy_(x0)
            else:
                x[...] = np.asarray(x0)
        if not graph:
            flags |= CG_NO_GRAPH
        o = self._opts(precision, long_recon, delta, max_iter, block_iters, flags, stream)
        st = CgStats()
        status = self._lib.cg_solve_full(self.handle, gauge_id, _ptr(s), float(mass), float(tol),
                                         ctypes.byref(o), _ptr(x), ctypes.byref(st))
        if check:
            _check(status, 'cg_solve_full')
        return x, st.as_dict()

    def bicgstab_solve_full(self, gauge_id, src, mass, tol, precision='f64', delta=-1.0,
                            max_iter=100000, x0=None, stream=None, check=True):
        """Solve (m + D) x = src on the whole lattice by BiCGstab on M itself:
        precision 'f64', or 'f32' (FP32 vectors and Dslash with FP64 reliable
        updates at |r| < delta max|r|, default delta 0.1).  Arrays as
        cg_solve_full.  Returns (x, stats dict)."""
        dev = _is_device(src)
        if dev:
            s = src.contiguous()
            x = s.new_zeros(s.shape)
        else:
            s = np.ascontiguousarray(src, dtype=np.complex128)
            x = np.zeros_like(s)
        flags = CG_DEVICE_PTRS if dev else 0
        if x0 is not None:
            flags |= CG_INITIAL_GUESS
            if dev:
                x.copy_(x0)
            else:
                x[...] = np.asarray(x0)
        o = self._opts(precision, 18, delta, max_iter, 16, flags, stream)
        st = CgStats()
        status = self._lib.bicgstab_solve_full(self.handle, gauge_id, _ptr(s), float(mass),
                                               float(tol), ctypes.byref(o), _ptr(x),
                                               ctypes.byref(st))
        if check:
            _check(status, 'bicgstab_solve_full')
        return x, st.as_dict()

    def dirac_apply(self, gauge_id, mass, in_dev, out_dev, stream=None):
        """out = (m + D) in on the whole lattice, FP64, device (V, 3) complex128."""
        _check(self._lib.dirac_apply(self.handle, gauge_id, float(mass), _ptr(in_dev),
                                     _ptr(out_dev), _stream(stream)), 'dirac_apply')

    # ------------------------------------------------- NPR operator (Eq. 1)
    NPR_MAX_OPS = 16   # operators per kernel launch (more are done in groups)

    def npr_four_fermion(self, dims, links_dev, props_dev, ops, out_dev, out_hc_dev=None,
                         stream=None):
        """The one-colour four-fermion operator of Eq. 1 on the device, FP64.

        links_dev: (V, 4, 3, 3) complex128; props_dev: four (V, 3, 3)
        complex128 propagators [site][colour][source colour]; ops: list of
        (S1, F1, S2, F2) 4-bit masks; out_dev: (nops, 3, 3, 3, 3) complex128,
        the sum over hypercubes; out_hc_dev: None or (V/16, nops, 3, 3, 3, 3)
        complex128 per hypercube.  Asynchronous on `stream` (None: the
        default stream, which torch's default stream is)."""
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        if len(props_dev) != 4:
            raise ValueError('four propagators')
        pp = (ctypes.c_void_p * 4)(*[_ptr(p) for p in props_dev])
        flat = [int(v) for op in ops for v in op]
        if len(flat) != 4 * len(ops):
            raise ValueError('ops are (S1, F1, S2, F2) tuples')
        oa = (ctypes.c_int * max(1, len(flat)))(*flat)
        _check(self._lib.npr_four_fermion(self.handle, d, _ptr(links_dev), pp, len(ops), oa,
                                          _ptr(out_dev), _ptr(out_hc_dev), _stream(stream)),
               'npr_four_fermion')

    # --------------------------------------------------------------- serving
    def serve_configure(self, slots_per_batch=8, block_iters=8):
        _check(self._lib.serve_configure(self.handle, int(slots_per_batch), int(block_iters)),
               'serve_configure')

    def serve_submit(self, gauge_id, src, mass, tol):
        src = np.ascontiguousarray(src, dtype=np.complex128)
        t = ctypes.c_uint64(0)
        _check(self._lib.serve_submit(self.handle, gauge_id, _ptr(src), float(mass), float(tol),
                                      ctypes.byref(t)), 'serve_submit')
        return t.value

    def serve_poll(self, ticket, vh=None, timeout_us=-1, want_x=True):
        """Returns (status, x or None, stats dict)."""
        x = np.zeros((vh, 3), dtype=np.complex128) if (want_x and vh) else None
        st = CgStats()
        status = self._lib.serve_poll(self.handle, ctypes.c_uint64(ticket), _ptr(x),
                                      ctypes.byref(st), int(timeout_us))
        return status, x, st.as_dict()

    def serve_cancel(self, ticket):
        return self._lib.serve_cancel(self.handle, ctypes.c_uint64(ticket))

    def serve_stats(self, reset=False):
        st = ServeStats()
        _check(self._lib.serve_stats(self.handle, ctypes.byref(st), int(bool(reset))),
               'serve_stats')
        return st.as_dict()


def spin_taste(s, f):
    """The hypercube spin-taste matrix (gamma_S x xi_F) as the library uses
    it: (partner, sign), row A having its one entry sign[A] at partner[A].
    Host only."""
    lib = load_library()
    partner = (ctypes.c_int * 16)()
    sign = (ctypes.c_int * 16)()
    _check(lib.sq_spin_taste(int(s), int(f), partner, sign), 'sq_spin_taste')
    return list(partner), list(sign)


def _forward(name):
    def f(ctx, *args, **kw):
        return getattr(ctx, name)(*args, **kw)
    f.__name__ = name
    f.__doc__ = 'Module-level form of Context.%s(ctx, ...).' % name
    return f


for _n in ('gauge_load', 'gauge_free', 'gauge_fatten', 'gauge_load_thin', 'gauge_fatten_asqtad',
           'dslash_apply', 'dslash_apply_multi', 'mdagm_apply', 'cg_solve',
           'cg_solve_multi', 'cg_solve_multishift', 'cg_solve_full', 'bicgstab_solve_full',
           'dirac_apply',
           'npr_four_fermion', 'serve_submit', 'serve_poll',
           'serve_cancel', 'serve_stats', 'serve_configure'):
    globals()[_n] = _forward(_n)
