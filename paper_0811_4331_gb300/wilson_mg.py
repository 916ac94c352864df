"""Thin ctypes binding of the C ABI in include/wilson_mg.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Host arrays are
numpy (C-contiguous); device arrays are torch CUDA tensors (contiguous).  No
arithmetic of the solver happens here: if the CUDA library is missing the
import of this module fails, there is no fallback.

Layouts (see the header): external spinors are complex128 arrays shaped
(nrhs, Lt, Lz, Ly, Lx, 4, 3) (or without the leading nrhs); internal fields
are complex in the precision named by ``prec``: complex128 (MG_F64),
complex64 (MG_F32), or a trailing pair of float16 / bfloat16 (MG_F16 /
MG_BF16), shaped (nrhs, 3, V, 4) on level 0 (component c = spin * 3 + colour
at [c // 4, site, c % 4]) and (nrhs, ncomp, V) on coarse levels.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwilsonmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ERANK, MG_ENOCONV, MG_EBREAKDOWN, MG_ENAN = range(8)
MG_F64, MG_F32, MG_F16, MG_BF16 = range(4)
MG_MAX_LEVELS = 4
STATUS_NAMES = ["MG_OK", "MG_EINVAL", "MG_ENOMEM", "MG_ECUDA", "MG_ERANK", "MG_ENOCONV", "MG_EBREAKDOWN", "MG_ENAN"]


class mg_params(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("block", (ctypes.c_int * 4) * (MG_MAX_LEVELS - 1)),
        ("nv", ctypes.c_int * (MG_MAX_LEVELS - 1)),
        ("setup_sweeps", ctypes.c_int * (MG_MAX_LEVELS - 1)),
        ("coarse_cycles", ctypes.c_int * (MG_MAX_LEVELS - 1)),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("gcr_restart", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("mixed", ctypes.c_int),
        ("fine_prec", ctypes.c_int),
        ("coarse_prec", ctypes.c_int),
        ("reliable_delta", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("use_graphs", ctypes.c_int),
        ("coarse_mma", ctypes.c_int),
        ("coarse_solver", ctypes.c_int),
        ("adapt_steps", ctypes.c_int),
        ("adapt_cycles", ctypes.c_int),
        ("adapt_nv", ctypes.c_int * 3),
        ("defer_coarsest", ctypes.c_int),
        ("fine_smoother", ctypes.c_int),
        ("coarsest_f64", ctypes.c_int),
    ]


class mg_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("fine_dslash", ctypes.c_longlong),
        ("fine_dslash_f64", ctypes.c_longlong),
        ("true_rel_residual", ctypes.c_double),
        ("solve_seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgError(RuntimeError):
    def __init__(self, status, msg, stats=None):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status
        self.stats = stats


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libwilsonmg.so is not built (run __graft_entry__.build()); no fallback exists")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, VP = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_default_params": (I, [P(mg_params)]),
        "mg_setup": (I, [P(VP), VP, I, P(I), D, P(mg_params), VP, VP]),
        "mg_destroy": (I, [VP]),
        "mg_retarget": (I, [VP, D, P(VP), VP]),
        "mg_retarget_batch": (I, [VP, P(D), I, P(VP), VP]),
        "mg_solve": (I, [VP, VP, VP, I, I, D, P(mg_stats), VP]),
        "mg_solve_masses": (I, [VP, P(D), VP, VP, I, I, D, P(mg_stats), VP]),
        "mg_solve_many": (I, [P(VP), I, P(VP), P(VP), I, I, D, P(mg_stats), P(VP)]),
        "krylov_solve": (I, [VP, I, VP, VP, I, I, D, I, P(mg_stats), VP]),
        "dslash_apply": (I, [VP, I, VP, VP, I, VP]),
        "eo_split": (I, [VP, I, VP, VP, VP, I, VP]),
        "eo_merge": (I, [VP, I, VP, VP, VP, I, VP]),
        "dslash_eo_apply": (I, [VP, I, I, VP, VP, VP, D, D, I, VP]),
        "schur_apply": (I, [VP, I, VP, VP, I, VP]),
        "coarse_apply": (I, [VP, I, I, VP, VP, I, VP]),
        "restrict_apply": (I, [VP, I, I, VP, VP, I, VP]),
        "prolong_apply": (I, [VP, I, I, VP, VP, I, VP]),
        "mr_apply": (I, [VP, I, I, VP, VP, VP, I, VP]),
        "mr_apply_noalloc": (I, [VP, I, I, VP, VP, VP, I, VP]),
        "vcycle_apply": (I, [VP, VP, VP, VP]),
        "mg_field_to_internal": (I, [VP, I, I, VP, I, VP, I, VP]),
        "mg_field_from_internal": (I, [VP, I, I, VP, VP, I, I, VP]),
        "mg_level_info": (I, [VP, I, P(I), P(I), P(I)]),
        "mg_get_prolongator": (I, [VP, I, VP]),
        "mg_get_coarse_op": (I, [VP, I, VP]),
        "mg_get_coarsest_inverse": (I, [VP, VP]),
        "mg_footprint": (ctypes.c_size_t, [P(I), P(mg_params), I]),
        "mg_profile": (I, [VP, ctypes.c_uint]),
        "mg_launch_count": (ctypes.c_ulonglong, []),
        "mg_alloc_count": (ctypes.c_ulonglong, []),
        "mg_trim_cache": (ctypes.c_size_t, []),
        "mg_handle_bytes": (ctypes.c_size_t, [VP]),
        "mg_release_work": (ctypes.c_size_t, [VP, VP]),
        "mg_profile_read": (I, [VP, I, I, P(ctypes.c_longlong), P(D)]),
        "mg_profile_bytes": (I, [VP, I, I, P(D)]),
        "mg_tune": (I, [I]),
        "mg_tune_report": (I, [ctypes.c_char_p, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()

# every entry point declared in include/wilson_mg.h
EXPORTS = ["mg_last_error", "mg_default_params", "mg_setup", "mg_retarget", "mg_destroy", "mg_solve", "dslash_apply",
           "coarse_apply", "restrict_apply", "prolong_apply", "mr_apply", "vcycle_apply", "mg_field_to_internal",
           "mg_field_from_internal", "mg_level_info", "mg_get_prolongator", "mg_get_coarse_op",
           "mg_get_coarsest_inverse", "mg_footprint", "mg_profile", "mg_profile_read", "mg_profile_bytes",
           "mg_launch_count", "mg_alloc_count", "mg_trim_cache", "mg_handle_bytes", "mg_release_work",
           "mr_apply_noalloc", "mg_tune", "mg_tune_report", "krylov_solve", "mg_retarget_batch", "eo_split", "eo_merge", "dslash_eo_apply",
           "schur_apply", "mg_solve_many", "mg_solve_masses"]

(MG_K_DSLASH, MG_K_COARSE, MG_K_RESTRICT, MG_K_PROLONG, MG_K_VECTOR, MG_K_COARSEST, MG_K_SETUP, MG_K_GALERKIN,
 MG_K_INVERSE, MG_K_GRAM) = range(10)
KERNEL_CLASS_NAMES = ["dslash", "coarse", "restrict", "prolong", "vector", "coarsest", "setup", "galerkin", "inverse",
                      "gram"]


def mg_last_error():
    return LIB.mg_last_error().decode()


def _check(status, stats=None):
    if status != MG_OK:
        raise MgError(status, mg_last_error(), stats)


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), 0
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def mg_default_params(**kw):
    p = mg_params()
    _check(LIB.mg_default_params(ctypes.byref(p)))
    for k, v in kw.items():
        if k in ("block",):
            for l, b in enumerate(v):
                for m in range(4):
                    p.block[l][m] = int(b[m])
        elif k in ("nv", "setup_sweeps", "coarse_cycles", "adapt_nv"):
            arr = getattr(p, k)
            for l, x in enumerate(v):
                arr[l] = int(x)
        else:
            setattr(p, k, v)
    return p


class Handle:
    """Owns an mg_handle*; freed by mg_destroy (explicitly or on garbage collection)."""

    def __init__(self, ptr, dims):
        self.ptr = ptr
        self.dims = tuple(dims)

    def __del__(self):
        try:
            if self.ptr:
                LIB.mg_destroy(self.ptr)
        except Exception:
            pass
        self.ptr = None


def mg_setup(gauge, dims, mass, params, starts=None, stream=None):
    """Build the hierarchy.  gauge: (4, Lt, Lz, Ly, Lx, 3, 3) complex128, numpy or CUDA tensor.

    starts: None or a list (one entry per coarsening) of numpy arrays of nv start
    vectors in the external layout of that level (None entries use the
    on-device generator).
    """
    gp, gdev = _ptr(gauge)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    keep = []
    sp = None
    if starts is not None:
        arr = (ctypes.c_void_p * (MG_MAX_LEVELS - 1))()
        for l, s in enumerate(starts):
            if s is None:
                arr[l] = None
            else:
                s = np.ascontiguousarray(s, dtype=np.complex128)
                keep.append(s)
                arr[l] = s.ctypes.data
        sp = ctypes.cast(arr, ctypes.c_void_p)
        keep.append(arr)
    h = ctypes.c_void_p()
    _check(LIB.mg_setup(ctypes.byref(h), gp, gdev, d, float(mass), ctypes.byref(params), sp, _stream(stream)))
    return Handle(h, dims)


def mg_retarget(src, mass, stream=None):
    """New handle for `mass` sharing the null vectors of `src` (coarse operators shifted)."""
    h = ctypes.c_void_p()
    _check(LIB.mg_retarget(src.ptr, float(mass), ctypes.byref(h), _stream(stream)))
    return Handle(h, src.dims)


def mg_retarget_batch(src, masses, stream=None):
    """New handles for several masses at once (one batched elimination builds all coarsest inverses)."""
    n = len(masses)
    ms = (ctypes.c_double * n)(*[float(m) for m in masses])
    hs = (ctypes.c_void_p * n)()
    _check(LIB.mg_retarget_batch(src.ptr, ms, n, hs, _stream(stream)))
    return [Handle(ctypes.c_void_p(hs[i]), src.dims) for i in range(n)]


def mg_destroy(h):
    if h.ptr:
        _check(LIB.mg_destroy(h.ptr))
        h.ptr = None


def mg_solve(h, b, x, tol, stream=None, raise_on_noconv=True):
    """Solve D x = b in place on x.  Returns (status, [stats dict per rhs])."""
    shp = b.shape
    nrhs = 1 if len(shp) == 6 else int(shp[0])
    st = (mg_stats * nrhs)()
    bp, bdev = _ptr(b)
    xp, xdev = _ptr(x)
    if bdev != xdev:
        raise ValueError("b and x must both be host arrays or both device tensors")
    status = LIB.mg_solve(h.ptr, bp, xp, nrhs, bdev, float(tol), st, _stream(stream))
    stats = [s.as_dict() for s in st]
    if status != MG_OK and (status != MG_ENOCONV or raise_on_noconv):
        raise MgError(status, mg_last_error(), stats)
    return status, stats


def mg_solve_many(hs, bs, xs, tol, streams=None, raise_on_noconv=True):
    """Independent solves on distinct handles at once (one host thread and stream each): hs[i] solves
    bs[i] -> xs[i] in place.  streams: None (a stream per solve is made for the call) or one per handle.
    Returns (status, [[stats dict per rhs] per handle])."""
    count = len(hs)
    if not (len(bs) == len(xs) == count) or count < 1:
        raise ValueError("need one b and one x per handle")
    shp = bs[0].shape
    nrhs = 1 if len(shp) == 6 else int(shp[0])
    bp, xp, dev = [], [], set()
    for b, x in zip(bs, xs):
        if b.shape != shp or x.shape != shp:
            raise ValueError("every b and x must have the same shape")
        pb, db = _ptr(b)
        px, dx = _ptr(x)
        bp.append(pb.value)
        xp.append(px.value)
        dev |= {db, dx}
    if len(dev) != 1:
        raise ValueError("b and x must all be host arrays or all device tensors")
    st = (mg_stats * (nrhs * count))()
    sp = None
    if streams is not None:
        sp = (ctypes.c_void_p * count)(*[_stream(q).value for q in streams])
    hp = [h.ptr.value if isinstance(h.ptr, ctypes.c_void_p) else h.ptr for h in hs]
    status = LIB.mg_solve_many((ctypes.c_void_p * count)(*hp), count,
                               (ctypes.c_void_p * count)(*bp), (ctypes.c_void_p * count)(*xp), nrhs, dev.pop(),
                               float(tol), st, sp)
    stats = [[st[i * nrhs + r].as_dict() for r in range(nrhs)] for i in range(count)]
    if status != MG_OK and (status != MG_ENOCONV or raise_on_noconv):
        raise MgError(status, mg_last_error(), stats)
    return status, stats


def mg_solve_masses(h, masses, b, x, tol, stream=None, raise_on_noconv=True):
    """One multi-RHS solve with a mass per right-hand side (masses[r] for b[r]), in place on x.
    Returns (status, [stats dict per rhs])."""
    shp = b.shape
    nrhs = 1 if len(shp) == 6 else int(shp[0])
    if len(masses) != nrhs:
        raise ValueError("one mass per right-hand side")
    ms = (ctypes.c_double * nrhs)(*[float(m) for m in masses])
    st = (mg_stats * nrhs)()
    bp, bdev = _ptr(b)
    xp, xdev = _ptr(x)
    if bdev != xdev:
        raise ValueError("b and x must both be host arrays or both device tensors")
    status = LIB.mg_solve_masses(h.ptr, ms, bp, xp, nrhs, bdev, float(tol), st, _stream(stream))
    stats = [s.as_dict() for s in st]
    if status != MG_OK and (status != MG_ENOCONV or raise_on_noconv):
        raise MgError(status, mg_last_error(), stats)
    return status, stats


MG_KRYLOV_BICGSTAB, MG_KRYLOV_CGNR, MG_KRYLOV_BICGSTAB_EO, MG_KRYLOV_CGNR_EO = 0, 1, 2, 3


def krylov_solve(h, method, b, x, tol, max_iter=100000, stream=None, raise_on_noconv=True):
    """Unpreconditioned BiCGstab or CG-on-the-normal-equations solve (FP64) in place on x, on the full
    system or (the *_EO methods) on its even-odd Schur complement.  Returns (status, [stats dict per rhs])."""
    shp = b.shape
    nrhs = 1 if len(shp) == 6 else int(shp[0])
    st = (mg_stats * nrhs)()
    bp, bdev = _ptr(b)
    xp, xdev = _ptr(x)
    if bdev != xdev:
        raise ValueError("b and x must both be host arrays or both device tensors")
    status = LIB.krylov_solve(h.ptr, int(method), bp, xp, nrhs, bdev, float(tol), int(max_iter), st, _stream(stream))
    stats = [s.as_dict() for s in st]
    if status != MG_OK and (status != MG_ENOCONV or raise_on_noconv):
        raise MgError(status, mg_last_error(), stats)
    return status, stats


def dslash_apply(h, prec, inp, out, nrhs=1, stream=None):
    _check(LIB.dslash_apply(h.ptr, prec, _ptr(inp)[0], _ptr(out)[0], nrhs, _stream(stream)))


def eo_split(h, prec, full, even, odd, nrhs=1, stream=None):
    _check(LIB.eo_split(h.ptr, prec, _ptr(full)[0], _ptr(even)[0], _ptr(odd)[0], nrhs, _stream(stream)))


def eo_merge(h, prec, even, odd, full, nrhs=1, stream=None):
    """full = merge(even, odd); None for a half means zero."""
    ep = _ptr(even)[0] if even is not None else None
    op = _ptr(odd)[0] if odd is not None else None
    _check(LIB.eo_merge(h.ptr, prec, ep, op, _ptr(full)[0], nrhs, _stream(stream)))


def dslash_eo_apply(h, prec, parity_out, x, inp, out, a, b, nrhs=1, stream=None):
    """out = a x + b H_{p,1-p} inp on half fields (x None: no a-term)."""
    xp = _ptr(x)[0] if x is not None else None
    _check(LIB.dslash_eo_apply(h.ptr, prec, int(parity_out), xp, _ptr(inp)[0], _ptr(out)[0], float(a), float(b),
                               nrhs, _stream(stream)))


def schur_apply(h, prec, inp, out, nrhs=1, stream=None):
    _check(LIB.schur_apply(h.ptr, prec, _ptr(inp)[0], _ptr(out)[0], nrhs, _stream(stream)))


def coarse_apply(h, level, prec, inp, out, nrhs=1, stream=None):
    _check(LIB.coarse_apply(h.ptr, level, prec, _ptr(inp)[0], _ptr(out)[0], nrhs, _stream(stream)))


def restrict_apply(h, level, prec, inp, out, nrhs=1, stream=None):
    _check(LIB.restrict_apply(h.ptr, level, prec, _ptr(inp)[0], _ptr(out)[0], nrhs, _stream(stream)))


def prolong_apply(h, level, prec, inp, out, nrhs=1, stream=None):
    _check(LIB.prolong_apply(h.ptr, level, prec, _ptr(inp)[0], _ptr(out)[0], nrhs, _stream(stream)))


def mr_apply(h, level, prec, b, x, r, steps, stream=None):
    _check(LIB.mr_apply(h.ptr, level, prec, _ptr(b)[0], _ptr(x)[0], _ptr(r)[0], steps, _stream(stream)))


def mr_apply_noalloc(h, level, prec, b, x, r, steps, stream=None):
    """mr_apply without device allocation (fixed in-library scratch, see the header)."""
    _check(LIB.mr_apply_noalloc(h.ptr, level, prec, _ptr(b)[0], _ptr(x)[0], _ptr(r)[0], steps, _stream(stream)))


def vcycle_apply(h, r, e, stream=None):
    _check(LIB.vcycle_apply(h.ptr, _ptr(r)[0], _ptr(e)[0], _stream(stream)))


def mg_field_to_internal(h, level, prec, ext, internal, nrhs=1, stream=None):
    ep, edev = _ptr(ext)
    _check(LIB.mg_field_to_internal(h.ptr, level, prec, ep, edev, _ptr(internal)[0], nrhs, _stream(stream)))


def mg_field_from_internal(h, level, prec, internal, ext, nrhs=1, stream=None):
    ep, edev = _ptr(ext)
    _check(LIB.mg_field_from_internal(h.ptr, level, prec, _ptr(internal)[0], ep, edev, nrhs, _stream(stream)))


def mg_level_info(h, level):
    d = (ctypes.c_int * 4)()
    nc = ctypes.c_int()
    nv = ctypes.c_int()
    _check(LIB.mg_level_info(h.ptr, level, d, ctypes.byref(nc), ctypes.byref(nv)))
    return tuple(d), nc.value, nv.value


def mg_get_prolongator(h, level):
    dims, nc, nv = mg_level_info(h, level)
    V = int(np.prod(dims))
    out = np.empty((nv, V, nc), dtype=np.complex128)
    _check(LIB.mg_get_prolongator(h.ptr, level, ctypes.c_void_p(out.ctypes.data)))
    return out


def mg_get_coarse_op(h, level):
    dims, nc, _ = mg_level_info(h, level)
    V = int(np.prod(dims))
    out = np.empty((9, V, nc, nc), dtype=np.complex128)
    _check(LIB.mg_get_coarse_op(h.ptr, level, ctypes.c_void_p(out.ctypes.data)))
    return out


def mg_get_coarsest_inverse(h):
    """Dense inverse of the coarsest operator, [N][N] complex in the external order (site-major,
    component fastest), N = sites x components of the coarsest level."""
    last = 0
    while LIB.mg_level_info(h.ptr, last + 1, (ctypes.c_int * 4)(), ctypes.byref(ctypes.c_int()),
                            ctypes.byref(ctypes.c_int())) == MG_OK:
        last += 1
    dims, nc, _ = mg_level_info(h, last)
    N = int(np.prod(dims)) * nc
    out = np.empty((N, N), dtype=np.complex128)
    _check(LIB.mg_get_coarsest_inverse(h.ptr, ctypes.c_void_p(out.ctypes.data)))
    return out


def mg_footprint(dims, params, nrhs):
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    return int(LIB.mg_footprint(d, ctypes.byref(params), int(nrhs)))


def mg_launch_count():
    return int(LIB.mg_launch_count())


def mg_alloc_count():
    """Device buffers the library has taken since it was loaded (from the driver or its cache)."""
    return int(LIB.mg_alloc_count())


def mg_handle_bytes(h):
    """Device bytes the handle holds now."""
    return int(LIB.mg_handle_bytes(h.ptr))


def mg_release_work(h, stream=None):
    """Hand the handle's solve buffers back to the library's cache (the hierarchy stays); returns the
    bytes released."""
    return int(LIB.mg_release_work(h.ptr, _stream(stream)))


def mg_trim_cache():
    """Hand the library's cached device memory back to the driver; returns the bytes freed."""
    return int(LIB.mg_trim_cache())


def mg_profile(h, mask):
    """Enable the per-launch event profiler of h (h None: default for handles created later)."""
    _check(LIB.mg_profile(h.ptr if h is not None else None, int(mask)))


def mg_profile_read(h, kclass, prec):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(LIB.mg_profile_read(h.ptr, kclass, prec, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def mg_tune(mode):
    """Launch-shape tuner mode (0 off, 1 on, 2 forget and on, 3 / 4 force last / first shape); returns the old mode."""
    r = LIB.mg_tune(int(mode))
    if r < 0:
        raise MgError(MG_EINVAL, "mg_tune: bad mode", None)
    return r


def mg_tune_report():
    """{key: (chosen shape, [microseconds per shape])} of the launch-shape tuner."""
    n = LIB.mg_tune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    LIB.mg_tune_report(buf, n + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        f = line.split()
        out[f[0]] = (int(f[1]), [float(x) for x in f[2:]])
    return out


def mg_profile_bytes(h, kclass, prec):
    b = ctypes.c_double()
    _check(LIB.mg_profile_bytes(h.ptr, kclass, prec, ctypes.byref(b)))
    return b.value


def internal_empty(h, level, prec, nrhs=1, device="cuda", half=False):
    """Allocate an internal-layout field of `level` (torch CUDA tensor); half=True: a level-0 half field
    (the V/2 sites of one parity)."""
    import torch
    dims, nc, _ = mg_level_info(h, level)
    V = int(np.prod(dims)) // (2 if half else 1)
    shape = (nrhs, 3, V, 4) if level == 0 else (nrhs, nc, V)
    if prec == MG_F64:
        return torch.empty(shape, dtype=torch.complex128, device=device)
    if prec == MG_F32:
        return torch.empty(shape, dtype=torch.complex64, device=device)
    dt = torch.float16 if prec == MG_F16 else torch.bfloat16
    return torch.empty(shape + (2,), dtype=dt, device=device)
