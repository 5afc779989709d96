"""Thin Python binding of libsparc.so (C ABI in include/sparc.h).

Argument marshalling only: every step of the CheFSI path runs in the CUDA
library.  The functions carry the C names (sparc_create, sparc_hpsi, ...);
`Handle` wraps them for convenience.  Orbital blocks are torch CUDA tensors
(or, where the C call allows host memory, numpy arrays) of shape (ns, ld):
row n of the array is orbital column n of the column-major Nd x Ns block.
Ns x Ns matrices are column-major on the C side; as (ns, ns) tensors they
are the transposes (symmetric Hs and Ms are unaffected; Z is returned as
its proper orientation).

If the library cannot be built or loaded this module raises at import of the
library (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SPARC_OK = 0
SPARC_ERR_INVALID_ARG = 1
SPARC_ERR_CUDA = 2
SPARC_ERR_OOM = 3
SPARC_ERR_NOT_SPD = 4
SPARC_ERR_NUMERIC = 5
SPARC_ERR_TIMEOUT = 6
SPARC_PERIODIC, SPARC_DIRICHLET = 0, 1
SPARC_F64, SPARC_F32, SPARC_C128 = 0, 1, 2
SPARC_PREC_FP64, SPARC_PREC_MIXED = 0, 1

_STATUS = {1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_SPD", 5: "NUMERIC", 6: "TIMEOUT"}


class SparcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"SPARC_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sparc_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("bc", ctypes.c_int * 3)]


class sparc_nonlocal(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("supp_ptr", ctypes.c_void_p),
                ("supp_idx", ctypes.c_void_p), ("nproj", ctypes.c_void_p),
                ("chi_ptr", ctypes.c_void_p), ("chi", ctypes.c_void_p),
                ("proj_ptr", ctypes.c_void_p), ("gamma", ctypes.c_void_p)]


class sparc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("ns_max", ctypes.c_int), ("device", ctypes.c_int),
                ("flags", ctypes.c_int), ("stencil_shape", ctypes.c_int),
                ("reserved", ctypes.c_int), ("timeout_cycles", ctypes.c_int64)]


class sparc_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("shape", "rows_per_thread", "planes_per_step", "slab_rows", "threads", "ns",
                 "candidates")] + [("candidate_ms", ctypes.c_float * 8)]


class sparc_timings(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("bounds_ms", "filter_ms", "hx_ms", "project_ms", "eig_ms", "rotate_ms",
                 "total_ms")] + [("launches", ctypes.c_int64)] + [
        (n, ctypes.c_float) for n in ("stage_in_ms", "stage_out_ms", "host_ms", "stencil_ms",
                                      "nonlocal_ms")] + [("stencil_launches", ctypes.c_int32)]


EXPORTS = ["sparc_create", "sparc_destroy", "sparc_last_error", "sparc_hpsi",
           "sparc_spectrum_bounds", "sparc_cheb_filter", "sparc_project", "sparc_subspace_eig",
           "sparc_rotate", "sparc_chefsi_step", "sparc_get_timings", "sparc_project_noalloc",
           "sparc_occupations", "sparc_density", "sparc_nonlocal_forces",
           "sparc_batch_create", "sparc_batch_destroy", "sparc_batch_last_error",
           "sparc_batch_chefsi_step", "sparc_batch_get_info", "sparc_get_tuning",
           "sparc_create_kpoint", "sparc_batch_subspace_eig"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) libsparc.so; raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsparc.so not found at {path}")
    L = ctypes.CDLL(path)
    vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.sparc_create.argtypes = [ctypes.POINTER(sparc_grid), vp, ctypes.POINTER(sparc_nonlocal),
                               ctypes.POINTER(sparc_options), ctypes.POINTER(vp)]
    L.sparc_create_kpoint.argtypes = [ctypes.POINTER(sparc_grid), vp,
                                      ctypes.POINTER(sparc_nonlocal), vp,
                                      ctypes.POINTER(sparc_options), vp, ctypes.POINTER(vp)]
    L.sparc_destroy.argtypes = [vp]
    L.sparc_last_error.argtypes = [vp]
    L.sparc_last_error.restype = ctypes.c_char_p
    L.sparc_hpsi.argtypes = [vp, vp, vp, i, i64, i, vp]
    L.sparc_spectrum_bounds.argtypes = [vp, i, ctypes.c_uint64, ctypes.POINTER(d),
                                        ctypes.POINTER(d), vp]
    L.sparc_cheb_filter.argtypes = [vp, vp, i, i64, i, i, d, d, d, vp]
    L.sparc_project.argtypes = [vp, vp, vp, i, i64, i, vp, vp, vp]
    L.sparc_subspace_eig.argtypes = [vp, vp, vp, i, vp, vp, vp]
    L.sparc_rotate.argtypes = [vp, vp, vp, vp, i, i64, i, vp]
    L.sparc_chefsi_step.argtypes = [vp, vp, i, i64, i, i, vp, vp, i, vp]
    L.sparc_get_timings.argtypes = [vp, ctypes.POINTER(sparc_timings)]
    L.sparc_get_tuning.argtypes = [vp, ctypes.POINTER(sparc_tuning)]
    L.sparc_project_noalloc.argtypes = [vp, vp, i, i64, i64, vp, vp, vp]
    L.sparc_occupations.argtypes = [vp, vp, i, d, d, vp, vp, vp]
    L.sparc_density.argtypes = [vp, vp, i, i64, i, vp, vp, vp]
    L.sparc_nonlocal_forces.argtypes = [vp, vp, i, i64, i, vp, vp, vp]
    L.sparc_batch_create.argtypes = [vp, i, ctypes.POINTER(vp)]
    L.sparc_batch_destroy.argtypes = [vp]
    L.sparc_batch_last_error.argtypes = [vp]
    L.sparc_batch_last_error.restype = ctypes.c_char_p
    L.sparc_batch_chefsi_step.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, vp]
    L.sparc_batch_get_info.argtypes = [vp, ctypes.POINTER(i64)]
    L.sparc_batch_subspace_eig.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("sparc_last_error", "sparc_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(h, rc):
    if rc != SPARC_OK:
        msg = load().sparc_last_error(h)
        raise SparcError(rc, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _block(X):
    """(pointer, ns, ld, dtype) of an (ns, ld) tensor or numpy array."""
    if isinstance(X, np.ndarray):
        if not X.flags.c_contiguous:
            raise ValueError("orbital block must be C-contiguous (ns, ld)")
        dt = SPARC_F64 if X.dtype == np.float64 else SPARC_F32 if X.dtype == np.float32 else None
        ptr = X.ctypes.data
    else:
        import torch
        if X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("orbital block must be a (ns, ld) tensor with unit inner stride")
        dt = {torch.float64: SPARC_F64, torch.float32: SPARC_F32,
              torch.complex128: SPARC_C128}.get(X.dtype)
        ptr = X.data_ptr()
        return ptr, X.shape[0], X.stride(0), dt
    if dt is None:
        raise ValueError("orbital blocks must be float64 or float32")
    return ptr, X.shape[0], X.shape[1], dt


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# -- C-named functions -------------------------------------------------------
def sparc_create(system, precision: int = SPARC_PREC_FP64, ns_max: int = 1, device: int = 0,
                 flags: int = 0, stencil_shape: int = 0, timeout_cycles: int = 0, kvec=None):
    """Create a handle for a `synth.System`-like object (grid, Veff, projectors).
    flags, stencil_shape and timeout_cycles are the sparc_options fields of the
    same names (flags bit 0 selects the generic stencil form).  With `kvec`
    (three components, 1/bohr) the handle is H(k) at that Bloch wavevector
    (sparc_create_kpoint; complex blocks)."""
    L = load()
    g = sparc_grid(system.nx, system.ny, system.nz, system.h, (ctypes.c_int * 3)(*system.bc))
    keep = [_arr(system.veff, np.float64), _arr(system.supp_ptr, np.int64),
            _arr(system.supp_idx, np.int32), _arr(system.nproj, np.int32),
            _arr(system.chi_ptr, np.int64), _arr(system.chi, np.float64),
            _arr(system.proj_ptr, np.int64), _arr(system.gamma, np.float64)]
    veff, sp, si, npj, cp, chi, pp, gam = keep
    nl = sparc_nonlocal(int(system.natoms), sp.ctypes.data, si.ctypes.data, npj.ctypes.data,
                        cp.ctypes.data, chi.ctypes.data, pp.ctypes.data, gam.ctypes.data)
    opt = sparc_options(precision, ns_max, device, flags, stencil_shape, 0, timeout_cycles)
    out = ctypes.c_void_p()
    if kvec is not None:
        pos = _arr(np.asarray(system.positions).reshape(-1, 3) if system.natoms else
                   np.zeros((1, 3)), np.float64)
        kv = _arr(kvec, np.float64).reshape(3)
        keep += [pos, kv]
        rc = L.sparc_create_kpoint(ctypes.byref(g), veff.ctypes.data, ctypes.byref(nl),
                                   pos.ctypes.data, ctypes.byref(opt), kv.ctypes.data,
                                   ctypes.byref(out))
    else:
        rc = L.sparc_create(ctypes.byref(g), veff.ctypes.data, ctypes.byref(nl),
                            ctypes.byref(opt), ctypes.byref(out))
    _check(None, rc)
    return out


def sparc_destroy(h):
    load().sparc_destroy(h)


def sparc_hpsi(h, X, Y, stream=None):
    px, ns, ld, dt = _block(X)
    py, ns2, ld2, dt2 = _block(Y)
    if (ns2, ld2, dt2) != (ns, ld, dt):
        raise ValueError("X and Y must have the same shape and dtype")
    _check(h, load().sparc_hpsi(h, px, py, ns, ld, dt, _stream(stream)))
    return Y


def sparc_spectrum_bounds(h, iters=32, seed=0, stream=None):
    a0, b = ctypes.c_double(), ctypes.c_double()
    _check(h, load().sparc_spectrum_bounds(h, iters, seed, ctypes.byref(a0), ctypes.byref(b),
                                           _stream(stream)))
    return a0.value, b.value


def sparc_cheb_filter(h, X, degree, a, b, a0, stream=None):
    px, ns, ld, dt = _block(X)
    _check(h, load().sparc_cheb_filter(h, px, ns, ld, dt, degree, a, b, a0, _stream(stream)))
    return X


def sparc_project(h, Xt, Yt, Hs, Ms, stream=None):
    px, ns, ld, dt = _block(Xt)
    py, *_ = _block(Yt)
    _check(h, load().sparc_project(h, px, py, ns, ld, dt, Hs.data_ptr(), Ms.data_ptr(),
                                   _stream(stream)))
    return Hs, Ms


def sparc_subspace_eig(h, Hs, Ms, lam, Zt, stream=None):
    ns = Hs.shape[0]
    _check(h, load().sparc_subspace_eig(h, Hs.data_ptr(), Ms.data_ptr(), ns, lam.data_ptr(),
                                        Zt.data_ptr(), _stream(stream)))
    return lam, Zt


def sparc_rotate(h, Xt, Xout, Zt, stream=None):
    px, ns, ld, dt = _block(Xt)
    po, *_ = _block(Xout)
    _check(h, load().sparc_rotate(h, px, po, Zt.data_ptr(), ns, ld, dt, _stream(stream)))
    return Xout


def sparc_chefsi_step(h, X, degree, bounds=None, eig=None, stream=None):
    """One CheFSI step; returns the Ritz values (numpy on the host, or the
    given device tensor `eig`, which then receives them on the device)."""
    px, ns, ld, dt = _block(X)
    eig = np.zeros(ns) if eig is None else eig
    on_host = isinstance(eig, np.ndarray)
    eptr = eig.ctypes.data if on_host else eig.data_ptr()
    bptr = None
    if bounds is not None:
        bb = (ctypes.c_double * 3)(*bounds)
        bptr = ctypes.cast(bb, ctypes.c_void_p)
    _check(h, load().sparc_chefsi_step(h, px, ns, ld, dt, degree, bptr, eptr, int(on_host),
                                       _stream(stream) if not isinstance(X, np.ndarray) else
                                       ctypes.c_void_p(0)))
    return eig


def sparc_occupations(h, lam, ne, kT, occ, mu, stream=None):
    """Fermi-Dirac occupations of device Ritz values `lam` into `occ`; the
    Fermi level goes to the one-element device tensor `mu`."""
    _check(h, load().sparc_occupations(h, lam.data_ptr(), lam.numel(), ctypes.c_double(ne),
                                       ctypes.c_double(kT), occ.data_ptr(), mu.data_ptr(),
                                       _stream(stream)))
    return occ, mu


def sparc_density(h, X, occ, rho, stream=None):
    px, ns, ld, dt = _block(X)
    _check(h, load().sparc_density(h, px, ns, ld, dt, occ.data_ptr(), rho.data_ptr(),
                                   _stream(stream)))
    return rho


def sparc_nonlocal_forces(h, X, occ, F, stream=None):
    """Nonlocal forces of the block X with occupations `occ` into the device
    tensor F (natoms x 3 doubles)."""
    px, ns, ld, dt = _block(X)
    _check(h, load().sparc_nonlocal_forces(h, px, ns, ld, dt, occ.data_ptr(), F.data_ptr(),
                                           _stream(stream)))
    return F


def sparc_get_timings(h):
    t = sparc_timings()
    _check(h, load().sparc_get_timings(h, ctypes.byref(t)))
    return {n: getattr(t, n) for n, _ in sparc_timings._fields_}


def sparc_get_tuning(h):
    t = sparc_tuning()
    _check(h, load().sparc_get_tuning(h, ctypes.byref(t)))
    d = {n: getattr(t, n) for n, _ in sparc_tuning._fields_ if n != "candidate_ms"}
    d["candidate_ms"] = list(t.candidate_ms)[: t.candidates]
    return d


class Handle:
    """Convenience wrapper owning one sparc_handle."""

    def __init__(self, system, precision="fp64", ns_max=1, device=0, options_flags=0,
                 stencil_shape=0, timeout_cycles=0, kvec=None):
        prec = SPARC_PREC_MIXED if precision == "mixed" else SPARC_PREC_FP64
        self.system = system
        self.precision = precision
        self.ns_max = ns_max
        self.kvec = kvec
        self.h = sparc_create(system, prec, ns_max, device, options_flags, stencil_shape,
                              timeout_cycles, kvec)

    @property
    def dtype(self):
        import torch
        if self.kvec is not None:
            return torch.complex128
        return torch.float32 if self.precision == "mixed" else torch.float64

    def close(self):
        if self.h:
            sparc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hpsi(self, X, Y=None, stream=None):
        import torch
        Y = torch.empty_like(X) if Y is None else Y
        return sparc_hpsi(self.h, X, Y, stream)

    def spectrum_bounds(self, iters=32, seed=0, stream=None):
        return sparc_spectrum_bounds(self.h, iters, seed, stream)

    def cheb_filter(self, X, degree, a, b, a0, stream=None):
        return sparc_cheb_filter(self.h, X, degree, a, b, a0, stream)

    def project(self, Xt, Yt, stream=None):
        """(Hs, Ms).  Real handles: the column-major results as (ns, ns) tensors
        (symmetric, so their orientation does not matter).  k-point handles:
        the complex Hermitian matrices in their proper orientation."""
        import torch
        ns = Xt.shape[0]
        dt = torch.complex128 if self.kvec is not None else torch.float64
        Hs = torch.empty((ns, ns), dtype=dt, device=Xt.device)
        Ms = torch.empty((ns, ns), dtype=dt, device=Xt.device)
        sparc_project(self.h, Xt, Yt, Hs, Ms, stream)
        if self.kvec is not None:
            return Hs.t(), Ms.t()
        return Hs, Ms

    def subspace_eig(self, Hs, Ms, stream=None):
        """Returns (lam, Z) with Z an ordinary (row, col) matrix."""
        import torch
        ns = Hs.shape[0]
        lam = torch.empty(ns, dtype=torch.float64, device=Hs.device)
        Zt = torch.empty((ns, ns), dtype=Hs.dtype, device=Hs.device)
        # column-major storage of a matrix is the row-major storage of its transpose
        sparc_subspace_eig(self.h, Hs.t().contiguous(), Ms.t().contiguous(), lam, Zt, stream)
        return lam, Zt.t()

    def rotate(self, Xt, Z, Xout=None, stream=None):
        import torch
        Xout = torch.empty_like(Xt) if Xout is None else Xout
        Zt = Z.t().contiguous()  # column-major ns x ns
        return sparc_rotate(self.h, Xt, Xout, Zt, stream)

    def chefsi_step(self, X, degree, bounds=None, stream=None, eig=None):
        return sparc_chefsi_step(self.h, X, degree, bounds, eig, stream)

    def occupations(self, lam, ne, kT=0.01, stream=None):
        """(occ, mu) as device tensors for device Ritz values `lam`."""
        import torch
        if not torch.is_tensor(lam):
            lam = torch.as_tensor(np.asarray(lam, dtype=np.float64), device="cuda")
        lam = lam.to(torch.float64).contiguous()
        occ = torch.empty_like(lam)
        mu = torch.empty(1, dtype=torch.float64, device=lam.device)
        return sparc_occupations(self.h, lam, ne, kT, occ, mu, stream)

    def density(self, X, occ, stream=None):
        """rho (device, Nd doubles) of the block X with occupations `occ`."""
        import torch
        rho = torch.empty(self.system.nd, dtype=torch.float64, device=X.device)
        return sparc_density(self.h, X, occ, rho, stream)

    def nonlocal_forces(self, X, occ, stream=None):
        """F (device, natoms x 3 doubles, Ha/bohr) of the block X with occupations `occ`."""
        import torch
        F = torch.zeros((max(self.system.natoms, 1), 3), dtype=torch.float64, device=X.device)
        sparc_nonlocal_forces(self.h, X, occ, F, stream)
        return F[: self.system.natoms]

    def timings(self):
        return sparc_get_timings(self.h)

    def tuning(self):
        return sparc_get_tuning(self.h)


class Batch:
    """A batch of handles stepped together (sparc_batch_* calls)."""

    def __init__(self, handles):
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        out = ctypes.c_void_p()
        rc = load().sparc_batch_create(arr, len(self.handles), ctypes.byref(out))
        _check(None, rc)
        self.b = out

    def close(self):
        if self.b:
            load().sparc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def chefsi_step(self, Xs, degrees, bounds=None, stream=None):
        """One batched step; Xs: list of (ns_i, ld_i) tensors; returns Ritz values."""
        L = load()
        n = len(Xs)
        blocks = [_block(X) for X in Xs]
        dt = blocks[0][3]
        ptrs = (ctypes.c_void_p * n)(*[b[0] for b in blocks])
        nss = (ctypes.c_int * n)(*[b[1] for b in blocks])
        lds = (ctypes.c_int64 * n)(*[b[2] for b in blocks])
        degs = (ctypes.c_int * n)(*degrees)
        eigs = [np.zeros(b[1]) for b in blocks]
        eptr = (ctypes.c_void_p * n)(*[e.ctypes.data for e in eigs])
        bptr = None
        if bounds is not None:
            flat = (ctypes.c_double * (3 * n))(*[v for t in bounds for v in t])
            bptr = ctypes.cast(flat, ctypes.c_void_p)
        rc = L.sparc_batch_chefsi_step(self.b, ptrs, nss, lds, dt, degs, bptr, eptr,
                                       _stream(stream))
        if rc != SPARC_OK:
            raise SparcError(rc, L.sparc_batch_last_error(self.b).decode())
        return eigs

    def subspace_eig(self, Hs, Ms, stream=None):
        """sparc_batch_subspace_eig on lists of device (n_i, n_i) FP64 tensors;
        returns (lams, Zs), each Z an ordinary (row, col) matrix."""
        import torch
        L = load()
        n = len(Hs)
        sizes = [int(H.shape[0]) for H in Hs]
        Hc = [H.t().contiguous() for H in Hs]  # column-major storage of H
        Mc = [M.t().contiguous() for M in Ms]
        lam = [torch.empty(k, dtype=torch.float64, device=H.device) for k, H in zip(sizes, Hs)]
        Zc = [torch.empty((k, k), dtype=torch.float64, device=H.device) for k, H in zip(sizes, Hs)]
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])  # noqa: E731
        rc = L.sparc_batch_subspace_eig(self.b, arr(Hc), arr(Mc), (ctypes.c_int * n)(*sizes),
                                        arr(lam), arr(Zc), _stream(stream))
        if rc != SPARC_OK:
            raise SparcError(rc, L.sparc_batch_last_error(self.b).decode())
        return lam, [z.t() for z in Zc]

    def launches(self):
        v = ctypes.c_int64()
        _check(None, load().sparc_batch_get_info(self.b, ctypes.byref(v)))
        return v.value
