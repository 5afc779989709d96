"""CPU oracle for one CheFSI step — test infrastructure, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``sparc_oracle.c`` (plain FP64 loops,
written from the paper's Algorithm 1 and Sec. II) through ctypes and adds the
occupation/density step in numpy.  It shares no code with the CUDA library and
never imports it.

Parity pins (see ``tests/test_oracle_*.py``): exact FD weights and polynomial
exactness, the free-electron closed form, dense brute-force diagonalisation
(periodic and Dirichlet), operator symmetry, the single-projector identity, the
Chebyshev scalar identity, extremal free-electron eigenvalues for Lanczos,
scipy's generalised eigensolver, and convergence of repeated steps to the exact
lowest eigenpairs.  The occupation/density step is pinned by its sum rule and
by the zero-temperature limit.

``oracle/kpoint.py`` holds the complex form of the step at a Bloch wavevector
k (numpy complex128, same restrictions), with its own pins in
``tests/test_oracle_kpoint.py``; ``oracle/forces.py`` the nonlocal
Hellmann-Feynman forces on the atoms (pins in ``tests/test_oracle_forces.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsparc_oracle.so")

OK, ERR_ARG, ERR_NOT_SPD, ERR_NUMERIC = 0, 1, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C99, -O2, OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.or_create.restype = ctypes.c_void_p
        L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip,
                                _dp, ctypes.c_int, _lp, _ip, _ip, _lp, _dp, _lp, _dp]
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_fd_weights.argtypes = [ctypes.c_int, _dp]
        L.or_hpsi.argtypes = [ctypes.c_void_p, _dp, ctypes.c_long, _dp, ctypes.c_long,
                              ctypes.c_int]
        L.or_cheb_filter.restype = ctypes.c_int
        L.or_cheb_filter.argtypes = [ctypes.c_void_p, _dp, ctypes.c_long, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double]
        L.or_uniform.restype = ctypes.c_double
        L.or_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_lanczos.restype = ctypes.c_int
        L.or_lanczos.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, _dp, _dp, _dp,
                                 _dp, _dp]
        L.or_project.argtypes = [_dp, ctypes.c_long, _dp, ctypes.c_long, ctypes.c_long,
                                 ctypes.c_int, _dp, _dp]
        L.or_cholesky.restype = ctypes.c_int
        L.or_cholesky.argtypes = [ctypes.c_int, _dp, _dp]
        L.or_householder_tridiag.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_tridiag_qr.restype = ctypes.c_int
        L.or_tridiag_qr.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
        L.or_sym_eig.restype = ctypes.c_int
        L.or_sym_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        L.or_gen_eig.restype = ctypes.c_int
        L.or_gen_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_rotate.argtypes = [_dp, ctypes.c_long, ctypes.c_long, ctypes.c_int, _dp, _dp,
                                ctypes.c_long]
        L.or_chefsi_step.restype = ctypes.c_int
        L.or_chefsi_step.argtypes = [ctypes.c_void_p, _dp, ctypes.c_long, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _dp]
        _lib = L
    return _lib


def _p(a, ct=_dp):
    return a.ctypes.data_as(ct)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def fd_weights(radius: int = 6) -> np.ndarray:
    w = np.zeros(radius + 1)
    lib().or_fd_weights(radius, _p(w))
    return w


def uniform(seed: int, i: int) -> float:
    """Counter-based splitmix64 uniform in [0, 1): value i of stream seed."""
    return lib().or_uniform(seed, i)


class Oracle:
    """FP64 CPU reference bound to one synthetic system (see paper Sec. II A)."""

    def __init__(self, system):
        self.system = system
        s = system
        self._keep = [np.ascontiguousarray(a) for a in (
            np.array(s.bc, np.int32), s.veff.astype(np.float64), s.supp_ptr.astype(np.int64),
            s.supp_idx.astype(np.int32), s.nproj.astype(np.int32), s.chi_ptr.astype(np.int64),
            s.chi.astype(np.float64), s.proj_ptr.astype(np.int64), s.gamma.astype(np.float64))]
        bc, veff, sp, si, npj, cp, chi, pp, gam = self._keep
        self._h = lib().or_create(s.nx, s.ny, s.nz, s.h, _p(bc, _ip), _p(veff), s.natoms,
                                  _p(sp, _lp), _p(si, _ip), _p(npj, _ip), _p(cp, _lp), _p(chi),
                                  _p(pp, _lp), _p(gam))
        self.nd = s.nd

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operator ---------------------------------------------------------
    def hpsi(self, X: np.ndarray) -> np.ndarray:
        """Y = H X for X of shape (ns, ld) (column-major Nd x Ns block)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.ndim == 1:
            X = X[None, :]
        ns, ld = X.shape
        Y = np.zeros((ns, self.nd))
        lib().or_hpsi(self._h, _p(X), ld, _p(Y), self.nd, ns)
        return Y

    def cheb_filter(self, X, degree, a, b, a0):
        X = np.array(X, dtype=np.float64, copy=True, order="C")
        ns, ld = X.shape
        st = lib().or_cheb_filter(self._h, _p(X), ld, ns, degree, a, b, a0)
        if st:
            raise OracleError(st, "cheb_filter")
        return X

    def lanczos(self, k, seed):
        """Returns (a0, b, alpha, beta): a0 = theta_min, b = theta_max + |beta_k|."""
        al, bt = np.zeros(k), np.zeros(k)
        tmin, tmax, bup = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = lib().or_lanczos(self._h, k, seed, _p(al), _p(bt), ctypes.byref(tmin),
                              ctypes.byref(tmax), ctypes.byref(bup))
        if st:
            raise OracleError(st, "lanczos")
        return tmin.value, bup.value, al, bt, tmax.value

    def chefsi_step(self, X, degree, a, b, a0):
        """One CheFSI step (Algorithm 1). Returns (X_new, ritz_values)."""
        X = np.array(X, dtype=np.float64, copy=True, order="C")
        ns, ld = X.shape
        lam = np.zeros(ns)
        st = lib().or_chefsi_step(self._h, _p(X), ld, ns, degree, a, b, a0, _p(lam))
        if st:
            raise OracleError(st, "chefsi_step")
        return X, lam


# -- dense pieces of the Rayleigh-Ritz step --------------------------------
def project(Xt: np.ndarray, Yt: np.ndarray, nd: int):
    """Hs = Xt^T Yt, Ms = Xt^T Xt (Algorithm 1, projection); inputs (ns, ld)."""
    Xt = np.ascontiguousarray(Xt, dtype=np.float64)
    Yt = np.ascontiguousarray(Yt, dtype=np.float64)
    ns = Xt.shape[0]
    Hs, Ms = np.zeros((ns, ns)), np.zeros((ns, ns))
    lib().or_project(_p(Xt), Xt.shape[1], _p(Yt), Yt.shape[1], nd, ns, _p(Hs), _p(Ms))
    # column-major ns x ns buffers -> return as ordinary (row, col) matrices
    return Hs.T.copy(), Ms.T.copy()


def cholesky(M: np.ndarray) -> np.ndarray:
    n = M.shape[0]
    Mf = np.asfortranarray(M, dtype=np.float64)
    L = np.zeros((n, n), order="F")
    st = lib().or_cholesky(n, Mf.ctypes.data_as(_dp), L.ctypes.data_as(_dp))
    if st:
        raise OracleError(st, "cholesky")
    return np.array(L)


def householder_tridiag(A: np.ndarray):
    n = A.shape[0]
    Af = np.asfortranarray(A, dtype=np.float64)
    d, e = np.zeros(n), np.zeros(max(n - 1, 1))
    Q = np.zeros((n, n), order="F")
    lib().or_householder_tridiag(n, Af.ctypes.data_as(_dp), _p(d), _p(e),
                                 Q.ctypes.data_as(_dp))
    return d, e[: n - 1], np.array(Q)


def tridiag_eigvals(d, e):
    d = np.array(d, dtype=np.float64)
    n = d.size
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = e
    st = lib().or_tridiag_qr(n, _p(d), _p(ee), None, 0, 0)
    if st:
        raise OracleError(st, "tridiag_qr")
    return np.sort(d)


def sym_eig(A: np.ndarray):
    n = A.shape[0]
    Af = np.asfortranarray(A, dtype=np.float64)
    lam = np.zeros(n)
    V = np.zeros((n, n), order="F")
    st = lib().or_sym_eig(n, Af.ctypes.data_as(_dp), _p(lam), V.ctypes.data_as(_dp))
    if st:
        raise OracleError(st, "sym_eig")
    return lam, np.array(V)


def gen_eig(Hs: np.ndarray, Ms: np.ndarray):
    """Hs Z = Ms Z D with Z^T Ms Z = I (Algorithm 1, diagonalisation)."""
    n = Hs.shape[0]
    Hf = np.asfortranarray(Hs, dtype=np.float64)
    Mf = np.asfortranarray(Ms, dtype=np.float64)
    lam = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    st = lib().or_gen_eig(n, Hf.ctypes.data_as(_dp), Mf.ctypes.data_as(_dp), _p(lam),
                          Z.ctypes.data_as(_dp))
    if st:
        raise OracleError(st, "gen_eig")
    return lam, np.array(Z)


def rotate(Xt: np.ndarray, Z: np.ndarray, nd: int) -> np.ndarray:
    """X = Xt Z (Algorithm 1, rotation); Xt of shape (ns, ld), Z an ns x ns matrix."""
    Xt = np.ascontiguousarray(Xt, dtype=np.float64)
    ns, ld = Xt.shape
    Zf = np.asfortranarray(Z, dtype=np.float64)
    out = np.zeros((ns, nd))
    lib().or_rotate(_p(Xt), ld, nd, ns, Zf.ctypes.data_as(_dp), _p(out), nd)
    return out


# -- occupations and density (metric for the mixed-precision comparison) ---
def fermi_occupations(lam: np.ndarray, ne: float, kT: float = 0.01, tol: float = 1e-12):
    """Fermi-Dirac f_n = 1/(1 + exp((lam_n - mu)/kT)), mu by bisection so that
    2 sum f_n = Ne.  Returns (f, mu)."""
    lam = np.asarray(lam, dtype=np.float64)

    def count(mu):
        t = np.clip((lam - mu) / kT, -700.0, 700.0)
        return 2.0 * np.sum(1.0 / (1.0 + np.exp(t)))

    lo, hi = lam.min() - 1.0, lam.max() + 1.0
    mu = 0.5 * (lo + hi)
    for _ in range(400):
        mu = 0.5 * (lo + hi)
        c = count(mu)
        if abs(c - ne) < tol:
            break
        if c < ne:
            lo = mu
        else:
            hi = mu
    t = np.clip((lam - mu) / kT, -700.0, 700.0)
    return 1.0 / (1.0 + np.exp(t)), mu


def density(X: np.ndarray, f: np.ndarray, nd: int, h: float) -> np.ndarray:
    """rho_i = 2 sum_n f_n X_{i n}^2 / h^3 for X of shape (ns, ld)."""
    X = np.asarray(X)[:, :nd]
    return 2.0 * np.einsum("n,ni->i", f, X * X) / h ** 3
