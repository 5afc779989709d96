"""Complex (Bloch wavevector) form of the CheFSI step — test infrastructure,
not product code.

Only ``tests/`` may import this module; it never imports the CUDA library.

The paper computes in real arithmetic at the Gamma point only. At any other
Bloch wavevector k of the Brillouin-zone sampling every operation is complex,
all in FP64 (Sec. III, introduction; the TiO2 slabs of Sec. IV use
Monkhorst-Pack grids). This module is the plain definition of that step for one
wavevector, in numpy complex128. The real oracle supplies two pieces, pinned on
their own: the exact FD weights and the real symmetric eigensolver.

Operator H(k) on grid values psi_i, with the Bloch condition
psi(r + L_d e_d) = exp(i k_d L_d) psi(r) on periodic axes (L_d = N_d h):

* Laplacian: the radius-6 central weights along each axis. A neighbour index
  j = i +- p is read at j mod N_d. On a periodic axis it is multiplied by
  exp(i k_d L_d q), with q = floor(j / N_d) the number of cell crossings.
  On a Dirichlet axis an index outside [0, N_d) reads 0, and k_d is ignored.
* Veff: the diagonal.
* Nonlocal: sum_J sum_lm gamma_Jl h^3 |chi^k_Jlm><chi^k_Jlm|.
  - The Bloch sum is chi^k_Jlm(r_i) = sum_T chi_Jlm(r_i - R_J - T) exp(i k.T).
  - With a cut-off below half of every periodic cell length, one image T_i
    contributes at each support point. That image is the one nearest r_i,
    T_i = L_d round((x_i - R_Jd) / L_d) per periodic axis.
  - So chi^k(r_i) = chi(d_i) exp(i k.T_i), with d_i = r_i - R_J - T_i the
    minimum-image displacement at which the tabulated value was taken.

The Rayleigh-Ritz step is Algorithm 1's, with ^T replaced by ^H.
Hs = Xt^H Yt and Ms = Xt^H Xt are Hermitian. The eigenproblem Hs Z = Ms Z Lam,
with Z^H Ms Z = I, is solved by these steps:
  1. Cholesky Ms = L L^H.
  2. A = L^-1 Hs L^-H.
  3. Householder tridiagonalisation T = Q^H A Q.
  4. A diagonal unitary D makes T's sub-diagonal real and nonnegative.
  5. The real oracle's symmetric eigensolver diagonalises D^H T D.
  6. Back-transformation Z = L^-H Q D V.

Pins (``tests/test_oracle_kpoint.py``):
* the free-electron closed form at any k, per plane wave and as a full dense
  spectrum;
* an independently assembled dense H(k): Kronecker sums of 1-D Bloch
  matrices, plus projectors rebuilt from their analytic form by an explicit
  sum over the 27 nearest images;
* the supercell identity: a real 3x supercell's spectrum is the union of
  H(k) over the three commensurate k;
* Hermiticity and time reversal, H(-k) = conj(H(k));
* k = 0 against the real oracle;
* the complex Cholesky, Householder and generalised eigensolver against
  numpy/scipy, including degenerate and ill-conditioned overlaps;
* the step's Ritz values against dense Rayleigh-Ritz on the filtered span;
* convergence of repeated steps to brute-force eigenvalues.
"""
from __future__ import annotations

import numpy as np

from . import OracleError, ERR_NOT_SPD, fd_weights, sym_eig, tridiag_eigvals, uniform

PERIODIC = 0


class KOracle:
    """H(k) and the complex CheFSI step for one system and one wavevector k
    (three components in 1/bohr; components on Dirichlet axes are ignored)."""

    def __init__(self, system, k):
        s = system
        self.system = s
        self.k = np.asarray(k, dtype=np.float64).reshape(3)
        self.nd = s.nd
        self.h = s.h
        self.w = fd_weights(6)
        self.dims = (s.nx, s.ny, s.nz)
        self.lengths = np.array(self.dims, dtype=np.float64) * s.h
        self.atoms = []
        nx, ny, nz = self.dims
        for J in range(s.natoms):
            lo, hi = int(s.supp_ptr[J]), int(s.supp_ptr[J + 1])
            idx = s.supp_idx[lo:hi].astype(np.int64)
            nproj = int(s.nproj[J])
            # column-major n_supp x nproj block: entry (i, p) at p * n_supp + i
            chi = s.chi[int(s.chi_ptr[J]):int(s.chi_ptr[J + 1])].reshape(nproj, hi - lo).T
            gam = s.gamma[int(s.proj_ptr[J]):int(s.proj_ptr[J + 1])]
            coords = (idx % nx, (idx // nx) % ny, idx // (nx * ny))
            T = np.zeros((idx.size, 3))
            for d in range(3):
                if s.bc[d] == PERIODIC:
                    x = coords[d] * s.h - s.positions[J, d]
                    T[:, d] = self.lengths[d] * np.round(x / self.lengths[d])
            phase = np.exp(1j * (T @ self.k))
            self.atoms.append((idx, chi * phase[:, None], gam))

    # -- operator ---------------------------------------------------------
    def _neighbour(self, G, axis, d, shift):
        """G shifted by `shift` points along grid axis d (array axis `axis`)
        with the Bloch phase or the Dirichlet zero for indices outside."""
        n = self.dims[d]
        j = np.arange(n) + shift
        q = np.floor_divide(j, n)
        if self.system.bc[d] == PERIODIC:
            f = np.exp(1j * self.k[d] * self.lengths[d] * q)
        else:
            f = (q == 0).astype(np.float64)
        shape = [1] * G.ndim
        shape[axis] = n
        return np.take(G, np.mod(j, n), axis=axis) * f.reshape(shape)

    def hpsi(self, X):
        """Y = H(k) X for X of shape (ns, ld) (one orbital per row)."""
        X = np.asarray(X, dtype=np.complex128)
        if X.ndim == 1:
            X = X[None, :]
        ns = X.shape[0]
        nx, ny, nz = self.dims
        G = X[:, : self.nd].reshape(ns, nz, ny, nx)
        Y = np.zeros_like(G)
        for d, axis in ((0, 3), (1, 2), (2, 1)):
            lap = self.w[0] * G
            for p in range(1, 7):
                lap = lap + self.w[p] * (self._neighbour(G, axis, d, p)
                                         + self._neighbour(G, axis, d, -p))
            Y += (-0.5 / self.h ** 2) * lap
        Y = Y.reshape(ns, self.nd) + self.system.veff[None, :] * X[:, : self.nd]
        h3 = self.h ** 3
        for idx, phi, gam in self.atoms:
            C = h3 * (X[:, idx] @ phi.conj())  # (ns, P): h^3 <chi^k_p | x_n>
            np.add.at(Y, (slice(None), idx), (C * gam[None, :]) @ phi.T)
        return Y

    def dense(self):
        """H(k) as a dense Nd x Nd matrix (columns H e_j); small grids only."""
        return self.hpsi(np.eye(self.nd)).T

    # -- Algorithm 1 -------------------------------------------------------
    def lanczos(self, k, seed):
        """k-step Lanczos from the splitmix64 start vector (uniform in
        [-1/2, 1/2), real, normalised).  Returns (a0, b, alpha, beta, theta_max)
        with a0 = theta_min and b = theta_max + |beta_k|."""
        v = np.array([uniform(seed, i) - 0.5 for i in range(self.nd)], dtype=np.complex128)
        v /= np.linalg.norm(v)
        vp = np.zeros_like(v)
        alpha, beta = np.zeros(k), np.zeros(k)
        bprev = 0.0
        for j in range(k):
            w = self.hpsi(v)[0] - bprev * vp
            al = float(np.real(np.vdot(v, w)))
            w = w - al * v
            bt = float(np.linalg.norm(w))
            alpha[j], beta[j] = al, bt
            vp, v = v, (w / bt if bt > 0.0 else np.zeros_like(w))
            bprev = bt
        theta = tridiag_eigvals(alpha, beta[: k - 1])
        return theta[0], theta[-1] + abs(beta[k - 1]), alpha, beta, theta[-1]

    def cheb_filter(self, X, degree, a, b, a0):
        """Scaled three-term Chebyshev recurrence of degree m on [a, b],
        normalised at a0 (the real oracle's recurrence in complex arithmetic)."""
        if degree < 1 or not (a0 < a < b):
            raise ValueError("need degree >= 1 and a0 < a < b")
        X = np.asarray(X, dtype=np.complex128)[:, : self.nd]
        e, c = (b - a) / 2.0, (b + a) / 2.0
        sigma = e / (a0 - c)
        tau = 2.0 / sigma
        prev = X.copy()
        cur = (self.hpsi(prev) - c * prev) * (sigma / e)
        for _ in range(2, degree + 1):
            sigma_new = 1.0 / (tau - sigma)
            nxt = (self.hpsi(cur) - c * cur) * (2.0 * sigma_new / e) - sigma * sigma_new * prev
            prev, cur = cur, nxt
            sigma = sigma_new
        return cur

    def chefsi_step(self, X, degree, a, b, a0):
        """One complex CheFSI step.  Returns (X_new, ritz_values ascending)."""
        Xt = self.cheb_filter(X, degree, a, b, a0)
        Yt = self.hpsi(Xt)
        Hs, Ms = project(Xt, Yt)
        lam, Z = gen_eig(Hs, Ms)
        return rotate(Xt, Z), lam


# -- dense pieces of the complex Rayleigh-Ritz step -------------------------
def project(Xt, Yt):
    """Hs = Xt^H Yt, Ms = Xt^H Xt for blocks of shape (ns, nd): entry (p, q) is
    sum_i conj(X_p(i)) Y_q(i)."""
    Xt = np.asarray(Xt, dtype=np.complex128)
    Yt = np.asarray(Yt, dtype=np.complex128)
    return Xt.conj() @ Yt.T, Xt.conj() @ Xt.T


def rotate(Xt, Z):
    """X_q = sum_p Xt_p Z[p, q] for Xt of shape (ns, nd)."""
    return np.asarray(Z).T @ np.asarray(Xt, dtype=np.complex128)


def cholesky(M):
    """Lower-triangular L with L L^H = M (Hermitian positive definite M)."""
    M = np.asarray(M, dtype=np.complex128)
    n = M.shape[0]
    L = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        djj = float(np.real(M[j, j] - np.vdot(L[j, :j], L[j, :j])))
        if not djj > 0.0:
            raise OracleError(ERR_NOT_SPD, "cholesky")
        L[j, j] = np.sqrt(djj)
        for i in range(j + 1, n):
            L[i, j] = (M[i, j] - L[i, :j] @ L[j, :j].conj()) / L[j, j]
    return L


def _solve_lower(L, B):
    """L^-1 B by forward substitution, row by row."""
    n = L.shape[0]
    W = np.zeros_like(B, dtype=np.complex128)
    for i in range(n):
        W[i] = (B[i] - L[i, :i] @ W[:i]) / L[i, i]
    return W


def _solve_upper_h(L, B):
    """L^-H B by back substitution on the upper-triangular L^H."""
    n = L.shape[0]
    U = L.conj().T
    W = np.zeros_like(B, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        W[i] = (B[i] - U[i, i + 1:] @ W[i + 1:]) / U[i, i]
    return W


def householder_tridiag(A):
    """T = Q^H A Q tridiagonal for Hermitian A.  Each reflector
    I - 2 v v^H (|v| = 1) maps column j below the diagonal onto
    alpha e_1 with alpha = -exp(i arg x_0) |x|.  Returns (d real, e complex
    sub-diagonal T[j+1, j], Q)."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    Q = np.eye(n, dtype=np.complex128)
    for j in range(n - 2):
        x = A[j + 1:, j].copy()
        xn = np.linalg.norm(x)
        if xn == 0.0:
            continue
        ph = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -ph * xn
        v = x
        v[0] -= alpha
        vn = np.linalg.norm(v)
        if vn == 0.0:
            continue
        v = v / vn
        A[j + 1:, :] -= 2.0 * np.outer(v, v.conj() @ A[j + 1:, :])
        A[:, j + 1:] -= 2.0 * np.outer(A[:, j + 1:] @ v, v.conj())
        Q[:, j + 1:] -= 2.0 * np.outer(Q[:, j + 1:] @ v, v.conj())
    return np.real(np.diag(A)).copy(), np.diag(A, -1).copy(), Q


def herm_eig(A):
    """Eigenpairs of Hermitian A: Householder, the unitary diagonal phase
    scaling to a real symmetric tridiagonal, the real oracle's eigensolver,
    back-transformation.  Returns (lam ascending, V) with A V = V diag(lam)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    d, e, Q = householder_tridiag(0.5 * (A + A.conj().T))
    D = np.ones(n, dtype=np.complex128)
    for j in range(n - 1):
        D[j + 1] = D[j] * (e[j] / abs(e[j])) if e[j] != 0 else D[j]
    Tr = np.diag(d)
    if n > 1:
        off = np.abs(e)
        Tr += np.diag(off, -1) + np.diag(off, 1)
    lam, V = sym_eig(Tr)
    order = np.argsort(lam, kind="stable")
    lam, V = lam[order], V[:, order]
    return lam, Q @ (D[:, None] * V)


def gen_eig(Hs, Ms):
    """Hs Z = Ms Z diag(lam), Z^H Ms Z = I (Hermitian Hs, positive definite Ms)."""
    Hs = np.asarray(Hs, dtype=np.complex128)
    L = cholesky(0.5 * (Ms + np.asarray(Ms).conj().T))
    W = _solve_lower(L, Hs)              # L^-1 Hs
    A = _solve_lower(L, W.conj().T)      # L^-1 (L^-1 Hs)^H = L^-1 Hs L^-H
    lam, V = herm_eig(A)
    return lam, _solve_upper_h(L, V)
