"""Nonlocal Hellmann-Feynman forces on the atoms — test infrastructure, not
product code.

Only ``tests/`` may import this module; it never imports the CUDA library.

The paper (Sec. III, end of the introduction) names the two kernels behind the
nonlocal force: the gradient operator applied to the orbitals, then the
nonlocal projectors applied to the result. Written out for real (Gamma-point)
orbitals psi_n with occupations f_n and spin degeneracy 2, the nonlocal band
energy is

    E_nl = 2 sum_n f_n sum_J sum_lm gamma_Jl (h^3 <chi_Jlm | psi_n>)^2 .

Moving atom J moves its projectors, and d chi(r - R_J) / dR_J = -grad chi.
Integration by parts moves the gradient onto the orbital. This gives

    F_J = -dE_nl/dR_J
        = -4 sum_n f_n sum_lm gamma_Jl (h^3 <chi_Jlm | psi_n>) (h^3 <chi_Jlm | D psi_n>),

with D the radius-6 central first-derivative operator, (D_d psi)_i =
(1/h) sum_p w'_p (psi_{i + p e_d} - psi_{i - p e_d}). The same boundary rules
as the Laplacian apply: a periodic axis wraps, a Dirichlet axis has zero
ghosts. The weights are the standard ones (Fornberg),
w'_p = (-1)^(p+1) (n!)^2 / (p (n - p)! (n + p)!) for n = 6.

Pins (``tests/test_oracle_forces.py``):
* exact weights from the Taylor moment system;
* the plane-wave symbol and polynomial exactness of D;
* a dense Kronecker assembly;
* forces against an independent dense evaluation with analytic projectors;
* invariance under rotations within equally occupied orbitals;
* zero force by inversion symmetry;
* F = -dE_nl/dR by central differences of the energy as the atom moves.
"""
from __future__ import annotations

from math import factorial

import numpy as np

PERIODIC = 0


def fd_first_weights(n: int = 6) -> np.ndarray:
    """w'_1..w'_n of the central first derivative of radius n (index 0 unused, 0)."""
    w = np.zeros(n + 1)
    for p in range(1, n + 1):
        w[p] = (-1) ** (p + 1) * factorial(n) ** 2 / (p * factorial(n - p) * factorial(n + p))
    return w


def gradient(system, X, d: int) -> np.ndarray:
    """D_d X along grid axis d (0 = x, 1 = y, 2 = z) for X of shape (ns, ld)."""
    s = system
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[None, :]
    ns = X.shape[0]
    nx, ny, nz = s.nx, s.ny, s.nz
    G = X[:, : s.nd].reshape(ns, nz, ny, nx)
    axis = 3 - d
    n = (nx, ny, nz)[d]
    w = fd_first_weights(6)
    out = np.zeros_like(G)
    i = np.arange(n)
    shape = [1, 1, 1, 1]
    shape[axis] = n
    for p in range(1, 7):
        for sgn in (1, -1):
            j = i + sgn * p
            if s.bc[d] == PERIODIC:
                mask = np.ones(n)
            else:
                mask = ((j >= 0) & (j < n)).astype(np.float64)
            val = np.take(G, np.mod(j, n), axis=axis) * mask.reshape(shape)
            out += sgn * w[p] * val
    return (out / s.h).reshape(ns, s.nd)


def nonlocal_forces(system, X, f) -> np.ndarray:
    """F_J (A x 3, Ha/bohr) for orbitals X of shape (ns, ld), occupations f."""
    s = system
    X = np.asarray(X, dtype=np.float64)[:, : s.nd]
    f = np.asarray(f, dtype=np.float64)
    h3 = s.h ** 3
    grads = [gradient(s, X, d) for d in range(3)]
    F = np.zeros((s.natoms, 3))
    for J in range(s.natoms):
        lo, hi = int(s.supp_ptr[J]), int(s.supp_ptr[J + 1])
        idx = s.supp_idx[lo:hi].astype(np.int64)
        nproj = int(s.nproj[J])
        chi = s.chi[int(s.chi_ptr[J]):int(s.chi_ptr[J + 1])].reshape(nproj, hi - lo).T
        gam = s.gamma[int(s.proj_ptr[J]):int(s.proj_ptr[J + 1])]
        c = h3 * (X[:, idx] @ chi)                 # (ns, P): h^3 <chi_p | psi_n>
        for d in range(3):
            g = h3 * (grads[d][:, idx] @ chi)      # (ns, P): h^3 <chi_p | D_d psi_n>
            F[J, d] = -4.0 * np.sum(f[:, None] * gam[None, :] * c * g)
    return F
