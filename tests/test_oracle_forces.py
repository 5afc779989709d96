"""Pins for the nonlocal-force oracle:
- the first-derivative weights as exact rationals from the Taylor moment system;
- the plane-wave symbol and polynomial exactness of the gradient;
- a dense Kronecker assembly;
- forces against a dense evaluation with analytic projectors;
- invariance under rotations of equally occupied orbitals;
- zero force by inversion symmetry;
- F = -dE_nl/dR by central differences of the nonlocal band energy."""
from fractions import Fraction

import numpy as np
import pytest

from analytic import analytic_projectors
from oracle import forces
from paper_2302_09708_gb300 import synth

P, D = synth.PERIODIC, synth.DIRICHLET


def first_derivative_by_moments(n):
    """Exact antisymmetric weights w_1..w_n of the central first derivative:
    sum_p 2 w_p p^(2k-1) = [k == 1] for k = 1..n (rational elimination)."""
    A = [[Fraction(2 * p ** (2 * k - 1)) for p in range(1, n + 1)] for k in range(1, n + 1)]
    rhs = [Fraction(1) if k == 1 else Fraction(0) for k in range(1, n + 1)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        rhs[c], rhs[piv] = rhs[piv], rhs[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
                rhs[r] -= f * rhs[c]
    return [rhs[i] / A[i][i] for i in range(n)]


def test_first_derivative_weights_exact():
    exact = first_derivative_by_moments(6)
    assert exact == [Fraction(6, 7), Fraction(-15, 56), Fraction(5, 63), Fraction(-1, 56),
                     Fraction(1, 385), Fraction(-1, 5544)]
    w = forces.fd_first_weights(6)
    assert w[0] == 0.0
    for got, ref in zip(w[1:], exact):
        assert abs(got - float(ref)) <= 2e-16 * abs(float(ref))


@pytest.mark.parametrize("deg", range(0, 14))
def test_gradient_exact_on_polynomials_in_the_interior(deg):
    """On a Dirichlet grid, points at least 6 away from the faces see no
    ghosts.  There D x^k = k x^(k-1) exactly for k <= 12 (order 12).  For
    k = 13 the whole error is the leading term, the constant
    h^12 (2 sum_p w_p p^13 - 13)."""
    s = synth.free_system((20, 15, 14), 0.5, (D, D, D))
    iz, iy, ix = np.meshgrid(np.arange(14), np.arange(15), np.arange(20), indexing="ij")
    coords = (ix.ravel() * 0.5 - 3.1, iy.ravel() * 0.5 - 2.2, iz.ravel() * 0.5 - 1.3)
    inner = ((ix >= 6) & (ix < 14) & (iy >= 6) & (iy < 9) & (iz >= 6) & (iz < 8)).ravel()
    for d in range(3):
        x = coords[d]
        g = forces.gradient(s, x ** deg, d)[0]
        ref = deg * x ** (deg - 1) if deg else np.zeros_like(x)
        scale = max(1.0, np.max(np.abs(x[inner])) + 3.0) ** deg
        if deg <= 12:
            assert np.max(np.abs(g[inner] - ref[inner])) < 1e-12 * scale
        else:
            w = first_derivative_by_moments(6)
            lead = float(2 * sum(w[p - 1] * Fraction(p) ** 13 for p in range(1, 7))
                         - 13) * 0.5 ** 12
            err = g[inner] - ref[inner]
            assert np.max(np.abs(err - lead)) < 1e-9 * scale, (err[:3], lead)


def test_gradient_plane_wave_symbol():
    """Periodic axes: D sin(theta i) = (2/h) sum_p w_p sin(p theta) cos(theta i)."""
    shape, h = (13, 16, 14), 0.4
    s = synth.free_system(shape, h, (P, P, P))
    w = [float(x) for x in first_derivative_by_moments(6)]
    iz, iy, ix = np.meshgrid(*[np.arange(n) for n in shape[::-1]], indexing="ij")
    grid = (ix.ravel(), iy.ravel(), iz.ravel())
    for d in range(3):
        for j in (1, 3, 6):
            th = 2 * np.pi * j / shape[d]
            x = np.sin(th * grid[d] + 0.3)
            sym = 2.0 / h * sum(w[p - 1] * np.sin(p * th) for p in range(1, 7))
            g = forces.gradient(s, x, d)[0]
            assert np.max(np.abs(g - sym * np.cos(th * grid[d] + 0.3))) < 1e-12


def fd_first_1d(n, periodic, h):
    w = [float(x) for x in first_derivative_by_moments(6)]
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(1, 7):
            for j, sgn in ((i + p, 1), (i - p, -1)):
                if 0 <= j < n or periodic:
                    A[i, j % n] += sgn * w[p - 1] / h
    return A


def dense_gradients(s):
    nx, ny, nz = s.shape
    Ax, Ay, Az = (fd_first_1d(n, s.bc[d] == P, s.h) for d, n in enumerate(s.shape))
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (np.kron(Iz, np.kron(Iy, Ax)), np.kron(Iz, np.kron(Ay, Ix)),
            np.kron(Az, np.kron(Iy, Ix)))


@pytest.mark.parametrize("shape,bc", [((13, 13, 6), (P, P, D)), ((7, 13, 14), (D, P, P))])
def test_gradient_matches_dense_kronecker(shape, bc):
    s = synth.free_system(shape, 0.5, bc)
    X = np.random.default_rng(3).standard_normal((2, s.nd))
    for d, Dm in enumerate(dense_gradients(s)):
        assert np.max(np.abs(forces.gradient(s, X, d) - X @ Dm.T)) < 1e-12


def edge_system(shape, bc, seed):
    h = 0.5
    L = np.array(shape) * h
    pos = np.array([[0.3, 0.2, 0.4], [L[0] - 0.4, 0.55 * L[1], 0.6 * L[2]],
                    [0.5 * L[0], L[1] - 0.1, L[2] - 0.35]])
    return synth.random_system(shape, h, bc, 3, seed, positions=pos)


@pytest.mark.parametrize("shape,bc", [((13, 13, 6), (P, P, D)), ((13, 14, 13), (P, P, P))])
def test_forces_match_dense_evaluation(shape, bc):
    s = edge_system(shape, bc, seed=11)
    rng = np.random.default_rng(12)
    ns = 5
    X = rng.standard_normal((ns, s.nd))
    f = rng.uniform(0.0, 1.0, ns)
    F = forces.nonlocal_forces(s, X, f)
    Ds = dense_gradients(s)
    h3 = s.h ** 3
    ref = np.zeros_like(F)
    for J, (phi, gam) in enumerate(analytic_projectors(s)):
        phi = phi.real
        c = h3 * X @ phi
        for d in range(3):
            g = h3 * (X @ Ds[d].T) @ phi
            ref[J, d] = -4.0 * np.sum(f[:, None] * gam[None, :] * c * g)
    assert np.max(np.abs(F - ref)) < 1e-11 * np.max(np.abs(ref))


def test_forces_invariant_under_rotation_of_equal_occupations():
    """F depends on the orbitals only through sum_n f_n psi_n psi_n^T."""
    s = edge_system((13, 13, 6), (P, P, D), seed=13)
    rng = np.random.default_rng(14)
    X = rng.standard_normal((6, s.nd))
    f = np.array([1.0, 1.0, 1.0, 0.4, 0.4, 0.0])
    F = forces.nonlocal_forces(s, X, f)
    Q3, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    R = np.eye(6)
    R[:3, :3], R[3:5, 3:5] = Q3, Q2
    Xr = R.T @ X
    Xr[5] = rng.standard_normal(s.nd)  # unoccupied: anything
    assert np.max(np.abs(forces.nonlocal_forces(s, Xr, f) - F)) < 1e-12 * np.max(np.abs(F))


def test_zero_force_by_inversion_symmetry():
    """Atom on a grid point, orbitals even or odd about it: each product
    <chi|psi><chi|D psi> pairs an even and an odd factor, so F = 0."""
    shape, h = (16, 16, 16), 0.5
    s = synth.random_system(shape, h, (P, P, P), 1, seed=15, positions=[[4.0, 4.0, 4.0]])
    iz, iy, ix = np.meshgrid(*[np.arange(n) for n in shape[::-1]], indexing="ij")
    dx, dy, dz = [(g.ravel() - 8) for g in (ix, iy, iz)]
    th = 2 * np.pi / 16
    X = np.stack([np.cos(th * dx) * np.cos(2 * th * dy),
                  np.sin(th * dx) * np.cos(th * dz),
                  np.sin(th * dx) * np.sin(th * dy) * np.sin(3 * th * dz)])
    F = forces.nonlocal_forces(s, X, np.array([1.0, 0.7, 0.3]))
    Fg = forces.nonlocal_forces(s, X + 0.3 * np.roll(X, 1, axis=1), np.array([1.0, 0.7, 0.3]))
    assert np.max(np.abs(F)) < 1e-12 * np.max(np.abs(Fg))
    assert np.max(np.abs(Fg)) > 1e-6


def test_force_is_minus_energy_derivative(monkeypatch):
    """F_J = -dE_nl/dR_J with E_nl = 2 sum_n f_n sum_p gamma_p (h^3 <chi_p|psi_n>)^2.
    Checked by central differences as the atom moves under fixed, smooth,
    periodic orbitals.
    - A cut-off of 7 bohr (Gaussian tail e^-24.5) makes E smooth in R: points
      crossing the cut-off sphere change it by ~1e-11.
    - Summation by parts is exact for the antisymmetric stencil on a periodic
      grid, so only the order-12 FD error on a smooth Gaussian remains
      (h / sigma = 0.35).
    - The difference step's own error is O(delta^2): about 4e-9 relative at
      delta = 1e-4, falling 10x per 3x smaller delta down to that point.
    A 6-bohr cut-off instead leaves a ~3e-6 floor from those crossings."""
    monkeypatch.setattr(synth, "RC", 7.0)
    shape, h = (44, 44, 44), 0.35
    L = 44 * h
    R0 = np.array([7.53, 7.31, 7.77])
    iz, iy, ix = np.meshgrid(*[np.arange(44)] * 3, indexing="ij")
    r = (ix.ravel() * h, iy.ravel() * h, iz.ravel() * h)
    modes = [((1, 0, 0), 0.2), ((0, 1, 1), 1.1), ((1, 1, 0), 2.0), ((2, 0, 1), 0.7),
             ((0, 0, 1), 2.9)]
    X = np.stack([np.cos(2 * np.pi * sum(m[d] * r[d] for d in range(3)) / L + ph)
                  for m, ph in modes])
    f = np.array([1.0, 0.8, 0.6, 0.5, 0.2])

    def system_at(R):
        return synth.random_system(shape, h, (P, P, P), 1, seed=16, positions=[R])

    def energy(s):
        nproj = int(s.nproj[0])
        chi = s.chi[: int(s.chi_ptr[1])].reshape(nproj, -1).T
        c = h ** 3 * (X[:, s.supp_idx.astype(np.int64)] @ chi)
        return 2.0 * np.sum(f[:, None] * s.gamma[None, :nproj] * c * c)

    F = forces.nonlocal_forces(system_at(R0), X, f)[0]
    delta = 1e-4
    Ffd = np.zeros(3)
    for d in range(3):
        e = np.zeros(3)
        e[d] = delta
        Ffd[d] = -(energy(system_at(R0 + e)) - energy(system_at(R0 - e))) / (2 * delta)
    assert np.max(np.abs(F - Ffd)) < 2e-8 * np.max(np.abs(F)), (F, Ffd)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_forces_covariant_under_a_lattice_translation(axis):
    """Periodic grid: moving every atom by one grid spacing along an axis and
    rolling the orbitals by one point the same way leaves every force
    unchanged (the projector tables, Veff and the gradient stencil all move
    with the lattice)."""
    shape, h = (13, 14, 12), 0.5
    L = np.array(shape) * h
    rng = np.random.default_rng(21)
    pos = rng.uniform(0.1, 0.9, size=(3, 3)) * (L - h)
    step = np.zeros(3)
    step[axis] = h
    s = synth.random_system(shape, h, (P, P, P), 3, seed=17, positions=pos)
    t = synth.random_system(shape, h, (P, P, P), 3, seed=17, positions=pos + step)
    ns = 4
    X = rng.standard_normal((ns, s.nd))
    Xt = np.roll(X.reshape(ns, shape[2], shape[1], shape[0]), 1, axis=3 - axis).reshape(ns, -1)
    f = np.array([1.0, 0.8, 0.5, 0.1])
    F = forces.nonlocal_forces(s, X, f)
    Ft = forces.nonlocal_forces(t, Xt, f)
    assert np.max(np.abs(F)) > 1e-6
    assert np.max(np.abs(Ft - F)) < 1e-12 * np.max(np.abs(F))
