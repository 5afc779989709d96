"""Pins for the oracle's Hamiltonian (paper Sec. II A): FD weights, the
free-electron closed form, an independently assembled dense H (periodic and
Dirichlet, with projectors), symmetry and the single-projector identity."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2302_09708_gb300 import synth


def fornberg_by_moments(n):
    """Exact central 2nd-derivative weights of radius n from the Taylor moment
    conditions  sum_p w_p p^(2k) = [k == 1]  (k = 1..n, symmetric weights
    counted once per side), solved with rational Gaussian elimination."""
    # unknowns w_1..w_n ; equation k: sum_p 2 w_p p^(2k) / (2k)! = [k == 1]
    A = [[Fraction(2 * p ** (2 * k)) for p in range(1, n + 1)] for k in range(1, n + 1)]
    rhs = [Fraction(2) if k == 1 else Fraction(0) for k in range(1, n + 1)]
    m = n
    for c in range(m):
        piv = next(r for r in range(c, m) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        rhs[c], rhs[piv] = rhs[piv], rhs[c]
        for r in range(m):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
                rhs[r] -= f * rhs[c]
    w = [rhs[i] / A[i][i] for i in range(m)]
    return [-2 * sum(w)] + w


def test_fd_weights_exact_rationals():
    exact = fornberg_by_moments(6)
    # the closed forms quoted for radius 6
    assert exact[0] == Fraction(-5369, 1800)
    assert exact[1:] == [Fraction(12, 7), Fraction(-15, 56), Fraction(10, 189),
                         Fraction(-1, 112), Fraction(2, 1925), Fraction(-1, 16632)]
    w = oracle.fd_weights(6)
    for got, ref in zip(w, exact):
        assert abs(got - float(ref)) <= 2e-16 * max(1.0, abs(float(ref)))
    assert abs(w[0] + 2 * w[1:].sum()) < 1e-15


@pytest.mark.parametrize("deg", range(0, 14))
def test_fd_exact_on_polynomials(deg):
    """The 12th-order operator differentiates x^k exactly for k <= 13."""
    w = [float(f) for f in fornberg_by_moments(6)]
    wo = oracle.fd_weights(6)
    x0 = Fraction(3, 7)
    for ww in (w, wo):
        got = ww[0] * float(x0) ** deg + sum(
            ww[p] * (float(x0 + p) ** deg + float(x0 - p) ** deg) for p in range(1, 7))
        ref = deg * (deg - 1) * float(x0) ** (deg - 2) if deg >= 2 else 0.0
        scale = max(1.0, sum(abs(c) * (abs(float(x0)) + 6) ** deg for c in ww))
        assert abs(got - ref) <= 1e-13 * scale


def _fd1d(n, bc, w):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] += w[0]
        for p in range(1, 7):
            for j in (i + p, i - p):
                if 0 <= j < n:
                    D[i, j] += w[p]
                elif bc == synth.PERIODIC:
                    D[i, j % n] += w[p]
    return D


def dense_hamiltonian(s):
    """H assembled as a dense matrix: Kronecker sum of 1-D FD matrices, diag(Veff),
    and the per-atom outer products gamma h^3 chi chi^T."""
    w = [float(f) for f in fornberg_by_moments(6)]
    Dx, Dy, Dz = (_fd1d(n, b, w) for n, b in zip(s.shape, s.bc))
    Ix, Iy, Iz = np.eye(s.nx), np.eye(s.ny), np.eye(s.nz)
    lap = (np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix))
           + np.kron(Dz, np.kron(Iy, Ix))) / s.h ** 2
    H = -0.5 * lap + np.diag(s.veff)
    for J in range(s.natoms):
        idx = s.supp_idx[s.supp_ptr[J]:s.supp_ptr[J + 1]]
        ns_ = idx.size
        chi = s.chi[s.chi_ptr[J]:s.chi_ptr[J + 1]].reshape(s.nproj[J], ns_).T
        gam = s.gamma[s.proj_ptr[J]:s.proj_ptr[J + 1]]
        full = np.zeros((s.nd, s.nproj[J]))
        full[idx, :] = chi
        H += s.h ** 3 * (full * gam) @ full.T
    return H


def free_electron_eigs(shape, h):
    w = [float(f) for f in fornberg_by_moments(6)]
    lam = 0.0
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for n, k in zip(shape, grids):
        th = 2 * np.pi * k / n
        S = w[0] + 2 * sum(w[p] * np.cos(p * th) for p in range(1, 7))
        lam = lam + (-0.5 / h ** 2) * S
    return np.sort(lam.ravel())


SMALL = [
    ((13, 13, 13), (0, 0, 0), 2),
    ((14, 13, 15), (0, 0, 1), 3),
    ((13, 15, 14), (1, 1, 1), 2),
]


@pytest.mark.parametrize("shape,bc,natoms", SMALL)
def test_hpsi_matches_dense_assembly(shape, bc, natoms):
    s = synth.random_system(shape, 0.5, bc, natoms, seed=11 + natoms)
    H = dense_hamiltonian(s)
    o = oracle.Oracle(s)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, s.nd))
    Y = o.hpsi(X)
    ref = X @ H.T
    assert np.max(np.abs(Y - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hpsi_symmetric():
    s = synth.random_system((16, 13, 14), 0.45, (0, 1, 0), 3, seed=5)
    o = oracle.Oracle(s)
    rng = np.random.default_rng(8)
    u, v = rng.standard_normal((2, s.nd))
    Hu, Hv = o.hpsi(u)[0], o.hpsi(v)[0]
    assert abs(u @ Hv - Hu @ v) < 1e-13 * np.abs(u @ Hv) + 1e-12


def test_free_electron_plane_waves():
    """Veff = V0, no atoms: plane waves are eigenvectors with the closed-form symbol."""
    shape, h, v0 = (24, 24, 24), 0.5, -0.7
    s = synth.free_system(shape, h, (0, 0, 0), v0=v0)
    o = oracle.Oracle(s)
    w = [float(f) for f in fornberg_by_moments(6)]
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for kv in [(0, 0, 0), (1, 0, 0), (2, 3, 1), (12, 12, 12), (5, 0, 7)]:
        phase = 2 * np.pi * (kv[0] * i / shape[0] + kv[1] * j / shape[1] + kv[2] * k / shape[2])
        x = np.cos(phase).transpose(2, 1, 0).ravel()  # x fastest
        lam = v0 + sum((-0.5 / h ** 2) * (w[0] + 2 * sum(
            w[p] * np.cos(p * 2 * np.pi * kk / n) for p in range(1, 7)))
            for kk, n in zip(kv, shape))
        y = o.hpsi(x)[0]
        assert np.max(np.abs(y - lam * x)) < 1e-11


def test_free_electron_shells():
    """Shell energies for 24^3, h = 0.5: the quoted closed-form values."""
    lam = free_electron_eigs((24, 24, 24), 0.5)
    shells = np.unique(np.round(lam[:100], 9))
    np.testing.assert_allclose(shells[:8], [0, 0.137078, 0.274156, 0.411234, 0.548311,
                                            0.685389, 0.822467, 1.096623], atol=2e-6)
    counts = [int(np.sum(np.abs(lam - e) < 1e-9)) for e in shells[:5]]
    assert np.cumsum(counts).tolist()[:5] == [1, 7, 19, 27, 33]
    # the largest eigenvalue is 3 |S(pi)| / (2 h^2) = 42.44 Ha
    assert abs(lam[-1] - 3 * 7.072939 / (2 * 0.25)) < 1e-4


@pytest.mark.parametrize("shape,bc", [((13, 13, 13), (0, 0, 0)), ((13, 14, 13), (1, 1, 1)),
                                      ((14, 13, 13), (0, 0, 1))])
def test_dense_spectrum_free_vs_closed_form(shape, bc):
    """The dense assembly itself reproduces the closed form where it applies."""
    s = synth.free_system(shape, 0.5, bc)
    H = dense_hamiltonian(s)
    ev = np.linalg.eigvalsh(H)
    if bc == (0, 0, 0):
        np.testing.assert_allclose(ev, free_electron_eigs(shape, 0.5), atol=1e-10)
    else:
        # Dirichlet: no closed form; the operator is symmetric negative-definite Laplacian
        assert ev.min() > 0 and np.allclose(H, H.T)


def test_single_projector_identity():
    """One atom on a grid point, Veff = 0: h^3 chi_q^T V_nl chi_q = gamma_q."""
    shape, h = (16, 16, 16), 0.4
    pos = np.array([[8 * h, 7 * h, 9 * h]])
    s = synth.build_system(shape, h, (0, 0, 0), pos, [0.0], [1.0], [0.37], [-0.81])
    free = synth.free_system(shape, h, (0, 0, 0))
    o, of = oracle.Oracle(s), oracle.Oracle(free)
    idx = s.supp_idx
    chi = s.chi.reshape(4, idx.size).T
    for q, gam in enumerate([0.37, -0.81, -0.81, -0.81]):
        x = np.zeros(s.nd)
        x[idx] = chi[:, q]
        vnl = o.hpsi(x)[0] - of.hpsi(x)[0]
        assert abs(h ** 3 * x @ vnl - gam) < 1e-13
        # discrete normalisation of the projector tables
        assert abs(h ** 3 * chi[:, q] @ chi[:, q] - 1.0) < 1e-13
