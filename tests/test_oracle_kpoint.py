"""Pins for the complex (Bloch wavevector) oracle: the free-electron closed form
at any k, an independently assembled dense H(k), the supercell identity
(spectrum of a real 3x supercell = union of the primitive cell's H(k) over the
commensurate k), Hermiticity and time reversal, the k = 0 reduction to the real
oracle, the complex dense eigen-pieces against numpy/scipy, and the complex
CheFSI step against dense Rayleigh-Ritz and brute-force eigenvalues."""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from analytic import analytic_projectors
from oracle import kpoint
from paper_2302_09708_gb300 import synth

P, D = synth.PERIODIC, synth.DIRICHLET
# radius-6 central second-derivative weights (exact rationals, pinned in
# test_oracle_operator.py by the Taylor moment system)
W = [-5369 / 1800, 12 / 7, -15 / 56, 10 / 189, -1 / 112, 2 / 1925, -1 / 16632]


def cheb_T(m, t):
    """Chebyshev polynomial of the first kind by its cos / cosh closed form."""
    if abs(t) <= 1:
        return math.cos(m * math.acos(t))
    return math.copysign(1.0, t) ** m * math.cosh(m * math.acosh(abs(t)))


def symbol(theta):
    """-(1/2) x the 1-D FD second-derivative symbol at phase theta (times h^2)."""
    return -0.5 * (W[0] + 2 * sum(W[p] * np.cos(p * theta) for p in range(1, 7)))


def bloch_fd1d(n, periodic, kL):
    """1-D radius-6 FD matrix: a neighbour beyond the cell is the wrapped value
    times exp(i k L) per crossing (periodic) or zero (Dirichlet)."""
    A = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        A[i, i] += W[0]
        for p in range(1, 7):
            for j in (i + p, i - p):
                if 0 <= j < n:
                    A[i, j] += W[p]
                elif periodic:
                    A[i, j % n] += W[p] * np.exp(1j * kL * (j // n))
    return A


def dense_hk(s, k):
    """H(k) assembled independently: Kronecker sum of 1-D Bloch FD matrices,
    diag(Veff) and explicit projector outer products."""
    k = np.asarray(k, dtype=np.float64)
    nx, ny, nz = s.shape
    L = np.array(s.shape) * s.h
    Ax, Ay, Az = (bloch_fd1d(n, s.bc[d] == P, k[d] * L[d]) for d, n in enumerate(s.shape))
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    lap = (np.kron(Iz, np.kron(Iy, Ax)) + np.kron(Iz, np.kron(Ay, Ix))
           + np.kron(Az, np.kron(Iy, Ix)))
    H = -0.5 / s.h ** 2 * lap + np.diag(s.veff)
    for phi, gam in analytic_projectors(s, k):
        H += s.h ** 3 * (phi * gam[None, :]) @ phi.conj().T
    return H


def edge_system(shape, bc, seed):
    """Atoms near the periodic faces, so that projector supports wrap."""
    h = 0.5
    L = np.array(shape) * h
    pos = np.array([[0.3, 0.2, 0.4], [L[0] - 0.4, 0.55 * L[1], 0.6 * L[2]],
                    [0.5 * L[0], L[1] - 0.1, L[2] - 0.35]])
    return synth.random_system(shape, h, bc, 3, seed, positions=pos)


# -- operator ------------------------------------------------------------------
@pytest.mark.parametrize("shape,bc,k", [
    ((13, 13, 6), (P, P, D), (0.31, -0.17, 0.0)),
    ((13, 7, 14), (P, D, P), (-0.23, 0.0, 0.41)),
    ((13, 13, 13), (P, P, P), (0.12, 0.29, -0.37)),
])
def test_hpsi_k_matches_dense_assembly(shape, bc, k):
    s = edge_system(shape, bc, seed=sum(shape))
    ko = kpoint.KOracle(s, k)
    H = dense_hk(s, k)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, s.nd)) + 1j * rng.standard_normal((3, s.nd))
    Y = ko.hpsi(X)
    ref = (H @ X.T).T
    assert np.max(np.abs(Y - ref)) < 1e-12 * np.max(np.abs(ref))


def test_free_electron_bloch_plane_waves():
    """Every exp(i (2 pi j / N + k h) . i) is an eigenvector of the free H(k)
    with eigenvalue sum_d symbol(2 pi j_d / N_d + k_d h) / h^2."""
    shape, h = (13, 14, 15), 0.5
    s = synth.free_system(shape, h, (P, P, P))
    k = np.array([0.21, -0.33, 0.07])
    ko = kpoint.KOracle(s, k)
    iz, iy, ix = np.meshgrid(*[np.arange(n) for n in shape[::-1]], indexing="ij")
    grid = (ix.ravel(), iy.ravel(), iz.ravel())
    for j in [(0, 0, 0), (1, 0, 0), (2, 5, 1), (6, 7, 7), (12, 13, 14)]:
        theta = [2 * np.pi * j[d] / shape[d] + k[d] * h for d in range(3)]
        x = np.exp(1j * sum(theta[d] * grid[d] for d in range(3)))
        lam = sum(symbol(t) for t in theta) / h ** 2
        y = ko.hpsi(x)[0]
        assert np.max(np.abs(y - lam * x)) < 1e-12 * max(1.0, lam)


def test_free_electron_dense_spectrum_closed_form():
    shape, h = (13, 13, 4), 0.45
    s = synth.free_system(shape, h, (P, P, D))
    k = np.array([0.4, -0.25, 0.9])
    ev = np.linalg.eigvalsh(kpoint.KOracle(s, k).dense())
    # x, y: Bloch plane waves; z (Dirichlet, 4 points): the 4 x 4 matrix's spectrum
    ez = np.linalg.eigvalsh(-0.5 * np.real(bloch_fd1d(4, False, 0.0))) / h ** 2
    ref = np.sort([(symbol(2 * np.pi * a / 13 + k[0] * h) + symbol(2 * np.pi * b / 13 + k[1] * h))
                   / h ** 2 + c for a in range(13) for b in range(13) for c in ez])
    assert np.max(np.abs(ev - ref)) < 1e-10 * ref[-1]


@pytest.mark.parametrize("axis", [0, 1])
def test_supercell_spectrum_is_union_over_k(axis):
    """A real 3x supercell along one periodic axis has exactly the eigenvalues
    of the primitive cell's H(k) at k = 0 and +-2 pi / (3 L): every supercell
    eigenvector is a sum of primitive Bloch functions. Non-real phases
    exp(+-2 pi i / 3) make a sign mismatch between the Laplacian's and the
    projectors' phases visible."""
    shape = [5, 5, 6]
    shape[axis] = 13
    bc = [D, D, D]
    bc[axis] = P
    s = edge_system(tuple(shape), tuple(bc), seed=40 + axis)
    L = shape[axis] * s.h
    # the supercell: same atoms repeated, Veff tiled, projectors rebuilt
    big = list(shape)
    big[axis] *= 3
    shift = np.zeros(3)
    shift[axis] = L
    pos3 = np.concatenate([s.positions + m * shift for m in range(3)])
    e0 = [s.gamma[int(s.proj_ptr[J])] for J in range(s.natoms)] * 3
    e1 = [s.gamma[int(s.proj_ptr[J]) + 1] for J in range(s.natoms)] * 3
    reps = [1, 1, 1]
    reps[2 - axis] = 3  # veff is (nz, ny, nx)
    v3 = np.tile(s.veff.reshape(shape[2], shape[1], shape[0]), reps).ravel()
    sp, si, npj, cp, chi, pp, gam = synth._projectors(tuple(big), s.h, tuple(bc), pos3, e0, e1)
    s3 = synth.System(big[0], big[1], big[2], s.h, tuple(bc), v3, pos3, sp, si, npj, cp, chi,
                      pp, gam, "supercell")
    o3 = oracle.Oracle(s3)
    H3 = o3.hpsi(np.eye(s3.nd)).T
    ev3 = np.linalg.eigvalsh(0.5 * (H3 + H3.T))
    evk = []
    for kk in (0.0, 2 * np.pi / (3 * L), -2 * np.pi / (3 * L)):
        k = np.zeros(3)
        k[axis] = kk
        evk.append(np.linalg.eigvalsh(kpoint.KOracle(s, k).dense()))
    union = np.sort(np.concatenate(evk))
    assert np.max(np.abs(ev3 - union)) < 1e-10 * np.max(np.abs(union))


def test_hermitian_time_reversal_and_k_periodicity():
    s = edge_system((13, 13, 6), (P, P, D), seed=9)
    k = np.array([0.37, -0.21, 0.0])
    H = kpoint.KOracle(s, k).dense()
    assert np.max(np.abs(H - H.conj().T)) < 1e-12 * np.max(np.abs(H))
    Hm = kpoint.KOracle(s, -k).dense()
    assert np.max(np.abs(Hm - H.conj())) < 1e-12 * np.max(np.abs(H))
    G = np.array([2 * np.pi / (13 * s.h), -2 * np.pi / (13 * s.h), 0.0])
    HG = kpoint.KOracle(s, k + G).dense()
    assert np.max(np.abs(HG - H)) < 1e-11 * np.max(np.abs(H))


@pytest.mark.parametrize("shape,bc", [((13, 13, 13), (P, P, P)), ((13, 17, 19), (P, D, P)),
                                      ((6, 7, 8), (D, D, D))])
def test_k_zero_matches_real_oracle(shape, bc):
    s = synth.random_system(shape, 0.5, bc, 4, seed=77)
    X = synth.random_orbitals(s.nd, 3, seed=2)
    Yr = oracle.Oracle(s).hpsi(X)
    Yk = kpoint.KOracle(s, (0.0, 0.0, 0.0)).hpsi(X)
    assert np.max(np.abs(Yk.imag)) == 0.0
    assert np.max(np.abs(Yk.real - Yr)) < 1e-13 * np.max(np.abs(Yr))


# -- dense eigen-pieces ---------------------------------------------------------
def _herm_pair(n, cond, rng, degenerate=0):
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = B + B.conj().T
    if degenerate:
        U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        lam = np.sort(rng.standard_normal(n))
        lam[:degenerate] = lam[0]
        H = (U * lam) @ U.conj().T
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sv = np.geomspace(1.0, 1.0 / cond, n)
    M = (U * sv) @ U.conj().T
    return 0.5 * (H + H.conj().T), 0.5 * (M + M.conj().T)


def test_complex_cholesky_and_not_spd():
    rng = np.random.default_rng(1)
    _, M = _herm_pair(12, 1e3, rng)
    L = kpoint.cholesky(M)
    assert np.max(np.abs(L - np.linalg.cholesky(M))) < 1e-12
    assert np.max(np.abs(np.triu(L, 1))) == 0.0
    with pytest.raises(oracle.OracleError):
        kpoint.cholesky(-M)


def test_complex_householder_tridiag():
    rng = np.random.default_rng(2)
    H, _ = _herm_pair(17, 1.0, rng)
    d, e, Q = kpoint.householder_tridiag(H)
    T = Q.conj().T @ H @ Q
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(17))) < 1e-13
    assert np.max(np.abs(np.tril(T, -2))) < 1e-12 and np.max(np.abs(np.triu(T, 2))) < 1e-12
    assert np.max(np.abs(np.diag(T) - d)) < 1e-12 and np.max(np.abs(np.diag(T, -1) - e)) < 1e-12
    assert np.max(np.abs(np.linalg.eigvalsh(H) - np.linalg.eigvalsh(T))) < 1e-12


@pytest.mark.parametrize("n,cond,deg", [(1, 1.0, 0), (2, 10.0, 0), (7, 1e3, 0), (40, 1e4, 0),
                                        (30, 1e8, 0), (25, 1e2, 6)])
def test_complex_gen_eig_vs_scipy(n, cond, deg):
    rng = np.random.default_rng(n + deg)
    H, M = _herm_pair(n, cond, rng, degenerate=deg)
    lam, Z = kpoint.gen_eig(H, M)
    ref = sl.eigh(H, M, eigvals_only=True)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(lam - ref)) < 1e-12 * cond * scale
    assert np.max(np.abs(Z.conj().T @ M @ Z - np.eye(n))) < 1e-12 * cond
    R = H @ Z - (M @ Z) * lam[None, :]
    assert np.max(np.abs(R)) < 1e-11 * cond * scale


def test_real_input_matches_real_gen_eig():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((15, 15))
    H = A + A.T
    B = rng.standard_normal((15, 15))
    M = B @ B.T + 15 * np.eye(15)
    lam_c, _ = kpoint.gen_eig(H, M)
    lam_r, _ = oracle.gen_eig(H, M)
    assert np.max(np.abs(lam_c - lam_r)) < 1e-12 * np.max(np.abs(lam_r))


# -- Algorithm 1 in complex arithmetic --------------------------------------------
def test_filter_scalar_identity_on_bloch_plane_waves():
    shape, h = (13, 14, 13), 0.5
    s = synth.free_system(shape, h, (P, P, P))
    k = np.array([0.17, 0.4, -0.3])
    ko = kpoint.KOracle(s, k)
    iz, iy, ix = np.meshgrid(*[np.arange(n) for n in shape[::-1]], indexing="ij")
    grid = (ix.ravel(), iy.ravel(), iz.ravel())
    a0, a, b = -0.05, 2.0, 60.0
    c, e = (b + a) / 2, (b - a) / 2
    for m in (1, 2, 9, 20):
        for j in [(0, 0, 0), (1, 2, 0), (3, 3, 1), (6, 7, 6)]:
            theta = [2 * np.pi * j[d] / shape[d] + k[d] * h for d in range(3)]
            x = np.exp(1j * sum(theta[d] * grid[d] for d in range(3)))
            lam = sum(symbol(t) for t in theta) / h ** 2
            ratio = cheb_T(m, (lam - c) / e) / cheb_T(m, (a0 - c) / e)
            y = ko.cheb_filter(x[None, :], m, a, b, a0)[0]
            assert np.max(np.abs(y - ratio * x)) < 1e-11 * max(1.0, abs(ratio))


def test_lanczos_bounds_bracket_spectrum():
    s = edge_system((13, 13, 5), (P, P, D), seed=12)
    ko = kpoint.KOracle(s, (0.3, -0.2, 0.0))
    ev = np.linalg.eigvalsh(ko.dense())
    a0, b, al, bt, tmax = ko.lanczos(32, 0)
    assert ev[0] - 1e-10 <= a0 < ev[0] + 0.5 * (ev[-1] - ev[0])
    assert tmax <= ev[-1] + 1e-10 and b >= ev[-1]


def _step_setup(seed=21):
    s = edge_system((13, 13, 5), (P, P, D), seed=seed)
    ko = kpoint.KOracle(s, (0.35, -0.15, 0.0))
    a0, b, *_ = ko.lanczos(32, 0)
    return s, ko, a0, b


def test_chefsi_step_ritz_values_equal_dense_rayleigh_ritz():
    s, ko, a0, b = _step_setup()
    ns, m = 10, 8
    a = a0 + 0.1 * (b - a0)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((ns, s.nd)) + 1j * rng.standard_normal((ns, s.nd))
    Xn, lam = ko.chefsi_step(X, m, a, b, a0)
    Xt = ko.cheb_filter(X, m, a, b, a0)
    Qb, _ = np.linalg.qr(Xt.T)
    H = ko.dense()
    ref = np.linalg.eigvalsh(Qb.conj().T @ H @ Qb)
    assert np.max(np.abs(lam - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(Xn.conj() @ Xn.T - np.eye(ns))) < 1e-10
    R = (H @ Xn.T) - Xn.T * lam[None, :]
    assert np.linalg.norm(R) < np.linalg.norm(H) * 10.0  # Ritz pairs, not eigenpairs yet


def test_chefsi_steps_converge_to_brute_force():
    s, ko, a0, b = _step_setup(seed=22)
    ev = np.linalg.eigvalsh(ko.dense())
    ns, m = 12, 12
    rng = np.random.default_rng(5)
    X = rng.standard_normal((ns, s.nd)) + 1j * rng.standard_normal((ns, s.nd))
    a = a0 + 0.1 * (b - a0)
    for _ in range(14):
        X, lam = ko.chefsi_step(X, m, a, b, a0)
        a = lam[-1]
    # the lowest states converge fastest; the top ones of the block lag
    assert np.max(np.abs(lam[:8] - ev[:8])) < 1e-8


def test_complex_step_depends_only_on_the_span_of_the_start():
    """As in the real step: a start block and the same block rotated by any
    unitary U give the same Ritz values and the same subspace."""
    s, ko, a0, b = _step_setup(seed=23)
    ns, m = 8, 8
    a = a0 + 0.1 * (b - a0)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((ns, s.nd)) + 1j * rng.standard_normal((ns, s.nd))
    U, _ = np.linalg.qr(rng.standard_normal((ns, ns)) + 1j * rng.standard_normal((ns, ns)))
    X1, lam1 = ko.chefsi_step(X, m, a, b, a0)
    X2, lam2 = ko.chefsi_step(U.T @ X, m, a, b, a0)
    assert np.max(np.abs(lam2 - lam1)) < 1e-10 * np.max(np.abs(lam1))
    P = X1.T @ X1.conj()  # projector onto span(X1) (columns X1.T)
    assert np.linalg.norm(X2.T - P @ X2.T) < 1e-8
