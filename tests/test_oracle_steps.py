"""Pins for the oracle's CheFSI steps (Algorithm 1): Chebyshev filter, Lanczos
bounds, projection, generalised eigensolve, rotation, the full step, the
occupations/density metric and the counter-based generator."""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2302_09708_gb300 import synth

from test_oracle_operator import dense_hamiltonian, free_electron_eigs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cheb_T(m, t):
    """Chebyshev polynomial of the first kind by its closed form."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
    return out


def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for seed, i, out in rows:
        z = int(out, 0)
        u = oracle.uniform(int(seed), int(i))
        assert u == (z >> 11) * 2.0 ** -53


def test_filter_scalar_identity_on_plane_waves():
    """Free electrons: filtering an eigenvector v (eigenvalue lam) gives
    T_m((lam - c)/e) / T_m((a0 - c)/e) v."""
    shape, h = (16, 16, 16), 0.5
    s = synth.free_system(shape, h, (0, 0, 0))
    o = oracle.Oracle(s)
    lam = free_electron_eigs(shape, h)
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    a0, a, b = -0.05, 2.0, lam[-1] + 0.3
    c, e = (b + a) / 2, (b - a) / 2
    for m in (1, 2, 7, 20):
        for kv in [(0, 0, 0), (1, 0, 0), (1, 2, 0), (3, 3, 1), (8, 8, 8)]:
            ph = 2 * np.pi * sum(kk * g / n for kk, g, n in zip(kv, (i, j, k), shape))
            x = np.cos(ph).transpose(2, 1, 0).ravel()
            lv = float(o.hpsi(x)[0] @ x / (x @ x))
            ratio = cheb_T(m, [(lv - c) / e])[0] / cheb_T(m, [(a0 - c) / e])[0]
            y = o.cheb_filter(x[None, :], m, a, b, a0)[0]
            assert np.max(np.abs(y - ratio * x)) < 1e-11 * max(1.0, abs(ratio))


def test_filter_rejects_bad_bounds():
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    o = oracle.Oracle(s)
    with pytest.raises(oracle.OracleError):
        o.cheb_filter(np.ones((1, s.nd)), 5, 1.0, 0.5, 0.0)


def test_lanczos_free_electron_bounds():
    shape, h = (24, 24, 24), 0.5
    s = synth.free_system(shape, h, (0, 0, 0))
    o = oracle.Oracle(s)
    a0, b, al, bt, tmax = o.lanczos(40, 7)
    lmax = 3 * 7.0729393 / (2 * h * h)
    assert b >= lmax  # safe upper bound
    assert tmax <= lmax + 1e-9  # Ritz values lie inside the spectrum
    assert tmax > 0.97 * lmax
    assert -1e-9 <= a0 < 0.2  # lambda_min = 0


def test_tridiag_qr_vs_library():
    rng = np.random.default_rng(1)
    for n in (1, 2, 5, 40, 150):
        d, e = rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))
        ref = scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True)
        np.testing.assert_allclose(oracle.tridiag_eigvals(d, e), ref, atol=1e-12)
    # degenerate: Wilkinson-type matrix with close pairs, and a split matrix
    n = 21
    d = np.abs(np.arange(n) - 10.0)
    e = np.ones(n - 1)
    np.testing.assert_allclose(oracle.tridiag_eigvals(d, e),
                               scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True),
                               atol=1e-12)
    d, e = np.ones(6), np.zeros(5)
    np.testing.assert_allclose(oracle.tridiag_eigvals(d, e), np.ones(6))


def test_householder_tridiag():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 30))
    A = A + A.T
    d, e, Q = oracle.householder_tridiag(A)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    np.testing.assert_allclose(Q.T @ Q, np.eye(30), atol=1e-13)
    np.testing.assert_allclose(Q @ T @ Q.T, A, atol=1e-12)


def test_cholesky_and_not_spd():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((25, 25))
    M = B @ B.T + 0.1 * np.eye(25)
    np.testing.assert_allclose(oracle.cholesky(M), np.linalg.cholesky(M), atol=1e-12)
    M[3, 3] = -1.0
    with pytest.raises(oracle.OracleError) as ei:
        oracle.cholesky(M)
    assert ei.value.status == oracle.ERR_NOT_SPD


def _spd_pair(n, cond, rng, degenerate=0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = np.logspace(0, -np.log10(cond), n)
    M = (Q * sv) @ Q.T
    M = 0.5 * (M + M.T)
    ev = np.sort(rng.uniform(-3, 40, n))
    if degenerate:
        ev[5:5 + degenerate] = ev[5]
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (P * ev) @ P.T
    L = np.linalg.cholesky(M)
    H = L @ A @ L.T
    return 0.5 * (H + H.T), M, ev


@pytest.mark.parametrize("n,cond,deg", [(8, 10, 0), (40, 1e4, 0), (60, 1e8, 0), (50, 1e3, 6),
                                        (120, 1e6, 0)])
def test_gen_eig_vs_scipy(n, cond, deg):
    rng = np.random.default_rng(n + deg)
    H, M, ev = _spd_pair(n, cond, rng, deg)
    lam, Z = oracle.gen_eig(H, M)
    ref = scipy.linalg.eigh(H, M, eigvals_only=True)
    np.testing.assert_allclose(lam, ref, atol=1e-9 * max(1, cond / 1e4), rtol=0)
    np.testing.assert_allclose(lam, ev, atol=1e-7 * max(1, cond / 1e4))
    np.testing.assert_allclose(Z.T @ M @ Z, np.eye(n), atol=1e-9 * max(1, cond / 1e4))
    R = H @ Z - M @ Z * lam
    assert np.max(np.abs(R)) < 1e-9 * np.max(np.abs(H)) * max(1, cond / 1e4)
    # sign convention: largest-magnitude entry of each column is positive
    cols = np.argmax(np.abs(Z), axis=0)
    assert np.all(Z[cols, np.arange(n)] > 0)


def test_projection_and_rotation_vs_numpy():
    rng = np.random.default_rng(4)
    nd, ld, ns = 301, 304, 9
    X, Y = rng.standard_normal((ns, ld)), rng.standard_normal((ns, ld))
    Hs, Ms = oracle.project(X, Y, nd)
    np.testing.assert_allclose(Hs, X[:, :nd] @ Y[:, :nd].T, atol=1e-12)
    np.testing.assert_allclose(Ms, X[:, :nd] @ X[:, :nd].T, atol=1e-12)
    Z = rng.standard_normal((ns, ns))
    R = oracle.rotate(X, Z, nd)
    np.testing.assert_allclose(R, (X[:, :nd].T @ Z).T, atol=1e-12)


def _cold_bounds(o):
    a0, b, *_ = o.lanczos(30, 99)
    return a0, b, a0 + 0.1 * (b - a0)


def test_chefsi_step_structure():
    """One step: X^T X = I after rotation, Ritz values inside [a0, b], ascending,
    and equal to the Rayleigh-Ritz values of span(filtered X)."""
    s = synth.random_system((13, 14, 15), 0.5, (0, 0, 1), 2, seed=21)
    o = oracle.Oracle(s)
    a0, b, a = _cold_bounds(o)
    X0 = synth.random_orbitals(s.nd, 10, seed=5)
    X1, lam = o.chefsi_step(X0, 12, a, b, a0)
    np.testing.assert_allclose(X1 @ X1.T, np.eye(10), atol=1e-10)
    assert np.all(np.diff(lam) >= 0)
    assert lam[0] >= a0 - 1e-8 and lam[-1] <= b
    # same Ritz values from the dense matrix restricted to the filtered span
    Xf = o.cheb_filter(X0, 12, a, b, a0)
    H = dense_hamiltonian(s)
    Q, _ = np.linalg.qr(Xf.T)
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(Q.T @ H @ Q), atol=1e-8)


def test_chefsi_converges_to_brute_force():
    """Repeated steps at fixed H converge to the exact lowest eigenpairs."""
    s = synth.random_system((13, 13, 13), 0.5, (0, 0, 0), 2, seed=31)
    o = oracle.Oracle(s)
    H = dense_hamiltonian(s)
    ev, V = np.linalg.eigh(H)
    ns, want = 16, 10
    a0, b, a = _cold_bounds(o)
    X = synth.random_orbitals(s.nd, ns, seed=9)
    for _ in range(12):
        X, lam = o.chefsi_step(X, 16, a, b, a0)
        a = lam[-1]
    np.testing.assert_allclose(lam[:want], ev[:want], atol=1e-9)
    # subspace of the wanted vectors
    P = X[:want].T
    err = np.linalg.norm(V[:, :want] - P @ (P.T @ V[:, :want]))
    assert err < 1e-6


def test_chefsi_free_electron_shells():
    """Free electrons, Ns at a shell closure: converged Ritz values are the
    closed-form shell energies."""
    shape, h = (14, 14, 14), 0.5
    s = synth.free_system(shape, h, (0, 0, 0), v0=0.25)
    o = oracle.Oracle(s)
    exact = free_electron_eigs(shape, h) + 0.25
    ns = 27 + 6  # shells 1 + 6 + 12 + 8, plus the next six
    a0, b, a = _cold_bounds(o)
    X = synth.random_orbitals(s.nd, ns, seed=3)
    for _ in range(8):
        X, lam = o.chefsi_step(X, 20, a, b, a0)
        a = lam[-1]
    np.testing.assert_allclose(lam[:27], exact[:27], atol=1e-9)


def test_occupations_and_density():
    rng = np.random.default_rng(6)
    lam = np.sort(rng.uniform(-2, 1, 40))
    ne = synth.electrons_for(40)
    assert ne == 58
    f, mu = oracle.fermi_occupations(lam, ne, kT=0.01)
    assert abs(2 * f.sum() - ne) < 1e-10
    assert np.all(np.diff(f) <= 0)
    # zero-temperature limit: the lowest Ne/2 levels are filled
    f0, _ = oracle.fermi_occupations(lam, ne, kT=1e-6)
    np.testing.assert_allclose(f0, (np.arange(40) < ne // 2).astype(float), atol=1e-9)
    # density of an orthonormal block integrates to Ne
    nd, h = 500, 0.4
    X = synth.random_orbitals(nd, 40, seed=2)
    rho = oracle.density(X, f, nd, h)
    assert abs(h ** 3 * rho.sum() - ne) < 1e-9


def test_occupations_two_level_and_degenerate_closed_forms():
    """Two levels lam1 < lam2 holding Ne = 2 electrons: by symmetry
    mu = (lam1 + lam2) / 2 and f_1,2 = 1 / (1 + exp(-+ (lam2 - lam1) / 2kT)).
    One degenerate level of Ns states: f = Ne / (2 Ns) at any kT."""
    for lam1, lam2, kT in ((-0.3, 0.1, 0.01), (0.0, 0.05, 0.02), (-1.0, -0.99, 0.1)):
        f, mu = oracle.fermi_occupations(np.array([lam1, lam2]), 2.0, kT=kT)
        assert abs(mu - 0.5 * (lam1 + lam2)) < 1e-12 * max(1.0, abs(lam1))
        half = (lam2 - lam1) / (2 * kT)
        assert abs(f[0] - 1 / (1 + np.exp(-half))) < 1e-12
        assert abs(f[1] - 1 / (1 + np.exp(half))) < 1e-12
    for ns, ne in ((7, 3.0), (12, 20.0)):
        f, _ = oracle.fermi_occupations(np.full(ns, -0.42), ne, kT=0.01)
        np.testing.assert_allclose(f, ne / (2 * ns), atol=1e-12)


def test_lanczos_full_krylov_gives_exact_extremes():
    """With k = Nd steps (no restarts, tiny system) the Krylov space is the
    whole space, so theta_min and theta_max are the exact extreme eigenvalues of
    the dense operator (up to the loss of orthogonality, which for Nd = 64
    and well separated ends stays far below 1e-8)."""
    s = synth.random_system((4, 4, 4), 0.5, (1, 1, 1), 2, seed=9)
    o = oracle.Oracle(s)
    H = o.hpsi(np.eye(s.nd)).T
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    a0, b, al, bt, tmax = o.lanczos(s.nd, 3)
    assert abs(a0 - ev[0]) < 1e-8 * np.max(np.abs(ev))
    assert abs(tmax - ev[-1]) < 1e-8 * np.max(np.abs(ev))
    assert b >= ev[-1] - 1e-8


def test_chefsi_step_depends_only_on_the_span_of_the_start():
    """The filter is linear and Rayleigh-Ritz sees only the span of its input,
    so a start block X0 and X0 rotated by any orthogonal Q (any basis of the
    same span) give the same Ritz values and the same subspace."""
    s = synth.random_system((13, 14, 13), 0.5, (0, 1, 0), 3, seed=41)
    o = oracle.Oracle(s)
    a0, b, a = _cold_bounds(o)
    ns = 9
    X0 = synth.random_orbitals(s.nd, ns, seed=12)
    Q, _ = np.linalg.qr(np.random.default_rng(13).standard_normal((ns, ns)))
    X1, lam1 = o.chefsi_step(X0, 10, a, b, a0)
    X2, lam2 = o.chefsi_step(Q.T @ X0, 10, a, b, a0)
    np.testing.assert_allclose(lam2, lam1, atol=1e-10)
    # the same span: the projector onto one basis reproduces the other
    P = X1.T @ X1
    assert np.linalg.norm(X2.T - P @ X2.T) < 1e-8


def test_chefsi_step_is_shift_covariant():
    """Veff + sigma with every bound moved by sigma leaves (H - c)/e unchanged,
    so the filtered block is the same and the Ritz values move by exactly
    sigma (to rounding)."""
    import dataclasses
    s = synth.random_system((13, 13, 14), 0.5, (0, 0, 1), 2, seed=43)
    sigma = 0.37
    t = dataclasses.replace(s, veff=s.veff + sigma)
    o, ot = oracle.Oracle(s), oracle.Oracle(t)
    a0, b, a = _cold_bounds(o)
    X0 = synth.random_orbitals(s.nd, 8, seed=14)
    X1, lam1 = o.chefsi_step(X0, 12, a, b, a0)
    X2, lam2 = ot.chefsi_step(X0, 12, a + sigma, b + sigma, a0 + sigma)
    np.testing.assert_allclose(lam2 - sigma, lam1, atol=1e-10)
    Xf1 = o.cheb_filter(X0, 12, a, b, a0)
    Xf2 = ot.cheb_filter(X0, 12, a + sigma, b + sigma, a0 + sigma)
    assert np.max(np.abs(Xf2 - Xf1)) < 1e-10 * np.max(np.abs(Xf1))
