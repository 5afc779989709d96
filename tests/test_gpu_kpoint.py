"""GPU parity of the complex step at a Bloch wavevector k (sparc_create_kpoint)
against the complex oracle (oracle/kpoint.py) on the same seeded inputs:
H(k) x, Lanczos bounds, the Chebyshev filter, the projection, the Hermitian
generalised eigensolver (including degenerate levels and an ill-conditioned
overlap) and the full step.  Also k = 0 against the real GPU path and time
reversal (the spectrum at -k equals the one at k).

Tolerances as in the real FP64 parity tests: H x 1e-13 relative (summation
order only), filter 1e-11, bounds 1e-9, projection 1e-12 of sum |x_k y_k|,
Ritz values 1e-8 Ha, subspace distance 1e-7."""
import numpy as np
import pytest

import oracle
from oracle import kpoint
from paper_2302_09708_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2302_09708_gb300 import sparc  # noqa: E402

DEV = torch.device("cuda:0")
P, D = synth.PERIODIC, synth.DIRICHLET

CASES = {
    # grid, h, bc, atoms, seed, k (1/bohr)
    "periodic": ((13, 14, 15), 0.5, (P, P, P), 3, 61, (0.21, -0.13, 0.37)),
    "dirichlet_z": ((14, 13, 16), 0.5, (P, P, D), 3, 62, (0.3, 0.1, 0.9)),
    "one_periodic_axis": ((15, 13, 13), 0.5, (P, D, D), 2, 63, (-0.41, 0.0, 0.0)),
    "zone_boundary": ((14, 14, 14), 0.5, (P, P, P), 2, 64, (np.pi / 7.0, 0.0, np.pi / 7.0)),
}


def system(name):
    shape, h, bc, na, seed, k = CASES[name]
    return synth.random_system(shape, h, bc, na, seed=seed), np.array(k)


def cplx(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.complex128)).to(DEV)


def rand_block(ns, nd, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((ns, nd)) + 1j * r.standard_normal((ns, nd))


def subspace_distance(A, B):
    Qa, _ = np.linalg.qr(A.T)
    Qb, _ = np.linalg.qr(B.T)
    return float(np.linalg.norm(Qb - Qa @ (Qa.conj().T @ Qb)))


@pytest.mark.parametrize("name", list(CASES))
def test_hpsi_kpoint(name):
    s, k = system(name)
    ko = kpoint.KOracle(s, k)
    X = rand_block(4, s.nd, 1)
    h = sparc.Handle(s, "fp64", ns_max=4, kvec=k)
    Y = h.hpsi(cplx(X)).cpu().numpy()
    ref = ko.hpsi(X)
    err = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    assert err < 1e-13, err
    h.close()


@pytest.mark.parametrize("name", ["periodic", "dirichlet_z"])
def test_bounds_and_filter_kpoint(name):
    s, k = system(name)
    ko = kpoint.KOracle(s, k)
    h = sparc.Handle(s, "fp64", ns_max=5, kvec=k)
    for seed in (0, 99):
        a0, b = h.spectrum_bounds(24, seed)
        ra0, rb, *_ = ko.lanczos(24, seed)
        assert abs(a0 - ra0) < 1e-9 * max(1, abs(ra0)) and abs(b - rb) < 1e-9 * abs(rb)
    ra0, rb, *_ = ko.lanczos(32, 0)
    a = ra0 + 0.1 * (rb - ra0)
    X = rand_block(5, s.nd, 2)
    Xd = cplx(X)
    h.cheb_filter(Xd, 9, a, rb, ra0)
    got = Xd.cpu().numpy()
    ref = ko.cheb_filter(X, 9, a, rb, ra0)
    for n in range(5):
        assert np.max(np.abs(got[n] - ref[n])) < 1e-11 * np.max(np.abs(ref[n]))
    h.close()


def test_project_and_rotate_kpoint():
    s, k = system("periodic")
    h = sparc.Handle(s, "fp64", ns_max=24, kvec=k)
    X, Y = rand_block(24, s.nd, 3), rand_block(24, s.nd, 4)
    Hs, Ms = h.project(cplx(X), cplx(Y))
    rH, rM = kpoint.project(X, Y)
    aX, aY = np.abs(X), np.abs(Y)
    bH, bM = 1e-12 * (aX @ aY.T), 1e-12 * (aX @ aX.T)
    # the GPU form makes Hs Hermitian from its upper triangle (real diagonal),
    # as it is in a step (Yt = H Xt): strict upper triangle and real diagonal
    iu = np.triu_indices(24, 1)
    Hg = Hs.cpu().numpy()
    assert np.all(np.abs(Hg[iu] - rH[iu]) <= bH[iu])
    assert np.all(np.abs(np.diag(Hg) - np.diag(rH).real) <= np.diag(bH))
    assert np.max(np.abs(Hg - Hg.conj().T)) == 0.0
    assert np.all(np.abs(Ms.cpu().numpy() - rM) <= bM)
    Z = np.random.default_rng(5).standard_normal((24, 24)) + 1j * np.random.default_rng(6).standard_normal((24, 24))
    R = h.rotate(cplx(X), cplx(Z)).cpu().numpy()
    ref = kpoint.rotate(X, Z)
    assert np.all(np.abs(R - ref) <= 1e-12 * (np.abs(Z).T @ aX))
    h.close()


def _hpd_pair(n, cond, rng, levels=None):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    M = (Q * np.logspace(0, -np.log10(cond), n)) @ Q.conj().T
    M = 0.5 * (M + M.conj().T)
    ev = np.sort(rng.uniform(-3, 40, n))
    for i0, mult in levels or ():
        ev[i0:i0 + mult] = ev[i0]
    ev = np.sort(ev)
    Pm, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    L = np.linalg.cholesky(M)
    H = L @ ((Pm * ev) @ Pm.conj().T) @ L.conj().T
    return 0.5 * (H + H.conj().T), M, ev


@pytest.mark.parametrize("n,cond,levels", [(1, 1, None), (7, 100, None), (40, 1e4, None),
                                           (64, 1e6, None), (48, 10, [(5, 12), (30, 6)])])
def test_subspace_eig_kpoint(n, cond, levels):
    rng = np.random.default_rng(n)
    H, M, ev = _hpd_pair(n, cond, rng, levels)
    s, k = system("periodic")
    h = sparc.Handle(s, "fp64", ns_max=max(n, 1), kvec=k)
    lam, Z = h.subspace_eig(cplx(H), cplx(M))
    lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
    rlam, rZ = kpoint.gen_eig(H, M)
    scale = max(1.0, cond / 1e4)
    amax = np.max(np.abs(rlam))
    assert np.max(np.abs(lam - rlam)) < 1e-9 * scale * amax
    assert np.max(np.abs(lam - ev)) < 1e-9 * scale * amax
    assert np.max(np.abs(Z.conj().T @ M @ Z - np.eye(n))) < 1e-9 * scale
    assert np.max(np.abs(H @ Z - M @ Z * lam)) < 1e-9 * scale * np.max(np.abs(H))
    for i0, mult in levels or ():
        c = np.abs(rlam - ev[i0]) < 1e-8 * amax
        assert c.sum() == mult
        Pg, Pr = Z[:, c] @ Z[:, c].conj().T, rZ[:, c] @ rZ[:, c].conj().T
        assert np.max(np.abs(Pg - Pr)) < 1e-9 * np.max(np.abs(Pr))
    h.close()


def test_subspace_eig_kpoint_not_spd():
    s, k = system("periodic")
    n = 10
    H, M, _ = _hpd_pair(n, 10, np.random.default_rng(7))
    M[3, 3] = -1.0
    h = sparc.Handle(s, "fp64", ns_max=n, kvec=k)
    with pytest.raises(sparc.SparcError) as ei:
        h.subspace_eig(cplx(H), cplx(M))
    assert ei.value.status == sparc.SPARC_ERR_NOT_SPD
    h.close()


@pytest.mark.parametrize("name,ns,degree", [("periodic", 16, 12), ("dirichlet_z", 12, 10),
                                            ("zone_boundary", 20, 15)])
def test_chefsi_step_kpoint_vs_oracle(name, ns, degree):
    s, k = system(name)
    ko = kpoint.KOracle(s, k)
    a0, b, *_ = ko.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    X0 = synth.random_orbitals(s.nd, ns, seed=17).astype(np.complex128)
    h = sparc.Handle(s, "fp64", ns_max=ns, kvec=k)
    Xd = cplx(X0)
    lam = h.chefsi_step(Xd, degree, bounds=(a, b, a0))
    X1 = Xd.cpu().numpy()
    rX, rlam = ko.chefsi_step(X0, degree, a, b, a0)
    assert np.max(np.abs(lam - rlam)) < 1e-8, np.max(np.abs(lam - rlam))
    assert subspace_distance(X1, rX) < 1e-7
    assert np.max(np.abs(X1.conj() @ X1.T - np.eye(ns))) < 1e-9
    # library bounds, then a second step from the first's cut-off
    lam2 = h.chefsi_step(Xd, degree)
    assert np.all(np.isfinite(lam2)) and lam2[0] <= lam[0] + 1e-9
    h.close()


def test_kpoint_gamma_matches_real_path_and_time_reversal():
    """k = 0: the complex path on a real start block gives the real path's Ritz
    values; the spectrum of H(-k) equals that of H(k) (H(-k) = conj H(k))."""
    s, k = system("periodic")
    ns, m = 10, 10
    X0 = synth.random_orbitals(s.nd, ns, seed=23)
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    hr = sparc.Handle(s, "fp64", ns_max=ns, options_flags=2)
    lr = hr.chefsi_step(torch.from_numpy(X0).to(DEV), m, bounds=(a, b, a0))
    hk = sparc.Handle(s, "fp64", ns_max=ns, kvec=(0.0, 0.0, 0.0))
    lk = hk.chefsi_step(cplx(X0), m, bounds=(a, b, a0))
    assert np.max(np.abs(lk - lr)) < 1e-9
    ko = kpoint.KOracle(s, k)
    ka0, kb, *_ = ko.lanczos(32, 0)
    ka = ka0 + 0.1 * (kb - ka0)
    Xc = X0.astype(np.complex128)
    lp = sparc.Handle(s, "fp64", ns_max=ns, kvec=k).chefsi_step(cplx(Xc), m, bounds=(ka, kb, ka0))
    lm = sparc.Handle(s, "fp64", ns_max=ns, kvec=-k).chefsi_step(cplx(Xc.conj()), m,
                                                                 bounds=(ka, kb, ka0))
    assert np.max(np.abs(lp - lm)) < 1e-9
    hr.close()
    hk.close()


def test_kpoint_rejects_real_blocks_and_real_only_calls():
    s, k = system("periodic")
    h = sparc.Handle(s, "fp64", ns_max=4, kvec=k)
    with pytest.raises(sparc.SparcError) as ei:
        h.hpsi(torch.zeros((4, s.nd), dtype=torch.float64, device=DEV))
    assert ei.value.status == sparc.SPARC_ERR_INVALID_ARG
    with pytest.raises(sparc.SparcError):
        h.density(torch.zeros((4, s.nd), dtype=torch.complex128, device=DEV),
                  torch.zeros(4, dtype=torch.float64, device=DEV))
    h.close()
    with pytest.raises(sparc.SparcError):
        sparc.Handle(s, "mixed", ns_max=4, kvec=k)
