"""Batched form: several independent systems of uneven size stepped by one
batched call (per-member filter chains on concurrent streams, the batched
eigensolver, one CUDA graph), against the oracle per member and against
per-member single steps; and the batched eigensolver alone
(sparc_batch_subspace_eig) against the oracle's generalised eigensolver on
problems that span every cluster size, the per-member path above 512,
degenerate levels and ill-conditioned overlaps.  FP64
members meet the FP64 targets (Ritz values within 1e-8 Ha); mixed members meet
the mixed ones against the FP64 oracle (occupied Ritz values within 1e-6 Ha,
density L1 within 1e-6 per electron)."""
import numpy as np
import pytest

import oracle
from paper_2302_09708_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2302_09708_gb300 import sparc  # noqa: E402

DEV = torch.device("cuda:0")

MEMBERS = [
    dict(shape=(24, 24, 24), bc=(0, 0, 0), natoms=5, ns=40, degree=16, seed=501),
    dict(shape=(26, 25, 27), bc=(0, 0, 0), natoms=9, ns=57, degree=20, seed=502),
    dict(shape=(18, 20, 22), bc=(0, 0, 1), natoms=4, ns=23, degree=24, seed=503),
    dict(shape=(30, 24, 28), bc=(1, 0, 0), natoms=12, ns=64, degree=17, seed=504),
]
# an FP64 member whose Rayleigh-Ritz step runs on a two-CTA cluster of the
# batched eigensolver (Ns > 128).  Mixed precision leaves it out: after one step
# from random orbitals its highest occupied Ritz values are still far from
# converged, and FP32 filtering moves them by about 2e-6 Ha, above the
# occupied-state target, whatever eigensolver runs after it.
BIG = dict(shape=(28, 26, 24), bc=(0, 0, 0), natoms=10, ns=150, degree=18, seed=505)


def _members(precision):
    return MEMBERS + ([BIG] if precision == "fp64" else [])


def _setup(precision):
    systems, handles, X0, bounds = [], [], [], []
    for m in _members(precision):
        s = synth.random_system(m["shape"], 0.5, m["bc"], m["natoms"], seed=m["seed"])
        o = oracle.Oracle(s)
        a0, b, *_ = o.lanczos(32, 0)
        bounds.append((a0 + 0.1 * (b - a0), b, a0))
        systems.append((s, o))
        handles.append(sparc.Handle(s, precision, ns_max=m["ns"]))
        X0.append(synth.random_orbitals(s.nd, m["ns"], seed=m["seed"] + 7))
    return systems, handles, X0, bounds


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_step_vs_oracle_and_single(precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    systems, handles, X0, bounds = _setup(precision)
    batch = sparc.Batch(handles)
    Xb = [torch.from_numpy(x).to(DEV, dt) for x in X0]
    members = _members(precision)
    degrees = [m["degree"] for m in members]
    for step in range(2):  # second call replays the captured graph
        lam_b = batch.chefsi_step(Xb, degrees, bounds=bounds)
        if step == 0:
            for i, ((s, o), m) in enumerate(zip(systems, members)):
                rX, rlam = o.chefsi_step(X0[i], m["degree"], *bounds[i])
                if precision == "fp64":
                    assert np.max(np.abs(lam_b[i] - rlam)) < 1e-8
                    continue
                ne = synth.electrons_for(m["ns"])
                rf, _ = oracle.fermi_occupations(rlam, ne, 0.01)
                occ = rf > 1e-6
                assert np.max(np.abs(lam_b[i] - rlam)[occ]) < 1e-6, (i, lam_b[i] - rlam)
                f, _ = handles[i].occupations(torch.from_numpy(lam_b[i]).to(DEV), ne, 0.01)
                rho = handles[i].density(Xb[i], f).cpu().numpy()
                rrho = oracle.density(rX, rf, s.nd, s.h)
                l1 = s.h ** 3 * np.sum(np.abs(rho - rrho)) / ne
                assert l1 < 1e-6, (i, l1)
        for i, ((s, o), m) in enumerate(zip(systems, members)):
            Xs = torch.from_numpy(X0[i]).to(DEV, dt)
            lam_s = handles[i].chefsi_step(Xs, m["degree"], bounds=bounds[i])
            assert np.max(np.abs(lam_b[i] - lam_s)) < (1e-10 if precision == "fp64" else 1e-5)
            X0[i] = Xs.double().cpu().numpy()
            Xb[i].copy_(Xs)
        assert batch.launches() > 0
    batch.close()


def _spd_pair(n, cond, rng, levels=()):
    """Hs, Ms with Ms of condition `cond` and generalised eigenvalues `ev`
    (levels: (first index, multiplicity) of exactly repeated eigenvalues)."""
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Q * np.logspace(0, -np.log10(cond), n)) @ Q.T
    M = 0.5 * (M + M.T)
    ev = np.sort(rng.uniform(-3, 40, n))
    for i0, mult in levels:
        ev[i0:i0 + mult] = ev[i0]
    ev = np.sort(ev)
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    L = np.linalg.cholesky(M)
    H = L @ ((P * ev) @ P.T) @ L.T
    return 0.5 * (H + H.T), M, ev


# n, cond(Ms), degenerate levels; cluster sizes 1 (n <= 128), 2, 4, 8 and the
# one-by-one path (n > 512)
EIG_CASES = [(1, 1, ()), (2, 10, ()), (7, 100, ()), (40, 1e4, ()), (33, 10, "all"),
             (50, 1e3, ((3, 8),)), (65, 1e6, ()), (130, 1e2, ()), (170, 1e3, ((9, 4),)),
             (200, 1e3, ((20, 5), (100, 3))), (300, 1e2, ((40, 12),)), (511, 10, ()),
             (520, 10, ())]


def _eig_batch_inputs(seed):
    rng = np.random.default_rng(seed)
    out = []
    for n, cond, levels in EIG_CASES:
        if levels == "all":  # fully degenerate: H = c M
            _, M, _ = _spd_pair(n, cond, rng)
            out.append((2.5 * M, M, np.full(n, 2.5), cond, ((0, n),)))
        else:
            H, M, ev = _spd_pair(n, cond, rng, levels)
            out.append((H, M, ev, cond, levels))
    return out


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).to(DEV)


def test_batch_subspace_eig_vs_oracle():
    s = synth.random_system((12, 12, 12), 0.5, (0, 0, 0), 2, seed=77)
    cases = _eig_batch_inputs(2024)
    handles = [sparc.Handle(s, "fp64", ns_max=H.shape[0]) for H, *_ in cases]
    batch = sparc.Batch(handles)
    lams, Zs = batch.subspace_eig([_dev(c[0]) for c in cases], [_dev(c[1]) for c in cases])
    for (H, M, ev, cond, levels), lam, Z, h in zip(cases, lams, Zs, handles):
        n = H.shape[0]
        lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
        rlam, rZ = oracle.gen_eig(H, M)
        scale = max(1.0, cond / 1e4)
        amax = np.max(np.abs(rlam))
        assert np.max(np.abs(lam - rlam)) < 1e-9 * scale * amax, n
        assert np.max(np.abs(lam - ev)) < 1e-9 * scale * amax, n
        assert np.max(np.abs(Z.T @ M @ Z - np.eye(n))) < 1e-9 * scale, n
        assert np.max(np.abs(H @ Z - M @ Z * lam)) < 1e-9 * scale * np.max(np.abs(H)), n
        cols = np.argmax(np.abs(Z), axis=0)
        assert np.all(Z[cols, np.arange(n)] > 0), n
        for i0, mult in levels:  # the eigenspace of a repeated level is unique
            c = np.abs(rlam - ev[i0]) < 1e-8 * amax
            assert c.sum() == mult, n
            Pg, Pr = Z[:, c] @ Z[:, c].T, rZ[:, c] @ rZ[:, c].T
            assert np.max(np.abs(Pg - Pr)) < 1e-9 * scale * np.max(np.abs(Pr)), n
        # the same problem through the single-handle solver
        lam1, _ = h.subspace_eig(_dev(H), _dev(M))
        assert np.max(np.abs(lam - lam1.cpu().numpy())) < 1e-10 * scale * amax, n
    batch.close()
    for h in handles:
        h.close()


def test_batch_subspace_eig_not_spd_names_member():
    s = synth.random_system((12, 12, 12), 0.5, (0, 0, 0), 2, seed=78)
    rng = np.random.default_rng(9)
    sizes = [20, 150, 260]
    pairs = [_spd_pair(n, 10, rng)[:2] for n in sizes]
    handles = [sparc.Handle(s, "fp64", ns_max=n) for n in sizes]
    batch = sparc.Batch(handles)
    bad = pairs[1][1].copy()
    bad[7, 7] = -2.0
    with pytest.raises(sparc.SparcError) as ei:
        batch.subspace_eig([_dev(H) for H, _ in pairs],
                           [_dev(pairs[0][1]), _dev(bad), _dev(pairs[2][1])])
    assert ei.value.status == sparc.SPARC_ERR_NOT_SPD and "system 1" in str(ei.value)
    # the batch and its handles stay usable
    lams, _ = batch.subspace_eig([_dev(H) for H, _ in pairs], [_dev(M) for _, M in pairs])
    for (H, M), lam in zip(pairs, lams):
        rlam, _ = oracle.gen_eig(H, M)
        assert np.max(np.abs(lam.cpu().numpy() - rlam)) < 1e-9 * np.max(np.abs(rlam))
    batch.close()
    for h in handles:
        h.close()
