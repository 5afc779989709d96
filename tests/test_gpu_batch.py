"""Batched form: several independent systems of uneven size stepped by one
batched call (one launch per Chebyshev degree for all members, CUDA graph),
against the oracle per member and against per-member single steps.  FP64
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


def _setup(precision):
    systems, handles, X0, bounds = [], [], [], []
    for m in MEMBERS:
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
    degrees = [m["degree"] for m in MEMBERS]
    for step in range(2):  # second call replays the captured graph
        lam_b = batch.chefsi_step(Xb, degrees, bounds=bounds)
        if step == 0:
            for i, ((s, o), m) in enumerate(zip(systems, MEMBERS)):
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
        for i, ((s, o), m) in enumerate(zip(systems, MEMBERS)):
            Xs = torch.from_numpy(X0[i]).to(DEV, dt)
            lam_s = handles[i].chefsi_step(Xs, m["degree"], bounds=bounds[i])
            assert np.max(np.abs(lam_b[i] - lam_s)) < (1e-10 if precision == "fp64" else 1e-5)
            X0[i] = Xs.double().cpu().numpy()
            Xb[i].copy_(Xs)
        assert batch.launches() > 0
    batch.close()
