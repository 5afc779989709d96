"""Parity at the benchmark's full size (96^3 periodic bulk, h = 0.4, 216 atoms,
Ns = 1300, the launch configuration bench.py times): the CUDA path runs on all
1300 orbitals; the oracle checks sampled columns (every operation here acts on
columns independently) and Rayleigh-Ritz invariants that hold at any size."""
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
NS = 1300
SAMPLE = [0, 1, 517, 1299]


@pytest.fixture(scope="module")
def system():
    return synth.make_workload_system("bulk96")


@pytest.fixture(scope="module")
def o(system):
    return oracle.Oracle(system)


@pytest.fixture(scope="module")
def X0(system):
    rng = np.random.default_rng(7)
    return rng.standard_normal((NS, system.nd))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hpsi_full_size_sampled(system, o, X0, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    h = sparc.Handle(system, precision, ns_max=NS)
    Xd = torch.from_numpy(X0).to(DEV, dt)
    Y = h.hpsi(Xd)
    torch.cuda.synchronize()
    xs = Xd[SAMPLE].double().cpu().numpy()
    ref = o.hpsi(xs)
    got = Y[SAMPLE].double().cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < (1e-13 if precision == "fp64" else 2e-6), err
    h.close()


def test_filter_full_size_sampled(system, o, X0):
    h = sparc.Handle(system, "fp64", ns_max=NS)
    a0, b = h.spectrum_bounds(32, 0)
    ra0, rb, *_ = o.lanczos(32, 0)
    assert abs(a0 - ra0) < 1e-9 and abs(b - rb) < 1e-9
    a = a0 + 0.1 * (b - a0)
    X = X0  # the filter acts column by column; no orthonormal start is needed
    Xd = torch.from_numpy(X).to(DEV)
    h.cheb_filter(Xd, 20, a, b, a0)
    torch.cuda.synchronize()
    got = Xd[SAMPLE].cpu().numpy()
    ref = o.cheb_filter(X[SAMPLE], 20, a, b, a0)
    for k in range(len(SAMPLE)):
        err = np.max(np.abs(got[k] - ref[k])) / np.max(np.abs(ref[k]))
        assert err < 1e-11, (SAMPLE[k], err)
    h.close()


def test_chefsi_step_full_size_invariants(system, o, X0):
    """Full step at Ns = 1300: X^T X = I on sampled pairs, Ritz values ascending,
    below the spectrum bound b, and equal to the oracle's Rayleigh quotients of
    the rotated columns.  (a0 from a short Lanczos run is only an estimate of the
    lowest eigenvalue from above, so Ritz values may lie below it.)"""
    h = sparc.Handle(system, "fp64", ns_max=NS)
    a0, b = h.spectrum_bounds(32, 0)
    a = a0 + 0.1 * (b - a0)
    Xd = torch.from_numpy(X0).to(DEV)  # Rayleigh-Ritz does not need an orthonormal start
    lam = h.chefsi_step(Xd, 20, bounds=(a, b, a0))
    torch.cuda.synchronize()
    assert np.all(np.diff(lam) >= 0) and lam[-1] <= b
    Xs = Xd[SAMPLE].cpu().numpy()
    G = Xs @ Xs.T
    assert np.max(np.abs(G - np.eye(len(SAMPLE)))) < 1e-9
    HX = o.hpsi(Xs)
    rq = np.einsum("ij,ij->i", Xs, HX)
    assert np.max(np.abs(rq - lam[SAMPLE])) < 1e-8
    h.close()
