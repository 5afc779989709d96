"""GPU parity of the occupation and density kernels (Fermi-Dirac occupations
of the Ritz values, rho = (2/h^3) sum_n f_n X_n^2) against the oracle, alone
and after a CheFSI step.

Tolerances: occupations and mu to 1e-10 (both sides bisect to |2 sum f - Ne|
< 1e-12; only the summation order differs); FP64 density to 1e-13 relative;
FP32 density to 1e-6 relative (FP32 products summed in groups of 16); after a
step, density L1 per electron h^3 sum |d rho| / Ne to 1e-8 (FP64) and 1e-6
(mixed, the stated mixed-precision target)."""
import numpy as np
import pytest

import oracle
from paper_2302_09708_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts skip via -m "not gpu"
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2302_09708_gb300 import sparc  # noqa: E402

DEV = torch.device("cuda:0")


def to_dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(X)).to(DEV, dtype)


@pytest.mark.parametrize("ns,kT", [(1, 0.01), (40, 0.01), (300, 0.02), (1300, 0.01),
                                   (4800, 0.01)])
def test_occupations_vs_oracle(ns, kT):
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    h = sparc.Handle(s, "fp64", ns_max=1)
    rng = np.random.default_rng(ns)
    lam = np.sort(rng.uniform(-2.0, 1.0, ns))
    ne = synth.electrons_for(ns) if ns > 5 else 1.0
    occ, mu = h.occupations(to_dev(lam), ne, kT)
    torch.cuda.synchronize()
    rf, rmu = oracle.fermi_occupations(lam, ne, kT)
    assert abs(float(mu) - rmu) < 1e-10, (float(mu), rmu)
    f = occ.cpu().numpy()
    assert np.max(np.abs(f - rf)) < 1e-10
    assert abs(2 * f.sum() - ne) < 1e-9


def test_occupations_degenerate_level():
    """All Ritz values equal: every state holds Ne / (2 Ns)."""
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    h = sparc.Handle(s, "fp64", ns_max=1)
    ns, ne = 12, 7.0
    occ, _ = h.occupations(to_dev(np.full(ns, -0.25)), ne, 0.01)
    assert np.allclose(occ.cpu().numpy(), ne / (2 * ns), atol=1e-12)


def test_occupations_reject_bad_arguments():
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    h = sparc.Handle(s, "fp64", ns_max=1)
    lam = to_dev(np.zeros(4))
    for ne, kT in ((8.0, 0.01), (0.0, 0.01), (2.0, 0.0), (2.0, -1.0)):
        with pytest.raises(sparc.SparcError) as ei:
            h.occupations(lam, ne, kT)
        assert ei.value.status == sparc.SPARC_ERR_INVALID_ARG


CASES = [  # (grid, bc, ns, ld padding): split and unsplit launches, ragged Nd, odd ld
    ((24, 24, 24), (0, 0, 0), 40, 0),
    ((15, 13, 14), (1, 1, 1), 17, 3),
    ((13, 17, 19), (0, 0, 0), 64, 1),
    ((96, 96, 72), (0, 0, 0), 3, 0),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("grid,bc,ns,pad", CASES)
def test_density_kernel_vs_oracle(grid, bc, ns, pad, precision):
    s = synth.free_system(grid, 0.45, bc)
    ld = s.nd + pad
    rng = np.random.default_rng(ns + pad)
    X = np.zeros((ns, ld))
    X[:, : s.nd] = rng.standard_normal((ns, s.nd))
    f = rng.uniform(0.0, 1.0, ns)
    dt = torch.float32 if precision == "mixed" else torch.float64
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)
    h = sparc.Handle(s, precision, ns_max=ns)
    rho = h.density(to_dev(X, dt), to_dev(f)).cpu().numpy()
    ref = oracle.density(X, f, s.nd, s.h)
    err = np.max(np.abs(rho - ref)) / np.max(np.abs(ref))
    assert err < (1e-6 if precision == "mixed" else 1e-13), err


def test_density_of_no_orbitals_is_zero():
    s = synth.free_system((13, 13, 13), 0.5, (0, 0, 0))
    h = sparc.Handle(s, "fp64", ns_max=2)
    rho = torch.full((s.nd,), 5.0, dtype=torch.float64, device=DEV)
    X = torch.zeros((1, s.nd), dtype=torch.float64, device=DEV)
    occ = torch.zeros(1, dtype=torch.float64, device=DEV)
    sparc.sparc_density(h.h, X[:0], occ[:0], rho)
    assert float(rho.abs().max()) == 0.0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_density_after_step_vs_oracle(precision, tol):
    """24^3 bulk system: one CheFSI step, occupations and density on the GPU
    against the oracle's step, occupations and density (the density is
    invariant under rotations within degenerate levels)."""
    s = synth.make_workload_system("bulk24")
    o = oracle.Oracle(s)
    ns, m = 40, 20
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    X0 = synth.random_orbitals(s.nd, ns, seed=synth.workload_seed("bulk24"))
    rX, rlam = o.chefsi_step(X0, m, a, b, a0)
    for _ in range(2):
        rX, rlam = o.chefsi_step(rX, m, rlam[-1], b, a0)
    ne = synth.electrons_for(ns)
    rf, _ = oracle.fermi_occupations(rlam, ne, 0.01)
    rrho = oracle.density(rX, rf, s.nd, s.h)

    dt = torch.float32 if precision == "mixed" else torch.float64
    h = sparc.Handle(s, precision, ns_max=ns)
    Xd = to_dev(X0, dt)
    lam = h.chefsi_step(Xd, m, bounds=(a, b, a0))
    for _ in range(2):
        lam = h.chefsi_step(Xd, m, bounds=(lam[-1], b, a0))
    occ, _ = h.occupations(to_dev(lam), ne, 0.01)
    rho = h.density(Xd, occ).cpu().numpy()
    l1 = s.h ** 3 * np.sum(np.abs(rho - rrho)) / ne
    assert l1 < tol, l1
    assert abs(s.h ** 3 * rho.sum() - ne) < 1e-6 * ne
