"""GPU parity of the nonlocal-force kernels (gradient of the orbitals at the
projector supports, then the projector contractions) against the oracle, on
periodic, Dirichlet and mixed grids with wrapped supports, ragged sizes and
padded leading dimensions, for FP64 and FP32 blocks, and after a CheFSI step.

Tolerance: 1e-12 of max |F| (both sides sum the same FP64 products in
different orders; FP32 blocks are compared against the oracle on the same
FP32-rounded values, which the kernel widens exactly)."""
import numpy as np
import pytest

from oracle import forces as oforces
from paper_2302_09708_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts skip via -m "not gpu"
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2302_09708_gb300 import sparc  # noqa: E402

DEV = torch.device("cuda:0")
P, D = synth.PERIODIC, synth.DIRICHLET


def to_dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(X)).to(DEV, dtype)


def edge_system(shape, bc, seed, h=0.5):
    L = np.array(shape) * h
    pos = np.array([[0.3, 0.2, 0.4], [L[0] - 0.4, 0.55 * L[1], 0.6 * L[2]],
                    [0.5 * L[0], L[1] - 0.1, L[2] - 0.35], [0.45 * L[0], 0.5 * L[1], 0.5 * L[2]]])
    return synth.random_system(shape, h, bc, 4, seed, positions=pos)


CASES = [  # (grid, bc, ns, ld padding)
    ((13, 13, 6), (P, P, D), 5, 0),
    ((13, 14, 13), (P, P, P), 17, 3),
    ((9, 10, 11), (D, D, D), 8, 0),
    ((15, 13, 14), (D, P, P), 33, 1),
    ((24, 24, 24), (P, P, P), 40, 0),
    ((13, 5, 4), (P, D, D), 3, 7),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("grid,bc,ns,pad", CASES)
def test_nonlocal_forces_vs_oracle(grid, bc, ns, pad, precision):
    s = edge_system(grid, bc, seed=sum(grid) + ns)
    ld = s.nd + pad
    rng = np.random.default_rng(ns + pad)
    X = np.zeros((ns, ld))
    X[:, : s.nd] = rng.standard_normal((ns, s.nd))
    f = rng.uniform(0.0, 1.0, ns)
    dt = torch.float32 if precision == "mixed" else torch.float64
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)
    h = sparc.Handle(s, precision, ns_max=ns)
    F = h.nonlocal_forces(to_dev(X, dt), to_dev(f)).cpu().numpy()
    ref = oforces.nonlocal_forces(s, X, f)
    assert F.shape == ref.shape == (s.natoms, 3)
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref)), (F, ref)


def test_nonlocal_forces_edge_cases():
    s = edge_system((13, 13, 6), (P, P, D), seed=3)
    h = sparc.Handle(s, "fp64", ns_max=4)
    X = to_dev(np.ones((1, s.nd)))
    occ = to_dev(np.ones(1))
    F = torch.full((s.natoms, 3), 7.0, dtype=torch.float64, device=DEV)
    sparc.sparc_nonlocal_forces(h.h, X[:0], occ[:0], F)
    assert float(F.abs().max()) == 0.0
    with pytest.raises(sparc.SparcError) as ei:
        sparc.sparc_nonlocal_forces(h.h, X.float(), occ, F)
    assert ei.value.status == sparc.SPARC_ERR_INVALID_ARG
    free = sparc.Handle(synth.free_system((13, 13, 13), 0.5, (P, P, P)), "fp64", ns_max=1)
    assert tuple(free.nonlocal_forces(to_dev(np.ones((1, 13 ** 3))), occ).shape) == (0, 3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonlocal_forces_after_step(precision):
    """Forces of the orbitals of a CheFSI step on the 24^3 bulk system (the
    GPU's own X, read back) against the oracle on the same X."""
    s = synth.make_workload_system("bulk24")
    ns, m = 40, 20
    h = sparc.Handle(s, precision, ns_max=ns)
    dt = torch.float32 if precision == "mixed" else torch.float64
    X = to_dev(synth.random_orbitals(s.nd, ns, seed=synth.workload_seed("bulk24")), dt)
    lam = None
    for _ in range(3):
        lam = h.chefsi_step(X, m)
    occ, _ = h.occupations(to_dev(lam), synth.electrons_for(ns), 0.01)
    F = h.nonlocal_forces(X, occ).cpu().numpy()
    ref = oforces.nonlocal_forces(s, X.double().cpu().numpy(), occ.cpu().numpy())
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(ref)) > 1e-6
