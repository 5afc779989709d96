"""Grids the TMA ring stencil does not fit, which take the generic local
stencil (y-slabs of whole rows) or, where a row is too narrow or too wide for
it, the tiled one, each followed by the tiled nonlocal pass: x shorter than the
stencil radius, x equal to it (Dirichlet), y shorter than the radius (halo rows
that wrap more than once), a last slab with fewer rows than the others, and a
row wider than one slab can hold.  H x, the Chebyshev filter and a full step
against the oracle, FP64 and FP32; tolerances as the other parity tests."""
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

GRIDS = {
    # shape, h, bc, atoms
    "tiny_x": ((5, 9, 11), 0.7, (0, 0, 0), 1),
    "short_y": ((7, 4, 10), 0.7, (0, 0, 1), 1),
    "x_equals_radius": ((6, 30, 8), 0.5, (1, 0, 0), 2),
    "ragged_slab": ((36, 31, 12), 0.5, (0, 0, 0), 3),
    "row_too_wide": ((520, 3, 4), 0.5, (0, 1, 0), 1),
}


def system(name):
    shape, h, bc, na = GRIDS[name]
    return synth.random_system(shape, h, bc, na, seed=71)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(GRIDS))
def test_hpsi_generic_grids(name, precision):
    s = system(name)
    o = oracle.Oracle(s)
    ns = 5
    dt = torch.float64 if precision == "fp64" else torch.float32
    X = np.random.default_rng(2).standard_normal((ns, s.nd))
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)  # the FP32 block's exact values
    h = sparc.Handle(s, precision, ns_max=ns)
    Y = h.hpsi(torch.from_numpy(X).to(DEV, dt)).double().cpu().numpy()
    ref = o.hpsi(X)
    err = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    assert err < (1e-13 if precision == "fp64" else 2e-6), err
    h.close()


@pytest.mark.parametrize("name", ["short_y", "ragged_slab", "row_too_wide"])
def test_cheb_filter_generic_grids(name):
    s = system(name)
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(24, 0)
    a = a0 + 0.1 * (b - a0)
    ns = 4
    X = np.random.default_rng(3).standard_normal((ns, s.nd))
    h = sparc.Handle(s, "fp64", ns_max=ns)
    Xd = torch.from_numpy(X).to(DEV)
    h.cheb_filter(Xd, 9, a, b, a0)
    got = Xd.cpu().numpy()
    ref = o.cheb_filter(X, 9, a, b, a0)
    for n in range(ns):
        assert np.max(np.abs(got[n] - ref[n])) < 1e-11 * np.max(np.abs(ref[n]))
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_ragged_slab_vs_oracle(precision):
    s = system("ragged_slab")
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    ns, m = 24, 12
    X0 = synth.random_orbitals(s.nd, ns, seed=5)
    dt = torch.float64 if precision == "fp64" else torch.float32
    h = sparc.Handle(s, precision, ns_max=ns)
    Xd = torch.from_numpy(X0).to(DEV, dt)
    lam = h.chefsi_step(Xd, m, bounds=(a, b, a0))
    _, rlam = o.chefsi_step(X0, m, a, b, a0)
    if precision == "fp64":
        assert np.max(np.abs(lam - rlam)) < 1e-8
    else:
        ne = synth.electrons_for(ns)
        rf, _ = oracle.fermi_occupations(rlam, ne, 0.01)
        occ = rf > 1e-6
        assert np.max(np.abs(lam - rlam)[occ]) < 1e-6
    h.close()


def test_dense_projectors_double_fp32_vs_oracle():
    """FP64 blocks in double-FP32 arithmetic (options bit 2) on a system whose
    projectors overlap many deep (more than four entries per grid point): the
    ring runs without its point-by-point nonlocal add and the tiled FP64 pass
    adds the nonlocal term (and, in the filter, the next degree's
    coefficients).  H x within 1e-12 and the filter within 1e-11 of the
    oracle, as the other double-FP32 parity tests."""
    s = synth.random_system((32, 32, 40), 0.35, (0, 0, 1), 30, seed=72)
    assert s.supp_ptr[-1] * 4 > 4 * s.nd  # > 4 projector entries per point
    o = oracle.Oracle(s)
    ns = 4
    X = np.random.default_rng(4).standard_normal((ns, s.nd))
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=4)
    Y = h.hpsi(torch.from_numpy(X).to(DEV)).cpu().numpy()
    ref = o.hpsi(X)
    assert np.max(np.abs(Y - ref)) / np.max(np.abs(ref)) < 1e-12
    a0, b, *_ = o.lanczos(24, 0)
    a = a0 + 0.1 * (b - a0)
    Xd = torch.from_numpy(X).to(DEV)
    h.cheb_filter(Xd, 8, a, b, a0)
    got = Xd.cpu().numpy()
    ref = o.cheb_filter(X, 8, a, b, a0)
    for n in range(ns):
        assert np.max(np.abs(got[n] - ref[n])) < 1e-11 * np.max(np.abs(ref[n]))
    h.close()
