"""GPU tests of the ring stencil's thread shapes and of the wait bound.

Every thread shape computes each point with the same operations in the same
order, so H x and the filter must agree bit for bit across shapes; the shape
the tuner picks is reported through sparc_get_tuning.  With the timeout test
hook (options flag bit 3) the stencil first waits on a barrier that nothing
completes: the wait runs out after timeout_cycles, the kernel stops once its
loads in flight have landed, the step returns SPARC_ERR_TIMEOUT, and the
context is still usable afterwards."""
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

SYSTEMS = {
    "ring_periodic": lambda: synth.random_system((32, 32, 64), 0.45, (0, 0, 0), 3, seed=45),
    "ring_dirichlet_y": lambda: synth.random_system((48, 20, 17), 0.5, (0, 1, 1), 3, seed=46),
    "ring_dirichlet_x": lambda: synth.random_system((32, 24, 20), 0.5, (1, 0, 1), 3, seed=47),
}


def _shapes(s, precision):
    """Shape indices (1-based option values) the handle accepts."""
    h = sparc.Handle(s, precision, ns_max=4)
    X = torch.zeros((4, s.nd), dtype=h.dtype, device=DEV)
    h.hpsi(X)
    torch.cuda.synchronize()
    n = h.tuning()["candidates"]
    h.close()
    return list(range(1, n + 1))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_stencil_shapes_are_bit_identical(name, precision):
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    ns = 5
    dt = torch.float32 if precision == "mixed" else torch.float64
    X = torch.from_numpy(np.random.default_rng(3).standard_normal((ns, s.nd))).to(DEV, dt)
    outs = []
    for k in _shapes(s, precision):
        h = sparc.Handle(s, precision, ns_max=ns, stencil_shape=k)
        Y = h.hpsi(X)
        F = X.clone()
        h.cheb_filter(F, 5, a, b, a0)
        torch.cuda.synchronize()
        t = h.tuning()
        assert t["shape"] == k - 1 and t["threads"] > 0 and t["slab_rows"] > 0
        outs.append((Y.cpu(), F.cpu()))
        h.close()
    assert len(outs) >= 2
    for Y, F in outs[1:]:
        assert torch.equal(Y, outs[0][0]) and torch.equal(F, outs[0][1])
    # and they are the right values: against the oracle
    ref = o.hpsi(X.double().cpu().numpy())
    err = np.max(np.abs(outs[0][0].double().numpy() - ref)) / np.max(np.abs(ref))
    assert err < (2e-6 if precision == "mixed" else 1e-13), err


def test_tuner_reports_timed_shapes():
    s = SYSTEMS["ring_periodic"]()
    h = sparc.Handle(s, "mixed", ns_max=16)
    X = torch.from_numpy(np.random.default_rng(4).standard_normal((16, s.nd))).to(DEV, torch.float32)
    h.hpsi(X)
    torch.cuda.synchronize()
    t = h.tuning()
    assert t["ns"] == 16 and 0 <= t["shape"] < t["candidates"]
    ms = t["candidate_ms"]
    assert ms[t["shape"]] > 0 and ms[t["shape"]] == min(m for m in ms if m > 0)
    h.close()


def test_wait_bound_runs_out_and_reports_timeout():
    """FP64 handle with SIMT GEMMs and ns < 64 (no other waiting kernel in the
    step), the timeout hook on and a wait bound of 2e6 cycles (about 1 ms):
    every stencil launch's hooked wait runs out and the step returns
    SPARC_ERR_TIMEOUT; a handle without the hook then steps the same system to
    the oracle's Ritz values."""
    s = SYSTEMS["ring_periodic"]()
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    ns, m = 16, 6
    X0 = synth.random_orbitals(s.nd, ns, seed=21)
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=2 | 8, timeout_cycles=2_000_000)
    with pytest.raises(sparc.SparcError) as ei:
        h.chefsi_step(torch.from_numpy(X0).to(DEV), m, bounds=(a, b, a0))
    assert ei.value.status == sparc.SPARC_ERR_TIMEOUT
    h.close()
    g = sparc.Handle(s, "fp64", ns_max=ns, options_flags=2)
    lam = g.chefsi_step(torch.from_numpy(X0).to(DEV), m, bounds=(a, b, a0))
    _, rlam = o.chefsi_step(X0, m, a, b, a0)
    assert np.max(np.abs(lam - rlam)) < 1e-8
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_switching_stencil_paths_vs_oracle(precision):
    """Leading dimension Nd + 3 on a ring grid: degrees that touch the caller's
    block (not 16-byte aligned rows) take the generic stencil, the others the
    ring stencil and the tiled nonlocal pass, so the step switches between the
    two layouts of the projector coefficients; it still meets the oracle."""
    s = SYSTEMS["ring_periodic"]()
    o = oracle.Oracle(s)
    a0, b, *_ = o.lanczos(32, 0)
    a = a0 + 0.1 * (b - a0)
    ns, m = 12, 8
    X0 = synth.random_orbitals(s.nd, ns, seed=31)
    ld = s.nd + 3
    dt = torch.float32 if precision == "mixed" else torch.float64
    Xd = torch.zeros((ns, ld), dtype=dt, device=DEV)
    Xd[:, : s.nd] = torch.from_numpy(X0).to(DEV, dt)
    h = sparc.Handle(s, precision, ns_max=ns)
    lam = h.chefsi_step(Xd, m, bounds=(a, b, a0))
    _, rlam = o.chefsi_step(X0, m, a, b, a0)
    tol = 1e-6 if precision == "mixed" else 1e-8
    assert np.max(np.abs(lam - rlam)) < tol, np.max(np.abs(lam - rlam))
    assert float(Xd[:, s.nd:].abs().max()) == 0.0  # rows beyond Nd untouched
    h.close()
