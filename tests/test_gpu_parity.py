"""GPU parity: every step of the CUDA path (through the C ABI) against the FP64
CPU oracle on the same seeded inputs.

Tolerances (FP64 mode): H application to 1e-13 relative in FP64 arithmetic
(summation order is the only difference) and 1e-12 in the double-FP32 stencil
(48-bit pairs), filter to 1e-11, Ritz values to 1e-8 Ha and subspace distance
to 1e-7 (the stated FP64 targets); mixed mode checks FP32 operator application
to single-precision rounding and its Ritz values to 1e-6 Ha."""
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

SYSTEMS = {
    "bulk24": lambda: synth.make_workload_system("bulk24"),
    "ragged_periodic": lambda: synth.random_system((13, 17, 19), 0.5, (0, 0, 0), 3, seed=41),
    "dirichlet_z": lambda: synth.random_system((20, 18, 27), 0.45, (0, 0, 1), 4, seed=42),
    "all_dirichlet_odd": lambda: synth.random_system((15, 13, 14), 0.5, (1, 1, 1), 2, seed=43),
    "wide_x": lambda: synth.random_system((70, 13, 16), 0.5, (0, 1, 0), 3, seed=44),
    "free": lambda: synth.free_system((16, 16, 16), 0.5, (0, 0, 0), v0=0.3),
    # grids the TMA plane-ring stencil handles (x a multiple of 16, z split in chunks)
    "ring_periodic": lambda: synth.random_system((32, 32, 64), 0.45, (0, 0, 0), 3, seed=45),
    "ring_dirichlet_y": lambda: synth.random_system((48, 20, 17), 0.5, (0, 1, 1), 3, seed=46),
}


def to_dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(X)).to(DEV, dtype)


def subspace_distance(A, B):
    """|(I - Qa Qa^T) Qb|_F for orthonormal bases Qa, Qb of span(A^T), span(B^T):
    the Frobenius norm of the sines of the principal angles, equal to
    sqrt(ns - |Qa^T Qb|_F^2) but without that form's cancellation (whose
    rounding floor, sqrt(ns * 2^-52), is ~1e-7 at ns = 40)."""
    Qa, _ = np.linalg.qr(A.T)
    Qb, _ = np.linalg.qr(B.T)
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb)))


@pytest.mark.parametrize("flags", [0, 4])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hpsi_fp64(name, flags):
    """flags 0 (default): FP64 arithmetic throughout (summation order is the
    only difference, 1e-13); flags 4: ring grids run the double-FP32 stencil
    (48-bit pairs, 1e-12)."""
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    ns = 5
    X = np.random.default_rng(1).standard_normal((ns, s.nd))
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=flags)
    Y = h.hpsi(to_dev(X)).cpu().numpy()
    ref = o.hpsi(X)
    err = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    assert err < (1e-12 if flags & 4 else 1e-13), err


@pytest.mark.parametrize("ld_pad", [0, 3, 32])
def test_hpsi_leading_dimension(ld_pad):
    s = SYSTEMS["ragged_periodic"]()
    o = oracle.Oracle(s)
    ns, ld = 3, s.nd + ld_pad
    X = np.zeros((ns, ld))
    X[:, : s.nd] = np.random.default_rng(2).standard_normal((ns, s.nd))
    h = sparc.Handle(s, "fp64", ns_max=ns)
    Yd = torch.full((ns, ld), 7.0, dtype=torch.float64, device=DEV)
    h.hpsi(to_dev(X), Yd)
    Y = Yd.cpu().numpy()
    ref = o.hpsi(X[:, : s.nd])
    assert np.max(np.abs(Y[:, : s.nd] - ref)) < 1e-13 * np.max(np.abs(ref))
    assert np.all(Y[:, s.nd:] == 7.0)  # rows beyond Nd are never written


@pytest.mark.parametrize("name", ["bulk24", "dirichlet_z", "wide_x", "ring_periodic",
                                  "ring_dirichlet_y"])
def test_hpsi_fp32(name):
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    ns = 4
    X = np.random.default_rng(3).standard_normal((ns, s.nd)).astype(np.float32)
    h = sparc.Handle(s, "mixed", ns_max=ns)
    Y = h.hpsi(to_dev(X, torch.float32)).double().cpu().numpy()
    ref = o.hpsi(X.astype(np.float64))
    err = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    assert err < 2e-6, err


def bounds_for(o):
    a0, b, *_ = o.lanczos(32, 0)
    return a0, b, a0 + 0.1 * (b - a0)


@pytest.mark.parametrize("name", ["bulk24", "dirichlet_z", "free"])
def test_spectrum_bounds(name):
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    h = sparc.Handle(s, "fp64", ns_max=1)
    for seed in (0, 12345):
        a0, b = h.spectrum_bounds(32, seed)
        ra0, rb, *_ = o.lanczos(32, seed)
        assert abs(a0 - ra0) < 1e-9 * max(1, abs(ra0)), (a0, ra0)
        assert abs(b - rb) < 1e-9 * max(1, abs(rb)), (b, rb)


@pytest.mark.parametrize("name,degree", [("bulk24", 20), ("dirichlet_z", 7), ("ragged_periodic", 1),
                                         ("wide_x", 12), ("ring_periodic", 9),
                                         ("ring_dirichlet_y", 4)])
def test_cheb_filter_fp64(name, degree):
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    ns = 6
    X = synth.random_orbitals(s.nd, ns, seed=7)
    h = sparc.Handle(s, "fp64", ns_max=ns)
    Xd = to_dev(X)
    h.cheb_filter(Xd, degree, a, b, a0)
    got = Xd.cpu().numpy()
    ref = o.cheb_filter(X, degree, a, b, a0)
    for n in range(ns):
        err = np.max(np.abs(got[n] - ref[n])) / np.max(np.abs(ref[n]))
        assert err < 1e-11, (n, err)


def test_cheb_filter_host_buffer_matches_device():
    s = SYSTEMS["bulk24"]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    X = synth.random_orbitals(s.nd, 4, seed=8)
    h = sparc.Handle(s, "fp64", ns_max=4)
    Xd = to_dev(X)
    h.cheb_filter(Xd, 9, a, b, a0)
    Xh = X.copy()
    h.cheb_filter(Xh, 9, a, b, a0)
    assert np.array_equal(Xh, Xd.cpu().numpy())


@pytest.mark.parametrize("flags", [0, 2])
def test_project_and_rotate_fp64(flags):
    """FP64 projection and rotation: flags 2 = FP64 SIMT pipe (summation order
    only differs from the oracle); flags 0 = six-digit tensor-core split, whose
    error is bounded by 2^-42 sum_k |x_k| |y_k| entrywise (about 2^-45 expected:
    the first dropped digit level is 2^-48 of the chunk maxima)."""
    s = SYSTEMS["bulk24"]()
    ns = 40
    rng = np.random.default_rng(4)
    X, Y = rng.standard_normal((2, ns, s.nd))
    Y = 0.5 * (Y + X)
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=flags)
    Hs, Ms = h.project(to_dev(X), to_dev(Y))
    rH, rM = oracle.project(X, Y, s.nd)
    # upper triangle of Hs is X_i . Y_j; lower is mirrored
    iu = np.triu_indices(ns)
    eH = np.abs(Hs.cpu().numpy().T - rH)
    eM = np.abs(Ms.cpu().numpy() - rM)
    Z = rng.standard_normal((ns, ns))
    R = h.rotate(to_dev(X), to_dev(Z)).cpu().numpy()
    rR = oracle.rotate(X, Z, s.nd)
    eR = np.abs(R - rR)
    if flags & 2:
        assert np.max(eH[iu]) < 1e-10 and np.max(eM) < 1e-10
        assert np.max(eR) < 1e-11 * np.max(np.abs(rR))
    else:
        bH = 2.0 ** -42 * (np.abs(X) @ np.abs(Y).T)
        bM = 2.0 ** -42 * (np.abs(X) @ np.abs(X).T)
        assert np.all(eH[iu] <= bH[iu]), np.max(eH[iu] / bH[iu])
        assert np.all(eM <= bM), np.max(eM / bM)
        bR = 2.0 ** -42 * (np.abs(Z).T @ np.abs(X))
        assert np.all(eR <= bR), np.max(eR / bR)


@pytest.mark.parametrize("name,ns", [("ragged_periodic", 200), ("bulk24", 129), ("wide_x", 1),
                                     ("dirichlet_z", 300)])
def test_project_rotate_fp64_tensor_cores_vs_simt(name, ns):
    """Six-digit tensor-core projection/rotation against the FP64 SIMT kernels
    on orbital-like blocks (orthonormal columns, one column decaying to 1e-127).
    Bound: 2^-42 sum_k |x_k| |y_k| plus an absolute floor of 1e-30 (the split's
    running sums are FP32 pairs, so results far below FP32's range are lost)."""
    s = SYSTEMS[name]()
    ns = min(ns, s.nd // 4)
    X = synth.random_orbitals(s.nd, ns, seed=ns)
    X[0, : s.nd] *= np.exp(-np.arange(s.nd) / 50.0)  # a strongly peaked column
    Y = X * 0.7 + synth.random_orbitals(s.nd, ns, seed=ns + 1)
    tc = sparc.Handle(s, "fp64", ns_max=ns)
    simt = sparc.Handle(s, "fp64", ns_max=ns, options_flags=2)
    Xd, Yd = to_dev(X), to_dev(Y)
    H1, M1 = tc.project(Xd, Yd)
    H2, M2 = simt.project(Xd, Yd)
    aX, aY = np.abs(X), np.abs(Y)
    bH = 2.0 ** -42 * (aX @ aY.T)
    bM = 2.0 ** -42 * (aX @ aX.T)
    iu = np.triu_indices(ns)
    assert np.all((H1 - H2).abs().cpu().numpy().T[iu] <= bH[iu] + 1e-30)
    assert np.all((M1 - M2).abs().cpu().numpy() <= bM + 1e-30)
    Z = np.linalg.qr(np.random.default_rng(ns).standard_normal((ns, ns)))[0]
    R1 = tc.rotate(Xd, to_dev(Z)).cpu().numpy()
    R2 = simt.rotate(Xd, to_dev(Z)).cpu().numpy()
    bR = 2.0 ** -42 * (np.abs(Z).T @ aX)
    assert np.all(np.abs(R1 - R2) <= bR + 1e-30)


def _spd_pair(n, cond, rng, degenerate=0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Q * np.logspace(0, -np.log10(cond), n)) @ Q.T
    M = 0.5 * (M + M.T)
    ev = np.sort(rng.uniform(-3, 40, n))
    if degenerate:
        ev[3:3 + degenerate] = ev[3]
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    L = np.linalg.cholesky(M)
    H = L @ ((P * ev) @ P.T) @ L.T
    return 0.5 * (H + H.T), M


@pytest.mark.parametrize("n,cond,deg", [(1, 1, 0), (2, 10, 0), (7, 100, 0), (40, 1e4, 0),
                                        (65, 1e6, 0), (50, 1e3, 8), (130, 1e2, 0), (33, 10, 33)])
def test_subspace_eig_vs_oracle(n, cond, deg):
    rng = np.random.default_rng(n * 7 + deg)
    if deg == n:  # fully degenerate: H = c M
        _, M = _spd_pair(n, cond, rng)
        H = 2.5 * M
    else:
        H, M = _spd_pair(n, cond, rng, deg)
    s = SYSTEMS["free"]()
    h = sparc.Handle(s, "fp64", ns_max=max(n, 1))
    lam, Z = h.subspace_eig(to_dev(H), to_dev(M))
    lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
    rlam, rZ = oracle.gen_eig(H, M)
    scale = max(1.0, cond / 1e4)
    assert np.max(np.abs(lam - rlam)) < 1e-9 * scale * np.max(np.abs(rlam))
    assert np.max(np.abs(Z.T @ M @ Z - np.eye(n))) < 1e-9 * scale
    assert np.max(np.abs(H @ Z - M @ Z * lam)) < 1e-9 * scale * np.max(np.abs(H))
    cols = np.argmax(np.abs(Z), axis=0)
    assert np.all(Z[cols, np.arange(n)] > 0)


def test_subspace_eig_not_spd():
    s = SYSTEMS["free"]()
    n = 12
    rng = np.random.default_rng(5)
    H, M = _spd_pair(n, 10, rng)
    M[4, 4] = -3.0
    h = sparc.Handle(s, "fp64", ns_max=n)
    with pytest.raises(sparc.SparcError) as ei:
        h.subspace_eig(to_dev(H), to_dev(M))
    assert ei.value.status == sparc.SPARC_ERR_NOT_SPD
    # the handle stays usable
    H, M = _spd_pair(n, 10, rng)
    lam, _ = h.subspace_eig(to_dev(H), to_dev(M))
    assert np.allclose(lam.cpu().numpy(), oracle.gen_eig(H, M)[0], atol=1e-10)


@pytest.mark.parametrize("name,ns,degree,flags", [("bulk24", 40, 20, 0), ("dirichlet_z", 24, 10, 0),
                                                  ("ragged_periodic", 9, 8, 0), ("free", 33, 15, 0),
                                                  ("wide_x", 1, 6, 0), ("bulk24", 40, 20, 2),
                                                  ("dirichlet_z", 24, 10, 2)])
def test_chefsi_step_fp64(name, ns, degree, flags):
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    X0 = synth.random_orbitals(s.nd, ns, seed=11)
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=flags)
    Xd = to_dev(X0)
    lam = h.chefsi_step(Xd, degree, bounds=(a, b, a0))
    X1 = Xd.cpu().numpy()
    rX, rlam = o.chefsi_step(X0, degree, a, b, a0)
    assert np.max(np.abs(lam - rlam)) < 1e-8, np.max(np.abs(lam - rlam))
    assert subspace_distance(X1, rX) < 1e-7
    assert np.max(np.abs(X1 @ X1.T - np.eye(ns))) < 1e-9
    t = h.timings()
    assert t["total_ms"] > 0 and t["filter_ms"] > 0


def test_chefsi_three_steps_bulk24_default_bounds():
    """Three steps with library-chosen bounds (cached Lanczos, cutoff = previous
    largest Ritz value) against the oracle fed the same bounds."""
    s = SYSTEMS["bulk24"]()
    o = oracle.Oracle(s)
    ns, m = 40, 20
    X0 = synth.random_orbitals(s.nd, ns, seed=synth.workload_seed("bulk24"))
    h = sparc.Handle(s, "fp64", ns_max=ns)
    a0, b = h.spectrum_bounds(32, 0)
    ra0, rb, *_ = o.lanczos(32, 0)
    assert abs(a0 - ra0) < 1e-9 and abs(b - rb) < 1e-9
    Xd = to_dev(X0)
    rX = X0
    a = a0 + 0.1 * (b - a0)
    for step in range(3):
        lam = h.chefsi_step(Xd, m)  # library bounds
        rX, rlam = o.chefsi_step(rX, m, a, b, a0)
        assert np.max(np.abs(lam - rlam)) < 1e-8, (step, np.max(np.abs(lam - rlam)))
        a = rlam[-1]
    assert subspace_distance(Xd.cpu().numpy(), rX) < 1e-7


def test_chefsi_step_host_buffer_and_determinism():
    s = SYSTEMS["dirichlet_z"]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    X0 = synth.random_orbitals(s.nd, 16, seed=3)
    h = sparc.Handle(s, "fp64", ns_max=16)
    outs = []
    for _ in range(2):
        Xd = to_dev(X0)
        lam = h.chefsi_step(Xd, 10, bounds=(a, b, a0))
        outs.append((Xd.cpu().numpy(), lam))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    Xh = X0.copy()
    lamh = h.chefsi_step(Xh, 10, bounds=(a, b, a0))
    assert np.array_equal(Xh, outs[0][0]) and np.array_equal(lamh, outs[0][1])
    # a page-locked host block (torch pinned memory)
    Xp = torch.from_numpy(X0.copy()).pin_memory().numpy()
    lamp = h.chefsi_step(Xp, 10, bounds=(a, b, a0))
    assert np.array_equal(Xp, outs[0][0]) and np.array_equal(lamp, outs[0][1])
    t = h.timings()
    assert t["stage_in_ms"] > 0 and t["stage_out_ms"] > 0 and t["host_ms"] >= t["total_ms"] * 0.999
    Xd = to_dev(X0)
    h.chefsi_step(Xd, 10, bounds=(a, b, a0))
    t = h.timings()
    assert t["stage_in_ms"] == 0 and t["stage_out_ms"] == 0 and t["host_ms"] > 0


def test_invalid_arguments():
    s = SYSTEMS["bulk24"]()
    h = sparc.Handle(s, "fp64", ns_max=4)
    X = to_dev(np.zeros((4, s.nd)))
    with pytest.raises(sparc.SparcError) as ei:
        sparc.sparc_hpsi(h.h, X, X)
    assert ei.value.status == sparc.SPARC_ERR_INVALID_ARG
    with pytest.raises(sparc.SparcError):
        h.cheb_filter(X, 5, 1.0, 0.5, 0.0)  # a > b
    with pytest.raises(sparc.SparcError):
        h.hpsi(to_dev(np.zeros((5, s.nd))))  # ns > ns_max
    with pytest.raises(sparc.SparcError):
        h.hpsi(X.float())  # dtype mismatch on an FP64 handle


# ---------------------------------------------------------------------------
# Mixed precision: FP32 orbitals, split-precision tensor-core projection and
# rotation (three BF16 slices per operand, six slice products, double-FP32
# accumulation) against the oracle evaluated on the same FP32 inputs.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,ns", [("bulk24", 40), ("ragged_periodic", 200), ("bulk24", 129),
                                     ("wide_x", 1)])
def test_project_mixed_tensor_cores(name, ns):
    s = SYSTEMS[name]()
    rng = np.random.default_rng(ns)
    X = rng.standard_normal((ns, s.nd)).astype(np.float32)
    Y = (0.3 * X + rng.standard_normal((ns, s.nd))).astype(np.float32)
    h = sparc.Handle(s, "mixed", ns_max=ns)
    Hs, Ms = h.project(to_dev(X, torch.float32), to_dev(Y, torch.float32))
    rH, rM = oracle.project(X.astype(np.float64), Y.astype(np.float64), s.nd)
    iu = np.triu_indices(ns)
    eH = np.max(np.abs(Hs.cpu().numpy().T[iu] - rH[iu])) / np.max(np.abs(rH))
    eM = np.max(np.abs(Ms.cpu().numpy() - rM)) / np.max(np.abs(rM))
    assert eH < 1e-7 and eM < 1e-7, (eH, eM)


@pytest.mark.parametrize("name,ns", [("bulk24", 40), ("ragged_periodic", 200), ("dirichlet_z", 7)])
def test_rotate_mixed_tensor_cores(name, ns):
    s = SYSTEMS[name]()
    rng = np.random.default_rng(ns + 1)
    X = rng.standard_normal((ns, s.nd)).astype(np.float32)
    Z = rng.standard_normal((ns, ns))
    h = sparc.Handle(s, "mixed", ns_max=ns)
    R = h.rotate(to_dev(X, torch.float32), to_dev(Z)).double().cpu().numpy()
    ref = oracle.rotate(X.astype(np.float64), Z, s.nd)
    err = np.max(np.abs(R - ref)) / np.max(np.abs(ref))
    assert err < 1e-6, err


@pytest.mark.parametrize("name,ns,degree", [("bulk24", 40, 20), ("dirichlet_z", 24, 10),
                                            ("ring_periodic", 30, 12)])
def test_chefsi_step_mixed_vs_oracle(name, ns, degree):
    """Mixed precision step against the FP64 oracle: the Ritz values of the
    occupied states agree to the stated 1e-6 Ha (FP32 filtering, FP64 Yt = H Xt,
    four-digit tensor-core projection and rotation)."""
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    X0 = synth.random_orbitals(s.nd, ns, seed=13)
    h = sparc.Handle(s, "mixed", ns_max=ns)
    Xd = to_dev(X0, torch.float32)
    lam = h.chefsi_step(Xd, degree, bounds=(a, b, a0))
    rX, rlam = o.chefsi_step(X0, degree, a, b, a0)
    ne = synth.electrons_for(ns)
    occ = np.arange(ns) < ne // 2
    err_occ = np.max(np.abs(lam - rlam)[occ])
    assert err_occ < 1e-6, err_occ
    X1 = Xd.double().cpu().numpy()
    assert np.max(np.abs(X1 @ X1.T - np.eye(ns))) < 1e-4


@pytest.mark.parametrize("name", ["ring_periodic", "ring_dirichlet_y", "bulk24"])
def test_ring_and_generic_stencil_agree(name):
    """The TMA plane-ring form and the generic form of the stencil kernel give
    the same H X: in FP64 arithmetic (default) up to summation order, in the
    double-FP32 form (flags 4) to the pairs' 48 bits; also with the Chebyshev
    recurrence term of the filter."""
    s = SYSTEMS[name]()
    ns = 6
    rng = np.random.default_rng(9)
    X = to_dev(rng.standard_normal((ns, s.nd)))
    ring64 = sparc.Handle(s, "fp64", ns_max=ns)
    ringdf = sparc.Handle(s, "fp64", ns_max=ns, options_flags=4)
    generic = sparc.Handle(s, "fp64", ns_max=ns, options_flags=1)
    Y1, Y2, Y3 = ring64.hpsi(X), generic.hpsi(X), ringdf.hpsi(X)
    torch.cuda.synchronize()
    scale = float(Y2.abs().max())
    assert float((Y1 - Y2).abs().max()) <= 1e-13 * scale
    assert float((Y3 - Y2).abs().max()) <= 1e-12 * scale
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    F = [X.clone() for _ in range(2)]
    ringdf.cheb_filter(F[0], 9, a, b, a0)
    generic.cheb_filter(F[1], 9, a, b, a0)
    torch.cuda.synchronize()
    assert float((F[0] - F[1]).abs().max()) <= 1e-11 * float(F[1].abs().max())


@pytest.mark.parametrize("name", ["bulk24", "ring_periodic"])
def test_chefsi_step_fp64_double_fp32_stencil(name):
    """FP64 handle with the double-FP32 stencil (options bit 2): Ritz values
    and subspace of a step stay within the FP64 targets (1e-8 Ha, 1e-7)."""
    s = SYSTEMS[name]()
    o = oracle.Oracle(s)
    a0, b, a = bounds_for(o)
    ns, m = 40, 20
    X0 = synth.random_orbitals(s.nd, ns, seed=11)
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=4)
    Xd = to_dev(X0)
    lam = h.chefsi_step(Xd, m, bounds=(a, b, a0))
    rX, rlam = o.chefsi_step(X0, m, a, b, a0)
    assert np.max(np.abs(lam - rlam)) < 1e-8, np.max(np.abs(lam - rlam))
    assert subspace_distance(Xd.cpu().numpy(), rX) < 1e-7
