"""sparc_project_noalloc: the FP64 projection for callers that may not allocate
device memory (their memory belongs to another allocator, or a cudaMalloc would
stall a latency-critical loop).  It keeps its split-K scratch in a static device
array, so this file checks it through the C ABI against sparc_project on a
handle and against the oracle's projection, on consecutive calls that reuse the
same scratch, including the largest size the scratch holds right after a call
that used more splits.  The file sorts last so that a run stopping at the first
failure has already run every other test."""
import ctypes

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
TOL = 1e-10  # the projection tolerance of the parity tests


def _noalloc(L, X, Y, ns, nd, ld):
    Hs = torch.full((ns, ns), float("nan"), dtype=torch.float64, device=DEV)
    Ms = torch.full((ns, ns), float("nan"), dtype=torch.float64, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.sparc_project_noalloc(X.data_ptr(), Y.data_ptr(), ns, nd, ld, Hs.data_ptr(),
                                 Ms.data_ptr(), stream)
    assert rc == sparc.SPARC_OK, L.sparc_last_error(None)
    torch.cuda.synchronize()
    return Hs, Ms


def test_project_noalloc_matches_handle_projection_on_consecutive_calls():
    L = sparc.load()
    s = synth.make_workload_system("bulk24")
    nd = s.nd
    # the handle projection on the FP64 SIMT pipe, the kernel sparc_project_noalloc runs
    h = sparc.Handle(s, "fp64", ns_max=64, options_flags=2)
    rng = np.random.default_rng(2302)
    for ns, pad in ((40, 0), (33, 5), (64, 32)):  # consecutive calls share the scratch
        ld = nd + pad
        X = torch.from_numpy(rng.standard_normal((ns, ld))).to(DEV)
        Y = torch.from_numpy(rng.standard_normal((ns, ld))).to(DEV)
        Hs, Ms = _noalloc(L, X, Y, ns, nd, ld)
        rH, rM = h.project(X, Y)
        torch.cuda.synchronize()
        assert torch.isfinite(Hs).all() and torch.isfinite(Ms).all()
        assert float((Hs - rH).abs().max()) < TOL
        assert float((Ms - rM).abs().max()) < TOL
        _check_vs_oracle(Hs, Ms, X[:, :nd].cpu().numpy(), Y[:, :nd].cpu().numpy(), nd)
    h.close()


def _check_vs_oracle(Hs, Ms, Xh, Yh, nd):
    """Against the oracle's FP64 sums in natural order: the two differ only in
    summation order, so each entry agrees to 1e-12 of sum_k |x_k y_k| (the
    rounding of an nd-term FP64 sum is far below that).  Hs is compared on its
    upper triangle, where the GPU form takes it from."""
    oH, oM = oracle.project(Xh, Yh, nd)
    aX, aY = np.abs(Xh), np.abs(Yh)
    bH, bM = 1e-12 * (aX @ aY.T) + 1e-30, 1e-12 * (aX @ aX.T) + 1e-30
    iu = np.triu_indices(Xh.shape[0])
    assert np.all(np.abs(Hs.cpu().numpy().T[iu] - oH[iu]) <= bH[iu])
    assert np.all(np.abs(Ms.cpu().numpy() - oM) <= bM)


def test_project_noalloc_largest_size_after_a_call_with_more_splits():
    """ns = 1448 fills the static scratch with a single split (2 ns^2 of its
    4194304 doubles), so the split count the size would otherwise get is
    clamped to 1.  It runs right after a call that spread its partials over many
    splits, whose stale values must not be read, and matches the oracle and the
    handle projection."""
    L = sparc.load()
    rng = np.random.default_rng(1448)
    nd0, ns0 = 200000, 40  # many splits: partials spread over the scratch
    X0 = torch.from_numpy(rng.standard_normal((ns0, nd0))).to(DEV)
    _noalloc(L, X0, X0, ns0, nd0, nd0)
    ns, nd = 1448, 4096
    X = torch.from_numpy(rng.standard_normal((ns, nd))).to(DEV)
    Y = torch.from_numpy(rng.standard_normal((ns, nd))).to(DEV)
    for _ in range(2):
        Hs, Ms = _noalloc(L, X, Y, ns, nd, nd)
        _check_vs_oracle(Hs, Ms, X.cpu().numpy(), Y.cpu().numpy(), nd)
        _noalloc(L, X0, X0, ns0, nd0, nd0)
    s = synth.free_system((16, 16, 16), 0.5, (0, 0, 0))
    h = sparc.Handle(s, "fp64", ns_max=ns, options_flags=2)
    rH, rM = h.project(torch.nn.functional.pad(X, (0, s.nd - nd)),
                       torch.nn.functional.pad(Y, (0, s.nd - nd)))
    torch.cuda.synchronize()
    assert float((Hs - rH).abs().max()) < TOL and float((Ms - rM).abs().max()) < TOL
    h.close()


def test_project_noalloc_rejects_sizes_beyond_its_scratch():
    L = sparc.load()
    X = torch.zeros((2, 64), dtype=torch.float64, device=DEV)
    rc = L.sparc_project_noalloc(X.data_ptr(), X.data_ptr(), 1449, 64, 64, X.data_ptr(),
                                 X.data_ptr(), ctypes.c_void_p(0))
    assert rc == sparc.SPARC_ERR_INVALID_ARG
    assert b"1448" in L.sparc_last_error(None)
