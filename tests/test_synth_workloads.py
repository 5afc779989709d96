"""The named synthetic workloads have the grid shapes, boundary conditions,
spacings, atom counts and orbital counts that stand in for the paper's
examples, and the input generators are deterministic per seed."""
import numpy as np

from paper_2302_09708_gb300 import synth


def test_bulk24_and_bulk96_shapes_and_atoms():
    s24 = synth.make_workload_system("bulk24")
    assert s24.shape == (24, 24, 24) and s24.h == 0.5 and s24.bc == (0, 0, 0)
    assert s24.natoms == 8 and s24.nd == 13824
    s96 = synth.make_workload_system("bulk96")
    assert s96.shape == (96, 96, 96) and s96.h == 0.4 and s96.nd == 884736
    assert s96.natoms == 216
    # every atom inside the periodic cell, all projectors normalised h^3 sum chi^2 = 1
    L = 96 * 0.4
    assert np.all((s96.positions >= -0.5) & (s96.positions < L + 0.5))
    for J in (0, 107, 215):
        n = int(s96.supp_ptr[J + 1] - s96.supp_ptr[J])
        chi = s96.chi[int(s96.chi_ptr[J]):int(s96.chi_ptr[J + 1])].reshape(4, n)
        np.testing.assert_allclose(s96.h ** 3 * np.sum(chi * chi, axis=1), 1.0, rtol=1e-12)


def test_workload_parameters():
    w = synth.WORKLOADS
    assert (w["bulk24"]["ns"], w["bulk24"]["degree"]) == (40, 20)
    assert (w["bulk96"]["ns"], w["bulk96"]["degree"]) == (1300, 20)
    assert (w["slab64x64x160"]["ns"], w["slab64x64x160"]["degree"]) == (4800, 24)
    m36 = synth.make_workload_system("member36")
    assert m36.shape == (36, 36, 36) and m36.natoms == 24 and w["member36"]["ns"] == 150
    assert 36 % 16 != 0  # a grid the TMA ring does not fit (nx not a multiple of 16)
    assert w["slab64x64x160"]["bc"] == (synth.PERIODIC, synth.PERIODIC, synth.DIRICHLET)
    seeds = {synth.workload_seed(k) for k in w}
    assert len(seeds) == len(w)


def test_batch_members_ranges():
    mem = synth.batch_members()
    assert len(mem) == 64
    for m in mem:
        n = m["shape"][0]
        assert 24 <= n <= 48 and 4 <= m["natoms"] <= 40 and 16 <= m["degree"] <= 24
        assert 1 <= m["ns"] <= min(300, n ** 3 // 4)
    assert mem == synth.batch_members()


def test_generators_are_deterministic_and_orthonormal():
    a = synth.random_orbitals(500, 12, seed=3)
    b = synth.random_orbitals(500, 12, seed=3)
    assert np.array_equal(a, b)
    np.testing.assert_allclose(a @ a.T, np.eye(12), atol=1e-13)
    s1 = synth.random_system((13, 14, 15), 0.5, (0, 1, 0), 3, seed=5)
    s2 = synth.random_system((13, 14, 15), 0.5, (0, 1, 0), 3, seed=5)
    assert np.array_equal(s1.veff, s2.veff) and np.array_equal(s1.chi, s2.chi)
    assert synth.electrons_for(1300) == 2158 and synth.electrons_for(40) == 58
