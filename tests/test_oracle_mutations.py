"""Planted mistakes in the oracle, on the CPU: each plausible slip (a dropped
term, a wrong sign, factor or index, a transposed operand, a missing complex
conjugate) is written into a copy of the oracle, and at least one of the pins
named beside it must fail on that copy.  This shows that the pins bind every
part of the oracle, not just its happy path.

* Mutants of the C oracle are compiled into a temporary library.  The oracle
  module is pointed at it for the one test, so the real and complex step (whose
  FD weights and real eigensolver come from the C library) both run on the
  mutant.
* Mutants of the Python parts (occupations and density, the complex k-point
  form, the nonlocal forces) are re-executed from patched source.  Only the
  top-level function or class holding the change is swapped in.
* A control runs every pin named here on an unchanged copy built the same way:
  all must pass, so a failure under a mutant is the mutant's doing.

The real oracle files are never written."""
import ast
import ctypes
import os
import subprocess
import types

import pytest

import oracle
from oracle import forces, kpoint

import test_oracle_forces as tf
import test_oracle_kpoint as tk
import test_oracle_operator as op
import test_oracle_steps as st

P, D = 0, 1
ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
C_SRC = os.path.join(ORACLE_DIR, "sparc_oracle.c")

# -- the pins a mutant is checked against (test function, arguments) ----------
FD_EXACT = (op.test_fd_weights_exact_rationals, ())
FD_POLY = (op.test_fd_exact_on_polynomials, (13,))
DENSE_PERIODIC = (op.test_hpsi_matches_dense_assembly, ((13, 13, 13), (0, 0, 0), 2))
DENSE_MIXED_BC = (op.test_hpsi_matches_dense_assembly, ((14, 13, 15), (0, 0, 1), 3))
DENSE_DIRICHLET = (op.test_hpsi_matches_dense_assembly, ((13, 15, 14), (1, 1, 1), 2))
PLANE_WAVES = (op.test_free_electron_plane_waves, ())
ONE_PROJECTOR = (op.test_single_projector_identity, ())
SPLITMIX = (st.test_splitmix64_published_vectors, ())
FILTER = (st.test_filter_scalar_identity_on_plane_waves, ())
LANCZOS_FREE = (st.test_lanczos_free_electron_bounds, ())
LANCZOS_FULL = (st.test_lanczos_full_krylov_gives_exact_extremes, ())
TRIDIAG = (st.test_tridiag_qr_vs_library, ())
HOUSEHOLDER = (st.test_householder_tridiag, ())
CHOLESKY = (st.test_cholesky_and_not_spd, ())
GEN_EIG = (st.test_gen_eig_vs_scipy, (40, 1e4, 0))
GEN_EIG_DEG = (st.test_gen_eig_vs_scipy, (50, 1e3, 6))
PROJ_ROT = (st.test_projection_and_rotation_vs_numpy, ())
STEP = (st.test_chefsi_step_structure, ())
OCC = (st.test_occupations_and_density, ())
OCC_CLOSED = (st.test_occupations_two_level_and_degenerate_closed_forms, ())
K_DENSE = (tk.test_hpsi_k_matches_dense_assembly, ((13, 13, 13), (P, P, P), (0.12, 0.29, -0.37)))
K_DENSE_D = (tk.test_hpsi_k_matches_dense_assembly, ((13, 13, 6), (P, P, D), (0.31, -0.17, 0.0)))
K_PLANE = (tk.test_free_electron_bloch_plane_waves, ())
K_HERM = (tk.test_hermitian_time_reversal_and_k_periodicity, ())
K_CHOL = (tk.test_complex_cholesky_and_not_spd, ())
K_HOUSE = (tk.test_complex_householder_tridiag, ())
K_GEN = (tk.test_complex_gen_eig_vs_scipy, (40, 1e4, 0))
K_FILTER = (tk.test_filter_scalar_identity_on_bloch_plane_waves, ())
K_LANCZOS = (tk.test_lanczos_bounds_bracket_spectrum, ())
K_STEP = (tk.test_chefsi_step_ritz_values_equal_dense_rayleigh_ritz, ())
F_WEIGHTS = (tf.test_first_derivative_weights_exact, ())
F_SYMBOL = (tf.test_gradient_plane_wave_symbol, ())
F_DENSE_GRAD = (tf.test_gradient_matches_dense_kronecker, ((7, 13, 14), (D, P, P)))
F_DENSE = (tf.test_forces_match_dense_evaluation, ((13, 13, 6), (P, P, D)))

# -- mutants of the C oracle: (id, original text, planted text, pins) ---------
C_MUTANTS = [
    ("fd_alternating_sign", "double sign = (p % 2 == 1) ? 1.0 : -1.0;",
     "double sign = (p % 2 == 0) ? 1.0 : -1.0;", [FD_EXACT]),
    ("fd_centre_weight_factor", "w[0] = -2.0 * s;", "w[0] = -s;", [FD_EXACT, FD_POLY]),
    ("fd_factorial_range", "for (int i = 2; i <= n + p; ++i) b *= i;",
     "for (int i = 2; i < n + p; ++i) b *= i;", [FD_EXACT]),
    ("periodic_wrap_off_by_one", "c[d] = ((c[d] % n[d]) + n[d]) % n[d];",
     "c[d] = ((c[d] % n[d]) + n[d] - 1) % n[d];", [DENSE_PERIODIC, PLANE_WAVES]),
    ("dirichlet_read_as_periodic", "if (s->bc[d] == 1) return 0.0;",
     "if (s->bc[d] == 2) return 0.0;", [DENSE_DIRICHLET, DENSE_MIXED_BC]),
    ("z_axis_steps_along_y", "if (d == 2) { kp += p; km -= p; }",
     "if (d == 2) { jp += p; jm -= p; }", [DENSE_MIXED_BC, PLANE_WAVES]),
    ("laplacian_sign", "y[g] = -0.5 * lap + s->veff[g] * xc;",
     "y[g] = 0.5 * lap + s->veff[g] * xc;", [PLANE_WAVES, DENSE_PERIODIC]),
    ("veff_dropped", "y[g] = -0.5 * lap + s->veff[g] * xc;", "y[g] = -0.5 * lap;",
     [DENSE_PERIODIC, PLANE_WAVES]),
    ("grid_spacing_power", "lap += acc / h2;", "lap += acc / s->h;", [PLANE_WAVES]),
    ("nonlocal_quadrature_weight_dropped", "c *= h3 * gam[q];", "c *= gam[q];",
     [ONE_PROJECTOR, DENSE_PERIODIC]),
    ("nonlocal_gamma_dropped", "c *= h3 * gam[q];", "c *= h3;", [ONE_PROJECTOR]),
    ("nonlocal_sign", "for (long t = 0; t < np_; ++t) y[s->supp_idx[p0 + t]] += col[t] * c;",
     "for (long t = 0; t < np_; ++t) y[s->supp_idx[p0 + t]] -= col[t] * c;",
     [ONE_PROJECTOR, DENSE_PERIODIC]),
    ("filter_sigma_recurrence_sign", "double sigma_new = 1.0 / (tau - sigma);",
     "double sigma_new = 1.0 / (tau + sigma);", [FILTER]),
    ("filter_three_term_dropped",
     "double next = (hy[t] - c * cur[t]) * (2.0 * sigma_new / e) - sigma * sigma_new * prev[t];",
     "double next = (hy[t] - c * cur[t]) * (2.0 * sigma_new / e);", [FILTER]),
    ("filter_first_degree_factor", "cur[t] = (hy[t] - c * prev[t]) * (sigma1 / e);",
     "cur[t] = (hy[t] - c * prev[t]) * (2.0 * sigma1 / e);", [FILTER]),
    ("filter_centre", "double e = (b - a) / 2.0, c = (b + a) / 2.0;",
     "double e = (b - a) / 2.0, c = (b - a) / 2.0;", [FILTER]),
    ("splitmix_multiplier", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;",
     "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B7ULL;", [SPLITMIX]),
    ("uniform_mantissa_shift", "return (double)(z >> 11) * (1.0 / 9007199254740992.0);",
     "return (double)(z >> 12) * (1.0 / 9007199254740992.0);", [SPLITMIX]),
    ("lanczos_beta_term_dropped", "for (long t = 0; t < nd; ++t) w[t] -= bprev * vp[t];",
     "for (long t = 0; t < nd; ++t) w[t] -= 0.0 * vp[t];", [LANCZOS_FULL, LANCZOS_FREE]),
    ("lanczos_bound_without_residual", "*b_upper = hi + fabs(beta[k - 1]);",
     "*b_upper = hi;", [LANCZOS_FREE]),
    ("lanczos_min_comparison", "if (d[j] < lo) lo = d[j];", "if (d[j] > lo) lo = d[j];",
     [LANCZOS_FULL, LANCZOS_FREE]),
    ("overlap_from_wrong_block",
     "Ms[i + (long)j * ns] = or_dot(Xt + (long)i * ldx, Xt + (long)j * ldx, nd);",
     "Ms[i + (long)j * ns] = or_dot(Xt + (long)i * ldx, Yt + (long)j * ldy, nd);", [PROJ_ROT]),
    ("projected_h_transposed",
     "Hs[i + (long)j * ns] = or_dot(Xt + (long)i * ldx, Yt + (long)j * ldy, nd);",
     "Hs[j + (long)i * ns] = or_dot(Xt + (long)i * ldx, Yt + (long)j * ldy, nd);", [PROJ_ROT]),
    ("cholesky_update_index",
     "for (int k = 0; k < j; ++k) t -= L[i + (long)k * n] * L[j + (long)k * n];",
     "for (int k = 0; k < j; ++k) t -= L[i + (long)k * n] * L[i + (long)k * n];", [CHOLESKY]),
    ("cholesky_no_spd_check", "if (!(s > 0.0)) return OR_ERR_NOT_SPD;",
     "if (s < -1e300) return OR_ERR_NOT_SPD;", [CHOLESKY]),
    ("householder_update_factor", "A[i + (long)j * n] -= 2.0 * (v[i] * p[j] + p[i] * v[j]);",
     "A[i + (long)j * n] -= (v[i] * p[j] + p[i] * v[j]);", [HOUSEHOLDER]),
    ("householder_correction_dropped", "for (int i = 0; i < n; ++i) p[i] -= vp * v[i];",
     "for (int i = 0; i < n; ++i) p[i] -= 0.0 * vp * v[i];", [HOUSEHOLDER]),
    ("householder_q_accumulation", "for (int j = k + 1; j < n; ++j) Q[i + (long)j * n] -= 2.0 * s * v[j];",
     "for (int j = k + 1; j < n; ++j) Q[i + (long)j * n] -= s * v[j];", [HOUSEHOLDER]),
    ("givens_diagonal_sign", "d[k + 1] = s * s * p + 2.0 * c * s * t + c * c * q;",
     "d[k + 1] = s * s * p - 2.0 * c * s * t + c * c * q;", [TRIDIAG]),
    ("givens_vector_sign", "zk1[r2] = s * u + c * v;", "zk1[r2] = -s * u + c * v;",
     [GEN_EIG]),
    ("eigenpairs_descending", "if (lam[j] < lam[m]) m = j;", "if (lam[j] > lam[m]) m = j;",
     [GEN_EIG]),
    ("eigenvector_sign_convention", "if (z[im] < 0.0)", "if (z[im] > 0.0)", [GEN_EIG]),
    ("forward_solve_transposed_factor",
     "for (int k = 0; k < i; ++k) s -= L[i + (long)k * n] * W[k + (long)c * n];",
     "for (int k = 0; k < i; ++k) s -= L[k + (long)i * n] * W[k + (long)c * n];", [GEN_EIG]),
    ("back_transform_transposed_factor",
     "for (int k = i + 1; k < n; ++k) s -= L[k + (long)i * n] * Z[k + (long)c * n];",
     "for (int k = i + 1; k < n; ++k) s -= L[i + (long)k * n] * Z[k + (long)c * n];",
     [GEN_EIG, GEN_EIG_DEG]),
    ("rotation_transposed", "s += Xt[t + (long)k * ld] * Z[k + (long)j * ns];",
     "s += Xt[t + (long)k * ld] * Z[j + (long)k * ns];", [PROJ_ROT]),
    ("step_rotation_not_stored",
     "for (int j = 0; j < ns; ++j) memcpy(X + (long)j * ld, Xn + (long)j * nd, sizeof(double) * nd);",
     "", [STEP]),
    ("step_filter_degree", "int st = or_cheb_filter(s, X, ld, ns, m, a, b, a0);",
     "int st = or_cheb_filter(s, X, ld, ns, m - 1, a, b, a0);", [STEP]),
]

# -- mutants of the Python parts: (id, module, original, planted, pins) -------
PY_MUTANTS = [
    ("occupations_spin_factor", oracle,
     "return 2.0 * np.sum(1.0 / (1.0 + np.exp(t)))", "return np.sum(1.0 / (1.0 + np.exp(t)))",
     [OCC, OCC_CLOSED]),
    ("occupations_bisection_direction", oracle, "if c < ne:", "if c > ne:", [OCC, OCC_CLOSED]),
    ("occupations_fermi_sign", oracle, "return 1.0 / (1.0 + np.exp(t)), mu",
     "return 1.0 / (1.0 + np.exp(-t)), mu", [OCC, OCC_CLOSED]),
    ("density_grid_power", oracle, 'return 2.0 * np.einsum("n,ni->i", f, X * X) / h ** 3',
     'return 2.0 * np.einsum("n,ni->i", f, X * X) / h ** 2', [OCC]),
    ("density_spin_factor", oracle, 'return 2.0 * np.einsum("n,ni->i", f, X * X) / h ** 3',
     'return np.einsum("n,ni->i", f, X * X) / h ** 3', [OCC]),
    ("project_result_transposed", oracle, "return Hs.T.copy(), Ms.T.copy()",
     "return Hs.copy(), Ms.copy()", [PROJ_ROT]),
    ("k_bloch_phase_sign", kpoint, "f = np.exp(1j * self.k[d] * self.lengths[d] * q)",
     "f = np.exp(-1j * self.k[d] * self.lengths[d] * q)", [K_PLANE, K_DENSE]),
    ("k_projector_phase_sign", kpoint, "phase = np.exp(1j * (T @ self.k))",
     "phase = np.exp(-1j * (T @ self.k))", [K_DENSE, K_DENSE_D]),
    ("k_projector_conjugate_dropped", kpoint, "C = h3 * (X[:, idx] @ phi.conj())",
     "C = h3 * (X[:, idx] @ phi)", [K_DENSE, K_HERM]),
    ("k_projection_conjugate_dropped", kpoint, "return Xt.conj() @ Yt.T, Xt.conj() @ Xt.T",
     "return Xt @ Yt.T, Xt.conj() @ Xt.T", [K_STEP]),
    ("k_cholesky_conjugate_dropped", kpoint,
     "L[i, j] = (M[i, j] - L[i, :j] @ L[j, :j].conj()) / L[j, j]",
     "L[i, j] = (M[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]", [K_CHOL]),
    ("k_householder_right_update", kpoint,
     "A[:, j + 1:] -= 2.0 * np.outer(A[:, j + 1:] @ v, v.conj())",
     "A[:, j + 1:] -= 2.0 * np.outer(A[:, j + 1:] @ v.conj(), v)", [K_HOUSE]),
    ("k_tridiagonal_phase_conjugated", kpoint,
     "D[j + 1] = D[j] * (e[j] / abs(e[j])) if e[j] != 0 else D[j]",
     "D[j + 1] = D[j] * (e[j].conj() / abs(e[j])) if e[j] != 0 else D[j]", [K_GEN]),
    ("k_back_transform_without_conjugate", kpoint, "U = L.conj().T", "U = L.T", [K_GEN]),
    ("k_lanczos_bound_without_residual", kpoint,
     "return theta[0], theta[-1] + abs(beta[k - 1]), alpha, beta, theta[-1]",
     "return theta[0], theta[-1], alpha, beta, theta[-1]", [K_LANCZOS]),
    ("k_filter_sigma_recurrence_sign", kpoint, "sigma_new = 1.0 / (tau - sigma)",
     "sigma_new = 1.0 / (tau + sigma)", [K_FILTER]),
    ("k_laplacian_sign", kpoint, "Y += (-0.5 / self.h ** 2) * lap",
     "Y += (0.5 / self.h ** 2) * lap", [K_PLANE]),
    ("k_veff_dropped", kpoint,
     "Y = Y.reshape(ns, self.nd) + self.system.veff[None, :] * X[:, : self.nd]",
     "Y = Y.reshape(ns, self.nd)", [K_DENSE]),
    ("k_dirichlet_ghost_read", kpoint, "f = (q == 0).astype(np.float64)", "f = np.ones(n)",
     [K_DENSE_D]),
    ("k_lanczos_three_term_dropped", kpoint, "w = self.hpsi(v)[0] - bprev * vp",
     "w = self.hpsi(v)[0]", [K_LANCZOS]),
    ("k_rotation_transposed", kpoint,
     "return np.asarray(Z).T @ np.asarray(Xt, dtype=np.complex128)",
     "return np.asarray(Z) @ np.asarray(Xt, dtype=np.complex128)", [K_STEP]),
    ("gradient_weight_sign", forces, "w[p] = (-1) ** (p + 1) * factorial(n) ** 2",
     "w[p] = (-1) ** p * factorial(n) ** 2", [F_WEIGHTS]),
    ("gradient_dirichlet_ghost_read", forces, "mask = ((j >= 0) & (j < n)).astype(np.float64)",
     "mask = ((j >= 0) & (j <= n)).astype(np.float64)", [F_DENSE_GRAD]),
    ("gradient_spacing_dropped", forces, "return (out / s.h).reshape(ns, s.nd)",
     "return out.reshape(ns, s.nd)", [F_SYMBOL]),
    ("force_prefactor", forces, "F[J, d] = -4.0 * np.sum(", "F[J, d] = -2.0 * np.sum(",
     [F_DENSE]),
    ("force_sign", forces, "F[J, d] = -4.0 * np.sum(", "F[J, d] = 4.0 * np.sum(", [F_DENSE]),
    ("force_gradient_axis", forces, "g = h3 * (grads[d][:, idx] @ chi)",
     "g = h3 * (grads[0][:, idx] @ chi)", [F_DENSE]),
    ("force_coefficient_from_gradient", forces, "c = h3 * (X[:, idx] @ chi)",
     "c = h3 * (grads[0][:, idx] @ chi)", [F_DENSE]),
]


def _compile(src_text, path):
    c = path.with_suffix(".c")
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared",
                          "-o", str(path), str(c), "-lm"])
    return str(path)


def _use_library(monkeypatch, so_path):
    """Point the oracle module at another build of the C oracle for one test."""
    ctypes.CDLL(so_path)  # fails here, not inside a pin, if the build is broken
    monkeypatch.setattr(oracle, "build", lambda force=False: so_path)
    monkeypatch.setattr(oracle, "_lib", None)


def _failures(pins):
    """Run each pin; return the names of those that failed (raised anything)."""
    failed = []
    for fn, args in pins:
        try:
            fn(*args)
        except (Exception, pytest.fail.Exception) as exc:  # incl. pytest.raises unmet
            failed.append(f"{fn.__name__}: {type(exc).__name__}")
    return failed


def _mutated_module(module, old, new):
    """Re-execute `module` from its source with `old` replaced by `new`; return
    the fresh module and the name of the top-level definition that changed."""
    path = module.__file__
    src = open(path).read()
    assert src.count(old) == 1, (module.__name__, old)
    line = src[:src.index(old)].count("\n") + 1
    owner = next(node.name for node in ast.parse(src).body
                 if isinstance(node, (ast.FunctionDef, ast.ClassDef))
                 and node.lineno <= line <= node.end_lineno)
    fresh = types.ModuleType(module.__name__ + "_mutant")
    fresh.__file__ = path
    fresh.__package__ = "oracle"
    exec(compile(src.replace(old, new), path, "exec"), fresh.__dict__)
    return fresh, owner


def test_every_c_function_has_a_mutant():
    """Each exported routine of the C oracle (and the boundary reader it uses)
    carries at least one planted mistake above."""
    src = open(C_SRC).read()
    covered = {
        "or_fd_weights": ["fd_"], "or_at": ["periodic_wrap", "dirichlet_read"],
        "or_hpsi": ["laplacian_sign", "veff_dropped", "nonlocal_"],
        "or_cheb_filter": ["filter_"], "or_mix64": ["splitmix"], "or_uniform": ["uniform"],
        "or_tridiag_qr": ["givens_"], "or_lanczos": ["lanczos_"],
        "or_project": ["overlap_", "projected_h"], "or_cholesky": ["cholesky_"],
        "or_householder_tridiag": ["householder_"], "or_sym_eig": ["eigenpairs_"],
        "or_fix_signs": ["eigenvector_sign"], "or_gen_eig": ["forward_solve", "back_transform"],
        "or_rotate": ["rotation_"], "or_chefsi_step": ["step_"],
    }
    ids = [m[0] for m in C_MUTANTS]
    for fn, prefixes in covered.items():
        assert f" {fn}(" in src, fn
        assert any(i.startswith(p) for p in prefixes for i in ids), fn


def test_control_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    """The harness itself: an unchanged copy built the same way passes all pins."""
    _use_library(monkeypatch, _compile(open(C_SRC).read(), tmp_path / "control.so"))
    pins = {(fn, args) for *_, ps in C_MUTANTS + PY_MUTANTS for fn, args in ps}
    assert _failures(sorted(pins, key=lambda p: (p[0].__name__, repr(p[1])))) == []


@pytest.mark.parametrize("mid,old,new,pins", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_caught(mid, old, new, pins, tmp_path, monkeypatch):
    src = open(C_SRC).read()
    assert src.count(old) == 1, old
    _use_library(monkeypatch, _compile(src.replace(old, new), tmp_path / f"{mid}.so"))
    assert _failures(pins), f"planted mistake {mid} passed every pin"


@pytest.mark.parametrize("mid,module,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_is_caught(mid, module, old, new, pins, monkeypatch):
    fresh, owner = _mutated_module(module, old, new)
    monkeypatch.setattr(module, owner, getattr(fresh, owner))
    assert _failures(pins), f"planted mistake {mid} passed every pin"
