"""The oracle's pins have teeth: each case plants one plausible mistake (a dropped term or factor, a wrong sign,
index or conjugation, a transposed operand, a skipped pass) in a copy of one oracle module, made from its source
text on the CPU, and runs the existing pin that should catch it with the mutant swapped in.  The pin must fail.
The oracle modules themselves are never modified; their unmutated pins run in the other test files."""
import importlib
import inspect
import types

import numpy as np
import pytest

import test_oracle_deflation as t_df
import test_oracle_estimators as t_est
import test_oracle_multigrid as t_mg
import test_oracle_nn as t_nn
import test_oracle_operator as t_op
import test_oracle_rng as t_rng
import test_oracle_tune_mass as t_tm
from oracle import multigrid as mg
from oracle import schwinger as osch
from synthetic import gauge


def mutant(name, old, new):
    """A fresh copy of oracle.<name> with the unique source text `old` replaced by `new`."""
    mod = importlib.import_module("oracle." + name)
    src = inspect.getsource(mod)
    assert src.count(old) == 1, "mutation site must occur once in oracle/%s.py: %r" % (name, old)
    m = types.ModuleType("oracle._mutant_" + name)
    m.__package__ = "oracle"
    m.__file__ = mod.__file__
    exec(compile(src.replace(old, new), "<mutant of oracle/%s.py>" % name, "exec"), m.__dict__)
    return m


def use_estimators(mp, m):
    """The estimator tests run Algorithm 2 with the mutant's level differences and estimator."""
    mp.setattr(t_est, "LevelDifference", m.LevelDifference)
    mp.setattr(t_est, "mgmlmc_pp", m.mgmlmc_pp)


def small():
    """The estimator tests' L = 16 operator and two-level hierarchy."""
    D = osch.dirac_sparse(gauge.links(gauge.field(16, 3.0, 0)), -0.05)
    return D, mg.Hierarchy(D, 16, ntv=4, setup_sweeps=3, seed=2)


def small3(mgm=mg):
    """The three-level L = 32 hierarchy (2x2 aggregates) of the multigrid and gamma5-trace tests, built by mgm."""
    U = gauge.links(gauge.field(32, 3.0, 3, sweeps=40))
    return mgm.Hierarchy(osch.dirac_sparse(U, -0.05), 32, levels=3, agg=2, ntv=2, setup_sweeps=2, seed=1)


def agg4(mgm):
    """A two-level L = 16 hierarchy with 4x4 aggregates and 4 test vectors per chirality, built by module mgm."""
    U = gauge.links(gauge.field(16, 3.0, 1, sweeps=30))
    return mgm.Hierarchy(osch.dirac_sparse(U, -0.05), 16, ntv=4, setup_sweeps=2, seed=3)


def deflation_op():
    D = osch.dirac_dense(gauge.links(gauge.field(16, 3.0, 0)), -0.05)
    return D, np.linalg.inv(D)


# (case id, oracle module, original text, planted mistake, pin: callable(monkeypatch, mutant module))
CASES = [
    # ---- operator (Section 4 reading of the Wilson formula): free-field closed form, gamma5-hermiticity, covariance
    ("periodic_t", "schwinger",
     "            eta_f = np.where(t == L - 1, -1.0, 1.0)\n            eta_b = np.where(t == 0, -1.0, 1.0)",
     "            eta_f = np.ones_like(t, dtype=float)\n            eta_b = np.ones_like(t, dtype=float)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_free_field_spectrum_and_trace(4, -0.05))),
    ("boundary_sign_forward_only", "schwinger",
     "            eta_f = np.where(t == L - 1, -1.0, 1.0)\n",
     "            eta_f = np.ones_like(t, dtype=float)\n",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_gamma5_hermiticity())),
    ("hop_factor_one", "schwinger", "vals.append(-0.5 * Pm[a, b] * Uf)", "vals.append(-1.0 * Pm[a, b] * Uf)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_free_field_spectrum_and_trace(6, 0.3))),
    ("backward_link_not_conjugated", "schwinger", "Ub = (np.conj(U[tb, xb, mu]) * eta_b)",
     "Ub = (U[tb, xb, mu] * eta_b)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_gamma5_hermiticity())),
    ("backward_link_wrong_site", "schwinger", "Ub = (np.conj(U[tb, xb, mu]) * eta_b)",
     "Ub = (np.conj(U[t, x, mu]) * eta_b)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_gamma5_hermiticity())),
    ("wrong_spin_projector", "schwinger", "Pp = eye + SIGMA[mu]", "Pp = eye - SIGMA[mu]",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_free_field_spectrum_and_trace(4, -0.05))),
    ("diagonal_term", "schwinger", "np.full(V, m0 + 2.0, dtype=complex)", "np.full(V, m0 + 1.0, dtype=complex)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_free_field_spectrum_and_trace(8, -0.4))),
    ("links_conjugated_everywhere", "schwinger", "Uf = (U[t, x, mu] * eta_f)", "Uf = (np.conj(U[t, x, mu]) * eta_f)",
     lambda mp, m: (mp.setattr(t_op, "osch", m), t_op.test_gamma5_hermiticity())),
    # ---- random numbers (SplitMix64, published outputs)
    ("splitmix_shift", "rng", "z = z ^ (z >> np.uint64(27))", "z = z ^ (z >> np.uint64(28))",
     lambda mp, m: (mp.setattr(t_rng, "rng", m), t_rng.test_splitmix64_reference_outputs())),
    # ---- QR (positive diagonal) and CholeskyQR2
    ("cholqr_single_pass", "linalg", "    return Q2, R2 @ R1", "    return Q1, R1",
     lambda mp, m: (mp.setattr(t_est, "cholesky_qr2", m.cholesky_qr2), t_est.test_cholesky_qr2_matches_householder())),
    ("cholqr_r_product_order", "linalg", "    return Q2, R2 @ R1", "    return Q2, R1 @ R2",
     lambda mp, m: (mp.setattr(t_est, "cholesky_qr2", m.cholesky_qr2), t_est.test_cholesky_qr2_matches_householder())),
    ("qr_phase_not_applied_to_r", "linalg", "    R = np.conj(ph)[:, None] * R\n", "    R = R\n",
     lambda mp, m: (mp.setattr(t_est, "qr_positive", m.qr_positive), t_est.test_cholesky_qr2_matches_householder())),
    # ---- Algorithm 2 stop rule (eqs. accuracy_opt / optimal_variance), hand-computed cases
    ("uniform_divides_by_L", "estimators", "rho2 = (eps * abs(tau_total)) ** 2 / nd",
     "rho2 = (eps * abs(tau_total)) ** 2 / (nd + 1)",
     lambda mp, m: (mp.setattr(t_est, "update_active", m.update_active), t_est.test_stop_rule_hand_computed())),
    ("cost_dropped_from_weight", "estimators", "w = math.sqrt(cost[l] * V[l]) / denom", "w = math.sqrt(V[l]) / denom",
     lambda mp, m: (mp.setattr(t_est, "update_active", m.update_active), t_est.test_stop_rule_hand_computed())),
    ("variance_not_divided_by_N", "estimators", "if V[l] / N[l] <= rho2:", "if V[l] <= rho2:",
     lambda mp, m: (mp.setattr(t_est, "update_active", m.update_active), t_est.test_stop_rule_hand_computed())),
    ("hutchinson_stop_without_s", "estimators", "if s >= min_samples and V / s <= (abs(tau) * eps) ** 2:",
     "if s >= min_samples and V <= (abs(tau) * eps) ** 2:",
     lambda mp, m: (mp.setattr(t_est, "hutchinson", m.hutchinson), t_est.test_hutchinson_algorithm1_stop(small()))),
    ("hutchinson_weight_dropped", "estimators", "            x = weight * x\n", "            x = x\n",
     lambda mp, m: (mp.setattr(t_est, "hutchinson", m.hutchinson), t_est.test_gamma5_weighted_hutchinson(small()))),
    ("noise_kind_ignored", "rng", "    if kind == NOISE_Z4:\n", "    if kind == -1:\n",
     lambda mp, m: (mp.setattr(t_est, "rng", m), t_est.test_gamma5_weighted_hutchinson(small()))),
    # ---- level differences (eqs. mlmc_decomp_matrix / mlmc_dec_trace_reduced) and Algorithm 2's samples
    ("accumulated_difference_sign", "estimators", "            Y = a - b\n", "            Y = a + b\n",
     lambda mp, m: (mp.setattr(t_est, "LevelDifference", m.LevelDifference),
                    t_est.test_level_difference_unbiased(small(), "accumulated"))),
    ("reduced_restriction_not_conjugated", "estimators", "P @ self.solvers[l + 1].solve(P.conj().T @ Z)",
     "P @ self.solvers[l + 1].solve(P.T @ Z)",
     lambda mp, m: (mp.setattr(t_est, "LevelDifference", m.LevelDifference),
                    t_est.test_level_difference_unbiased(small(), "reduced"))),
    ("projection_sign", "estimators", "z = zeta if Q[l] is None else zeta - Q[l] @ (Q[l].conj().T @ zeta)",
     "z = zeta if Q[l] is None else zeta + Q[l] @ (Q[l].conj().T @ zeta)",
     lambda mp, m: (use_estimators(mp, m),
                    t_est.test_full_sketch_gives_the_exact_trace(small(), "accumulated", 0))),
    ("low_rank_trace_not_conjugated", "estimators", "tau_lr[l] = complex(np.sum(np.conj(S) * ld.apply(l, S)))",
     "tau_lr[l] = complex(np.sum(S * ld.apply(l, S)))",
     lambda mp, m: (use_estimators(mp, m),
                    t_est.test_full_sketch_gives_the_exact_trace(small(), "reduced", 1))),
    ("coarsest_term_not_conjugated", "estimators", "M = (Ph.conj().T @ W @ Ph).toarray()",
     "M = (Ph.T @ W @ Ph).toarray()",
     lambda mp, m: (use_estimators(mp, m),
                    t_est.test_algorithm2_end_to_end(small(), 0))),
    ("level_weight_dropped", "estimators", "        return Y if W is None else W @ Y\n", "        return Y\n",
     lambda mp, m: (mp.setattr(t_est, "LevelDifference", m.LevelDifference),
                    t_est.test_gamma5_telescoping_and_unbiased(small3(), "reduced"))),
    # ---- multigrid (Section 3.1): orthonormal aggregation, Galerkin operator, SAP, V-cycle
    ("prolongator_not_orthonormalised", "multigrid", "                Q, _ = qr_positive(V[I, :])\n",
     "                Q = V[I, :]\n",
     lambda mp, m: t_mg.test_orthonormal_and_aggregate_support(agg4(m))),
    ("chirality_blocks_interleaved", "multigrid", "ks = np.arange(dc) + c * dc if d > 2 else np.array([c])",
     "ks = 2 * np.arange(dc) + c if d > 2 else np.array([c])",
     lambda mp, m: t_mg.test_orthonormal_and_aggregate_support(three_level_agg4(m))),
    ("stencil_directions_swapped", "multigrid", "enumerate(((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)))",
     "enumerate(((0, 0), (-1, 0), (1, 0), (0, 1), (0, -1)))",
     lambda mp, m: (mp.setattr(t_mg, "mg", m), t_mg.test_stencil_blocks_direction_convention())),
    ("check_prolongator_ignores_chirality", "multigrid",
     "chiral = bool(np.all(chirality(fk, d) == chirality(ck, dc)))", "chiral = True",
     lambda mp, m: (mp.setattr(t_mg, "mg", m),
                    t_mg.test_imported_prolongators_rebuild_the_hierarchy(three_level_agg4(mg)))),
    ("check_prolongator_ignores_orthonormality", "multigrid",
     "orth = float(np.abs(G.data).max()) if G.nnz else 0.0", "orth = 0.0",
     lambda mp, m: (mp.setattr(t_mg, "mg", m),
                    t_mg.test_imported_prolongators_rebuild_the_hierarchy(three_level_agg4(mg)))),
    ("galerkin_transpose_not_adjoint", "multigrid", "Dc = (P.conj().T @ self.D[l] @ P).tocsr()",
     "Dc = (P.T @ self.D[l] @ P).tocsr()",
     lambda mp, m: t_mg.test_gamma5_coarse(small3(m))),
    ("sap_residual_not_refreshed", "multigrid",
     "        for I, inv in self.sets:\n            r = f - self.D @ x\n",
     "        r = f - self.D @ x\n        for I, inv in self.sets:\n",
     lambda mp, m: (mp.setattr(t_mg, "mg", m), t_mg.test_sap_residual_vanishes_on_updated_colour())),
    ("vcycle_restriction_not_conjugated", "multigrid", "e = e + P @ self.vcycle(l + 1, P.conj().T @ res, pre, post)",
     "e = e + P @ self.vcycle(l + 1, P.T @ res, pre, post)",
     lambda mp, m: (mp.setattr(t_mg, "mg", m), t_mg.test_vcycle_error_propagator(small3(), 1, 1))),
    ("vcycle_correction_sign", "multigrid", "e = e + P @ self.vcycle(l + 1, P.conj().T @ res, pre, post)",
     "e = e - P @ self.vcycle(l + 1, P.conj().T @ res, pre, post)",
     lambda mp, m: (mp.setattr(t_mg, "mg", m), t_mg.test_vcycle_error_propagator(small3(), 2, 1))),
    # ---- exact deflation (Section 2): singular triplets from gamma5 D and the direct trace part
    ("deflation_trace_times_mu", "deflation", 'np.einsum("ik,i,ik->k", np.conj(V), g5, V) / mu',
     'np.einsum("ik,i,ik->k", np.conj(V), g5, V) * mu',
     lambda mp, m: (mp.setattr(t_df, "odf", m), t_df.test_singular_values_and_trace_split(deflation_op()))),
    ("deflation_largest_not_smallest", "deflation", "idx = np.argsort(np.abs(mu))[:k]", "idx = np.argsort(mu)[:k]",
     lambda mp, m: (mp.setattr(t_df, "odf", m), t_df.test_singular_values_and_trace_split(deflation_op()))),
    ("z4_table_not_zero_mean", "rng", "np.array([1.0, 1j, -1.0, -1j])[q]", "np.array([1.0, 1j, 1.0, -1j])[q]",
     lambda mp, m: (mp.setattr(t_rng, "rng", m), t_rng.test_z4_values_isotropy_and_second_moment())),
    ("complex_test_vector_same_bit", "rng", "return s[0::2] + 1j * s[1::2]", "return s[0::2] + 1j * s[0::2]",
     lambda mp, m: (mp.setattr(t_rng, "rng", m), t_rng.test_complex_rademacher_test_vectors())),
    ("stream_counter_fields_overlap", "rng", "ctr = np.uint64((level << 56) | (phase << 48) | sample)",
     "ctr = np.uint64((level << 48) | (phase << 48) | sample)",
     lambda mp, m: (mp.setattr(t_rng, "rng", m), t_rng.test_streams_are_distinct())),
    ("sigma_without_division_by_N", "estimators", "sigma = math.sqrt(sum(V[l] / N[l] for l in range(nd) if N[l] >= 2))",
     "sigma = math.sqrt(sum(V[l] for l in range(nd) if N[l] >= 2))",
     lambda mp, m: (use_estimators(mp, m),
                    t_est.test_algorithm2_end_to_end(small(), 0))),
    ("sap_block_inverse_transposed", "multigrid", "inv = np.stack([np.linalg.inv(Dd[i][:, i].toarray()) for i in I])",
     "inv = np.stack([np.linalg.inv(Dd[i][:, i].toarray()).T for i in I])",
     lambda mp, m: (mp.setattr(t_mg, "mg", m), t_mg.test_sap_residual_vanishes_on_updated_colour())),
    ("mass_shift_sign", "tune_mass", "    return target - lam_c.real", "    return target + lam_c.real",
     lambda mp, m: (mp.setattr(t_tm, "otm", m), t_tm.test_interacting_field_matches_dense_spectrum_and_target())),
    ("deflated_sample_sign", "deflation", "taus.append(complex(np.vdot(z, y) - np.vdot(c, g)))",
     "taus.append(complex(np.vdot(z, y) + np.vdot(c, g)))",
     lambda mp, m: (mp.setattr(t_df, "odf", m), t_df.test_deflated_hutchinson_unbiased_with_smaller_variance(
         deflation_op()))),
    ("subspace_iteration_without_gamma5", "deflation", "V, _ = qr_positive(solve(g5[:, None] * V))",
     "V, _ = qr_positive(solve(V))",
     lambda mp, m: (mp.setattr(t_df, "odf", m), t_df.test_subspace_iteration_converges_to_the_exact_subspace(
         deflation_op()))),
    # ---- learned preconditioner: backward pass against finite differences
    ("nn_input_gradient_not_conjugated", "nn", 'gu = np.einsum("dkc,rxk->rxdc", np.conj(self.W[l]), gz)',
     'gu = np.einsum("dkc,rxk->rxdc", self.W[l], gz)',
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_backward_matches_finite_differences())),
    ("nn_transport_not_conjugated", "nn", "contrib = np.conj(self.T)[None, :, :, None] * gu",
     "contrib = self.T[None, :, :, None] * gu",
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_backward_matches_finite_differences())),
    ("nn_activation_radial_term_dropped", "nn", "gz = np.where(on, rad * ph + scale * (g - rad * ph), 0)",
     "gz = np.where(on, scale * (g - rad * ph), 0)",
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_backward_matches_finite_differences())),
    ("nn_activation_bias_outside", "nn",
     "s = np.where(mag > 0, np.maximum(0.0, mag + self.b[l][None, None, :]) / np.where(mag > 0, mag, 1), 0)",
     "s = np.where(mag > 0, (np.maximum(0.0, mag) + self.b[l][None, None, :]) / np.where(mag > 0, mag, 1), 0)",
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_backward_matches_finite_differences())),
    ("nn_diagonal_single_path", "nn", "T = 0.5 * (Tx[dx] * sh(Tt[dt], dx, 0) + Tt[dt] * sh(Tx[dx], 0, dt))",
     "T = Tx[dx] * sh(Tt[dt], dx, 0)",
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_reversed_path_identity())),
    ("nn_transport_periodic_t", "nn", "sgn_f = np.where(t == L - 1, -1.0, 1.0)", "sgn_f = np.ones((L, L))",
     lambda mp, m: (mp.setattr(t_nn, "onn", m), t_nn.test_transport_of_constant_field_is_trivial())),
]


def three_level_agg4(m):
    """A hierarchy whose level 1 has 8 dof per site (4 test vectors per chirality) and is aggregated again, so
    that the coarse chirality split of level 1 -> 2 is exercised (L = 64, 4x4 aggregates, 3 levels)."""
    U = gauge.links(gauge.field(64, 3.0, 0, sweeps=40))
    return m.Hierarchy(osch.dirac_sparse(U, -0.05), 64, ntv=4, setup_sweeps=1, seed=5)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(case, monkeypatch):
    _, name, old, new, pin = case
    m = mutant(name, old, new)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        pin(monkeypatch, m)
