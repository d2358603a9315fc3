"""Plant plausible mistakes in the oracle (CPU only) and check that a pin catches each one.

A pin that a dropped term, a wrong sign, a missing exchange or a wrong share would still pass is
no pin; these tests run the pins of test_oracle.py against deliberately broken oracles.
"""
import numpy as np
import pytest

import test_oracle as T
from conftest import load_golden
from oracle import evs, matching, theory
from oracle import vtm as ovtm


def _fails(fn, *args):
    try:
        fn(*args)
    except (AssertionError, np.linalg.LinAlgError, ValueError):
        return True
    return False


def test_dropped_line_admittance_is_caught(monkeypatch):
    """eq. 5.8 without the Z^{-1} port term."""
    monkeypatch.setattr(ovtm, "local_matrix", lambda split, ends, j: split.subgraphs[j].A.tocsr())
    assert _fails(T.test_example_5_1_local_matrices, load_golden)
    assert _fails(T.test_example_5_1_converges_to_direct_solution, load_golden)


def test_missing_exchange_is_caught(monkeypatch):
    """Table 1 step 5 forgotten: every end reads its own old values instead of its twin's."""
    orig = ovtm.ends_of

    def no_exchange(split, Z):
        e = orig(split, Z)
        e.twin = np.arange(len(e.twin))
        return e

    monkeypatch.setattr(ovtm, "ends_of", no_exchange)
    assert _fails(T.test_example_5_1_converges_to_direct_solution, load_golden)
    assert _fails(T.test_a38_operator_reproduces_iteration, 0)


def test_asymmetric_impedance_is_caught(monkeypatch):
    """The two ends of one line must see the same Z (Table 1 step 1)."""
    orig = ovtm.ends_of

    def skewed(split, Z):
        e = orig(split, Z)
        e.Z = e.Z.copy()
        e.Z[1::2] *= 2.0
        return e

    monkeypatch.setattr(ovtm, "ends_of", skewed)
    assert _fails(T.test_example_5_1_local_matrices, load_golden)


def test_unsplit_source_is_caught(monkeypatch):
    """Step 3 forgetting to split b_i between the copies of a boundary vertex."""
    monkeypatch.setattr(evs.SplitGraph, "local_rhs",
                        lambda self, b, j: np.atleast_2d(b)[:, self.subgraphs[j].vertices].astype(float))
    assert _fails(T.test_config1_oracle_reaches_1e10)


def test_unsplit_edge_is_caught(monkeypatch):
    """Step 3 forgetting to split an edge along the boundary (KCL broken)."""
    orig = evs.split_by_owners

    def keep_edges(A, owners, pairs):
        s = orig(A, owners, pairs)
        for g in s.subgraphs:
            g.A = g.A.tolil()
            for r in range(g.A.shape[0]):
                for c in range(g.A.shape[1]):
                    if r != c and g.A[r, c] != 0 and len(owners[g.vertices[r]]) > 1 and len(owners[g.vertices[c]]) > 1:
                        g.A[r, c] = g.A[r, c] * 2
            g.A = g.A.tocsr()
        return s

    monkeypatch.setattr(evs, "split_by_owners", keep_edges)
    assert _fails(T.test_equal_share_rule_on_example_3_1)


def test_input_impedance_without_inverse_is_caught(monkeypatch):
    """Def. 7.1 read as 1 / a_cc instead of (Ã^{-1})_cc."""
    import scipy.sparse as sp
    monkeypatch.setattr(matching, "input_impedance_open",
                        lambda A, c: 1.0 / (A.toarray() if sp.issparse(A) else np.asarray(A))[c, c])
    assert _fails(T.test_example_7_1_input_impedances, load_golden)


def test_operator_without_exchange_is_caught(monkeypatch):
    """eq. A3.8 with J = I: the operator no longer reproduces the iteration."""
    orig_block = np.block

    def fake_block(rows):
        out = orig_block(rows)
        if out.shape[0] == out.shape[1] and np.all(np.diag(out) == 0) and np.allclose(out, out.T):
            return np.eye(out.shape[0])
        return out

    monkeypatch.setattr(theory.np, "block", fake_block)
    assert _fails(T.test_a38_operator_reproduces_iteration, 0)


# ---------------------------------------------------------------- coupled lines (§7.2)
import test_oracle_coupled as TC  # noqa: E402
from oracle import coupled  # noqa: E402


def _coupled_pins_fail():
    return (_fails(TC.test_bundle_reflection_law) and _fails(TC.test_matched_bundle_is_exact_after_three_sweeps)
            and _fails(TC.test_theorem_7_1_random_spd_bundles_converge, (20, 20), (7, 7), 1.0))


def test_coupling_dropped_from_local_matrix_is_caught(monkeypatch):
    """eq. 5.8 with only the diagonal of Y_j in K_j (the right-hand side still coupled)."""
    orig = coupled.local_matrix
    monkeypatch.setattr(coupled, "local_matrix", lambda A, loc, Yj: orig(A, loc, np.diag(np.diag(Yj))))
    assert _coupled_pins_fail()


# the planted mistake makes the iteration diverge: the overflow it meets is the expected outcome
@pytest.mark.filterwarnings("ignore:overflow encountered:RuntimeWarning")
def test_coupling_dropped_from_inflow_is_caught(monkeypatch):
    """The incoming waves injected through the diagonal of Y_j only."""
    orig = coupled.inflow
    monkeypatch.setattr(coupled, "inflow", lambda u, om, Yj: orig(u, om, np.diag(np.diag(Yj))))
    assert _coupled_pins_fail()


# the planted mistake makes the iteration diverge: the overflow it meets is the expected outcome
@pytest.mark.filterwarnings("ignore:overflow encountered:RuntimeWarning")
def test_coupled_current_sign_is_caught(monkeypatch):
    """The twin's current added instead of subtracted in the current update."""
    monkeypatch.setattr(coupled, "current_update", lambda ut, omt, un, Yj: (ut - un) @ Yj + omt)
    assert _coupled_pins_fail()


# ---------------------------------------------------------------- general conformal split (App. 1)
import test_oracle_conformal as TF  # noqa: E402
from oracle import conformal  # noqa: E402


def _conformal_pins_fail():
    return (_fails(TF.test_app1_two_vertex_construction)
            and _fails(TF.test_kcl_and_spd_where_the_diagonal_rule_fails, 12, 10, 2, 2, 0.6))


def test_schur_share_not_divided_is_caught(monkeypatch):
    """Both new subgraphs take lam S: the pieces no longer sum back to A."""
    monkeypatch.setattr(conformal, "boundary_blocks", lambda Ta, Tb, S, lam: (Ta + lam * S, Tb + lam * S))
    assert _conformal_pins_fail()


def test_dropped_completing_square_term_is_caught(monkeypatch):
    """The beta boundary block without M_Bb M_bb^{-1} M_bB."""
    orig = conformal.schur_terms

    def no_tb(M, Ia, Ib, B):
        Ta, Tb, S = orig(M, Ia, Ib, B)
        return Ta, 0 * Tb, S

    monkeypatch.setattr(conformal, "schur_terms", no_tb)
    assert _conformal_pins_fail()


@pytest.mark.parametrize("mistake", ["diag_in_coupling", "own_weight_as_twin", "inverse_size_ratio",
                                     "equal_share_weight"])
def test_line_feature_mistakes_are_caught(monkeypatch, mistake):
    """Feature 4 with the copy's own diagonal, feature 5 from the copy instead of its twin,
    feature 7 as log(n_j / n), feature 1 as a_ii / |O(i)| (an equal share instead of §4 step 3)."""
    import test_oracle_mlp as M
    from oracle import features
    orig = features.line_features

    def broken(split, A):
        f = orig(split, A).copy()
        if mistake == "diag_in_coupling":
            f[:, 4] = np.log(np.exp(f[:, 4]) + np.exp(f[:, 1]))
        elif mistake == "own_weight_as_twin":
            f[:, 5] = f[:, 1]
        elif mistake == "inverse_size_ratio":
            f[:, 7] = -f[:, 7]
        else:
            f[:, 1] = f[:, 0] - f[:, 2]
        return f

    monkeypatch.setattr(features, "line_features", broken)
    assert _fails(M.test_line_features_hand_computed) or _fails(M.test_line_features_ragged_subgraph_sizes)
