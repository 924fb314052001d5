"""Planted mistakes: each test swaps one plausible bug into the oracle (on the
CPU, through monkeypatch) and checks that one of the oracle's pins fails."""
import numpy as np
import pytest

import oracle.philox as ph
from oracle import dpar2 as od
import test_oracle_als as T_als
import test_oracle_philox as T_ph
import test_oracle_rsvd as T_rsvd
import test_oracle_sketch as T_sk


def _fails(fn, *a):
    with pytest.raises((AssertionError, ValueError)):
        fn(*a)


def test_swapped_khatri_rao_operands_caught(monkeypatch):
    orig = od.khatri_rao
    monkeypatch.setattr(od, "khatri_rao", lambda A, B: orig(B, A) if A.shape[0] == B.shape[0] else orig(A, B)[::-1])
    _fails(T_als.test_mttkrp_matches_brute_force_definition)


def test_transposed_unfolding_caught(monkeypatch):
    monkeypatch.setattr(od, "unfold", lambda T, m: np.moveaxis(T, m, 0).reshape(T.shape[m], -1, order="C"))
    _fails(T_als.test_mttkrp_matches_brute_force_definition)


def test_transposed_polar_factor_caught(monkeypatch):
    def bad(T):
        Z, s, Pt = np.linalg.svd(T)
        return Pt.T @ Z.T
    monkeypatch.setattr(od, "_polar_from_svd", bad)
    _fails(T_als.test_polar_factor_closed_form)


def test_wrong_truncation_order_caught(monkeypatch):
    orig_svd = np.linalg.svd

    def ascending(B, full_matrices=True, compute_uv=True):
        U, s, Vt = orig_svd(B, full_matrices=full_matrices)
        return U[:, ::-1], s[::-1], Vt[::-1]
    monkeypatch.setattr(od.np.linalg, "svd", ascending)
    _fails(T_rsvd.test_truncation_is_eckart_young_when_sketch_spans_range)


def test_gradient_sign_error_caught(monkeypatch):
    orig = od.sketch_loss_grad
    monkeypatch.setattr(od, "sketch_loss_grad", lambda X, O: -orig(X, O))
    _fails(T_sk.test_gradient_matches_central_finite_differences)


def test_missing_e_in_compressed_slices_caught(monkeypatch):
    monkeypatch.setattr(od, "compressed_slices",
                        lambda comp: [a @ f @ comp["D"].T for a, f in zip(comp["A"], comp["Fk"])])
    _fails(T_rsvd.test_stage2_identity_and_compressed_slices_exact_on_lowrank)


def test_wrong_philox_multiplier_caught(monkeypatch):
    monkeypatch.setattr(ph, "M1", np.uint64(0xCD9E8D55))
    ctr, key, out = T_ph._kat()[2]
    _fails(T_ph.test_known_answer_vectors, ctr, key, out)


def test_missing_key_bump_caught(monkeypatch):
    monkeypatch.setattr(ph, "W0", np.uint64(0))
    ctr, key, out = T_ph._kat()[0]
    _fails(T_ph.test_known_answer_vectors, ctr, key, out)
