"""Pins for the oracle's PST sampling (Sec. 4, "PST pre-sampling") and the PST
update of Sec. 3.3 (APS, Eq. ebs, Eq. wafit, Eq. rsdir, Eq. rsinter,
Eq. momentum, the empty-APS corner case of Sec. 4).

Philox4x32-10 is checked against the known-answer vectors published with the
generator (Salmon et al., SC 2011, Random123 distribution); the update against
hand-derived cases in tests/golden/pst_update.json."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pst_update.json")

# (counter, key) -> output, Philox4x32 with 10 rounds (Random123 known-answer vectors)
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(oracle, ctr, key, out):
    assert tuple(oracle.philox4x32_10(ctr, key)) == out


def test_pst_uniform_invariants(oracle):
    n = 5000
    P = oracle.pst_uniform(n, seed=7)
    assert P.shape == (6, n) and P.dtype == np.float32
    assert np.all(P[:, 0] == 0)  # row 0 is the origin (the PST centre)
    r = np.linalg.norm(P.astype(np.float64), axis=0)
    assert r.max() <= 1.0
    scaled = P.astype(np.float64) * 2 ** 24  # exact odd integers (2 m + 1 - 2^24)
    assert np.all(scaled[:, 1:] == np.round(scaled[:, 1:])) and np.all(np.mod(scaled[:, 1:], 2) == 1)
    np.testing.assert_array_equal(P, oracle.pst_uniform(n, seed=7))
    assert not np.array_equal(P, oracle.pst_uniform(n, seed=8))
    # prefixes are consistent: particle i does not depend on n
    np.testing.assert_array_equal(oracle.pst_uniform(100, seed=7), P[:, :100])


def test_pst_uniform_distribution(oracle):
    from scipy import stats

    n = 20000
    P = oracle.pst_uniform(n, seed=1).astype(np.float64)[:, 1:]
    r = np.linalg.norm(P, axis=0)
    # uniform in the unit 6D ball: P(|x| <= a) = a^6
    assert stats.kstest(r, lambda a: np.clip(a, 0, 1) ** 6).pvalue > 1e-3
    # E[x_d] = 0 and E[x_d^2] = 1 / (d + 2) = 1/8 per coordinate
    se = np.sqrt(1 / 8 / P.shape[1])
    assert np.all(np.abs(P.mean(axis=1)) < 5 * se)
    assert np.all(np.abs((P ** 2).mean(axis=1) - 0.125) < 0.01)


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_pst_update_golden(oracle, case):
    n_aps, dbar, rho_t, r = oracle.pst_update(np.array(case["rho"]), np.array(case["delta"], float),
                                              case["rho_ref"], np.array(case["r_prev"], float), 0.1, 1e-3)
    assert n_aps == case["expect_n_aps"]
    np.testing.assert_allclose(dbar, case["expect_delta_bar"], atol=1e-15)
    assert rho_t == pytest.approx(case["expect_rho_tilde"], abs=1e-15)
    np.testing.assert_allclose(r, case["expect_r"], atol=1e-15)


def test_pst_update_weight_scale_invariance(oracle):
    # wbar is a normalised weight: shifting every APS member's excess by the same
    # factor (rho_i - rho_ref -> c (rho_i - rho_ref)) keeps delta_bar (Eq. ebs)
    rng = np.random.default_rng(0)
    delta = rng.normal(size=(50, 6)) * 0.05
    rho = rng.uniform(0.5, 0.9, size=50)
    ref = 0.7
    n1, d1, _, _ = oracle.pst_update(rho, delta, ref, np.ones(6))
    rho2 = ref + 0.5 * (rho - ref)
    n2, d2, _, _ = oracle.pst_update(rho2, delta, ref, np.ones(6))
    assert n1 == n2 == int((rho > ref).sum())
    np.testing.assert_allclose(d1, d2, atol=1e-14)
