"""Wetting theory: the oracle's contact angles pinned, and the product's host-side
functions (closed form and inversion) checked against the oracle.

Pins of the oracle (Sec. Surface Thermodynamics, Sec. Inverting the contact
angle relations):
- neutral walls (h = 0) give 90 degrees for every pair;
- binary limit: with only fluids m and n present, equal kappa and
  h_m = -h_n = h, the surface term is -h (C_m - C_n) on the binary order
  parameter, and the angle must be the binary free-energy model's Cahn result
  cos theta = [(1 + W)^{3/2} - (1 - W)^{3/2}] / 2 with W = 4h / (alpha kappa);
- the majority and minority integrals agree with the closed forms the paper
  prints for them (Eq. integral_max and the J_n expression);
- Girifalco-Good: gamma_12 cos theta_12 + gamma_23 cos theta_23 + gamma_31 cos theta_31 = 0;
- swapping the labels of two fluids (with their kappa and h) swaps the angles;
- a fluid that is attracted (h_m > 0 against h_n < 0) wets: theta_mn < 90.
"""
import numpy as np
import pytest

from oracle import wetting as OW


def test_neutral_wall_gives_right_angles():
    for kap in ((0.01, 0.01, 0.01), (0.01, 0.02, 0.03), (0.05, 0.005, 0.02)):
        for alpha in (1.0, 1.5):
            assert np.allclose(OW.contact_angles(kap, alpha, (0, 0, 0)), 90.0, atol=1e-9)


@pytest.mark.parametrize("alpha", [1.0, 1.5, 2.0])
@pytest.mark.parametrize("W_", [-0.9, -0.5, -0.1, 0.2, 0.6, 0.95])
def test_binary_limit_is_the_cahn_result(alpha, W_):
    kap = 0.013
    h = W_ * alpha * kap / 4
    want = ((1 + W_) ** 1.5 - (1 - W_) ** 1.5) / 2
    for m, n in ((0, 1), (1, 2), (2, 0)):
        hh = [0.0, 0.0, 0.0]
        hh[m], hh[n] = h, -h
        k = [kap, kap, 0.031]  # the absent fluid's parameters must not matter
        k[m] = k[n] = kap
        l = 3 - m - n
        hh[l] = 0.3 * 0.031 * alpha / 4
        c = OW.contact_cosines(k, alpha, hh)
        pair = {(0, 1): 0, (1, 2): 1, (2, 0): 2}[(m, n)]
        assert c[pair] == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("h", [-0.0024, -0.001, 0.0, 0.0007, 0.0024])
def test_integrals_match_the_printed_closed_forms(h):
    kap, alpha = 0.01, 1.0
    sp = np.sqrt(1 + 4 * h / (alpha * kap))
    sm = np.sqrt(1 - 4 * h / (alpha * kap))
    cmax, cmin = OW.wall_roots(kap, alpha, h)
    I_printed = -h * cmax + alpha / 12 * (kap + sp * (2 * h / alpha - kap))
    J_printed = -h * cmin + alpha / 12 * (kap - sm * (2 * h / alpha + kap))
    assert OW.majority_term(kap, alpha, h) == pytest.approx(I_printed, abs=1e-15)
    assert OW.minority_term(kap, alpha, h) == pytest.approx(J_printed, abs=1e-15)


def _draws(n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        kap = rng.uniform(0.005, 0.05, 3)
        alpha = rng.uniform(0.8, 2.0)
        h = rng.uniform(-0.24, 0.24, 3) * alpha * kap
        yield kap, alpha, h


def test_girifalco_good_and_relabelling():
    for kap, alpha, h in _draws(40, 1):
        c = OW.contact_cosines(kap, alpha, h)
        g = [OW.fluid_tension(kap, alpha, m, n) for m, n in OW.PAIRS]
        assert abs(sum(gi * ci for gi, ci in zip(g, c))) <= 1e-15
        # swap fluids 1 and 2: theta_12 -> theta_21 = 180 - theta_12, theta_23 <-> theta_13
        perm = [1, 0, 2]
        c2 = OW.contact_cosines(kap[perm], alpha, h[perm])
        assert c2[0] == pytest.approx(-c[0], abs=1e-12)
        assert c2[1] == pytest.approx(-c[2], abs=1e-12)  # cos theta_13 = -cos theta_31
        assert c2[2] == pytest.approx(-c[1], abs=1e-12)


def test_attracted_fluid_wets():
    kap = (0.01, 0.02, 0.03)
    t = OW.contact_angles(kap, 1.0, (0.002, -0.002, 0.0))
    assert t[0] < 90 and t[2] > 90  # fluid 1 attracted: theta_12 < 90, theta_31 > 90


def test_oracle_inversion_round_trip():
    kap = (0.01, 0.02, 0.03)
    for t12, t13 in ((45, 70), (120, 100), (90, 90), (60, 30)):
        h = OW.wetting_from_angles(kap, 1.0, t12, t13)
        assert h is not None
        assert abs(h[0] / kap[0] + h[1] / kap[1] + h[2] / kap[2]) <= 1e-15
        th = OW.contact_angles(kap, 1.0, h)
        assert th[0] == pytest.approx(t12, abs=1e-8)
        assert 180 - th[2] == pytest.approx(t13, abs=1e-8)


# ---- product host functions against the oracle (host code only, no GPU)

tl = pytest.importorskip("paper_1511_02155_gb300")


def _lib_or_skip():
    try:
        tl.load_library(build_if_missing=True)
    except Exception as e:  # pragma: no cover - no toolkit
        pytest.skip(f"libtlbm.so unavailable: {e}")


def test_product_angles_match_oracle():
    _lib_or_skip()
    for kap, alpha, h in _draws(60, 2):
        got = tl.contact_angles(kap, alpha, h)
        want = OW.contact_angles(kap, alpha, h)
        assert np.allclose(got, want, atol=1e-9), (got, want)


def test_product_inversion_matches_oracle_and_gauge():
    _lib_or_skip()
    rng = np.random.default_rng(3)
    done = 0
    while done < 25:
        kap = rng.uniform(0.005, 0.05, 3)
        t12, t13 = rng.uniform(30, 150, 2)
        try:
            h = tl.wetting_from_angles(kap, 1.0, t12, t13)
        except tl.TLBMError:
            # infeasible pair: the oracle must not find a solution either
            assert OW.wetting_from_angles(kap, 1.0, t12, t13) is None
            continue
        ho = OW.wetting_from_angles(kap, 1.0, t12, t13)
        assert ho is not None
        assert np.allclose(h, ho, atol=1e-12)
        assert abs(sum(hm / km for hm, km in zip(h, kap))) <= 1e-14
        th = OW.contact_angles(kap, 1.0, h)
        assert th[0] == pytest.approx(t12, abs=1e-7) and 180 - th[2] == pytest.approx(t13, abs=1e-7)
        done += 1


def test_product_rejects_unreachable_angles_and_bad_arguments():
    _lib_or_skip()
    with pytest.raises(tl.TLBMError):
        tl.wetting_from_angles((0.01, 0.01, 0.01), 1.0, 20.0, 170.0)  # theta_23 would not exist
    with pytest.raises(tl.TLBMError):
        tl.wetting_from_angles((0.01, 0.01, 0.01), 1.0, 0.0, 90.0)
    with pytest.raises(tl.TLBMError):
        tl.contact_angles((0.01, 0.01, 0.01), 1.0, (0.0026, 0.0, 0.0))  # |4h| > alpha kappa
    assert tl.contact_angles((0.01, 0.02, 0.03), 1.0, (0, 0, 0)) == pytest.approx((90.0, 90.0, 90.0))
