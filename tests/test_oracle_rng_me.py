"""Oracle pins: the Philox4x32-10 generator and the LO e+e- -> q qbar matrix
element (App. B).  CPU only."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Electroweak inputs adopted by this build (the paper names none).
MZ, GZ, ALPHA, SW2 = 91.1876, 2.4952, 1.0 / 128.802, 0.222
GEV2PB = 0.389379e9


def test_philox_known_answers(oracle_mod):
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle_mod.philox(v[0:4], v[4:6]) == v[6:10]


def test_unit_double_open_interval(oracle_mod):
    """u = (m + 1/2) 2^-52 from the top 26 bits of two words: strictly inside
    (0, 1), and the two halves of a draw are different words of one block."""
    us = np.array([oracle_mod.uniform_pair(7, e, 3, 5, 2) for e in range(4000)])
    assert np.all(us > 0) and np.all(us < 1)
    # mean and variance of U(0,1) within 5 sigma
    for col in range(2):
        assert abs(us[:, col].mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(us))
    assert abs(np.corrcoef(us[:, 0], us[:, 1])[0, 1]) < 0.1
    # the pair is built from words (0,1) and (2,3) of the block
    w = oracle_mod.philox([11, 3, 5, 2], [7, 0])
    m0 = ((w[0] >> 6) << 26) | (w[1] >> 6)
    m1 = ((w[2] >> 6) << 26) | (w[3] >> 6)
    u = oracle_mod.uniform_pair(7, 11, 3, 5, 2)
    assert u[0] == (m0 + 0.5) * 2.0 ** -52 and u[1] == (m1 + 0.5) * 2.0 ** -52


def _couplings(f):
    up = f in (2, 4)
    q = 2 / 3 if up else -1 / 3
    t3 = 0.5 if up else -0.5
    return q, t3 - 2 * q * SW2, t3


def _chis(s):
    kappa = 1 / (4 * SW2 * (1 - SW2))
    den = (s - MZ ** 2) ** 2 + GZ ** 2 * MZ ** 2
    return kappa * s * (s - MZ ** 2) / den, kappa ** 2 * s ** 2 / den


def sigma_total_closed(s, f):
    """Total LO cross section for one flavour (Ellis-Stirling-Webber), pb."""
    qe, ve, ae = -1.0, -0.5 + 2 * SW2, -0.5
    qf, vf, af = _couplings(f)
    c1, c2 = _chis(s)
    bracket = qe ** 2 * qf ** 2 + 2 * qe * qf * ve * vf * c1 + (ae ** 2 + ve ** 2) * (af ** 2 + vf ** 2) * c2
    return 4 * math.pi * ALPHA ** 2 / (3 * s) * 3 * bracket * GEV2PB


def _gl_integral(fun, a, b, n=8):
    x, w = np.polynomial.legendre.leggauss(n)
    xm, xr = 0.5 * (a + b), 0.5 * (b - a)
    return xr * sum(wi * fun(xm + xr * xi) for xi, wi in zip(x, w))


@pytest.mark.parametrize("sqrt_s", [10.0, 91.2, 133.0, 200.0])
def test_dsigma_integrates_to_closed_form(oracle_mod, sqrt_s):
    p = oracle_mod.make_params(sqrt_s=sqrt_s)
    for f in range(1, 6):
        num = _gl_integral(lambda c: oracle_mod.dsigma_dcos(p, f, c), -1.0, 1.0)
        assert num == pytest.approx(sigma_total_closed(sqrt_s ** 2, f), rel=1e-12)


def test_forward_backward_asymmetry_at_pole(oracle_mod):
    """At s = m_Z^2 the gamma-Z interference vanishes (chi_1 = 0) and
    A_FB = 3/4 * Ae * Af * Z / (Z + G), with A_f = 2 V_f A_f / (V_f^2 + A_f^2),
    Z = (Ae^2 + Ve^2)(Af^2 + Vf^2) chi_2 and G = Qe^2 Qf^2 the pure-photon part."""
    p = oracle_mod.make_params(sqrt_s=MZ)
    qe, ve, ae = -1.0, -0.5 + 2 * SW2, -0.5
    chi2 = _chis(MZ ** 2)[1]
    for f in range(1, 6):
        fwd = _gl_integral(lambda c: oracle_mod.dsigma_dcos(p, f, c), 0.0, 1.0)
        bwd = _gl_integral(lambda c: oracle_mod.dsigma_dcos(p, f, c), -1.0, 0.0)
        qf, vf, af = _couplings(f)
        zpart = (ae ** 2 + ve ** 2) * (af ** 2 + vf ** 2) * chi2
        afb = 0.75 * (2 * ve * ae / (ve ** 2 + ae ** 2)) * (2 * vf * af / (vf ** 2 + af ** 2))
        afb *= zpart / (zpart + qe ** 2 * qf ** 2)
        assert (fwd - bwd) / (fwd + bwd) == pytest.approx(afb, rel=1e-11)


def test_qed_limit_charge_ratio(oracle_mod):
    """Far below the Z the cross section goes as Q_f^2: u/d = 4."""
    p = oracle_mod.make_params(sqrt_s=2.0)
    assert oracle_mod.dsigma_dcos(p, 2, 0.3) / oracle_mod.dsigma_dcos(p, 1, 0.3) == pytest.approx(4.0, rel=2e-3)


@pytest.mark.parametrize("sqrt_s,mutation,ok", [(91.2, 0, True), (133.0, 0, True), (200.0, 0, True),
                                               (133.0, 1 << 5, False)])
def test_mean_weight_is_total_cross_section(oracle_mod, sqrt_s, mutation, ok):
    """The mean ME weight estimates sum_f sigma_f (within 4 sigma_MC).  The
    planted mistake (no gamma-Z interference) must fail it."""
    n = 40000
    p = oracle_mod.make_params(sqrt_s=sqrt_s, seed=11, mutation=mutation, max_emissions=1)
    ev = oracle_mod.run(p, 0, n, threads=oracle_mod.threads_available(), want_obs=False,
                        want_hist=False)["events"]
    w = ev["weight"]
    expect = sum(sigma_total_closed(sqrt_s ** 2, f) for f in range(1, 6))
    pull = (w.mean() - expect) / (w.std() / math.sqrt(n))
    assert (abs(pull) < 4) == ok
    # every flavour is drawn uniformly
    counts = np.bincount(ev["me_flavour"], minlength=6)[1:]
    assert np.all(np.abs(counts - n / 5) < 5 * math.sqrt(n / 5))
