"""Pins of the oracle's per-dipole trial mode (trial_mode 1): one trial per
dipole with the summed overestimate of its kernels, the kernel drawn in
proportion to its share.  App. A generates one trial per (dipole, kernel);
the first of independent exponential trials is distributed as one trial
with the summed rate whose kind has probability rate / sum, so both modes
give the same distribution.  These tests check that equivalence on the full
shower, the exact Sudakov factor of the first emission, and that a planted
uniform kernel choice is caught."""
import numpy as np
import pytest

from tests.test_oracle_shower import _first_emission_chi2, _threads

N = 100_000


def _run(O, trial_mode, seed, mutation=0, n=N):
    p = O.make_params(seed=seed, trial_mode=trial_mode, mutation=mutation)
    return O.run(p, 0, n, threads=_threads(O))


def _two_sample_chi2(a, b):
    """chi^2 / ndf of two histograms of event counts from independent samples
    of equal size (bins empty in both skipped)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    m = (a + b) > 0
    return float(np.sum((a[m] - b[m]) ** 2 / (a[m] + b[m])) / max(1, m.sum() - 1))


def _multiplicity(ev):
    return np.bincount(ev["n_partons"], minlength=64)[:64]


@pytest.fixture(scope="module")
def samples(oracle_mod):
    return {m: _run(oracle_mod, m, seed=31 + m) for m in (0, 1)}


def test_one_trial_per_dipole(oracle_mod, samples):
    """Every trial is a dipole's: n_trials equals n_dipoles (one trial per
    dipole with phase space, every cycle); per kernel there are more."""
    ev1, ev0 = samples[1]["events"], samples[0]["events"]
    assert np.array_equal(ev1["n_trials"], ev1["n_dipoles"])
    assert np.all(ev0["n_trials"] >= ev0["n_dipoles"]) and ev0["n_trials"].sum() > 2 * ev0["n_dipoles"].sum()


def test_modes_agree_in_distribution(oracle_mod, samples):
    """Multiplicity and every observable histogram of the two modes agree
    within statistics (independent draws: the modes use different random
    numbers)."""
    h0, h1 = samples[0]["hist"], samples[1]["hist"]
    assert _two_sample_chi2(_multiplicity(samples[0]["events"]), _multiplicity(samples[1]["events"])) < 1.6
    for h in range(oracle_mod.N_OBS):
        assert _two_sample_chi2(h0[h, :, 2], h1[h, :, 2]) < 1.6, h
    # mean emissions per event within 4 sigma
    e0 = samples[0]["events"]["n_emissions"].astype(float)
    e1 = samples[1]["events"]["n_emissions"].astype(float)
    sigma = np.sqrt(e0.var() / len(e0) + e1.var() / len(e1))
    assert abs(e0.mean() - e1.mean()) < 4 * sigma


def test_g_to_qqbar_rate_agrees(oracle_mod):
    """The fraction of gluon splittings into a quark pair (the kernels'
    shares) is the same in both modes: quark pairs counted from the final
    flavours."""
    n = 20_000
    rates = []
    for m in (0, 1):
        p = oracle_mod.make_params(seed=41 + m, trial_mode=m, capacity=64)
        r = oracle_mod.run(p, 0, n, threads=_threads(oracle_mod), want_momenta=True, want_obs=False,
                           want_hist=False)
        flav = r["info"][:, :, 0]
        quarks = np.sum((flav != 0) & (flav != 21), axis=1)
        pairs = (quarks - 2) / 2.0
        rates.append((pairs.mean(), pairs.std() / np.sqrt(n)))
    (m0, s0), (m1, s1) = rates
    assert m0 > 0.0
    assert abs(m0 - m1) < 4 * np.hypot(s0, s1), rates


def test_uniform_kernel_choice_is_caught(oracle_mod, samples):
    """Drawing the kernel uniformly (5 of 6 gluon splittings into quarks)
    changes the multiplicity distribution far beyond statistics."""
    bad = _run(oracle_mod, 1, seed=32, mutation=oracle_mod.MUT_KERNEL_UNIFORM)
    assert _two_sample_chi2(_multiplicity(samples[0]["events"]), _multiplicity(bad["events"])) > 20.0


@pytest.mark.parametrize("fixed", [1, 0])
def test_first_emission_matches_exact_sudakov_per_dipole(oracle_mod, fixed):
    """The first emission of the two-parton state against the exact Sudakov
    factor, in the per-dipole mode."""
    chi2, ndf, ks = _first_emission_chi2(_Mode1(oracle_mod), fixed)
    assert chi2 / ndf < 2.0, (chi2, ndf)
    assert ks > 1e-3


class _Mode1:
    """The oracle module with make_params defaulting to trial_mode 1."""

    def __init__(self, O):
        self._O = O

    def __getattr__(self, name):
        return getattr(self._O, name)

    def make_params(self, **kw):
        kw.setdefault("trial_mode", 1)
        return self._O.make_params(**kw)
