"""Oracle pins for the shower (Sec. 2, App. A, App. C): event invariants, the
splitting kernels and z generation, the final-final dipole map, and the
first-emission distribution against the exact Sudakov form factor.  Planted
mistakes (oracle mutations) must fail at least one pin each.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, interpolate, stats

CF, CA, TR = 4 / 3, 3.0, 0.5
MZ = 91.1876


def _threads(O):
    return O.threads_available()


# ------------------------------------------------------------ invariants
@pytest.mark.parametrize("kw", [
    dict(sqrt_s=91.2, t_cutoff=1.0, seed=1),
    dict(sqrt_s=133.0, t_cutoff=0.5, seed=2),
    dict(sqrt_s=200.0, t_cutoff=2.0, seed=3),
    dict(sqrt_s=91.2, t_cutoff=1.0, seed=4, n_flavours=3),
    dict(sqrt_s=91.2, t_cutoff=1.0, seed=5, fixed_alphas=1),
])
def test_every_event_is_physical(oracle_mod, kw):
    """Momentum conserved to 1e-10 GeV, massless positive-energy partons,
    valid colour chains (each line once as colour and once as anticolour,
    chains from quark to antiquark, no loops), flavour balance."""
    p = oracle_mod.make_params(**kw)
    r = oracle_mod.run(p, 0, 3000, threads=_threads(oracle_mod), want_momenta=True)
    ev = r["events"]
    assert np.all(ev["status"] == oracle_mod.DONE)
    assert np.all(ev["valid"] == 0)
    # the record really is conserved (independent re-check in numpy)
    for j in range(0, 3000, 97):
        n = ev["n_partons"][j]
        m = r["mom"][j, :n]
        tot = m.sum(axis=0)
        assert np.allclose(tot, [kw["sqrt_s"], 0, 0, 0], atol=1e-10, rtol=0)
        m2 = m[:, 0] ** 2 - (m[:, 1:] ** 2).sum(axis=1)
        assert np.all(np.abs(m2) <= 1e-10 * m[:, 0] * kw["sqrt_s"])
    assert ev["n_emissions"].sum() > 2000
    assert np.all(ev["n_partons"] == 2 + ev["n_emissions"])


@pytest.mark.parametrize("mutation,bit", [(1 << 2, 1), (1 << 8, 1), (1 << 3, 8)])
def test_invariants_catch_planted_mistakes(oracle_mod, mutation, bit):
    """No recoil / wrong k_perp sign break conservation; swapped colour lines
    break the colour chain."""
    p = oracle_mod.make_params(seed=1, mutation=mutation)
    ev = oracle_mod.run(p, 0, 500, threads=_threads(oracle_mod), want_obs=False, want_hist=False)["events"]
    emitted = ev["n_emissions"] > 0
    assert np.mean((ev["valid"][emitted] & bit) != 0) > 0.9


def test_counter_rng_makes_events_independent_of_batching(oracle_mod):
    """An event's history depends only on (seed, event id): a range and the
    same events showered one by one agree bit for bit."""
    p = oracle_mod.make_params(seed=9)
    whole = oracle_mod.run(p, 100, 50, want_momenta=True)
    for j in (0, 17, 49):
        one = oracle_mod.run(p, 100 + j, 1, want_momenta=True)
        assert one["events"][0].tobytes() == whole["events"][j].tobytes()
        assert np.array_equal(one["mom"][0], whole["mom"][j])
        assert np.array_equal(one["obs"][0], whole["obs"][j])


def test_overflow_flag(oracle_mod):
    """With a small parton capacity the event stops with the overflow status
    at exactly that many partons; larger capacities reproduce the same
    history up to that point."""
    small = oracle_mod.run(oracle_mod.make_params(seed=3, capacity=4), 0, 400,
                           want_momenta=True)["events"]
    big = oracle_mod.run(oracle_mod.make_params(seed=3, capacity=128), 0, 400)["events"]
    over = small["status"] == oracle_mod.OVERFLOW
    assert over.sum() > 50
    assert np.all(small["n_partons"][over] == 4)
    assert np.all(big["n_partons"][over] > 4)
    ok = ~over
    assert np.array_equal(small["hash"][ok], big["hash"][ok])


def test_step_limit_flag(oracle_mod):
    ev = oracle_mod.run(oracle_mod.make_params(seed=3, max_steps=5), 0, 200,
                        want_obs=False, want_hist=False)["events"]
    assert np.all((ev["status"] == oracle_mod.STEP_LIMIT) | (ev["n_steps"] <= 5))
    assert np.any(ev["status"] == oracle_mod.STEP_LIMIT)


def test_param_validation(oracle_mod):
    O = oracle_mod
    assert O.check_params(O.make_params()) == 0
    assert O.check_params(O.make_params(t_cutoff=0.0)) != 0
    assert O.check_params(O.make_params(t_cutoff=91.2 ** 2 / 4)) != 0
    assert O.check_params(O.make_params(n_flavours=6)) != 0
    assert O.check_params(O.make_params(sqrt_s=-1)) != 0
    assert O.check_params(O.make_params(t_cutoff=0.001)) != 0  # below the Landau pole


# ---------------------------------------------- kernels and z generation
def test_estimates_bound_kernels(oracle_mod):
    zs = np.linspace(1e-4, 1 - 1e-4, 301)
    for kind in range(3):
        for y in (1e-6, 0.1, 0.5, 0.99):
            for z in zs:
                assert (1 - y) * oracle_mod.kernel_value(kind, z, y) <= oracle_mod.kernel_estimate(kind, z) + 1e-12


def test_kernel_soft_and_collinear_limits(oracle_mod):
    """Textbook limits: y -> 0 gives the collinear splitting functions
    (C_F (1+z^2)/(1-z), half of C_A [2z/(1-z) + z(1-z)] on the z -> 1 side,
    T_R/2 [z^2 + (1-z)^2])."""
    for z in (0.1, 0.5, 0.9):
        assert oracle_mod.kernel_value(0, z, 0.0) == pytest.approx(CF * (1 + z * z) / (1 - z), rel=1e-13)
        assert oracle_mod.kernel_value(1, z, 0.0) == pytest.approx(CA / 2 * (2 * z / (1 - z) + z * (1 - z)), rel=1e-13)
        assert oracle_mod.kernel_value(2, z, 0.0) == pytest.approx(TR / 2 * (z * z + (1 - z) ** 2), rel=1e-13)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_integral_and_inversion(oracle_mod, kind):
    """I(zp) - I(zm) is the integral of P^over; z(r) inverts its cumulative
    integral (Eq. A.8), and samples follow the normalised P^over (KS test)."""
    zm, zp = 0.013, 0.987
    num, _ = integrate.quad(lambda z: oracle_mod.kernel_estimate(kind, z), zm, zp, epsabs=0, epsrel=1e-13)
    assert oracle_mod.kernel_integral(kind, zm, zp) == pytest.approx(num, rel=1e-11)
    for r in (0.0, 0.1, 0.37, 0.5, 0.93, 1.0):
        z = oracle_mod.kernel_generate_z(kind, zm, zp, r)
        part, _ = integrate.quad(lambda x: oracle_mod.kernel_estimate(kind, x), zm, z, epsabs=1e-14, epsrel=1e-13)
        assert part == pytest.approx(r * num, rel=1e-9, abs=1e-12)
    # KS against the textbook CDF of 1/(1-z) (kinds 0, 1) or a constant (kind 2)
    us = np.random.default_rng(kind).random(20000)
    zs = np.array([oracle_mod.kernel_generate_z(kind, zm, zp, u) for u in us])
    if kind == 2:
        cdf = lambda z: (z - zm) / (zp - zm)
    else:
        cdf = lambda z: np.log((1 - zm) / (1 - z)) / np.log((1 - zm) / (1 - zp))
    assert stats.kstest(zs, cdf).pvalue > 1e-3
    zs_bad = np.array([oracle_mod.kernel_generate_z(kind, zm, zp, u, 1 << 1) for u in us])
    if kind != 2:
        assert stats.kstest(zs_bad, cdf).pvalue < 1e-6


# ------------------------------------------------------- kinematic map
def _random_massless(rng, e):
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    return np.concatenate([[e], e * v])


def _mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


@pytest.mark.parametrize("mutation,expect_ok", [(0, True), (1 << 9, False)])
def test_splitting_map_round_trip(oracle_mod, mutation, expect_ok):
    """The final-final map conserves momentum, keeps partons massless, and
    its inverse y = pi.pj / (pi.pj + pi.pk + pj.pk), z = pi.pk / (pi.pk +
    pj.pk) recovers (y, z); the emission's k_T^2 = z(1-z) y Q^2."""
    rng = np.random.default_rng(5)
    bad = 0
    for _ in range(300):
        pij = _random_massless(rng, rng.uniform(1, 45))
        pk = _random_massless(rng, rng.uniform(1, 45))
        if _mdot(pij, pk) < 1e-3:
            continue
        z, y, phi = rng.uniform(0.01, 0.99), rng.uniform(1e-4, 0.95), rng.uniform(0, 2 * math.pi)
        pi, pj, pkn = oracle_mod.splitting_map(pij, pk, z, y, phi, mutation)
        q2 = 2 * _mdot(pij, pk)
        assert np.allclose(pi + pj + pkn, pij + pk, atol=1e-12 * q2 ** 0.5, rtol=0)
        for v in (pi, pj, pkn):
            assert abs(_mdot(v, v)) < 1e-11 * q2
        yij = _mdot(pi, pj) / (_mdot(pi, pj) + _mdot(pi, pkn) + _mdot(pj, pkn))
        zi = _mdot(pi, pkn) / (_mdot(pi, pkn) + _mdot(pj, pkn))
        assert yij == pytest.approx(y, rel=1e-10)
        if not (abs(zi - z) < 1e-9 and abs(2 * _mdot(pi, pj) * zi * (1 - zi) - z * (1 - z) * y * q2) < 1e-9 * q2):
            bad += 1
    assert (bad == 0) == expect_ok


def test_azimuth_is_uniform_around_the_dipole(oracle_mod):
    """The emitted k_perp sweeps a full circle: p_i at phi and phi + pi are
    mirror images about the dipole plane, and the transverse vectors for
    phi = 0 and pi/2 are orthogonal."""
    rng = np.random.default_rng(8)
    pij = _random_massless(rng, 30.0)
    pk = _random_massless(rng, 20.0)
    z, y = 0.3, 0.2
    base = z * pij + (1 - z) * y * pk
    k0 = oracle_mod.splitting_map(pij, pk, z, y, 0.0)[0] - base
    k1 = oracle_mod.splitting_map(pij, pk, z, y, math.pi / 2)[0] - base
    k2 = oracle_mod.splitting_map(pij, pk, z, y, math.pi)[0] - base
    assert np.allclose(k2, -k0, atol=1e-12)
    assert abs(_mdot(k0, k1)) < 1e-10
    assert _mdot(k0, k0) == pytest.approx(-z * (1 - z) * y * 2 * _mdot(pij, pk), rel=1e-12)
    assert abs(_mdot(k0, pij)) < 1e-10 and abs(_mdot(k0, pk)) < 1e-10


# ----------------------------------------- first emission vs exact Sudakov
def _alphas(t, as_mz, fixed, nf=5):
    if fixed:
        return as_mz
    b0 = (33 - 2 * nf) / (12 * math.pi)
    return as_mz / (1 + as_mz * b0 * math.log(t / MZ ** 2))


def _emission_density(t, s, as_mz, fixed):
    """(1/t) (alpha_s(t)/2pi) int dz (1-y) P_qq(z, y) over the physical z range
    at scale t, for a q qbar dipole of mass^2 s (App. A, Eq. A.1 with the
    Catani-Seymour (1-y) phase-space factor)."""
    if t >= s / 4:
        return 0.0
    root = math.sqrt(1 - 4 * t / s)
    zlo, zhi = 0.5 * (1 - root), 0.5 * (1 + root)

    def f(z):
        y = t / (s * z * (1 - z))
        return (1 - y) * CF * (2 / (1 - z * (1 - y)) - (1 + z))

    inner, _ = integrate.quad(f, zlo, zhi, epsabs=1e-13, epsrel=1e-11, limit=200)
    return _alphas(t, as_mz, fixed) / (2 * math.pi) * inner / t


def _log_sudakov_grid(edges, s, as_mz, fixed):
    """ln Delta(t) for one dipole at every edge: -int_t^{s/4} density."""
    tops = list(edges) + [s / 4]
    pieces = []
    for a, b in zip(tops[:-1], tops[1:]):
        # integrate in ln t for smoothness
        val, _ = integrate.quad(lambda lt: _emission_density(math.exp(lt), s, as_mz, fixed) * math.exp(lt),
                                math.log(a), math.log(b), epsabs=1e-12, epsrel=1e-10, limit=200)
        pieces.append(val)
    cum = np.cumsum(pieces[::-1])[::-1]
    return -cum  # ln Delta at each edge


def _first_emission_chi2(O, fixed, mutation=0, n=200000, seed=21):
    sqrt_s, tc, as_mz = 91.2, 1.0, 0.118
    s = sqrt_s ** 2
    p = O.make_params(sqrt_s=sqrt_s, t_cutoff=tc, alphas_mz=as_mz, seed=seed, fixed_alphas=fixed,
                      max_emissions=1, mutation=mutation)
    ev = O.run(p, 0, n, threads=_threads(O), want_obs=False, want_hist=False)["events"]
    t1 = ev["t_first"]
    edges = np.exp(np.linspace(math.log(tc), math.log(s / 4), 25))
    ln_delta = _log_sudakov_grid(edges[:-1], s, as_mz, fixed)
    ln_delta = np.append(ln_delta, 0.0)  # Delta(s/4) = 1
    # two identical dipoles: P(t1 < t) = Delta(t)^2
    cdf2 = np.exp(2 * ln_delta)
    probs = np.diff(cdf2)
    p_none = cdf2[0]
    counts, _ = np.histogram(t1[t1 > 0], bins=edges)
    n_none = np.sum(t1 == 0)
    obs = np.append(counts, n_none)
    exp = np.append(probs, p_none) * n
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    # KS on the emitted events against the normalised CDF
    spline = interpolate.CubicSpline(np.log(edges), 2 * ln_delta)
    cdf = lambda t: (np.exp(spline(np.log(t))) - p_none) / (1 - p_none)
    ks = stats.kstest(t1[t1 > 0], cdf).pvalue
    return chi2, len(obs) - 1, ks


@pytest.mark.parametrize("fixed", [1, 0])
def test_first_emission_matches_exact_sudakov(oracle_mod, fixed):
    """P(t1 < t) = Delta(t)^2 from the 2-parton state (two q qbar dipoles of
    mass^2 s), with ln Delta by adaptive quadrature; the veto algorithm
    reproduces it (App. A: proven to give the correct Sudakov factor)."""
    chi2, ndf, ks = _first_emission_chi2(oracle_mod, fixed)
    assert chi2 / ndf < 2.0, (chi2, ndf)
    assert ks > 1e-3


@pytest.mark.parametrize("fixed,mutation", [(1, 1 << 0), (1, 1 << 1), (1, 1 << 11), (0, 1 << 4)])
def test_sudakov_pin_catches_planted_mistakes(oracle_mod, fixed, mutation):
    """Dropping (1-y), a wrong z inversion, restarting vetoed trials from the
    old scale, or an alpha_s^over below alpha_s(t) all move the first-emission
    distribution away from the exact Sudakov factor."""
    chi2, ndf, ks = _first_emission_chi2(oracle_mod, fixed, mutation=mutation)
    assert chi2 / ndf > 10.0 or ks < 1e-6, (chi2, ndf, ks)


def test_paper_scale_run_is_qualitatively_like_the_paper(oracle_mod):
    """Most events end within a few tens of veto cycles (the paper's Fig. 7
    shows 40-50 for its conventions); 50 parton slots almost never overflow
    (App. C sets 50 for LEP)."""
    ev = oracle_mod.run(oracle_mod.make_params(seed=2, capacity=50), 0, 20000,
                        threads=_threads(oracle_mod), want_obs=False, want_hist=False)["events"]
    assert 15 <= np.median(ev["n_steps"]) <= 60
    assert ev["n_steps"].max() < 250
    assert np.mean(ev["status"] == oracle_mod.OVERFLOW) < 1e-3


# ------------------- first emission from a q g qbar state (gluon branches)
# A fixed three-parton state at sqrt(s) = 91.2 GeV with energy fractions
# x_q = 0.8, x_qbar = 0.7, x_g = 0.5, colour-ordered q - g - qbar: four
# dipoles, (q | g) and (g | q) of mass^2 0.3 s, (g | qbar) and (qbar | g) of
# mass^2 0.2 s.  Each quark end has the q -> qg kernel; the gluon has, on each
# of its two dipoles, half of g -> gg and half of g -> q qbar for every
# flavour (App. A: competing kernels, each with its own overestimate and
# veto).  The first emission then has P(t1 < t) = prod over dipoles and
# kernels of Delta_{d,k}(t), and the kind of the first emission has the
# density rho_k(t) Delta(t), both computed here by quadrature.
QGQ_X = (0.8, 0.5, 0.7)  # x_q, x_g, x_qbar


def _qgq_state(sqrt_s, flavour=1):
    xq, xg, xqb = QGQ_X
    s = sqrt_s ** 2
    eq, eqb = 0.5 * xq * sqrt_s, 0.5 * xqb * sqrt_s
    cos_qqb = 1.0 - (1.0 - xg) * s / (2.0 * eq * eqb)
    sin_qqb = math.sqrt(1.0 - cos_qqb ** 2)
    pq = np.array([eq, 0.0, 0.0, eq])
    pqb = np.array([eqb, eqb * sin_qqb, 0.0, eqb * cos_qqb])
    pg = np.array([sqrt_s - eq - eqb, -(pq[1] + pqb[1]), -(pq[2] + pqb[2]), -(pq[3] + pqb[3])])
    mom = np.stack([pq, pg, pqb])
    info = np.array([[flavour, 1, 0], [21, 2, 1], [-flavour, 0, 2]], dtype=np.int32)
    return mom, info


def _z_integral(t, q2, kind):
    """int dz (1 - y) P(z, y) over the z range with y = t / (Q^2 z (1-z)) < 1;
    P as pinned by its collinear limits: 0 q->qg (C_F), 1 half g->gg, 2 half
    g->q qbar of one flavour."""
    if t >= q2 / 4:
        return 0.0
    root = math.sqrt(1 - 4 * t / q2)
    zlo, zhi = 0.5 * (1 - root), 0.5 * (1 + root)

    def f(z):
        y = t / (q2 * z * (1 - z))
        if kind == 0:
            p = CF * (2 / (1 - z * (1 - y)) - (1 + z))
        elif kind == 1:
            p = 0.5 * CA * (2 / (1 - z * (1 - y)) - 2 + z * (1 - z))
        else:
            p = 0.5 * TR * (1 - 2 * z * (1 - z))
        return (1 - y) * p

    val, _ = integrate.quad(f, zlo, zhi, epsabs=1e-13, epsrel=1e-11, limit=200)
    return val


def _qgq_prediction(sqrt_s, tc, as_mz, fixed, nf, n_bins, sub=60):
    """Bin edges in t (log-uniform from t_C to the largest dipole's s/4-like
    end), and per bin the probability of a first emission of each kind
    (q->qg, g->gg, g->q qbar summed over flavours) plus the probability of
    none above t_C; the emission CDF on the fine grid for a KS test."""
    s = sqrt_s ** 2
    xq, xg, xqb = QGQ_X
    q2a, q2b = s * (1 - xqb), s * (1 - xq)  # (q|g) and (g|qbar) masses
    tmax = max(q2a, q2b) / 4
    lt = np.linspace(math.log(tc), math.log(tmax), n_bins * sub + 1)
    t = np.exp(lt)
    rho = np.zeros((3, len(t)))  # per kind, d P / d ln t
    for j, tj in enumerate(t):
        a = _alphas(tj, as_mz, fixed, nf) / (2 * math.pi)
        for q2 in (q2a, q2b):
            rho[0, j] += a * _z_integral(tj, q2, 0)
            rho[1, j] += a * _z_integral(tj, q2, 1)
            rho[2, j] += a * nf * _z_integral(tj, q2, 2)
    tot = rho.sum(axis=0)
    # F(L) = int_L^Lmax tot dL': cumulative trapezoid from the top
    h = np.diff(lt)
    seg = 0.5 * h * (tot[1:] + tot[:-1])
    F = np.append(np.cumsum(seg[::-1])[::-1], 0.0)
    delta = np.exp(-F)
    dens = rho * delta  # joint density of (ln t1, kind)
    seg_k = 0.5 * h * (dens[:, 1:] + dens[:, :-1])  # per fine interval
    probs = seg_k.reshape(3, n_bins, sub).sum(axis=2)
    edges = t[::sub]
    p_none = delta[0]
    return edges, probs, p_none, lt, delta


def _qgq_first_emission(O, fixed, mutation=0, n=200000, seed=31, nf=5):
    sqrt_s, tc, as_mz = 91.2, 1.0, 0.118
    mom, info = _qgq_state(sqrt_s)
    p = O.make_params(sqrt_s=sqrt_s, t_cutoff=tc, alphas_mz=as_mz, seed=seed, fixed_alphas=fixed, n_flavours=nf,
                      max_emissions=1, mutation=mutation, capacity=8)
    r = O.run_from_state(p, mom, info, 0, n, threads=_threads(O), want_momenta=True)
    ev, fin = r["events"], r["info"]
    t1 = ev["t_first"]
    emitted = ev["n_emissions"] == 1
    assert np.all(emitted == (t1 > 0))
    new = fin[:, 3]  # the emitted parton (flavour, colour, anticolour)
    m = 3  # the first new colour line: the state uses lines 1 and 2
    kind = np.full(n, -1)
    gluon = emitted & (new[:, 0] == 21)
    split_g = (fin[:, 1, 1] == m) | (fin[:, 1, 2] == m)  # the gluon took the new line: it split
    kind[gluon & ~split_g] = 0
    kind[gluon & split_g] = 1
    kind[emitted & (new[:, 0] < 0)] = 2
    assert np.all(kind[emitted] >= 0)
    qq = kind == 2
    # g -> q qbar: the gluon (slot 1) became the quark of the new antiquark's flavour
    assert np.all(fin[qq, 1, 0] == -new[qq, 0])
    flavours = np.bincount(-new[qq, 0], minlength=nf + 1)[1:]
    edges, probs, p_none, lt, delta = _qgq_prediction(sqrt_s, tc, as_mz, fixed, nf, n_bins=24)
    obs = np.zeros_like(probs)
    for k in range(3):
        obs[k], _ = np.histogram(t1[kind == k], bins=edges)
    exp = probs * n
    cells = exp > 5
    chi2 = float(np.sum((obs[cells] - exp[cells]) ** 2 / exp[cells]))
    chi2 += (np.sum(~emitted) - p_none * n) ** 2 / (p_none * n)
    ndf = int(cells.sum())
    spline = interpolate.CubicSpline(lt, np.log(delta))
    cdf = lambda t: (np.exp(spline(np.log(t))) - p_none) / (1 - p_none)
    ks = stats.kstest(t1[emitted], cdf).pvalue
    flav_p = stats.chisquare(flavours).pvalue
    return {"chi2_ndf": chi2 / ndf, "ndf": ndf, "ks": ks, "flavour_p": flav_p, "flavours": flavours,
            "kinds": np.bincount(kind[emitted], minlength=3), "expected_kinds": probs.sum(axis=1) * n}


@pytest.mark.parametrize("fixed", [1, 0])
def test_gluon_branches_match_exact_sudakov(oracle_mod, fixed):
    """From the q g qbar state, the first emission's scale and kind (q->qg,
    g->gg, g->q qbar) follow rho_k(t) prod Delta, binned chi^2/ndf < 2 and KS
    p > 1e-3, at fixed and running alpha_s; the g->q qbar flavours are equally
    shared (chi^2 p > 1e-3)."""
    r = _qgq_first_emission(oracle_mod, fixed)
    assert r["chi2_ndf"] < 2.0, r
    assert r["ks"] > 1e-3, r
    assert r["flavour_p"] > 1e-3, r
    assert r["kinds"][2] > 2000, r  # the g->q qbar branch is well populated


@pytest.mark.parametrize("mutation", [1 << 14, 1 << 15, 1 << 16])
def test_gluon_pin_catches_planted_mistakes(oracle_mod, mutation):
    """n_f - 1 g->q qbar kernels, both kernels of a trial slot drawing the
    same uniform, or g->gg without the half weight each break the pin."""
    r = _qgq_first_emission(oracle_mod, 1, mutation=mutation)
    assert r["chi2_ndf"] > 10.0 or r["ks"] < 1e-6 or r["flavour_p"] < 1e-6, r
