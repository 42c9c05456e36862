"""GPU validation stage ("Validate Events", Table 1) on broken records: the
validation bits of gaps_validate equal the oracle's for records with one
planted defect each -- a 1e-9 GeV momentum offset, a parton off shell,
negative energy, a swapped or dangling colour line, a closed gluon loop, an
unbalanced flavour, a NaN -- and stay zero for clean records and for a valid
renumbering of the colour lines.  Requires a GB300."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08692_gb300 as g
    g.load()
    return g


NO_LINK = 255


def _links(info, n):
    """Colour-partner slots from colour and anticolour lines: side 0 the
    first other parton whose anticolour is this parton's colour, side 1 the
    first whose colour is its anticolour (255 = none)."""
    link = np.full((2, n), NO_LINK, dtype=np.uint8)
    for i in range(n):
        c, a = info[i, 1], info[i, 2]
        for k in range(n):
            if k == i:
                continue
            if c > 0 and link[0, i] == NO_LINK and info[k, 2] == c:
                link[0, i] = k
            if a > 0 and link[1, i] == NO_LINK and info[k, 1] == a:
                link[1, i] = k
    return link


def _plant(case, mom, info, rng, sqrt_s=91.2):
    """One defect of kind `case` in an event (mom [n][4], info [n][3]);
    returns False when the event cannot carry it."""
    n = len(mom)
    gluons = np.nonzero(info[:, 0] == 21)[0]
    quarks = np.nonzero((info[:, 0] >= 1) & (info[:, 0] <= 5))[0]
    if case == "offset":
        mom[0, 1] += 1e-9
    elif case == "off_shell":
        d = 1e-6 * mom[0, 0]
        mom[0, 0] += d
        mom[1, 0] -= d
    elif case == "negative_energy":
        mom[1] = -mom[1]
    elif case == "zero_energy":
        mom[1, 0] = 0.0
    elif case == "swapped_colour":
        if len(gluons) == 0:
            return False
        k = gluons[0]
        info[k, 1], info[k, 2] = info[k, 2], info[k, 1]
    elif case == "dangling":
        if len(gluons) == 0:
            return False
        info[gluons[0], 1] = 999
    elif case == "gluon_loop":
        # one quark line q -> ... -> qbar through all but two gluons, which
        # close on each other
        antiq = np.nonzero(info[:, 0] < 0)[0]
        if len(gluons) < 2 or len(quarks) != 1 or len(antiq) != 1:
            return False
        loop, chain = gluons[:2], gluons[2:]
        order = [quarks[0], *chain, antiq[0]]
        line = 100
        info[order[0], 1:] = (line, 0)
        for k in order[1:-1]:
            info[k, 1:] = (line + 1, line)
            line += 1
        info[order[-1], 1:] = (0, line)
        info[loop[0], 1:] = (500, 501)
        info[loop[1], 1:] = (501, 500)
    elif case == "flavour":
        if len(quarks) == 0:
            return False
        f = info[quarks[0], 0]
        info[quarks[0], 0] = f % 5 + 1
    elif case == "nan":
        mom[n - 1, 2] = np.nan
    elif case == "near_shell":
        # parton 0 given a small mass^2 m2 on either side of where the
        # kernel's exponent screen of the on-shell test stops deciding
        # (2^(u_e + u_s - 36)) and on either side of the bound 1e-10 E sqrt(s)
        e0, p2 = mom[0, 0], float(np.dot(mom[0, 1:], mom[0, 1:]))
        u = np.frexp(e0)[1] - 1 + np.frexp(sqrt_s)[1] - 1
        m2 = rng.choice([1.5 * 2.0 ** (u - 36), 1.99 * 2.0 ** (u - 36), 1.01 * 2.0 ** (u - 35),
                         0.5e-10 * e0 * sqrt_s, 3e-10 * e0 * sqrt_s])
        mom[0, 0] = np.sqrt(p2 + m2)
    elif case == "tiny_energy":
        # a subnormal energy: the bound underflows and the FP64 test decides
        mom[0] = (1e-310, 0.0, 0.0, 0.0)
    elif case == "renumbered":
        # a valid record: every colour line renamed by one permutation
        lines = np.unique(info[:, 1:][info[:, 1:] > 0])
        new = dict(zip(lines, rng.permutation(len(lines)) + 40))
        for k in range(n):
            for c in (1, 2):
                if info[k, c] > 0:
                    info[k, c] = new[info[k, c]]
    return True


CASES = ["clean", "offset", "off_shell", "negative_energy", "zero_energy", "swapped_colour", "dangling",
         "gluon_loop", "flavour", "nan", "renumbered", "near_shell", "tiny_energy"]


@pytest.mark.parametrize("sqrt_s", [91.2, 200.0])
def test_validate_bits_match_oracle_on_broken_records(g, oracle_mod, sqrt_s):
    import torch
    n_ev, cap = 4000, 128
    p = g.make_params(seed=31, sqrt_s=sqrt_s)
    ws = g.Workspace(n_ev, cap)
    g.generate_me(p, ws)
    g.shower(p, ws)
    torch.cuda.synchronize()
    sc = ws.scalars()
    npart = sc["n_partons"].cpu().numpy()
    mom_v, col_v = ws.momenta(), ws.colours()
    mom = np.stack([mom_v[c].cpu().numpy() for c in ("e", "px", "py", "pz")], axis=-1)  # [cap][n][4]
    info = np.stack([col_v["flav"].cpu().numpy().astype(np.int32), col_v["col"].cpu().numpy().astype(np.int32),
                     col_v["acol"].cpu().numpy().astype(np.int32)], axis=-1)  # [cap][n][3]
    link = col_v["link"].cpu().numpy()  # [2][cap][n]
    rng = np.random.default_rng(5)
    planted = {}
    for j in range(n_ev):
        case = CASES[j % len(CASES)]
        if case == "clean":
            continue
        k = npart[j]
        m, i = mom[:k, j].copy(), info[:k, j].copy()
        if not _plant(case, m, i, rng, sqrt_s):
            continue
        mom[:k, j], info[:k, j] = m, i
        link[:, :k, j] = _links(i, k)
        planted[j] = case
    for c, v in zip(("e", "px", "py", "pz"), np.moveaxis(mom, -1, 0)):
        mom_v[c].copy_(torch.from_numpy(np.ascontiguousarray(v)))
    col_v["flav"].copy_(torch.from_numpy(info[..., 0].astype(np.int8)))
    col_v["col"].copy_(torch.from_numpy(info[..., 1].astype(np.int16)))
    col_v["acol"].copy_(torch.from_numpy(info[..., 2].astype(np.int16)))
    col_v["link"].copy_(torch.from_numpy(link))
    g.validate(p, ws)
    bits = sc["valid"].cpu().numpy()
    want = np.array([oracle_mod.validate(mom[:npart[j], j], info[:npart[j], j], sqrt_s) for j in range(n_ev)])
    assert np.array_equal(bits, want), [(j, planted.get(j), bits[j], want[j]) for j in np.nonzero(bits != want)[0][:10]]
    by_case = {c: bits[[j for j, cc in planted.items() if cc == c]] for c in CASES[1:]}
    for c in CASES[1:]:
        assert len(by_case[c]) > 50, c  # every defect was planted many times
    expected_bit = {"offset": 1, "off_shell": 2, "negative_energy": 4, "zero_energy": 4, "swapped_colour": 8,
                    "dangling": 8, "gluon_loop": 8, "flavour": 16, "nan": 32}
    for c, b in expected_bit.items():
        assert np.all(by_case[c] & b), c
    assert np.all(by_case["renumbered"] == 0)
    # the near-shell partons fall on both sides of the bound
    assert np.any(by_case["near_shell"] & 2) and np.any((by_case["near_shell"] & 2) == 0)
    clean = [j for j in range(n_ev) if j not in planted]
    assert np.all(bits[clean] == 0)
