"""Seeded synthetic final states for the observables tests (input generation
only: nothing here computes an observable).

Events are massless n-parton final states with total momentum (sqrt(s), 0,
0, 0), drawn with the RAMBO algorithm (R. Kleiss, W. J. Stirling, S. D.
Ellis, Comput. Phys. Commun. 40 (1986) 359): n isotropic massless momenta
with energies from -ln(r1 r2), then the Lorentz boost and scaling that take
their sum to the centre-of-mass frame at energy sqrt(s).  A few constructions
add the degenerate cases the observables' searches must handle: exactly
collinear pairs and nearly symmetric planar events whose best thrust
partitions differ by a relative 1e-8.
"""
import numpy as np


def rambo(rng, n, sqrt_s):
    """One massless n-parton event, [n][4] = (E, px, py, pz)."""
    r = rng.random((n, 4))
    c = 2.0 * r[:, 0] - 1.0
    phi = 2.0 * np.pi * r[:, 1]
    q0 = -np.log(r[:, 2] * r[:, 3])
    st = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    q = np.stack([q0, q0 * st * np.cos(phi), q0 * st * np.sin(phi), q0 * c], axis=1)
    Q = q.sum(axis=0)
    M = np.sqrt(Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2)
    b = -Q[1:] / M
    x = sqrt_s / M
    gamma = Q[0] / M
    a = 1.0 / (1.0 + gamma)
    bq = q[:, 1:] @ b
    p = np.empty_like(q)
    p[:, 0] = x * (gamma * q[:, 0] + bq)
    p[:, 1:] = x * (q[:, 1:] + np.outer(q[:, 0], b) + a * np.outer(bq, b))
    return p


def split_collinear(p, i, z):
    """Replace parton i by two exactly collinear partons z p_i and (1 - z) p_i."""
    return np.concatenate([p[:i], [z * p[i]], [(1.0 - z) * p[i]], p[i + 1:]], axis=0)


def planar_polygon(n, sqrt_s, eps, rng):
    """n >= 3 partons on a regular polygon in a randomly oriented plane, each
    angle moved by a relative eps of the spacing and each energy by a
    relative eps, then the energies corrected along cos and sin of the angles
    so that the momenta still sum to zero, and rescaled to sum to sqrt(s):
    several thrust partitions, and several Durham pairs, are then equal to a
    relative ~eps (the angle jitter keeps pairs from tying exactly)."""
    ang = 2.0 * np.pi * (np.arange(n) + eps * rng.uniform(-1.0, 1.0, n)) / n
    cs, sn = np.cos(ang), np.sin(ang)
    e = (sqrt_s / n) * (1.0 + eps * rng.uniform(-1.0, 1.0, n))
    m = np.array([[np.sum(cs * cs), np.sum(sn * cs)], [np.sum(cs * sn), np.sum(sn * sn)]])
    uv = np.linalg.solve(m, -np.array([np.sum(e * cs), np.sum(e * sn)]))
    e = e + uv[0] * cs + uv[1] * sn
    e *= sqrt_s / e.sum()
    v = np.stack([e * cs, e * sn, np.zeros(n)], axis=1)
    return np.concatenate([e[:, None], v @ random_rotation(rng).T], axis=1)


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1.0
    return q


def events_with_multiplicities(seed, counts, sqrt_s):
    """A list of events, one per entry of counts (parton numbers)."""
    rng = np.random.default_rng(seed)
    return [rambo(rng, int(n), sqrt_s) for n in counts]


def pack_slot_major(events, capacity):
    """Events [n_i][4] -> slot-major arrays e, px, py, pz of [capacity][n_events]
    (zero beyond each event's partons) and the parton counts."""
    n_ev = len(events)
    out = np.zeros((4, capacity, n_ev))
    counts = np.zeros(n_ev, dtype=np.int32)
    for j, p in enumerate(events):
        k = min(len(p), capacity)
        out[:, :k, j] = p[:k].T
        counts[j] = len(p)
    return {"e": out[0], "px": out[1], "py": out[2], "pz": out[3]}, counts
