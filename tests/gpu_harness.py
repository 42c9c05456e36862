"""Shared helpers of the GPU tests: run the CUDA pipeline through the C ABI and
compare it with the oracle event by event."""
import numpy as np

# Tolerances.  FP64 rounding through ~10 emissions leaves ~1e-13 relative on
# the momenta; 1e-9 leaves four orders of margin while still catching any
# FP32 value leaking into the kinematics (~1e-7).
MOM_REL = 1e-9       # per component, relative to the parton energy
MOM_ABS = 1e-12      # GeV
OBS_REL = 1e-9
OBS_ABS = 1e-12
AGREE_MIN = 0.999    # fraction of events with the identical decision sequence


def gpu_params(g, **kw):
    return g.make_params(**kw)


def oracle_params(O, capacity, **kw):
    kw = dict(kw)
    max_steps = kw.pop("max_steps", 100000)
    return O.make_params(capacity=capacity, max_steps=max_steps, **kw)


def run_gpu(g, params, n_events, capacity=128, first_event=0, stages=("me", "shower", "validate", "obs")):
    """Run the requested stages and copy everything back to numpy."""
    import torch
    ws = g.Workspace(n_events, capacity, first_event)
    out = {"ws": ws}
    if "me" in stages:
        g.generate_me(params, ws)
    if "shower" in stages:
        rc, launches = g.shower(params, ws)
        out["rc"], out["launches"] = rc, launches
    if "validate" in stages:
        g.validate(params, ws)
    if "obs" in stages:
        g.observables(params, ws)
    torch.cuda.synchronize()
    sc = {k: v.cpu().numpy() for k, v in ws.scalars().items()}
    sc["hash"] = sc["hash"].view(np.uint64)
    out["scalars"] = sc
    mom = ws.momenta()
    out["mom"] = np.stack([mom["e"].cpu().numpy(), mom["px"].cpu().numpy(), mom["py"].cpu().numpy(),
                           mom["pz"].cpu().numpy()], axis=-1).transpose(1, 0, 2)  # [n][cap][4]
    col = ws.colours()
    out["info"] = np.stack([col["flav"].cpu().numpy().astype(np.int32), col["col"].cpu().numpy().astype(np.int32),
                            col["acol"].cpu().numpy().astype(np.int32)], axis=-1).transpose(1, 0, 2)
    out["obs"] = ws.obs().cpu().numpy().T.copy()  # [n][6]
    return out


def compare_events(gpu, orc, n_check=None):
    """Event-by-event comparison.  Returns a dict of agreement figures and
    asserts the per-event tolerances on the events whose decision sequences
    agree."""
    sc = gpu["scalars"]
    ev = orc["events"]
    n = len(ev)
    same = ((sc["hash"] == ev["hash"]) & (sc["n_partons"] == ev["n_partons"]) &
            (sc["status"] == ev["status"]) & (sc["n_steps"] == ev["n_steps"]) &
            (sc["n_emissions"] == ev["n_emissions"]) & (sc["n_trials"] == ev["n_trials"]) &
            (sc["n_winners"] == ev["n_winners"]) & (sc["n_dipoles"] == ev["n_dipoles"]))
    res = {"n": n, "agree": float(same.mean()) if n else 1.0, "n_differ": int((~same).sum())}
    # The matrix element has no decisions: it must agree for every event.
    assert np.array_equal(sc["me_flavour"], ev["me_flavour"])
    np.testing.assert_allclose(sc["weight"], ev["weight"], rtol=1e-12, atol=0)
    idx = np.nonzero(same)[0]
    if n_check is not None:
        idx = idx[:n_check]
    worst_mom = 0.0
    for j in idx:
        k = ev["n_partons"][j]
        gm, om = gpu["mom"][j, :k], orc["mom"][j, :k]
        tol = MOM_REL * np.abs(om[:, :1]) + MOM_ABS
        err = np.abs(gm - om)
        worst_mom = max(worst_mom, float((err / (np.abs(om[:, :1]) + 1e-300)).max()))
        assert np.all(err <= tol), (j, gm, om)
        assert np.array_equal(gpu["info"][j, :k], orc["info"][j, :k]), j
        go, oo = gpu["obs"][j], orc["obs"][j]
        assert np.all(np.abs(go - oo) <= OBS_REL * np.abs(oo) + OBS_ABS), (j, go, oo)
    res["worst_mom_rel"] = worst_mom
    return res


def hist_chi2(h1, h2):
    """chi^2 / ndf between two weighted histograms [6][102][3], using the
    summed variances; bins empty in both are skipped."""
    chi2, ndf = 0.0, 0
    for h in range(h1.shape[0]):
        w1, v1 = h1[h, :, 0], h1[h, :, 1]
        w2, v2 = h2[h, :, 0], h2[h, :, 1]
        var = v1 + v2
        m = var > 0
        chi2 += float(np.sum((w1[m] - w2[m]) ** 2 / var[m]))
        ndf += int(m.sum())
    return chi2 / max(ndf, 1), ndf
