"""Comparison of CUDA results with the oracle (test helper).

Bit-exact: selection mask, number of surviving variations, cut flow and
histogram counts.  Reconstructed per-event means: relative 1e-5 (the
accuracy target for reconstructed masses and momenta) of the magnitude of
the averaged terms, i.e. of the mean of |value| over the surviving
variations (the oracle's reco_abs); for masses this is the mean itself, for
the signed p_z it is the scale of its terms (a mean of values of both signs
can be much smaller than each of them).
"""
import numpy as np

RTOL = 1e-5


def assert_parity(gpu, orc, *, model="semilep", what=""):
    assert np.array_equal(gpu["cutflow"].astype(np.uint64), orc["cutflow"]), \
        "%s cutflow\n gpu %s\n orc %s" % (what, gpu["cutflow"], orc["cutflow"])
    assert np.array_equal(gpu["hist"].astype(np.uint64), orc["hist"]), \
        "%s hist differs at bins %s" % (what, np.nonzero(gpu["hist"].astype(np.uint64) != orc["hist"])[0])
    bad = np.nonzero(gpu["mask"] != orc["mask"])[0]
    assert bad.size == 0, "%s mask differs at events %s" % (what, bad[:20])
    ns = gpu["n_surv"].astype(np.uint16)
    bad = np.nonzero(ns != orc["n_surv"])[0]
    assert bad.size == 0, "%s n_surv differs at events %s (gpu %s orc %s)" % (
        what, bad[:20], ns[bad[:5]], orc["n_surv"][bad[:5]])
    assert_reco(gpu["reco"], orc["reco"], orc.get("reco_abs"), model=model, what=what)


def assert_reco(g, o, oabs=None, *, model="semilep", what=""):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    oabs = np.abs(o) if oabs is None else np.asarray(oabs, dtype=np.float64)
    for k in range(4):
        scale = np.maximum(oabs[:, k], np.abs(o[:, k]))
        if model == "semilep" and k == 2:
            # p_z: relative to the neutrino momentum, |p_z| + pT(nu) = |p_z| + |MET|
            scale = oabs[:, 2] + oabs[:, 3]
        err = np.abs(g[:, k] - o[:, k])
        bad = np.nonzero(err > RTOL * scale)[0]
        assert bad.size == 0, "%s reco[%d] differs at events %s: gpu %s orc %s" % (
            what, k, bad[:10], g[bad[:5], k], o[bad[:5], k])


def max_rel_err(g, o):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    sel = o != 0
    if not sel.any():
        return 0.0
    return float(np.max(np.abs(g[sel] - o[sel]) / np.abs(o[sel])))


def assert_records(g, o, an, *, what=""):
    """Per-cut records: same (event, level) pairs; measured variables
    bit-equal (both sides round the same FP64 value to float); reconstructed
    means within RTOL of the oracle's, as in assert_reco."""
    names = list(an["record"].get("vars", ()))
    names += ["none"] * (4 - len(names))
    assert g.shape[0] == o["event"].shape[0], "%s: %d records, oracle %d" % (what, g.shape[0], o["event"].shape[0])
    assert np.array_equal(g["event"], o["event"]), "%s: record events differ" % what
    assert np.array_equal(g["level"], o["level"]), "%s: record levels differ" % what
    oabs = o["run"]["reco_abs"]
    for i, name in enumerate(names):
        gv = g["value"][:, i].astype(np.float64)
        ov = o["value"][:, i]
        if name.startswith("reco"):
            k = int(name[4])
            scale = np.maximum(oabs[o["event"], k], np.abs(ov))
            if an["model"] == "semilep" and k == 2:
                scale = oabs[o["event"], 2] + oabs[o["event"], 3]
            bad = np.nonzero(np.abs(gv - ov) > RTOL * scale)[0]
        else:
            bad = np.nonzero(g["value"][:, i] != ov.astype(np.float32))[0]
        assert bad.size == 0, "%s: value %d (%s) differs at records %s: gpu %s orc %s" % (
            what, i, name, bad[:5], gv[bad[:5]], ov[bad[:5]])
