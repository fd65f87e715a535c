"""Host logic of the learned order (no GPU): the risk rule's choice over a calibration sweep,
the class weights, the class lookup and the assembly of an ensemble checkpoint."""
import numpy as np
import pytest

from paper_1703_09619_gb300 import learned as LN
from paper_1703_09619_gb300 import p2s


def sweep(*rows):
    return [{"risk": r, "above_tol": n, "max_err": 0.0, "mean_G3": 0.0} for r, n in rows]


def test_choose_risk_takes_the_largest_risk_without_failures():
    assert LN.choose_risk(sweep((0.05, 7), (0.02, 2), (0.01, 0), (0.005, 0), (0.001, 0))) == 0.01


def test_choose_risk_when_no_risk_is_clean_keeps_the_fewest_failures():
    # a confident mistake that no risk removes: the largest risk with that one failure
    assert LN.choose_risk(sweep((0.05, 8), (0.02, 2), (0.01, 1), (0.002, 1), (0.0001, 1))) == 0.01


def test_choose_risk_ignores_sweep_order():
    t = sweep((0.001, 0), (0.05, 3), (0.002, 0), (0.01, 1))
    assert LN.choose_risk(t) == 0.002
    assert LN.choose_risk(list(reversed(t))) == 0.002


def test_balanced_weights_favour_rare_classes_within_bounds():
    y = np.array([1] * 1000 + [2] * 4000 + [3] * 1500 + [4] * 20)
    w = LN.balanced_weights(y)
    assert w.shape == (6,) and np.all(w >= 0.5) and np.all(w <= 10.0)
    assert w[4] > w[3] > w[2] and w[1] > w[2]
    assert w[0] == 10.0 and w[5] == 10.0  # classes without samples take the cap


def test_classes_of_inverts_the_class_table():
    assert LN.classes_of(np.array(LN.CLASS_NPTS)).tolist() == list(range(6))


def test_committed_checkpoint_carries_its_calibration():
    P, meta = LN.load_checkpoint()
    n = meta.get("n_nets", 1)  # an ensemble stores its networks one after another
    assert 1 <= n <= 8 and P.shape == (n * 41478,) and LN.n_nets_of(P) == n
    if n > 1:
        assert len(meta["members"]) == n
    cal = meta["risk_calibration"]
    assert meta["risk"] == LN.choose_risk(cal["sweep"])
    assert cal["tol"] <= 1e-8 and "shard 1" in cal["holdout"]
    assert meta["evaluation"]["above_tol"] == 0


def test_combine_ensemble_concatenates_members():
    a = (LN.init_params(1), {"seed": 1, "epochs": 150, "risk": 0.001, "extra": "dropped"})
    b = (LN.init_params(2), {"seed": 2, "epochs": 150, "risk": 0.0005})
    P, meta = LN.combine_ensemble([a, b])
    assert P.dtype == np.float32 and P.shape == (2 * p2s.MLP_PARAMS,)
    assert np.array_equal(P[:p2s.MLP_PARAMS], a[0]) and np.array_equal(P[p2s.MLP_PARAMS:], b[0])
    assert meta["n_nets"] == LN.n_nets_of(P) == 2
    assert [m["seed"] for m in meta["members"]] == [1, 2] and "extra" not in meta["members"][0]
    # an ensemble can take an ensemble as a member; sizes outside 2..MLP_MAX_NETS are refused
    P3, meta3 = LN.combine_ensemble([(P, meta), (LN.init_params(3), {})])
    assert meta3["n_nets"] == 3
    with pytest.raises(ValueError):
        LN.combine_ensemble([a])
    with pytest.raises(ValueError):
        LN.combine_ensemble([(LN.init_params(s), {}) for s in range(p2s.MLP_MAX_NETS + 1)])
    with pytest.raises(AssertionError):
        LN.n_nets_of(np.zeros(p2s.MLP_PARAMS + 1, dtype=np.float32))


def test_binding_mlp_constants_match_header():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "p2s.h")).read()
    defs = dict(re.findall(r"#define\s+(P2S_MLP_\w+)\s+(\d+)", hdr))
    assert int(defs["P2S_MLP_MAX_NETS"]) == p2s.MLP_MAX_NETS
    assert int(defs["P2S_MLP_PARAMS"]) == p2s.MLP_PARAMS
    assert int(defs["P2S_MLP_IN"]) == p2s.MLP_IN and int(defs["P2S_MLP_CLASSES"]) == p2s.MLP_CLASSES
