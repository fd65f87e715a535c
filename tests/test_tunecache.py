"""The autotuner's pick cache (host logic): signatures and the JSON round trip."""
import json

import numpy as np

from paper_1703_09619_gb300 import tunecache as TC
from paper_1703_09619_gb300 import workloads as W


def test_signature_depends_on_shape_not_element_order():
    wl = W.make("c4", 64)
    k = TC.signature(wl.orders, 16, 1, 0xF, "GB300")
    perm = np.random.default_rng(0).permutation(wl.n_elem)
    assert TC.signature(wl.orders[perm], 16, 1, 0xF, "GB300") == k
    assert TC.signature(wl.orders, 12, 1, 0xF, "GB300") != k        # another rule
    assert TC.signature(wl.orders, 16, 0, 0xF, "GB300") != k        # another precision
    assert TC.signature(wl.orders, 16, 1, 0x3, "GB300") != k        # other types
    assert TC.signature(wl.orders, 16, 1, 0xF, "B200") != k         # another device
    assert TC.signature(wl.orders[:63], 16, 1, 0xF, "GB300") != k   # another batch
    o2 = wl.orders.copy()
    o2[0, 0, 0] = 9 - o2[0, 0, 0] if o2[0, 0, 0] != 4 else 5
    assert TC.signature(o2, 16, 1, 0xF, "GB300") != k               # another order histogram
    g = np.full(wl.n_elem, 16)
    assert TC.signature(wl.orders, g, 1, 0xF, "GB300") == k          # a per-element rule of one size


def test_tuned_tile_tunes_once_then_hits(tmp_path, monkeypatch):
    path = tmp_path / "tiles.json"
    monkeypatch.setenv("P2S_TUNE_CACHE", str(path))
    calls = []

    def tune():
        calls.append(1)
        return {"combo_target": 512, "unit_kbytes": 100, "threads": 512, "kernel": 2}, 1.25, 40

    wl = W.make("c4", 32)
    key = TC.signature(wl.orders, 16, 1, 0xF, "GB300")
    tile, info = TC.tuned_tile(tune, key, workload="c4")
    assert info["cache"] == "miss" and len(calls) == 1
    tile2, info2 = TC.tuned_tile(tune, key, workload="c4")
    assert info2["cache"] == "hit" and len(calls) == 1 and tile2 == tile
    d = json.loads(path.read_text())
    assert d[key]["tile"]["kernel"] == 2 and d[key]["candidates"] == 40


def test_shipped_table_is_valid():
    """The shipped picks parse and name tile shapes the library accepts."""
    d = json.loads(open(TC.SHIPPED).read())
    assert d
    for key, e in d.items():
        assert key.count("|") == 5 and key.split("|")[1] in ("p0", "p1")
        t = e["tile"]
        assert 0 <= t["combo_target"] <= 4096 and 0 <= t["unit_kbytes"] <= 227
        assert t["threads"] == 0 or (64 <= t["threads"] <= 512 and t["threads"] % 32 == 0)
        assert t["kernel"] in (0, 1, 2)
