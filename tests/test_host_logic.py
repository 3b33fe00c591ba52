"""Host-side logic of the package that needs no GPU: the work-item count of a
catalog, the autotuner's grid-length classes and its JSON cache, and the
argument checks of the per-event routing entry point that return before any
device work."""
import json
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def gw():
    from paper_2207_06910_gb300 import build
    build.build()
    import paper_2207_06910_gb300 as g
    return g


def test_work_items_counts_whole_items(gw):
    # ceil(npts / points per item), summed over events
    npts = np.array([1, 256, 257, 512, 0], dtype=np.int32)
    assert gw.work_items(npts) == 1 + 1 + 2 + 2 + 0
    assert gw.work_items(npts, gw.TC_ITEM_POINTS) == 1 + 2 + 3 + 4 + 0
    assert gw.work_items(np.zeros(0, dtype=np.int32)) == 0


def test_length_classes_follow_mean_items_per_event(gw):
    from paper_2207_06910_gb300 import autotune
    # mean items per event of ITEM_POINTS points: <= 1.5 short, <= 12 medium, else long
    assert autotune.length_class_of(np.full(10, 256)) == 0            # 1 item
    assert autotune.length_class_of(np.array([256, 512])) == 0        # 1.5 items
    assert autotune.length_class_of(np.array([257, 512])) == 1        # 2 items
    assert autotune.length_class_of(np.full(4, 12 * 256)) == 1        # 12 items
    assert autotune.length_class_of(np.full(4, 12 * 256 + 1)) == 2   # 13 items
    assert len(gw.LENGTH_CLASSES) == 3


def test_autotune_cache_round_trip_and_bad_files(tmp_path):
    from paper_2207_06910_gb300 import autotune
    p = str(tmp_path / "sub" / "cache.json")
    assert autotune.load(p) == {}                       # missing file
    c = {"GB300|152|abi7": {"mixed/short": {"group": 8, "blocks_per_sm": 2}}}
    autotune.save(c, p)
    assert autotune.load(p) == c
    assert not os.path.exists(p + ".tmp")              # written through a rename
    with open(p, "w") as f:
        f.write("{not json")
    assert autotune.load(p) == {}                       # unreadable file: no entries
    with open(p, "w") as f:
        json.dump({"a": 1}, f)
    assert autotune.load(p) == {"a": 1}


def test_autotune_cache_path_from_environment(monkeypatch, tmp_path):
    from paper_2207_06910_gb300 import autotune
    monkeypatch.setenv("GWFISH_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("GWFISH_AUTOTUNE_CACHE")
    assert autotune.cache_path().endswith(os.path.join(".cache", "gwfish", "autotune.json"))


def test_routed_and_refine_refuse_a_null_context(gw):
    lib = gw.load_library()
    n64 = gw.ctypes.c_int64(-1)
    m64 = gw.ctypes.c_int64(-1)
    st = lib.gw_fisher_routed(None, None, None, 11, 2, 1e7, 1e50, None, None, None, None, None,
                              None, None, None, None, gw.ctypes.byref(n64),
                              gw.ctypes.byref(m64), None)
    assert st == 1                                      # GW_EINVAL, before any device work
    st = lib.gw_fisher_refine(None, None, None, 11, 1e7, 1e50, None, None, None, None, None,
                              None, None, None, None, None, gw.ctypes.byref(n64), None)
    assert st == 1
