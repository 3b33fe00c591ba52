"""Fisher-pass tiles and the autotuner: every tile (lanes per work item 4, 8,
16 x CTAs per SM 1, 2) gives the default tile's Fisher matrices within
rounding: the FP64 path only sums in a different order; in the mixed path the
lanes also start their FP32 recurrences at other points, so every point's
tangents round differently (elementwise differences ~1e-9 of
sqrt(Gamma_ii Gamma_jj), well inside its ~1e-7 accuracy); gw_autotune times the six
on a catalog, installs the fastest for its grid-length class, and the JSON
cache reinstalls it without timing."""
import numpy as np
import pytest
import torch

import gwcat
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")
from paper_2207_06910_gb300 import autotune  # noqa: E402


@pytest.fixture
def fresh_tiles():
    yield
    for prec in (gw.GW_FP64, gw.GW_MIXED):
        for cls in range(3):
            gw.gw_set_tile(prec, cls, 8, 2)


@pytest.mark.parametrize("name,n,cap", [("c3", 40, None), ("c1", 5, 1400)])
def test_every_tile_gives_the_same_fisher(fresh_tiles, name, n, cap):
    cat, d, p = oracle_catalog(name, n, max_npts=cap)
    net = gw.Network(*gwcat.network(name))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    cls = autotune.length_class_of(gcat.npts)
    for prec, tol in ((gw.GW_FP64, 1e-12), (gw.GW_MIXED, 1e-7)):
        F0, s0, st0 = gw.gw_fisher(gcat, net, 11, prec)
        dg = torch.sqrt(torch.stack([F0[i * 11 - i * (i - 1) // 2] for i in range(11)]))
        iu = np.triu_indices(11)
        norm = dg[torch.as_tensor(iu[0])] * dg[torch.as_tensor(iu[1])]
        for g, b in gw.TILES:
            gw.gw_set_tile(prec, cls, g, b)
            F, s, st = gw.gw_fisher(gcat, net, 11, prec)
            assert torch.equal(st, st0)
            assert torch.max(torch.abs(F - F0) / norm).item() < tol, (prec, g, b)
        gw.gw_set_tile(prec, cls, 8, 2)


def test_autotune_and_cache(fresh_tiles, tmp_path):
    d = gwcat.draw("c3", 2000, grid="stress")
    cat = gw.gw_prepare_catalog(d, d["npts_rule"])
    net = gw.Network(*gwcat.network("c3"))
    path = str(tmp_path / "tiles.json")
    e = autotune.tune(cat, net, 11, gw.GW_MIXED, reps=2, path=path)
    assert not e["cached"] and e["length_class"] == 2
    assert (e["group"], e["blocks_per_sm"]) in gw.TILES and len(e["ms"]) == 6
    assert min(e["ms"].values()) == e["ms"][f"{e['group']}x{e['blocks_per_sm']}"]
    print("\nstress catalog, mixed: tile ms", e["ms"], "->", e["group"], e["blocks_per_sm"])
    e2 = autotune.tune(cat, net, 11, gw.GW_MIXED, reps=2, path=path)
    assert e2["cached"] and (e2["group"], e2["blocks_per_sm"]) == (e["group"], e["blocks_per_sm"])
    assert autotune.apply(autotune.load(path)) == 1
    with pytest.raises(gw.GWError):
        gw.gw_set_tile(gw.GW_MIXED, 0, 6, 2)
