"""Autotuned row tiling of the tensor-core Legendre GEMMs (sht_plan_create):
every tiling gives bitwise the same transforms (tiles split output rows, not
the sums over degrees or latitudes), the choice per launch width is reported
by sht_plan_query, and the JSON-lines cache file receives the timings."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from _lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
FORMS = [f for f in ("bf16x3", "bf16") if f in ps.available_precisions()]


def transforms(T, nf, form):
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, nf, form)
    spec = torch.tensor(syn.random_spectrum(T, (nf,), seed=T, nmin=0), dtype=torch.complex128, device=DEV)
    grid = torch.empty((nf, nlat, nlon), dtype=torch.float32, device=DEV)
    back = torch.empty_like(spec)
    ps.sht_inverse(plan, spec, grid)
    ps.sht_forward(plan, grid, back)
    ps.pfsh_sync_status()
    tiles = plan.tc_tiles
    plan.close()
    return grid.cpu().numpy(), back.cpu().numpy(), tiles


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("T,nf", [(255, 80), (127, 40), (511, 24)])
def test_every_tiling_gives_the_same_transforms(form, T, nf, monkeypatch):
    monkeypatch.setenv("PFSH_TC_TILES", "1")
    g1, b1, t1 = transforms(T, nf, form)
    monkeypatch.setenv("PFSH_TC_TILES", "2")
    g2, b2, t2 = transforms(T, nf, form)
    monkeypatch.delenv("PFSH_TC_TILES")
    ga, ba, ta = transforms(T, nf, form)
    nb = (2 * nf + 127) // 128
    assert t2[0][nb - 1] > t1[0][nb - 1] or t2[1][nb - 1] > t1[1][nb - 1]   # a second tiling exists
    assert np.array_equal(g1, g2) and np.array_equal(b1, b2)
    assert np.array_equal(g1, ga) and np.array_equal(b1, ba)
    for d in range(2):
        assert ta[d][nb - 1] in (t1[d][nb - 1], t2[d][nb - 1])
    print(f"\n{form} T{T} {nf} fields: row tiles chosen (synthesis, analysis) {ta[0][nb - 1]}, {ta[1][nb - 1]}")


def test_tuning_cache_file(tmp_path, monkeypatch):
    if not FORMS:
        pytest.skip("no tensor-core form built")
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("PFSH_TUNE_CACHE", str(path))
    T = 95                                        # a shape no other test tunes
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 200, FORMS[0])
    tiles = plan.tc_tiles
    plan.close()
    rows = [json.loads(line) for line in path.read_text().splitlines()]
    assert {r["dir"] for r in rows} == {0, 1}
    assert all(r["T"] == T and r["nlat"] == nlat and r["tile_mult"] in (1, 2) and len(r["us"]) == 2 for r in rows)
    for r in rows:     # the plan uses what was measured faster: 1 tile per order below 256 rows, or 2
        assert tiles[r["dir"]][r["nb"] - 1] == r["tile_mult"]
        chosen, other = r["us"][r["tile_mult"] - 1], r["us"][2 - r["tile_mult"]]
        assert chosen <= other        # (times are printed to 0.01 us; a tie may go either way)
    print("\n" + "\n".join(json.dumps(r) for r in rows))
