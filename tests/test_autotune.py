"""The launch autotuner: the tuning table's C ABI (ranges, defaults), the nearest-size rule that
spreads tuned sizes over all size classes, the JSON cache's device check and validation (CPU);
and on the GPU that a tuning run keeps only measured gains and that outputs do not depend on the
grids chosen."""
import json

import pytest
import torch

from paper_1704_00513_gb300 import autotune, fqbfs
from paper_1704_00513_gb300 import build as fqbuild


@pytest.fixture(autouse=True)
def _clean_table():
    fqbuild.build()
    autotune.reset()
    yield
    autotune.reset()


def test_table_ranges_and_defaults():
    assert fqbfs.tune_get("bu_sweep", 24) == 0
    fqbfs.tune_set("bu_sweep", 24, 6)
    assert fqbfs.tune_get("bu_sweep", 24) == 6 and fqbfs.tune_get("bu_sweep", 23) == 0
    for bad in [(len(fqbfs.TUNE_SITES), 0, 1), (0, fqbfs.TUNE_MAX_CLASS + 1, 1), (0, 10, 33)]:
        assert fqbfs.lib().fq_tune_set(*bad) == fqbfs.FQ_EINVAL
    assert fqbfs.lib().fq_tune_get(99, 0) == 0


def test_nearest_tuned_size_governs_every_class():
    entries = [{"site": "enc_pack", "class": 20, "ctas_per_sm": 2}, {"site": "enc_pack", "class": 26, "ctas_per_sm": 8}]
    autotune.apply(entries)
    got = [fqbfs.tune_get("enc_pack", c) for c in range(fqbfs.TUNE_MAX_CLASS + 1)]
    assert got[:23] == [2] * 23   # classes 0..22 are nearer to 20
    assert got[23:] == [8] * (fqbfs.TUNE_MAX_CLASS + 1 - 23)  # 23 ties (3 and 3): the larger size wins
    assert fqbfs.tune_get("enc_widths", 20) == 0  # untouched sites keep the built-in grid


def test_cache_is_device_keyed_and_validated(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "device_key", lambda dev: {"name": "GPU-A", "sms": 152})
    path = str(tmp_path / "tune.json")
    autotune.save(path, None, [{"site": "bu_sweep", "class": 24, "ctas_per_sm": 4}])
    assert autotune.load(path, None) is not None and fqbfs.tune_get("bu_sweep", 24) == 4
    autotune.reset()
    monkeypatch.setattr(autotune, "device_key", lambda dev: {"name": "GPU-B", "sms": 152})
    assert autotune.load(path, None) is None and fqbfs.tune_get("bu_sweep", 24) == 0
    doc = json.load(open(path))
    doc["device"] = {"name": "GPU-B", "sms": 152}
    doc["entries"][0]["ctas_per_sm"] = 99
    json.dump(doc, open(path, "w"))
    with pytest.raises(ValueError):
        autotune.load(path, None)


@pytest.mark.gpu
def test_tuning_keeps_only_gains_and_outputs_do_not_depend_on_grids():
    dev = torch.device("cuda")
    entries = autotune.tune_codec(dev, log_sizes=(16, 18), reps=2)
    for e in entries:
        assert e["ctas_per_sm"] == 0 or e["ms"] <= e["default_ms"] * (1 - autotune.MIN_GAIN) + 1e-9
    from paper_1704_00513_gb300 import inputs
    v = inputs.geometric_set(300_000, 9.0, seed=5, device=dev).to(torch.int32)
    ref, _ = fqbfs.fq_frontier_encode(v)
    ref = ref.clone()
    for c in (1, 3, 16):
        for site in ("enc_widths", "enc_pack", "dec_unpack"):
            fqbfs.tune_set(site, 18, c)
        out, _ = fqbfs.fq_frontier_encode(v)
        assert torch.equal(out, ref)
        assert torch.equal(fqbfs.fq_frontier_decode(out, cap=v.numel()), v)


@pytest.mark.gpu
def test_batched_and_bfs_tuning_run_and_keep_results():
    dev = torch.device("cuda")
    entries = autotune.tune_batch(dev, S=64, hi=1 << 14, reps=1)
    assert {e["site"] for e in entries} == {"bat_encode", "bat_dunpack"}
    from paper_1704_00513_gb300 import inputs
    off, cols = inputs.rmat_csr(14, 16, seed=20170402, device="cuda")
    g = fqbfs.Graph(off, cols)
    roots = inputs.pick_roots(off, 2, seed=1)
    ref = g.bfs(roots[0], flags=fqbfs.FQ_BFS_DEVICE_LOOP).depth.clone()
    e2 = autotune.tune_bfs(g, roots)
    assert {e["site"] for e in e2} == {"bu_sweep", "td_hub"}
    fqbfs.tune_set("bu_sweep", 14, 1)   # the device-loop graph rebuilds with the new grid
    assert torch.equal(g.bfs(roots[0], flags=fqbfs.FQ_BFS_DEVICE_LOOP).depth, ref)
    g.close()
