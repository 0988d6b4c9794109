"""The on-disk cache of autotuned launch shapes (host logic, no GPU)."""
import json
import multiprocessing as mp

from paper_1810_04201_gb300 import wd


def test_key_names_every_input():
    k = wd.tile_cache_key((16, 16, 16, 16), 0, 18, 1, "GPU|sm_103")
    assert k == "16x16x16x16|prec0|recon18|nrhs1|GPU|sm_103"
    others = [wd.tile_cache_key((16, 16, 16, 8), 0, 18, 1, "GPU|sm_103"),
              wd.tile_cache_key((16, 16, 16, 16), 1, 18, 1, "GPU|sm_103"),
              wd.tile_cache_key((16, 16, 16, 16), 0, 12, 1, "GPU|sm_103"),
              wd.tile_cache_key((16, 16, 16, 16), 0, 18, 4, "GPU|sm_103"),
              wd.tile_cache_key((16, 16, 16, 16), 0, 18, 1, "GPU|sm_100")]
    assert len(set(others + [k])) == 6


def test_round_trip_and_merge(tmp_path):
    p = tmp_path / "tiles.json"
    c = wd.TileCache(p)
    assert c.get("a") is None
    c.put("a", (64, 1))
    c.put("b", (32, 4))
    assert wd.TileCache(p).get("a") == (64, 1) and wd.TileCache(p).get("b") == (32, 4)
    assert json.loads(p.read_text()) == {"a": [64, 1], "b": [32, 4]}
    c.put("a", (128, 2))
    assert wd.TileCache(p).get("a") == (128, 2)


def test_bad_files_count_as_empty(tmp_path):
    p = tmp_path / "tiles.json"
    p.write_text("{not json")
    assert wd.TileCache(p).get("a") is None
    p.write_text(json.dumps({"a": [64], "b": "x", "c": [32, 2]}))
    c = wd.TileCache(p)
    assert c.get("a") is None and c.get("b") is None and c.get("c") == (32, 2)
    c.put("d", (16, 2))
    assert json.loads(p.read_text())["d"] == [16, 2]


def _writer(path, i):
    wd.TileCache(path).put(f"k{i}", (32, i))


def test_concurrent_writers_leave_a_valid_file(tmp_path):
    p = str(tmp_path / "tiles.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_writer, args=(p, i)) for i in range(1, 5)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(60)
    d = json.loads(open(p).read())  # whole file, never a partial write
    assert all(d[k][0] == 32 for k in d) and len(d) >= 1
