"""The autotuner's JSON cache (host logic, no GPU): a miss tunes and stores, a hit
applies the stored choice, an unreadable file counts as empty, and processes
that write the file at once never leave a partial file for a reader."""
import json
import multiprocessing as mp

from paper_1603_09493_gb300 import api


class _FakeBatch:
    """Stands in for a batch: the key, the tuner and the setter the cache calls."""

    def __init__(self, key):
        self.key, self.applied, self.tuned = key, None, 0

    def tuning_key(self, device_name=""):
        return f"{device_name}|{self.key}"

    def autotune(self, reps):
        self.tuned += 1
        return {"gemm_tile_n": 256, "stage_threads": 256, "gemm_raster": 0,
                "stage_islands": 2, "gemm_k_block": 32}

    def set_tuning(self, **kw):
        self.applied = kw


def test_miss_then_hit(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    b = _FakeBatch("npad=1568|B=4096|prec=1")
    first = api.Batch.autotune_cached(b, path, "GB300")
    assert first["cached"] is False and b.tuned == 1
    c = _FakeBatch("npad=1568|B=4096|prec=1")
    second = api.Batch.autotune_cached(c, path, "GB300")
    assert second["cached"] is True and c.tuned == 0
    assert c.applied == {k: v for k, v in first.items() if k != "cached"}
    # another key in the same file keeps the first entry
    d = _FakeBatch("npad=160|B=64|prec=0")
    api.Batch.autotune_cached(d, path, "GB300")
    with open(path) as f:
        assert len(json.load(f)) == 2


def test_unreadable_file_counts_as_empty(tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text('{"GB300|npad=1568": {"gemm_tile')               # cut short
    b = _FakeBatch("npad=1568|B=1|prec=1")
    assert api.Batch.autotune_cached(b, str(path), "GB300")["cached"] is False
    with open(path) as f:
        assert list(json.load(f)) == ["GB300|npad=1568|B=1|prec=1"]


def _writer(path, rank, n):
    for i in range(n):
        api.Batch.autotune_cached(_FakeBatch(f"r{rank}|i{i}"), path, "GB300")


def test_concurrent_writers_leave_whole_files(tmp_path):
    path = str(tmp_path / "tuning.json")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_writer, args=(path, r, 60)) for r in range(2)]
    for p in procs:
        p.start()
    reads = 0
    while any(p.is_alive() for p in procs):
        try:
            with open(path) as f:
                text = f.read()
        except FileNotFoundError:
            continue
        json.loads(text)                                              # never a partial write
        reads += 1
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    with open(path) as f:
        final = json.load(f)
    # a key lost to a concurrent read-merge-replace is only tuned again on its next use
    assert all(k.startswith("GB300|r") for k in final) and len(final) >= 60
    assert not list(tmp_path.glob("*.tmp"))
