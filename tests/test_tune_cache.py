"""The tuning-cache file of MOLC_AUTOTUNE on the host (no GPU): molc_tune_cache reads a JSON cache, counts its
entries, accepts a missing file as empty and rejects what this library did not write.  The GPU side (entries
written by tuning, applied without timing) is tests/test_gpu_tune.py."""
import json

import pytest

import paper_2305_11998_gb300 as molc


def entry(key="16x16 cells", depth=4, **kw):
    e = {"key": key, "device": "dev, 152 SMs, sm_103", "build": "b0123456789abcdef", "sweep_depth": depth,
         "tile_cells": 0, "tile_groups": 0, "block_threads": 0, "best_ms": 0.25}
    e.update(kw)
    return e


def cache(entries, **kw):
    d = {"format": "molc-tune-cache", "version": 1, "entries": entries}
    d.update(kw)
    return d


@pytest.fixture
def path(tmp_path):
    yield tmp_path / "tune.json"
    molc.tune_cache(None)


def test_missing_file_is_an_empty_cache(path):
    assert molc.tune_cache(str(path)) == 0
    assert not path.exists()              # nothing is written until a plan is tuned
    assert molc.tune_cache(None) == 0


def test_entries_are_counted(path):
    es = [entry(), entry(key='quoted "key" \\ with escapes é', depth=6),
          entry(key="tiled", depth=0, tile_cells=16, tile_groups=2, block_threads=256, extra={"later": [1, 2]})]
    path.write_text(json.dumps(cache(es, note="members this version does not know are ignored")))
    assert molc.tune_cache(str(path)) == 3
    path.write_text(json.dumps(cache([])))
    assert molc.tune_cache(str(path)) == 0


@pytest.mark.parametrize("text", [
    "{bad",                                                         # not JSON
    json.dumps(cache([entry()])) + " trailing",                     # trailing characters
    json.dumps({"version": 1, "entries": []}),                      # no format
    json.dumps(cache([entry()], format="something else")),
    json.dumps(cache([entry()], version=2)),                        # another version
    json.dumps(cache({"key": "not an array"})),
    json.dumps(cache([{"device": "d", "build": "b"}])),             # entry without key
    json.dumps(cache([entry(depth=4.5)])),                          # non-integer field
    json.dumps(cache([entry(depth=-1)])),                           # out of range
    json.dumps(cache([entry(block_threads="256")])),                # wrong type
    "[" * 100 + "]" * 100,                                          # nested too deep
])
def test_foreign_or_malformed_files_are_rejected(path, text):
    path.write_text(text)
    with pytest.raises(molc.MolcError) as e:
        molc.tune_cache(str(path))
    assert e.value.code == 1 and "tune_cache" in str(e.value)
    assert path.read_text() == text      # left as it was


def test_unreadable_path_is_rejected(tmp_path):
    d = tmp_path / "a_directory"
    d.mkdir()
    with pytest.raises(molc.MolcError):
        molc.tune_cache(str(d))
    molc.tune_cache(None)


def test_host_only_plans_are_not_tuned(path):
    # MOLC_AUTOTUNE on a host-only plan times nothing and writes no entry
    assert molc.tune_cache(str(path)) == 0
    q = molc.quadrature_product(2, 8)
    P = molc.Plan(8, 8, 1.0, 1.0, *q, 2, 0.05, host_only=True, autotune=True)
    assert P.info.tuned_from_cache == 0
    P.close()
    assert not path.exists()
