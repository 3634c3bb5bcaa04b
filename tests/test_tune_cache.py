"""The batch autotuner's JSON cache (host code of the C library; no GPU needed):
entries round-trip, several keys coexist, a key is replaced in place, a missing
or malformed file reads as empty, keys with quotes and control characters
survive, unknown tiles are refused, and the file is valid JSON written without
leftovers."""

import json
import os

import pytest

from paper_2510_01190_gb300 import _binding as B


@pytest.fixture(scope="module")
def lib():
    try:
        B.load()
    except RuntimeError as e:
        pytest.skip(f"library not buildable here: {e}")
    return B


def test_round_trip_and_miss(lib, tmp_path):
    path = tmp_path / "tune.json"
    assert lib.lcp_tune_cache_lookup(path, "a") is None  # no file yet
    lib.lcp_tune_cache_store(path, "a", (32, 64), [1.5, 2.5, 0.75, 3.0])
    tile, ms = lib.lcp_tune_cache_lookup(path, "a")
    assert tile == (32, 64)
    assert ms == pytest.approx([1.5, 2.5, 0.75, 3.0])
    assert lib.lcp_tune_cache_lookup(path, "b") is None


def test_several_keys_and_replacement(lib, tmp_path):
    path = tmp_path / "tune.json"
    lib.lcp_tune_cache_store(path, "a", (64, 64), [1, 2, 3, 4])
    lib.lcp_tune_cache_store(path, "b", (16, 128), [4, 3, 2, 1])
    lib.lcp_tune_cache_store(path, "a", (32, 128))  # replaced, times zero
    assert lib.lcp_tune_cache_lookup(path, "a") == ((32, 128), [0.0, 0.0, 0.0, 0.0])
    assert lib.lcp_tune_cache_lookup(path, "b")[0] == (16, 128)
    doc = json.loads(path.read_text())
    assert doc["lcp_tune_cache"] == 1
    assert [e["key"] for e in doc["entries"]] == ["a", "b"]
    assert doc["entries"][0]["tile"] == [32, 128]
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]  # the temporary file was renamed over it


def test_malformed_file_reads_as_empty_and_is_rewritten(lib, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json at all")
    assert lib.lcp_tune_cache_lookup(path, "a") is None
    lib.lcp_tune_cache_store(path, "a", (32, 64))
    assert json.loads(path.read_text())["entries"][0]["key"] == "a"
    path.write_text("")
    assert lib.lcp_tune_cache_lookup(path, "a") is None


def test_keys_with_quotes_and_control_characters(lib, tmp_path):
    path = tmp_path / "tune.json"
    key = 'GPU "X"\\9|sm152|tab\there'
    lib.lcp_tune_cache_store(path, key, (64, 64))
    assert lib.lcp_tune_cache_lookup(path, key)[0] == (64, 64)
    assert json.loads(path.read_text())["entries"][0]["key"] == key


def test_unknown_tiles_are_refused(lib, tmp_path):
    path = tmp_path / "tune.json"
    with pytest.raises(lib.LcpError) as e:
        lib.lcp_tune_cache_store(path, "a", (7, 7))
    assert e.value.status == -1
    assert not path.exists()
    # an entry written by hand with a shape the kernel does not have is a miss
    path.write_text('{"lcp_tune_cache": 1, "entries": [{"key": "a", "tile": [7, 7], "ms": [1, 1, 1, 1]}]}')
    assert lib.lcp_tune_cache_lookup(path, "a") is None


def test_null_path_is_an_argument_error(lib):
    with pytest.raises(lib.LcpError) as e:
        lib.lcp_tune_cache_lookup(None, "a")
    assert e.value.status == -1
    with pytest.raises(lib.LcpError):
        lib.lcp_tune_cache_store(None, "a", (32, 64))


def test_unwritable_path_is_an_argument_error(lib, tmp_path):
    with pytest.raises(lib.LcpError) as e:
        lib.lcp_tune_cache_store(tmp_path / "no_such_dir" / "tune.json", "a", (32, 64))
    assert e.value.status == -1
