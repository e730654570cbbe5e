"""The autotuners' persisted cache (dsrg_tune_cache_get / _put): a flat JSON
object of integer choices in a file, read and written through the C ABI with
no GPU. The GPU side (the autotuners applying a stored choice without timing)
is in tests/test_gpu_batch.py."""
import json
import os

import pytest


@pytest.fixture(scope="module")
def pk():
    import paper_1603_00561_gb300 as pk
    from paper_1603_00561_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        pytest.skip("library not built")
    return pk


def test_put_then_get_round_trip(pk, tmp_path):
    path = tmp_path / "tune.json"
    assert pk.tune_cache_get(path, "ccvv-schedule|NVIDIA GB300 sm_103|bf16x3|c24-t10-k112-w1") is None
    pk.tune_cache_put(path, "ccvv-schedule|NVIDIA GB300 sm_103|bf16x3|c24-t10-k112-w1", 4)
    pk.tune_cache_put(path, "batch-branches|NVIDIA GB300 sm_103|bf16x3|n64-i15360-q2112", 2)
    pk.tune_cache_put(path, "ccvv-schedule|NVIDIA GB300 sm_103|bf16x3|c24-t10-k112-w1", 17)
    assert pk.tune_cache_get(path, "ccvv-schedule|NVIDIA GB300 sm_103|bf16x3|c24-t10-k112-w1") == 17
    assert pk.tune_cache_get(path, "batch-branches|NVIDIA GB300 sm_103|bf16x3|n64-i15360-q2112") == 2
    # the file is plain JSON that other tools can read, with no temporary file left behind
    data = json.loads(path.read_text())
    assert data == {"ccvv-schedule|NVIDIA GB300 sm_103|bf16x3|c24-t10-k112-w1": 17,
                    "batch-branches|NVIDIA GB300 sm_103|bf16x3|n64-i15360-q2112": 2}
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]


def test_large_and_negative_values(pk, tmp_path):
    path = tmp_path / "t.json"
    pk.tune_cache_put(path, "a", (12 << 16) | 9)
    pk.tune_cache_put(path, "b", -1)
    assert pk.tune_cache_get(path, "a") == (12 << 16) | 9
    assert pk.tune_cache_get(path, "b") == -1


def test_reads_a_file_written_by_hand(pk, tmp_path):
    path = tmp_path / "t.json"
    path.write_text('{ "x|y": 3 ,\n\t"z": 42}')
    assert pk.tune_cache_get(path, "x|y") == 3
    assert pk.tune_cache_get(path, "z") == 42
    path.write_text("{}")
    assert pk.tune_cache_get(path, "z") is None


def test_malformed_file_is_reported_and_replaced(pk, tmp_path):
    path = tmp_path / "t.json"
    path.write_text('{"a": "not a number"}')
    with pytest.raises(ValueError):
        pk.tune_cache_get(path, "a")
    pk.tune_cache_put(path, "a", 5)     # a store starts a fresh object
    assert pk.tune_cache_get(path, "a") == 5


def test_bad_keys_and_paths(pk, tmp_path):
    with pytest.raises(pk.DSRGError):
        pk.tune_cache_put(tmp_path / "t.json", 'with "quote"', 1)
    with pytest.raises(pk.DSRGError):
        pk.tune_cache_put(tmp_path / "no_such_dir" / "t.json", "k", 1)
    assert pk.tune_cache_get(tmp_path / "absent.json", "k") is None
