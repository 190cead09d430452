"""Launch-shape table and its cache file (host-only: no device work, so these run on the CPU;
with no device the SM count in every key is 0)."""
import json
import os
import subprocess
import sys

import pytest

import paper_2410_02408_gb300 as pc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = {"spmv_ctas_per_sm": 3, "ring_stages": 2, "bin_pipe": -1, "fuse_update": 2, "us_per_iteration": 97.5}


def _sms(tmp_path):
    """The SM count the library puts in keys on this machine (0 without a device)."""
    pc.tune_set(1, "fp64", 1, 1, SHAPE)
    path = str(tmp_path / "probe.jsonl")
    pc.tune_save(path)
    sms = json.loads(open(path).read().splitlines()[0])["sms"]
    pc.tune_clear()
    return sms


@pytest.fixture(autouse=True)
def _clean():
    pc.load()
    pc.tune_clear()
    yield
    pc.tune_clear()


def test_set_get_and_key_buckets():
    n, nnz = 2_097_152, 14_581_760
    pc.tune_set(16, "fp32", n, nnz, SHAPE)
    assert pc.tune_get(16, "fp32", n, nnz) == SHAPE
    # same key: ceil(log2 n) = 21 and round(log2(nnz / n)) = 3
    assert pc.tune_get(16, "fp32", 1_500_000, 10_000_000) == SHAPE
    # another size bucket, degree bucket, block size or precision: no entry
    assert pc.tune_get(16, "fp32", 4_194_305, 29_000_000) is None
    assert pc.tune_get(16, "fp32", n, 2 * nnz) is None
    assert pc.tune_get(32, "fp32", n, nnz) is None
    assert pc.tune_get(16, "fp64", n, nnz) is None
    # a second set replaces the entry
    pc.tune_set(16, "fp32", n, nnz, dict(SHAPE, ring_stages=4))
    assert pc.tune_get(16, "fp32", n, nnz)["ring_stages"] == 4


def test_save_load_round_trip(tmp_path):
    path = str(tmp_path / "tune.jsonl")
    pc.tune_set(16, "fp32", 2_097_152, 14_581_760, SHAPE)
    pc.tune_set(32, "tf32", 8_000_000, 255_734_998, {"spmv_ctas_per_sm": 0, "ring_stages": 3, "bin_pipe": 0})
    pc.tune_save(path)
    lines = [json.loads(x) for x in open(path).read().splitlines()]
    assert len(lines) == 2 and all(x["kind"] == "cg" for x in lines)
    assert {x["bs"] for x in lines} == {16, 32}
    assert not os.path.exists(path + ".tmp")
    pc.tune_clear()
    assert pc.tune_get(16, "fp32", 2_097_152, 14_581_760) is None
    assert pc.tune_load(path) == 2
    assert pc.tune_get(16, "fp32", 2_097_152, 14_581_760) == SHAPE
    assert pc.tune_get(32, "tf32", 8_000_000, 255_734_998)["bin_pipe"] == 0


def test_load_skips_malformed_lines(tmp_path):
    sms = _sms(tmp_path)
    path = tmp_path / "tune.jsonl"
    good = ('{"kind": "cg", "bs": 8, "prec": 1, "log2n": 12, "log2deg": 2, "sms": %d, "spmv_ctas_per_sm": 6, '
            '"ring_stages": 3, "bin_pipe": -1, "us_per_iteration": 12.5}' % sms)
    batch = ('{"kind": "batch", "n_sys": 4, "n_rows": 1000, "nnz": 9000, "prec": 1, "sms": %d, "ctas_per_sm": 1, '
             '"team_max": 8, "setup_kb": 70, "split": 2}' % sms)
    path.write_text("\n".join([
        "not json at all",
        '{"kind": "cg", "bs": 8}',                                    # missing fields
        good.replace('"ring_stages": 3', '"ring_stages": 1'),        # out of range
        good.replace('"bs": 8', '"bs": 8.5'),                        # not an integer
        good.replace('"bin_pipe": -1', '"bin_pipe": -1, "fuse_update": 3'),   # out of range
        '{"kind": "other", "x": 1}',
        good,
        batch,
        "",
    ]) + "\n")
    assert pc.tune_load(str(path)) == 2
    got = pc.tune_get(8, "fp32", 4096, 4 * 4096)
    # a line without fuse_update (files written before the field existed) takes the default 0
    assert got == {"spmv_ctas_per_sm": 6, "ring_stages": 3, "bin_pipe": -1, "fuse_update": 0,
                   "us_per_iteration": 12.5}
    # the batch line is kept and written back
    out = tmp_path / "again.jsonl"
    pc.tune_save(str(out))
    kinds = sorted(json.loads(x)["kind"] for x in out.read_text().splitlines())
    assert kinds == ["batch", "cg"]


def test_invalid_arguments(tmp_path):
    with pytest.raises(pc.PcError) as ei:
        pc.tune_set(16, "fp32", 1000, 7000, dict(SHAPE, ring_stages=1))
    assert ei.value.name == "invalid_arg"
    for bad in (dict(SHAPE, spmv_ctas_per_sm=9), dict(SHAPE, bin_pipe=3), dict(SHAPE, ring_stages=5),
                dict(SHAPE, fuse_update=3), dict(SHAPE, fuse_update=-1)):
        with pytest.raises(pc.PcError):
            pc.tune_set(16, "fp32", 1000, 7000, bad)
    with pytest.raises(pc.PcError):
        pc.tune_set(0, "fp32", 1000, 7000, SHAPE)
    with pytest.raises(pc.PcError):
        pc.tune_load(str(tmp_path / "missing.jsonl"))
    with pytest.raises(pc.PcError):
        pc.tune_save(str(tmp_path / "no_such_dir" / "t.jsonl"))


def test_cache_file_named_by_environment_is_loaded_once(tmp_path):
    sms = _sms(tmp_path)
    path = tmp_path / "tune.jsonl"
    path.write_text('{"kind": "cg", "bs": 16, "prec": 0, "log2n": 10, "log2deg": 2, "sms": %d, '
                    '"spmv_ctas_per_sm": 2, "ring_stages": 2, "bin_pipe": 1, "us_per_iteration": 0}\n' % sms)
    code = ("import paper_2410_02408_gb300 as pc; pc.load(); "
            "print(pc.tune_get(16, 'fp64', 1000, 4000))")
    env = dict(os.environ, PC_TUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert "'spmv_ctas_per_sm': 2" in out.stdout and "'bin_pipe': 1" in out.stdout
