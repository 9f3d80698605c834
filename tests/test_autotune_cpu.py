"""The autotuner's cache file (no GPU needed: the cache lives on the host).

tu_autotune_cache_load merges the entries of a file written in the
one-entry-per-line JSON format of tu_autotune_cache_save; the saved file is
valid JSON with the same entries; a malformed file or a shape value outside
the documented ranges is refused with TU_ERR_INVALID_ARG and merges nothing.
"""

import json

import pytest

import paper_2411_19214_gb300 as tu


@pytest.fixture()
def lib():
    try:
        return tu.load()
    except (OSError, RuntimeError) as e:  # pragma: no cover
        pytest.skip(f"library not built: {e}")


def _entry(nb, mb, kp, dtype, sms, small, split, ms, ms0):
    return (f'{{"n_bucket": {nb}, "m_bucket": {mb}, "kp": {kp}, "dtype": {dtype}, "sms": {sms}, '
            f'"small_tiles": {small}, "split": {split}, "ms": {ms}, "ms_default": {ms0}}}')


def test_cache_roundtrip(lib, tmp_path):
    tu.tu_autotune_cache_clear()
    src = tmp_path / "in.json"
    entries = [(66, 66, 128, 0, 148, 0, 3, 4.1, 4.6), (53, 60, 256, 2, 148, 2, 1, 0.2, 0.25)]
    src.write_text('{"tu_autotune": 1, "entries": [\n' + ",\n".join(_entry(*e) for e in entries) + "\n]}\n")
    tu.tu_autotune_cache_load(str(src))
    out = tmp_path / "out.json"
    tu.tu_autotune_cache_save(str(out))
    doc = json.loads(out.read_text())
    got = sorted((d["n_bucket"], d["m_bucket"], d["kp"], d["dtype"], d["sms"], d["small_tiles"], d["split"],
                  d["ms"], d["ms_default"]) for d in doc["entries"])
    assert got == sorted(entries)
    tu.tu_autotune_cache_clear()
    tu.tu_autotune_cache_save(str(out))
    assert json.loads(out.read_text())["entries"] == []


@pytest.mark.parametrize("bad", [
    '{"n_bucket": 66, "m_bucket": 66, "kp": 128}',                     # fields missing
    _entry(66, 66, 128, 0, 148, 3, 1, 1.0, 1.0),                         # no such tile mode
    _entry(66, 66, 128, 0, 148, 0, 9, 1.0, 1.0),                         # split beyond 8
])
def test_cache_load_refuses_malformed_entries(lib, tmp_path, bad):
    tu.tu_autotune_cache_clear()
    p = tmp_path / "bad.json"
    p.write_text('{"tu_autotune": 1, "entries": [\n' + _entry(1, 1, 64, 0, 148, 0, 1, 1.0, 1.0) + ",\n" + bad
                 + "\n]}\n")
    with pytest.raises(tu.TuError) as e:
        tu.tu_autotune_cache_load(str(p))
    assert e.value.status == tu.TU_ERR_INVALID_ARG
    out = tmp_path / "out.json"
    tu.tu_autotune_cache_save(str(out))
    assert json.loads(out.read_text())["entries"] == []  # nothing merged
    with pytest.raises(tu.TuError):
        tu.tu_autotune_cache_load(str(tmp_path / "missing.json"))
