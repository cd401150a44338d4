"""The autotuner's persisted cache (rs_tune_cache_*): host-side file handling,
no GPU needed.  Lines naming shapes this build compiles are merged, others
(unknown shapes, digit widths out of range, bad key sizes, garbage) are
skipped; a saved file reads back to the same entries."""
import os


def _line(gpu="NVIDIA GB300", algo=0, kb=4, vals=0, kbits=32, l2n=26, d=8, block=256, items=22):
    return (f'{{"gpu": "{gpu}", "algo": {algo}, "key_bytes": {kb}, "values": {vals}, "key_bits": {kbits}, '
            f'"log2n": {l2n}, "digit_bits": {d}, "block_threads": {block}, "items_per_thread": {items}}}')


def test_round_trip_and_stale_lines(tmp_path):
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    _lib.rs_tune_cache_clear()
    assert _lib.rs_tune_cache_size() == 0
    src = tmp_path / "tune.json"
    lines = [
        _line(),                                             # radix u32 keys only, a compiled shape
        _line(algo=0, kb=8, vals=1, kbits=64, l2n=20, block=384, items=10),
        _line(algo=2, kb=4, l2n=32, block=256, items=24),    # segmented: compiled at 8-bit digits
        _line(algo=2, kb=4, l2n=31, d=9, block=256, items=24),  # segmented passes are 8-bit only: skipped
        _line(block=999, items=7),                           # not compiled: skipped
        _line(d=12),                                         # digit width out of range: skipped
        _line(kb=3),                                         # bad key size: skipped
        "not json at all",
        "",
    ]
    src.write_text("\n".join(lines) + "\n")
    assert _lib.rs_tune_cache_load(str(src)) == 3
    assert _lib.rs_tune_cache_size() == 3
    assert _lib.rs_tune_cache_load(str(src)) == 3  # merging the same entries again adds none
    assert _lib.rs_tune_cache_size() == 3
    out = tmp_path / "saved.json"
    assert _lib.rs_tune_cache_save(str(out)) == 3
    saved = [ln for ln in out.read_text().splitlines() if ln]
    assert len(saved) == 3 and not os.path.exists(str(out) + ".tmp")
    assert any('"block_threads": 384' in ln and '"items_per_thread": 10' in ln for ln in saved)
    _lib.rs_tune_cache_clear()
    assert _lib.rs_tune_cache_load(str(out)) == 3
    _lib.rs_tune_cache_clear()


def test_missing_file_and_unwritable_path(tmp_path):
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    assert _lib.rs_tune_cache_load(str(tmp_path / "absent.json")) == -1
    assert _lib.rs_tune_cache_save(str(tmp_path / "no_such_dir" / "x.json")) == -1


def test_check_failed_status_has_a_name():
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    assert _lib.STATUS[10] == "RS_ERR_CHECK_FAILED"
    assert "RS_ERR_CHECK_FAILED" in _lib.rs_status_string(10)
